"""Thin ctypes binding of libldg.so (see include/ldg.h for every contract).

Functions carry the C names and only marshal arguments: torch CUDA tensors
are passed as raw device pointers together with torch's current CUDA
stream, host numpy arrays as host pointers. There is no fallback: if the
library is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libldg.so")

EQ = {"poisson": 0, "euler": 1, "ns": 2, "advection": 3}
FLUX = {"roe": 0, "lf": 1}
BC = {"dirichlet": 0, "wall": 1, "neumann": 2}
PREC_FP32, PREC_FP64 = 0, 1
MODE_FP64, MODE_MIXED = 0, 1
PRED_EXTRAP, PRED_GIVEN, PRED_CHECKED = 0, 1, 2
ERRORS = {-1: "LDG_ERR_ARG", -2: "LDG_ERR_CUDA", -3: "LDG_ERR_MESH", -4: "LDG_ERR_NONFINITE",
          -5: "LDG_ERR_GMRES_BREAKDOWN", -6: "LDG_ERR_NEWTON_MAXIT", -7: "LDG_ERR_NOT_BUILT",
          -8: "LDG_ERR_UNSUPPORTED", -9: "LDG_ERR_TOO_LARGE"}


class LdgError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {ERRORS.get(code, code)}")
        self.code = code


class ldg_mesh_t(C.Structure):
    _fields_ = [("D", C.c_int32), ("p", C.c_int32), ("n_elem", C.c_int64),
                ("s", C.c_void_p), ("nodes", C.c_void_p), ("vertices", C.c_void_p),
                ("btag", C.c_void_p), ("switches", C.c_void_p)]


class ldg_equations_t(C.Structure):
    _fields_ = [("kind", C.c_int32), ("flux", C.c_int32), ("gamma", C.c_double),
                ("mu", C.c_double), ("Pr", C.c_double), ("C11", C.c_double),
                ("C11_b", C.c_double), ("adv", C.c_double * 3), ("n_bc", C.c_int32),
                ("bc_kind", C.c_void_p), ("g_D", C.c_void_p), ("source", C.c_void_p),
                ("g_N", C.c_void_p), ("C22", C.c_double)]


class ldg_solver_opts_t(C.Structure):
    _fields_ = [("mode", C.c_int32), ("predictor", C.c_int32), ("first_step", C.c_int32),
                ("restart", C.c_int32), ("max_newton", C.c_int32), ("reuse", C.c_int32),
                ("max_refine", C.c_int32), ("force_rebuild", C.c_int32),
                ("rtol", C.c_double), ("gmres_tol", C.c_double), ("stall_rebuild", C.c_int32),
                ("forcing", C.c_int32), ("ortho", C.c_int32), ("reorth_factor", C.c_double)]


class ldg_step_stats_t(C.Structure):
    _fields_ = [("newton_its", C.c_int32), ("gmres_its", C.c_int32), ("jac_builds", C.c_int32),
                ("refine_sweeps", C.c_int32), ("res0", C.c_double), ("res_final", C.c_double),
                ("res_pred", C.c_double), ("t_residual_ms", C.c_double),
                ("t_jacobian_ms", C.c_double), ("t_precond_ms", C.c_double),
                ("t_linear_ms", C.c_double), ("res_extrap", C.c_double), ("pred_weight", C.c_double),
                ("reorth_its", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = C.c_void_p
_I = C.c_int
_SIGS = {
    "ldg_setup": [C.POINTER(ldg_mesh_t), C.POINTER(ldg_equations_t), C.POINTER(_P)],
    "ldg_setup_host": [C.POINTER(ldg_mesh_t), C.POINTER(ldg_equations_t), _P, _P, _P, _P, _P, _P],
    "ldg_destroy": [_P],
    "ldg_info": [_P, _P],
    "ldg_export_tables": [_P, _P, _P],
    "ldg_residual": [_P, _P, _P, _P],
    "ldg_gradient": [_P, _P, _P, _P],
    "ldg_residual_uq": [_P, _P, _P, _P, _P],
    "ldg_norm2": [_P, _P, C.c_int64, C.POINTER(C.c_double), _P],
    "ldg_jacobian": [_P, _P, _I, C.POINTER(_P), _P],
    "ldg_jac_destroy": [_P],
    "ldg_jac_export": [_P, _P, _P, _P],
    "ldg_jacvec": [_P, _P, C.c_double, C.c_double, _P, _P, _I, _P],
    "ldg_precond": [_P, _P, C.c_double, C.c_double, C.POINTER(_P), _P],
    "ldg_precond_apply": [_P, _P, _P, _P, _I, _P],
    "ldg_pc_destroy": [_P],
    "ldg_pc_export": [_P, _P],
    "ldg_launch_count": [C.POINTER(C.c_longlong)],
    "ldg_kernel_timer": [C.c_int32],
    "ldg_kernel_timer_read": [C.c_int32, C.c_int32, C.POINTER(C.c_longlong), C.POINTER(C.c_double),
                              C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "ldg_residual_noalloc": [_P, _P, _P, _P],
    "ldg_fp64_fma_probe": [C.c_int32, _P, C.c_int64, C.POINTER(C.c_double), _P],
    "ldg_k21_apply": [_P, _P, _P, _P, _I, _P],
    "ldg_jacvec_g": [_P, _P, C.c_double, C.c_double, _P, _P, _P, _I, _P],
    "ldg_jacobian_uq": [_P, _P, _P, _I, C.POINTER(_P), _P],
    "ldg_set_viscosity": [_P, C.c_double],
    "ldg_mlp_create": [C.c_int32, C.c_int32, C.POINTER(_P)],
    "ldg_mlp_destroy": [_P],
    "ldg_mlp_params": [_P, _P, C.c_int32],
    "ldg_mlp_set_scaling": [_P, _P, _P, _P],
    "ldg_mlp_forward": [_P, _P, C.c_int64, _P, _P],
    "ldg_mlp_grad": [_P, _P, _P, C.c_int64, _P, _P, _P],
    "ldg_mlp_train_step": [_P, _P, _P, C.c_int64, C.c_double, _P, _P],
    "ldg_line_features": [_P, _P, _P, _P, _P, _P, _P],
    "ldg_line_targets": [_P, _P, _P, _P, _P, _P, _P],
    "ldg_mlp_predict": [_P, _P, _P, _P, _P, _P, _P],
    "ldg_newton_step": [_P, _P, _P, _P, _P, C.c_double, C.POINTER(ldg_solver_opts_t),
                        C.POINTER(ldg_step_stats_t), _P],
    "ldg_dirk3_step": [_P, _P, _P, C.c_double, C.POINTER(ldg_solver_opts_t), C.POINTER(ldg_step_stats_t), _P],
    "ldg_rk4_step": [_P, _P, _P, C.c_double, _P],
    "ldg_steady_solve": [_P, _P, C.c_double, C.c_double, C.c_int32, C.POINTER(ldg_solver_opts_t),
                         C.POINTER(ldg_step_stats_t), _P],
    "ldg_gradient_uq": [_P, _P, _P, _P, _P],
    "ldg_coupled_solve": [_P, _P, _P, C.c_double, C.c_int32, C.c_int32, C.POINTER(ldg_step_stats_t), _P],
}


def lib():
    """Load libldg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1204_1533_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.argtypes = args
            f.restype = C.c_int
        _lib = L
    return _lib


def declared_symbols():
    """Names of the entry points declared in include/*.h."""
    import re
    inc = os.path.join(os.path.dirname(HERE), "include")
    names = set()
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            txt = open(os.path.join(inc, fn)).read()
            names.update(re.findall(r"^int\s+(ldg_\w+)\s*\(", txt, re.M))
    return sorted(names)


def _check(rc, where):
    if rc != 0:
        raise LdgError(rc, where)


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# marshalling of mesh / equations dictionaries
# ---------------------------------------------------------------------------
class _Marshal:
    """Holds the host arrays alive while the C structures point at them."""

    def __init__(self, mesh, eq):
        self.s = np.ascontiguousarray(mesh["s"], dtype=np.float64)
        self.nodes = np.ascontiguousarray(mesh["nodes"], dtype=np.float64)
        self.verts = np.ascontiguousarray(mesh["vertices"], dtype=np.int64)
        self.btag = np.ascontiguousarray(mesh["btag"], dtype=np.int32)
        self.sw = None if mesh.get("switches") is None else np.ascontiguousarray(mesh["switches"], dtype=np.int8)
        if self.sw is not None and self.sw.size != self.nodes.shape[0] * int(mesh["D"]) * 2:
            raise ValueError("switches: expected [n_elem, D, 2]")
        self.mesh = ldg_mesh_t(int(mesh["D"]), int(mesh["p"]), int(self.nodes.shape[0]),
                               self.s.ctypes.data, self.nodes.ctypes.data, self.verts.ctypes.data,
                               self.btag.ctypes.data, None if self.sw is None else self.sw.ctypes.data)
        bc = eq.get("bc", {0: "dirichlet"})
        nbc = (max(bc) + 1) if bc else 0
        self.bck = np.zeros(max(nbc, 1), dtype=np.int32)
        for t, k in bc.items():
            self.bck[t] = BC[k]
        self.gD = None if eq.get("gD") is None else np.ascontiguousarray(eq["gD"], dtype=np.float64)
        self.src = None if eq.get("source") is None else np.ascontiguousarray(eq["source"], dtype=np.float64)
        self.gN = None if eq.get("gN") is None else np.ascontiguousarray(eq["gN"], dtype=np.float64)
        D, npe = int(mesh["D"]), self.nodes.shape[1]
        nc = D + 2 if eq["kind"] in ("euler", "ns") else 1
        for name, a, per in (("gD", self.gD, nc), ("source", self.src, nc), ("gN", self.gN, nc * D)):
            if a is not None and a.size != self.nodes.shape[0] * per * npe:
                raise ValueError(f"{name}: expected {self.nodes.shape[0] * per * npe} values, got {a.size}")
        adv = list(eq.get("adv", [0.0, 0.0, 0.0])) + [0.0] * 3
        self.eq = ldg_equations_t(
            EQ[eq["kind"]], FLUX[eq.get("flux", "roe")], float(eq.get("gamma", 1.4)),
            float(eq.get("mu", 0.0)), float(eq.get("Pr", 0.72)), float(eq.get("C11", 0.0)),
            float(eq.get("C11b", 1.0)), (C.c_double * 3)(*adv[:3]), nbc, self.bck.ctypes.data,
            None if self.gD is None else self.gD.ctypes.data,
            None if self.src is None else self.src.ctypes.data,
            None if self.gN is None else self.gN.ctypes.data, float(eq.get("C22", 0.0)))


def ldg_setup_host(mesh, eq):
    """Host-only set-up; returns dict of tables and metrics (numpy)."""
    m = _Marshal(mesh, eq)
    D, p = int(mesh["D"]), int(mesh["p"])
    E = m.nodes.shape[0]
    nl, npe, nq = (p + 1) ** (D - 1), (p + 1) ** D, (3 * p + 2) // 2
    out = {"nbr": np.zeros((E, D, nl, 2), np.int64), "sw": np.zeros((E, D, 2), np.int8),
           "ng": np.zeros((E, D, nl, nq, D)), "nend": np.zeros((E, D, nl, 2, D)),
           "invJ": np.zeros((E, npe)), "tables": np.zeros(nq * (p + 1) * 2 + 2 * (p + 1))}
    _check(lib().ldg_setup_host(C.byref(m.mesh), C.byref(m.eq), *[_hptr(out[k]) for k in
                                ("nbr", "sw", "ng", "nend", "invJ", "tables")]), "ldg_setup_host")
    t = out.pop("tables")
    n = p + 1
    out["Phi"] = t[:nq * n].reshape(nq, n)
    out["Kd"] = t[nq * n:2 * nq * n].reshape(n, nq)
    out["L0"] = t[2 * nq * n:2 * nq * n + n]
    out["L1"] = t[2 * nq * n + n:]
    return out


class Handle:
    """Owns an ldg_handle_t; `h.ptr` is the C pointer."""

    def __init__(self, ptr):
        self.ptr = ptr
        info = (C.c_int64 * 10)()
        _check(lib().ldg_info(ptr, info), "ldg_info")
        (self.D, self.p, self.nc, self.E, self.npe, self.nl, self.nq, self.ndof,
         self.k11_len, self.k12_len) = [int(v) for v in info]

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.ldg_destroy(self.ptr)
            self.ptr = None

    @property
    def shape(self):
        return (self.E, self.nc, self.npe)

    @property
    def nlines(self):
        return self.E * self.D * self.nl

    @property
    def ntiles(self):
        return (self.nlines + 31) // 32

    @property
    def nk11(self):
        return self.k11_len // self.nlines

    @property
    def nk12(self):
        return self.k12_len // self.nlines


def ldg_setup(mesh, eq):
    m = _Marshal(mesh, eq)
    ptr = C.c_void_p()
    _check(lib().ldg_setup(C.byref(m.mesh), C.byref(m.eq), C.byref(ptr)), "ldg_setup")
    return Handle(ptr)


def ldg_export_tables(h):
    nbr = np.zeros((h.E, h.D, h.nl, 2), np.int64)
    sw = np.zeros((h.E, h.D, 2), np.int8)
    _check(lib().ldg_export_tables(h.ptr, _hptr(nbr), _hptr(sw)), "ldg_export_tables")
    return nbr, sw


def ldg_residual(h, U, R, stream=None):
    _check(lib().ldg_residual(h.ptr, _dptr(U), _dptr(R), _stream(stream)), "ldg_residual")
    return R


def ldg_gradient(h, U, Q, stream=None):
    _check(lib().ldg_gradient(h.ptr, _dptr(U), _dptr(Q), _stream(stream)), "ldg_gradient")
    return Q


def ldg_gradient_uq(h, U, Q, Qout, stream=None):
    """D(U, Q) of the stabilised scheme (Q may be None when C22 = 0)."""
    _check(lib().ldg_gradient_uq(h.ptr, _dptr(U), _dptr(Q), _dptr(Qout), _stream(stream)), "ldg_gradient_uq")
    return Qout


def ldg_coupled_solve(h, U, Q, rtol=1e-10, restart=64, max_cycles=200, stream=None):
    """Solve (R(U, Q), Q - D(U, Q)) = 0 in place (Poisson, stabilised scheme)."""
    st = ldg_step_stats_t()
    _check(lib().ldg_coupled_solve(h.ptr, _dptr(U), _dptr(Q), float(rtol), int(restart), int(max_cycles),
                                   C.byref(st), _stream(stream)), "ldg_coupled_solve")
    return st.as_dict()


def ldg_residual_uq(h, U, Q, R, stream=None):
    _check(lib().ldg_residual_uq(h.ptr, _dptr(U), _dptr(Q), _dptr(R), _stream(stream)),
           "ldg_residual_uq")
    return R


def ldg_norm2(h, x, stream=None):
    out = C.c_double()
    _check(lib().ldg_norm2(h.ptr, _dptr(x), x.numel(), C.byref(out), _stream(stream)), "ldg_norm2")
    return out.value


class Jacobian:
    def __init__(self, h, ptr, prec):
        self.h, self.ptr, self.prec = h, ptr, prec

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.ldg_jac_destroy(self.ptr)
            self.ptr = None


def ldg_jacobian(h, U, prec=PREC_FP32, J=None, stream=None):
    ptr = C.c_void_p(None if J is None else J.ptr.value)
    _check(lib().ldg_jacobian(h.ptr, _dptr(U), prec, C.byref(ptr), _stream(stream)), "ldg_jacobian")
    if J is None:
        J = Jacobian(h, ptr, prec)
    return J


def ldg_jacobian_uq(h, U, Q, prec=PREC_FP32, J=None, stream=None):
    """ldg_jacobian at a given gradient Q (see ldg.h)."""
    ptr = C.c_void_p(None if J is None else J.ptr.value)
    _check(lib().ldg_jacobian_uq(h.ptr, _dptr(U), None if Q is None else _dptr(Q), prec, C.byref(ptr),
                                 _stream(stream)), "ldg_jacobian_uq")
    if J is None:
        J = Jacobian(h, ptr, prec)
    return J


def ldg_jac_export(J):
    h = J.h
    dt = np.float32 if J.prec == PREC_FP32 else np.float64
    n = h.p + 1
    NL = h.E * h.D * h.nl
    K11 = np.zeros((h.k11_len // NL, NL), dt)
    K12 = np.zeros((max(h.k12_len // NL, 1), NL), dt) if h.k12_len else None
    K21 = np.zeros(((n * n + n) * h.D, NL), dt) if h.k12_len else None
    _check(lib().ldg_jac_export(J.ptr, _hptr(K11), _hptr(K12), _hptr(K21)), "ldg_jac_export")
    return K11, K12, K21


def ldg_jacvec(h, J, shift, scale, x, y, prec=PREC_FP32, stream=None):
    _check(lib().ldg_jacvec(h.ptr, J.ptr, float(shift), float(scale), _dptr(x), _dptr(y), prec,
                            _stream(stream)), "ldg_jacvec")
    return y


def ldg_k21_apply(h, J, x, g, prec=PREC_FP32, stream=None):
    """g = K21 x, the first half of the split product (see ldg.h)."""
    _check(lib().ldg_k21_apply(h.ptr, J.ptr, _dptr(x), _dptr(g), prec, _stream(stream)), "ldg_k21_apply")
    return g


def ldg_jacvec_g(h, J, shift, scale, x, g, y, prec=PREC_FP32, stream=None):
    """y = shift x + scale (K11 x + K12 g), the second half (see ldg.h)."""
    _check(lib().ldg_jacvec_g(h.ptr, J.ptr, float(shift), float(scale), _dptr(x), None if g is None else _dptr(g),
                              _dptr(y), prec, _stream(stream)), "ldg_jacvec_g")
    return y


class Precond:
    def __init__(self, h, ptr):
        self.h, self.ptr = h, ptr

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.ldg_pc_destroy(self.ptr)
            self.ptr = None


def ldg_precond(h, J, shift, scale, P=None, stream=None):
    ptr = C.c_void_p(None if P is None else P.ptr.value)
    _check(lib().ldg_precond(h.ptr, J.ptr, float(shift), float(scale), C.byref(ptr), _stream(stream)),
           "ldg_precond")
    if P is None:
        P = Precond(h, ptr)
    return P


def ldg_precond_apply(h, P, r, z, prec=PREC_FP32, stream=None):
    _check(lib().ldg_precond_apply(h.ptr, P.ptr, _dptr(r), _dptr(z), prec, _stream(stream)),
           "ldg_precond_apply")
    return z


def ldg_pc_export(P, prec):
    h = P.h
    dt = np.float32 if prec == PREC_FP32 else np.float64
    F = np.zeros((h.E, h.npe, h.D * h.p + 1, h.nc, h.nc), dt)
    _check(lib().ldg_pc_export(P.ptr, _hptr(F)), "ldg_pc_export")
    return F


FORCING_FIXED, FORCING_TARGET = 0, 1
ORTHO_CGS2, ORTHO_SELECTIVE = 0, 1


def solver_opts(mode=MODE_MIXED, predictor=PRED_EXTRAP, first_step=False, restart=30,
                max_newton=50, reuse=15, max_refine=10, force_rebuild=True, rtol=1e-8,
                gmres_tol=1e-3, stall_rebuild=True, forcing=FORCING_FIXED, ortho=ORTHO_SELECTIVE,
                reorth_factor=0.0):
    return ldg_solver_opts_t(mode, predictor, int(first_step), restart, max_newton, reuse,
                             max_refine, int(force_rebuild), rtol, gmres_tol, int(stall_rebuild), int(forcing),
                             int(ortho), float(reorth_factor))


def ldg_newton_step(h, U_next, U_n, U_nm1, U_nm2, dt, opts, stream=None):
    st = ldg_step_stats_t()
    _check(lib().ldg_newton_step(h.ptr, _dptr(U_next), _dptr(U_n), _dptr(U_nm1), _dptr(U_nm2),
                                 float(dt), C.byref(opts), C.byref(st), _stream(stream)),
           "ldg_newton_step")
    return st.as_dict()


def ldg_dirk3_step(h, U_next, U_n, dt, opts, stream=None):
    st = ldg_step_stats_t()
    _check(lib().ldg_dirk3_step(h.ptr, _dptr(U_next), _dptr(U_n), float(dt), C.byref(opts), C.byref(st),
                                _stream(stream)), "ldg_dirk3_step")
    return st.as_dict()


def ldg_rk4_step(h, U_next, U_n, dt, stream=None):
    _check(lib().ldg_rk4_step(h.ptr, _dptr(U_next), _dptr(U_n), float(dt), _stream(stream)), "ldg_rk4_step")


def ldg_steady_solve(h, U, dt0, growth, n_steps, opts, stream=None):
    st = ldg_step_stats_t()
    _check(lib().ldg_steady_solve(h.ptr, _dptr(U), float(dt0), float(growth), int(n_steps), C.byref(opts),
                                  C.byref(st), _stream(stream)), "ldg_steady_solve")
    return st.as_dict()


def paper_policy_opts(mode=MODE_FP64, rtol=1e-8, max_newton=50):
    """The paper's Newton policy for DIRK3 (Sec. 5.5): a fixed five GMRES
    iterations per Newton step, Jacobian and preconditioner re-used until the
    Newton iterations since the last rebuild exceed 15."""
    return solver_opts(mode=mode, restart=5, max_refine=1, gmres_tol=0.0, reuse=15, force_rebuild=False,
                       rtol=rtol, max_newton=max_newton, stall_rebuild=False)


def ldg_launch_count():
    v = C.c_longlong()
    _check(lib().ldg_launch_count(C.byref(v)), "ldg_launch_count")
    return v.value


KT_APPLY, KT_JACVEC, KT_ORTHO = 0, 1, 2


def ldg_kernel_timer(enable=True):
    _check(lib().ldg_kernel_timer(int(bool(enable))), "ldg_kernel_timer")


def ldg_kernel_timer_read(kernel, prec):
    """(launches, summed device ms, summed bytes, summed FLOPs) of one timed
    kernel at one vector precision."""
    n, ms, by, fl = C.c_longlong(), C.c_double(), C.c_double(), C.c_double()
    _check(lib().ldg_kernel_timer_read(kernel, prec, C.byref(n), C.byref(ms), C.byref(by), C.byref(fl)),
           "ldg_kernel_timer_read")
    return n.value, ms.value, by.value, fl.value


def ldg_fp64_fma_probe(iters, sink, stream=None):
    """Enqueue the FP64 FMA-throughput kernel (see ldg.h); returns the number
    of FMAs it performs. sink: CUDA float64 tensor of >= 4 x SMs values."""
    f = C.c_double()
    _check(lib().ldg_fp64_fma_probe(int(iters), _dptr(sink), sink.numel(), C.byref(f), _stream(stream)),
           "ldg_fp64_fma_probe")
    return f.value


def ldg_residual_noalloc(h, U, R, stream=None):
    """ldg_residual without allocation (fixed device scratch; see ldg.h)."""
    _check(lib().ldg_residual_noalloc(h.ptr, _dptr(U), _dptr(R), _stream(stream)),
           "ldg_residual_noalloc")
    return R


MLP_INP = 96


class Mlp:
    def __init__(self, ptr, n_in, n_out):
        self.ptr, self.n_in, self.n_out = ptr, n_in, n_out
        self.n_params = n_in * 128 + 128 + 2 * (128 * 128 + 128) + 128 * n_out + n_out

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.ldg_mlp_destroy(self.ptr)
            self.ptr = None


def ldg_mlp_create(n_in, n_out):
    ptr = C.c_void_p()
    _check(lib().ldg_mlp_create(int(n_in), int(n_out), C.byref(ptr)), "ldg_mlp_create")
    return Mlp(ptr, n_in, n_out)


def ldg_mlp_params(m, theta=None):
    """Return the FP32 master parameters (as float64) or set them."""
    if theta is None:
        out = np.zeros(m.n_params)
        _check(lib().ldg_mlp_params(m.ptr, _hptr(out), 0), "ldg_mlp_params")
        return out
    th = np.ascontiguousarray(theta, dtype=np.float64)
    _check(lib().ldg_mlp_params(m.ptr, _hptr(th), 1), "ldg_mlp_params")
    return th


def ldg_mlp_set_scaling(m, in_mean, in_std, out_scale):
    a, b, c = (np.ascontiguousarray(x, dtype=np.float64) for x in (in_mean, in_std, out_scale))
    _check(lib().ldg_mlp_set_scaling(m.ptr, _hptr(a), _hptr(b), _hptr(c)), "ldg_mlp_set_scaling")


def ldg_mlp_forward(m, X, Y, stream=None):
    _check(lib().ldg_mlp_forward(m.ptr, _dptr(X), X.shape[0], _dptr(Y), _stream(stream)), "ldg_mlp_forward")
    return Y


def ldg_mlp_grad(m, X, T, grad, loss=None, stream=None):
    _check(lib().ldg_mlp_grad(m.ptr, _dptr(X), _dptr(T), X.shape[0], _dptr(grad), _dptr(loss),
                              _stream(stream)), "ldg_mlp_grad")
    return grad


def ldg_mlp_train_step(m, X, T, lr, loss=None, stream=None):
    _check(lib().ldg_mlp_train_step(m.ptr, _dptr(X), _dptr(T), X.shape[0], float(lr), _dptr(loss),
                                    _stream(stream)), "ldg_mlp_train_step")


def ldg_line_features(h, m, Un, Unm1, Unm2, X, stream=None):
    _check(lib().ldg_line_features(h.ptr, m.ptr, _dptr(Un), _dptr(Unm1), _dptr(Unm2), _dptr(X),
                                   _stream(stream)), "ldg_line_features")
    return X


def ldg_line_targets(h, m, Unext, Un, Unm1, T, stream=None):
    _check(lib().ldg_line_targets(h.ptr, m.ptr, _dptr(Unext), _dptr(Un), _dptr(Unm1), _dptr(T),
                                  _stream(stream)), "ldg_line_targets")
    return T


def ldg_mlp_predict(h, m, Un, Unm1, Unm2, U0, stream=None):
    _check(lib().ldg_mlp_predict(h.ptr, m.ptr, _dptr(Un), _dptr(Unm1), _dptr(Unm2), _dptr(U0),
                                 _stream(stream)), "ldg_mlp_predict")
    return U0


def ldg_set_viscosity(h, mu):
    _check(lib().ldg_set_viscosity(h.ptr, float(mu)), "ldg_set_viscosity")
