"""The C-ABI library without a GPU: it builds, loads, exports every symbol
include/*.h declares, and its host-side set-up (tables, switches, metrics,
1-D operators) matches the oracle (bit-exact for integers)."""
import numpy as np
import pytest

from paper_1204_1533_gb300 import inputs as I
from paper_1204_1533_gb300 import ldg
from oracle.residual import Discretization

EULER = {"kind": "euler", "gamma": 1.4, "flux": "roe"}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1204_1533_gb300 import build
    build.build()


def test_exports_every_declared_symbol():
    L = ldg.lib()
    names = ldg.declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def _meshes():
    m2 = I.reorient(I.vortex_mesh(4, 3, perturb=0.15))[0]
    m3 = I.reorient(I.structured_mesh((3, 3, 3), 2, (0,) * 3, (1,) * 3, (True,) * 3, perturb=0.1))[0]
    mp = I.poisson_square_mesh(4, 3)
    mc = I.channel_mesh(4, 4, 3, 2)
    mu2 = I.unstructured_quad_mesh(2, 3, perturb=0.15)
    mu3 = I.unstructured_hex_mesh(3, 2, periodic=True, perturb=0.1)
    return [("vortex2d", m2, EULER), ("box3d", m3, EULER),
            ("poisson", mp, {"kind": "poisson", "bc": {0: "dirichlet"}}),
            ("channel", mc, {"kind": "ns", "mu": 0.01, "Pr": 0.72, "bc": {1: "wall"}}),
            ("unstructured_quads", mu2, {"kind": "poisson", "bc": {0: "dirichlet"}}),
            ("unstructured_hexes", mu3, EULER)]


@pytest.mark.parametrize("case", range(6))
def test_tables_bit_exact_and_metrics_match_oracle(case):
    name, m, eq = _meshes()[case]
    host = ldg.ldg_setup_host(m, eq)
    disc = Discretization(m, dict(eq, bc={0: "dirichlet", 1: "wall"}))
    assert np.array_equal(host["nbr"], disc.conn.nbr), name
    assert np.array_equal(host["sw"], disc.S), name
    scale = max(np.abs(disc.met.ng[d]).max() for d in range(m["D"]))
    for d in range(m["D"]):
        assert np.allclose(host["ng"][:, d], disc.met.ng[d], rtol=0, atol=1e-13 * scale)
        assert np.allclose(host["nend"][:, d, :, 1], disc.met.nplus[d], rtol=0, atol=1e-13 * scale)
        assert np.allclose(host["nend"][:, d, :, 0], disc.met.nminus[d], rtol=0, atol=1e-13 * scale)
    assert np.allclose(host["invJ"], 1.0 / disc.met.J, rtol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_one_d_operators_match_oracle(p):
    m = I.vortex_mesh(3, p)
    host = ldg.ldg_setup_host(m, EULER)
    r = Discretization(m, EULER).rules
    Kd = r.mass_solve(r.dPhi * r.wq[:, None]).T            # M^-1 dPhi^T W
    assert np.allclose(host["Phi"], r.Phi, atol=1e-15)
    assert np.allclose(host["Kd"], Kd, rtol=0, atol=1e-12 * np.abs(Kd).max())
    assert np.allclose(host["L1"], r.mass_solve(np.eye(p + 1)[p]), atol=1e-12 * (p + 1) ** 2)
    assert np.allclose(host["L0"], r.mass_solve(np.eye(p + 1)[0]), atol=1e-12 * (p + 1) ** 2)


def test_rejects_bad_meshes():
    m = I.vortex_mesh(3, 2)
    bad = dict(m, s=np.array([0.0, 0.4, 1.0]))          # not symmetric
    with pytest.raises(ldg.LdgError) as e:
        ldg.ldg_setup_host(bad, EULER)
    assert e.value.code == -3
    bad = dict(m, btag=np.zeros_like(m["btag"]))        # matched faces tagged as boundary
    with pytest.raises(ldg.LdgError):
        ldg.ldg_setup_host(bad, EULER)
    nodes = m["nodes"].copy()
    n1 = m["p"] + 1                                       # mirror element 0 along i: J < 0
    nodes[0] = nodes[0].reshape(n1, n1, 2)[:, ::-1].reshape(-1, 2)
    with pytest.raises(ldg.LdgError):
        ldg.ldg_setup_host(dict(m, nodes=nodes), EULER)
    with pytest.raises(ldg.LdgError) as e:
        ldg.ldg_setup_host(I.vortex_mesh(3, 6), EULER)   # p not compiled in
    assert e.value.code == -8


def test_stabilised_scheme_is_poisson_only():
    m = I.poisson_square_mesh(3, 2)
    ldg.ldg_setup_host(m, {"kind": "poisson", "C22": 0.05, "bc": {0: "dirichlet"}})
    with pytest.raises(ldg.LdgError) as e:
        ldg.ldg_setup_host(m, {"kind": "poisson", "C22": -0.05, "bc": {0: "dirichlet"}})
    assert e.value.code == -1
    with pytest.raises(ldg.LdgError) as e:
        ldg.ldg_setup_host(I.vortex_mesh(3, 2), dict(EULER, C22=0.05))
    assert e.value.code == -8


def _header_structs():
    """Field (name, C type) lists of every `typedef struct { ... } NAME;` in
    include/ldg.h, comments stripped."""
    import pathlib
    import re
    src = (pathlib.Path(__file__).resolve().parents[1] / "include" / "ldg.h").read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            m = re.match(r"(.*?)(\w+)(\[\d+\])?$", decl)
            fields.append((m.group(2), m.group(1).replace(" ", "") + (m.group(3) or "")))
        out[name] = fields
    return out


def test_binding_structs_and_constants_match_header():
    # every ctypes struct of the binding lists the header's fields in order
    # with the same widths, and the binding's option constants equal the
    # header's #defines
    import ctypes as C
    import pathlib
    import re
    scalar = {"int32_t": C.c_int32, "int64_t": C.c_int64, "double": C.c_double}
    hdr = _header_structs()
    for name in ("ldg_mesh_t", "ldg_equations_t", "ldg_solver_opts_t", "ldg_step_stats_t"):
        fields = getattr(ldg, name)._fields_
        assert [f[0] for f in fields] == [h[0] for h in hdr[name]], name
        for (fname, ftype), (_, ctype) in zip(fields, hdr[name]):
            if ctype.endswith("*"):
                assert C.sizeof(ftype) == C.sizeof(C.c_void_p), (name, fname)
            elif "[" in ctype:
                base, n = ctype[:-1].split("[")
                assert C.sizeof(ftype) == int(n) * C.sizeof(scalar[base]), (name, fname)
            else:
                assert ftype == scalar[ctype], (name, fname)
    src = (pathlib.Path(__file__).resolve().parents[1] / "include" / "ldg.h").read_text()
    defs = {k: int(v) for k, v in re.findall(r"#define LDG_(\w+) \(?(-?\d+)\)?", src)}
    for key in ("PREC_FP32", "PREC_FP64", "MODE_FP64", "MODE_MIXED", "PRED_EXTRAP", "PRED_GIVEN",
                "PRED_CHECKED", "FORCING_FIXED", "FORCING_TARGET", "ORTHO_CGS2", "ORTHO_SELECTIVE",
                "KT_APPLY", "KT_JACVEC", "KT_ORTHO"):
        assert getattr(ldg, key) == defs[key], key
