// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ldg.h"

namespace ldg {

// number of kernels this library has launched (host-side counter)
void count_launch(int n = 1);

// Event timing of selected kernels (ldg_kernel_timer): while enabled, each
// timed launch is bracketed by two events on its stream and carries its
// algorithmic bytes and FLOPs.
enum { KT_APPLY = 0, KT_JACVEC = 1, KT_ORTHO = 2, KT_COUNT = 3 };
int timer_begin(int kernel, int vprec, cudaStream_t st, double bytes, double flops);  // slot or -1
void timer_end(int slot, cudaStream_t st);
struct TimedScope {
  int slot;
  cudaStream_t st;
  TimedScope(int k, int vprec, cudaStream_t s, double bytes, double flops)
      : slot(timer_begin(k, vprec, s, bytes, flops)), st(s) {}
  ~TimedScope() {
    if (slot >= 0) timer_end(slot, st);
  }
};

// Raise a kernel's dynamic shared-memory limit to `bytes` on the current
// device, calling the runtime only the first time a larger size is needed.
cudaError_t smem_attr_cached(const void* fn, size_t bytes);
template <typename K>
inline cudaError_t set_smem_once(K kern, size_t bytes) {
  return smem_attr_cached(reinterpret_cast<const void*>(kern), bytes);
}

constexpr int MAXP = 7;
constexpr int MAXP1 = MAXP + 1;
constexpr int MAXQ = (3 * MAXP + 2) / 2;
constexpr int MAXBC = 8;

// 1-D operators of the reference line (Sec. 2.2), passed by value to kernels.
//   Phi[q][j] = phi_j(xi_q)               interpolation to Gauss points
//   Kd[i][q]  = (M^-1 dPhi^T W)[i][q]     mass-inverse weighted derivative
//   L0 = M^-1 e_0, L1 = M^-1 e_p           lifting of the end fluxes
struct Tab {
  double Phi[MAXQ][MAXP1];
  double Kd[MAXP1][MAXQ];
  double L0[MAXP1];
  double L1[MAXP1];
  float Phif[MAXQ][MAXP1];
  float Kdf[MAXP1][MAXQ];
  float L0f[MAXP1];
  float L1f[MAXP1];
};

struct PhysArgs {
  double gamma, mu, Pr, C11, C11b;
  double C22;  // LDG flux-jump penalty (Poisson only; 0 = minimal dissipation)
  double adv[3];
  int flux;
  int nbc;
  int bck[MAXBC];
};

// Geometry and tables as the kernels see them.
struct Geo {
  const int32_t* nbr;   // [E][D][nl][2]
  const int8_t* sw;     // [E][D][2]
  const double* ng;     // [E][D][nl][nq][D]
  const double* nend;   // [E][D][nl][2][D]
  const double* invJ;   // [E][npe]
  const double* gD;     // [E][nc][npe] or null
  const double* src;    // [E][nc][npe] or null
  const double* gN;     // [E][nc][D][npe] or null (Neumann flux vector)
  int64_t E;
};

// Arnoldi column of GMRES by CGS2 (reorth_k <= 0), or by classical
// Gram-Schmidt re-orthogonalised only where one pass shrank w by more than
// a factor reorth_k (ldg_ortho.cu): orthogonalises w against the kv basis vectors
// Vb[0..kv) (stride n) and normalises it. Device scratch: part
// [GS_PART_LEN], gs [GS_SCRATCH_LEN] doubles. Host col [2 kv + 2]: on
// return col[0..kv) = Hessenberg entries, col[kv] = the norm before
// normalisation (0: w lies in the span); *passes (if not null) = the
// Gram-Schmidt passes made (1 or 2). pin: null, or pinned host memory of
// GS_PIN_LEN doubles with ev an event, for a read-back that lets the last
// update sweep run while the host waits. Synchronises on st (on ev).
constexpr int GS_KMAX = 32;        // basis vectors per fused sweep
constexpr int GS_MAX_BASIS = 66;   // largest basis (restart 64 + 2)
constexpr int GS_MAX_BLOCKS = 320;
constexpr size_t GS_PART_LEN = (size_t)(GS_KMAX + 1) * GS_MAX_BLOCKS;
constexpr size_t GS_SCRATCH_LEN = 4 * (GS_MAX_BASIS + 2) + 4;
constexpr size_t GS_PIN_LEN = GS_MAX_BASIS + 4;  // host read-back of one column
template <typename V>
int arnoldi_column(const V* Vb, int kv, int64_t n, V* w, double* part, double* gs, double* col, double reorth_k,
                   int* passes, double* pin, cudaEvent_t ev, cudaStream_t st);

cudaError_t launch_gradient(const struct ::ldg_handle* h, const double* U, double* Q,
                            cudaStream_t st);
// D(U, Qs) of the stabilised scheme (C22 != 0): the trace also takes the
// jump of the normal flux of the given gradient Qs (Qs may not alias Q)
cudaError_t launch_gradient_uq(const struct ::ldg_handle* h, const double* U, const double* Qs, double* Q,
                               cudaStream_t st);
cudaError_t launch_residual(const struct ::ldg_handle* h, const double* U, const double* Q,
                            double* R, cudaStream_t st);
bool residual_supported(int D, int p, int kind);

}  // namespace ldg

struct ldg_handle {
  int D, p, nc, npe, nl, nq, kind;
  int64_t E, ndof;
  ldg::PhysArgs phys;
  ldg::Tab tab;
  std::vector<int32_t> nbr_h;
  std::vector<int8_t> sw_h;
  // device buffers (owned)
  int32_t* nbr = nullptr;
  int8_t* sw = nullptr;
  double* ng = nullptr;
  double* nend = nullptr;
  double* invJ = nullptr;
  double* gD = nullptr;
  double* src = nullptr;
  double* gN = nullptr;      // prescribed Neumann flux [E][nc][D][npe]
  int8_t* nbf = nullptr;     // neighbour face id per element face [E][2D] (-1: boundary)
  std::vector<int8_t> nbf_h;
  int16_t* pat = nullptr;    // element Line-DG pattern: sorted columns of each row [npe][Dp+1]
  int8_t* slot = nullptr;    // column slot of node j in row i, or -1 [npe][npe]
  int16_t* lvl = nullptr;    // rows sorted by wavefront level (sum of indices) [npe]
  int32_t* lvl_ptr = nullptr; // level start offsets [D p + 2]
  bool has_wall = false;
  float* linemet = nullptr;  // per direction-1 line: line-averaged G / h, [E nl][D D]
  // Newton-Krylov state kept across time steps (Jacobian re-use, Sec. 4.3)
  struct ldg_jac* Jn = nullptr;
  struct ldg_pc* Pn = nullptr;
  int jac_age = 0;
  int jac_mode = -1;
  double pc_adt = 0.0;
  void* ws = nullptr;        // solver workspace
  size_t ws_bytes = 0;
  double* Qbuf = nullptr;    // LDG gradient of the last residual [E][nc][D][npe]
  double* dirk = nullptr;    // DIRK3 stage vectors K1..K3, B, U_i [5][ndof]
  double* red = nullptr;     // reduction scratch (doubles)
  struct ldg_cpl* cpl = nullptr;  // coupled (U, Q) solver state of the stabilised scheme
  int64_t red_len = 0;
  double* gs_pin = nullptr;    // pinned host read-back of GMRES columns [GS_PIN_LEN]
  cudaEvent_t gs_ev = nullptr; // marks that read-back
  ldg::Geo geo() const {
    ldg::Geo g;
    g.nbr = nbr;
    g.sw = sw;
    g.ng = ng;
    g.nend = nend;
    g.invJ = invJ;
    g.gD = gD;
    g.src = src;
    g.gN = gN;
    g.E = E;
    return g;
  }
  bool viscous() const { return kind == LDG_EQ_NAVIER_STOKES || kind == LDG_EQ_POISSON; }
  int64_t nlines() const { return E * D * nl; }
  int64_t ntiles() const { return (nlines() + 31) / 32; }
  int pat_w() const { return D * p + 1; }
  int nk11() const { return ((p + 1) * (p + 1) + 2 * (p + 1)) * nc * nc; }
  int nk12() const { return viscous() ? ((p + 1) * (p + 1) + (p + 1)) * nc * nc * D : 0; }
  int nk21() const { return viscous() ? ((p + 1) * (p + 1) + (p + 1)) * D : 0; }
};

// Line-sparse Jacobian: K11, K12, K21 in 32-line tiles, entry-major inside a
// tile: value k of line L sits at ((L / 32) nk + k) 32 + L % 32.
struct ldg_jac {
  ldg_handle* h = nullptr;
  int prec = 0;
  bool built = false;
  bool k21_built = false;
  void* K11 = nullptr;
  void* K12 = nullptr;
  void* K21 = nullptr;
  void* Kw = nullptr;     // wall ends: energy row of the wall-state derivative, 2 n_c per line (tiles)
  void* gbuf = nullptr;   // K21 x workspace [E][nc][D][npe] in the vector precision (double)
  void* ucvt = nullptr;   // FP32 Jacobians: FP32 copies of U [ndof] and Q [ndof D] for the assembly
  void* geof = nullptr;   // FP32 Jacobians: FP32 copies of ng, nend, invJ (made at the first build)
  bool geof_ready = false;
};

// Element-block ILU(0) factors [E][npe][Dp+1][nc][nc] at the Jacobian's
// precision: L below the diagonal, U above it, and in each row's diagonal
// slot the inverse of U's diagonal block (what the triangular solves use);
// the diagonal blocks U_ii themselves [E][npe][nc][nc] are kept aside for
// the export.
struct ldg_pc {
  ldg_handle* h = nullptr;
  int prec = 0;
  bool built = false;
  void* F = nullptr;
  void* Udiag = nullptr;
};

namespace ldg {
cudaError_t launch_jacobian(const ldg_handle* h, const double* U, const double* Q, ldg_jac* J,
                            cudaStream_t st);
cudaError_t launch_k21(const ldg_handle* h, ldg_jac* J, cudaStream_t st);
cudaError_t launch_jacvec(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                          const void* x, void* y, int vprec, cudaStream_t st);
cudaError_t launch_precond(const ldg_handle* h, const ldg_jac* J, double shift, double scale,
                           ldg_pc* P, cudaStream_t st);
cudaError_t launch_precond_apply(const ldg_handle* h, const ldg_pc* P, const void* r, void* z,
                                 int vprec, cudaStream_t st);
}  // namespace ldg

// releases the coupled-solver state of a handle (ldg_solver.cu)
void free_coupled(struct ldg_cpl* c);

#define LDG_CUDA_TRY(x)                      \
  do {                                       \
    cudaError_t _e = (x);                    \
    if (_e != cudaSuccess) return LDG_ERR_CUDA; \
  } while (0)
