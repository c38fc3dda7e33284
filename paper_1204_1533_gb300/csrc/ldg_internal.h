// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ldg.h"

namespace ldg {

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
  int64_t E;
};

cudaError_t launch_gradient(const struct ::ldg_handle* h, const double* U, double* Q,
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
  double* Qbuf = nullptr;    // LDG gradient of the last residual [E][nc][D][npe]
  double* red = nullptr;     // reduction scratch (doubles)
  int64_t red_len = 0;
  ldg::Geo geo() const {
    ldg::Geo g;
    g.nbr = nbr;
    g.sw = sw;
    g.ng = ng;
    g.nend = nend;
    g.invJ = invJ;
    g.gD = gD;
    g.src = src;
    g.E = E;
    return g;
  }
  bool viscous() const { return kind == LDG_EQ_NAVIER_STOKES || kind == LDG_EQ_POISSON; }
};

#define LDG_CUDA_TRY(x)                      \
  do {                                       \
    cudaError_t _e = (x);                    \
    if (_e != cudaSuccess) return LDG_ERR_CUDA; \
  } while (0)
