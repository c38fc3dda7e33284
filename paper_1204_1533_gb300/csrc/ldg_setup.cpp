// Host set-up of a Line-DG handle: 1-D rules, face matching with general
// orientations, neighbour-node tables, switch function and metric terms.
//
//   * Sec. 2.2: Gauss-Legendre integration of precision 3p with
//     ceil((3p+1)/2) points; the mass matrix is line-, component- and
//     element-independent, factorised once (Cholesky) and folded into
//     Kd = M^-1 dPhi^T W, L0 = M^-1 e_0, L1 = M^-1 e_p (computed in long
//     double, rounded once).
//   * Sec. 2.1, Eqs. 2, 4-6: isoparametric G = grad_X x, J = det G,
//     contravariant normals n_d = J G^-T N_d (columns of the cofactor
//     matrix) at the Gauss points of every line and at both line ends.
//   * Sec. 2.1: the outside trace of each line end is the coincident node of
//     the neighbouring element; faces are matched by their corner vertex ids
//     and the node correspondence follows from the corner permutation.
//   * Sec. 3: switches S^+-_d with S^+ = -S^- and opposite signs across each
//     shared face, propagated along globally connected lines of elements.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <atomic>
#include <thread>
#include <vector>

#include "ldg_internal.h"

namespace {

using ld = long double;

// Gauss-Legendre on [0,1]: Newton iteration on P_n from its recurrence.
void gauss01(int n, std::vector<ld>& x, std::vector<ld>& w) {
  x.assign(n, 0);
  w.assign(n, 0);
  const ld pi = 3.141592653589793238462643383279502884L;
  for (int k = 0; k < n; ++k) {
    ld t = std::cos(pi * (k + 0.75L) / (n + 0.5L));
    ld dp = 0;
    for (int it = 0; it < 200; ++it) {
      ld p0 = 1, p1 = t;
      for (int m = 2; m <= n; ++m) {
        ld p2 = ((2 * m - 1) * t * p1 - (m - 1) * p0) / m;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (t * p1 - p0) / (t * t - 1);
      ld step = p1 / dp;
      t -= step;
      if (std::fabs(step) < 1e-30L) break;
    }
    ld p0 = 1, p1 = t;
    for (int m = 2; m <= n; ++m) {
      ld p2 = ((2 * m - 1) * t * p1 - (m - 1) * p0) / m;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (t * p1 - p0) / (t * t - 1);
    x[k] = (1 - t) / 2;  // ascending on [0,1]
    w[k] = 1 / ((1 - t * t) * dp * dp);
  }
}

// Barycentric Lagrange basis on nodes s: values and derivatives at xq.
void barycentric(const std::vector<ld>& s, const std::vector<ld>& xq, std::vector<ld>& phi,
                 std::vector<ld>& dphi) {
  const int n = (int)s.size(), m = (int)xq.size();
  std::vector<ld> bw(n, 1);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) bw[j] /= (s[j] - s[k]);
  // nodal differentiation matrix Dn[i][j] = phi_j'(s_i)
  std::vector<ld> Dn(n * n, 0);
  for (int i = 0; i < n; ++i) {
    ld diag = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      Dn[i * n + j] = (bw[j] / bw[i]) / (s[i] - s[j]);
      diag -= Dn[i * n + j];
    }
    Dn[i * n + i] = diag;
  }
  phi.assign(m * n, 0);
  dphi.assign(m * n, 0);
  for (int q = 0; q < m; ++q) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (std::fabs(xq[q] - s[j]) < 1e-13L) hit = j;
    if (hit >= 0) {  // the point is a node: exact delta and nodal derivative
      for (int j = 0; j < n; ++j) {
        phi[q * n + j] = (j == hit) ? 1 : 0;
        dphi[q * n + j] = Dn[hit * n + j];
      }
      continue;
    }
    std::vector<ld> a(n);
    ld den = 0;
    for (int j = 0; j < n; ++j) {
      a[j] = bw[j] / (xq[q] - s[j]);
      den += a[j];
    }
    for (int j = 0; j < n; ++j) phi[q * n + j] = a[j] / den;
    for (int mm = 0; mm < n; ++mm) {
      ld acc = 0;
      for (int j = 0; j < n; ++j)
        acc += a[j] * (phi[q * n + mm] - (j == mm ? 1 : 0)) / (xq[q] - s[j]);
      dphi[q * n + mm] = acc / den;
    }
  }
}

int build_tables(const std::vector<ld>& s, int p, ldg::Tab& tab, std::vector<ld>& Dnode,
                 int& nq) {
  const int n = p + 1;
  nq = (3 * p + 2) / 2;
  std::vector<ld> xq, wq, phi, dphi, phin, dphin;
  gauss01(nq, xq, wq);
  barycentric(s, xq, phi, dphi);
  barycentric(s, s, phin, dphin);
  Dnode.assign(n * n, 0);
  for (int i = 0; i < n * n; ++i) Dnode[i] = dphin[i];
  // mass matrix and its Cholesky factor
  std::vector<ld> M(n * n, 0), L(n * n, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld acc = 0;
      for (int q = 0; q < nq; ++q) acc += wq[q] * phi[q * n + i] * phi[q * n + j];
      M[i * n + j] = acc;
    }
  for (int j = 0; j < n; ++j) {
    ld d = M[j * n + j];
    for (int k = 0; k < j; ++k) d -= L[j * n + k] * L[j * n + k];
    if (d <= 0) return LDG_ERR_MESH;
    L[j * n + j] = std::sqrt(d);
    for (int i = j + 1; i < n; ++i) {
      ld v = M[i * n + j];
      for (int k = 0; k < j; ++k) v -= L[i * n + k] * L[j * n + k];
      L[i * n + j] = v / L[j * n + j];
    }
  }
  auto chol_solve = [&](std::vector<ld>& b) {
    for (int i = 0; i < n; ++i) {
      for (int k = 0; k < i; ++k) b[i] -= L[i * n + k] * b[k];
      b[i] /= L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      for (int k = i + 1; k < n; ++k) b[i] -= L[k * n + i] * b[k];
      b[i] /= L[i * n + i];
    }
  };
  std::memset(&tab, 0, sizeof(tab));
  for (int q = 0; q < nq; ++q) {
    std::vector<ld> b(n);
    for (int i = 0; i < n; ++i) b[i] = dphi[q * n + i] * wq[q];
    chol_solve(b);
    for (int i = 0; i < n; ++i) tab.Kd[i][q] = (double)b[i];
    for (int j = 0; j < n; ++j) tab.Phi[q][j] = (double)phi[q * n + j];
  }
  for (int end = 0; end < 2; ++end) {
    std::vector<ld> b(n, 0);
    b[end ? p : 0] = 1;
    chol_solve(b);
    for (int i = 0; i < n; ++i) (end ? tab.L1 : tab.L0)[i] = (double)b[i];
  }
  for (int q = 0; q < ldg::MAXQ; ++q)
    for (int j = 0; j < ldg::MAXP1; ++j) {
      tab.Phif[q][j] = (float)tab.Phi[q][j];
      tab.Kdf[j][q] = (float)tab.Kd[j][q];
    }
  for (int i = 0; i < ldg::MAXP1; ++i) {
    tab.L0f[i] = (float)tab.L0[i];
    tab.L1f[i] = (float)tab.L1[i];
  }
  return LDG_OK;
}

int ipow(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// local node index of line l of direction d at position t
inline int line_node(int D, int p, int d, int l, int t) {
  const int n = p + 1, stride = ipow(n, d);
  const int base = (l % stride) + (l / stride) * stride * n;
  return base + t * stride;
}

struct FaceRef {
  int64_t e;
  int f;
};

// corner ids of face f in face-local order (tangential dims ascending)
void face_corner_ids(const int64_t* verts, int D, int f, int64_t* out) {
  const int d = f / 2, end = f % 2;
  int tang[2], nt = 0;
  for (int b = 0; b < D; ++b)
    if (b != d) tang[nt++] = b;
  for (int c = 0; c < (1 << (D - 1)); ++c) {
    int corner = end << d;
    for (int k = 0; k < nt; ++k)
      if ((c >> k) & 1) corner |= 1 << tang[k];
    out[c] = verts[corner];
  }
}

}  // namespace

// Everything of the set-up that runs on the host. On success *hp owns a new
// handle without device buffers and ng/nend/invJ hold the metric terms.
static int host_setup(const ldg_mesh_t* mesh, const ldg_equations_t* eq, ldg_handle_t** hp,
                      std::vector<double>& ng, std::vector<double>& nend,
                      std::vector<double>& invJ, std::vector<float>& linemet) {
  *hp = nullptr;
  const int D = mesh->D, p = mesh->p;
  const int64_t E = mesh->n_elem;
  if ((D != 2 && D != 3) || p < 1 || p > ldg::MAXP || E < 1) return LDG_ERR_ARG;
  if (!mesh->s || !mesh->nodes || !mesh->vertices || !mesh->btag) return LDG_ERR_ARG;
  if (eq->kind < 0 || eq->kind > 3) return LDG_ERR_ARG;
  if (eq->n_bc < 0 || eq->n_bc > ldg::MAXBC) return LDG_ERR_ARG;
  if (!(eq->C22 >= 0.0)) return LDG_ERR_ARG;
  if (eq->C22 != 0.0 && eq->kind != LDG_EQ_POISSON) return LDG_ERR_UNSUPPORTED;
  for (int t = 0; t < eq->n_bc && eq->bc_kind; ++t)
    if (eq->bc_kind[t] < LDG_BC_DIRICHLET || eq->bc_kind[t] > LDG_BC_NEUMANN) return LDG_ERR_ARG;
  if (!ldg::residual_supported(D, p, eq->kind)) return LDG_ERR_UNSUPPORTED;
  const int n = p + 1, npe = ipow(n, D), nl = ipow(n, D - 1);
  // node set: increasing, end points 0 and 1, symmetric
  std::vector<ld> s(n);
  for (int i = 0; i < n; ++i) s[i] = mesh->s[i];
  if (mesh->s[0] != 0.0 || mesh->s[p] != 1.0) return LDG_ERR_MESH;
  for (int i = 0; i < p; ++i)
    if (!(mesh->s[i + 1] > mesh->s[i])) return LDG_ERR_MESH;
  for (int i = 0; i <= p; ++i)
    if (std::fabs(mesh->s[i] + mesh->s[p - i] - 1.0) > 1e-14) return LDG_ERR_MESH;

  ldg_handle_t* h = new ldg_handle_t();
  h->D = D;
  h->p = p;
  h->E = E;
  h->npe = npe;
  h->nl = nl;
  h->kind = eq->kind;
  h->nc = (eq->kind == LDG_EQ_EULER || eq->kind == LDG_EQ_NAVIER_STOKES) ? D + 2 : 1;
  h->ndof = E * h->nc * npe;
  h->phys.gamma = eq->gamma;
  h->phys.mu = eq->mu;
  h->phys.Pr = eq->Pr;
  h->phys.C11 = eq->C11;
  h->phys.C11b = eq->C11_b;
  h->phys.C22 = eq->C22;
  for (int a = 0; a < 3; ++a) h->phys.adv[a] = eq->adv[a];
  h->phys.flux = eq->flux;
  h->phys.nbc = eq->n_bc;
  for (int t = 0; t < ldg::MAXBC; ++t)
    h->phys.bck[t] = (t < eq->n_bc && eq->bc_kind) ? eq->bc_kind[t] : LDG_BC_DIRICHLET;
  for (int64_t k = 0; k < E * 2 * D; ++k)
    if (mesh->btag[k] >= 0 && mesh->btag[k] < ldg::MAXBC && h->phys.bck[mesh->btag[k]] == LDG_BC_WALL)
      h->has_wall = true;
  std::vector<ld> Dnode;
  int rc = build_tables(s, p, h->tab, Dnode, h->nq);
  if (rc != LDG_OK) {
    delete h;
    return rc;
  }
  const int nq = h->nq;

  // ---- face matching -----------------------------------------------------
  const int nfc = 1 << (D - 1);
  std::map<std::vector<int64_t>, std::vector<FaceRef>> faces;
  for (int64_t e = 0; e < E; ++e)
    for (int f = 0; f < 2 * D; ++f) {
      int64_t ids[4];
      face_corner_ids(mesh->vertices + e * (1 << D), D, f, ids);
      std::vector<int64_t> key(ids, ids + nfc);
      std::sort(key.begin(), key.end());
      for (int k = 1; k < nfc; ++k)
        if (key[k] == key[k - 1]) {
          delete h;
          return LDG_ERR_MESH;
        }
      faces[key].push_back({e, f});
    }
  std::vector<int64_t> nb_e(E * 2 * D, -1);
  std::vector<int> nb_f(E * 2 * D, -1);
  for (auto& kv : faces) {
    if (kv.second.size() > 2) {
      delete h;
      return LDG_ERR_MESH;
    }
    if (kv.second.size() == 2) {
      FaceRef a = kv.second[0], b = kv.second[1];
      nb_e[a.e * 2 * D + a.f] = b.e;
      nb_f[a.e * 2 * D + a.f] = b.f;
      nb_e[b.e * 2 * D + b.f] = a.e;
      nb_f[b.e * 2 * D + b.f] = a.f;
    }
  }
  for (int64_t k = 0; k < E * 2 * D; ++k) {
    const bool matched = nb_e[k] >= 0, tagged = mesh->btag[k] >= 0;
    if (matched == tagged || (tagged && mesh->btag[k] >= ldg::MAXBC)) {
      delete h;
      return LDG_ERR_MESH;
    }
  }
  // ---- neighbour node of every line end ------------------------------------
  h->nbr_h.assign(E * D * nl * 2, 0);
  for (int64_t e = 0; e < E; ++e)
    for (int d = 0; d < D; ++d)
      for (int end = 0; end < 2; ++end) {
        const int f = 2 * d + end;
        const int64_t en = nb_e[e * 2 * D + f];
        if (en < 0) {
          for (int l = 0; l < nl; ++l)
            h->nbr_h[((e * D + d) * nl + l) * 2 + end] = -1 - mesh->btag[e * 2 * D + f];
          continue;
        }
        const int fn = nb_f[e * 2 * D + f], dn = fn / 2, endn = fn % 2;
        int64_t mine[4], theirs[4];
        face_corner_ids(mesh->vertices + e * (1 << D), D, f, mine);
        face_corner_ids(mesh->vertices + en * (1 << D), D, fn, theirs);
        int perm[4];
        for (int c = 0; c < nfc; ++c) {
          perm[c] = -1;
          for (int c2 = 0; c2 < nfc; ++c2)
            if (theirs[c2] == mine[c]) perm[c] = c2;
          if (perm[c] < 0) {
            delete h;
            return LDG_ERR_MESH;
          }
        }
        // my tangential axis k maps to their axis ax[k], reversed if flip[k]
        int ax[2] = {0, 0}, flip[2] = {0, 0};
        for (int k = 0; k < D - 1; ++k) {
          const int diff = perm[1 << k] ^ perm[0];
          if (__builtin_popcount(diff) != 1) {
            delete h;
            return LDG_ERR_MESH;
          }
          ax[k] = __builtin_ctz(diff);
          flip[k] = (perm[0] >> ax[k]) & 1;
        }
        // the corner map must be a symmetry of the face
        for (int c = 0; c < nfc; ++c) {
          int img = 0;
          for (int k = 0; k < D - 1; ++k) img |= (((c >> k) & 1) ^ flip[k]) << ax[k];
          if (img != perm[c] || (D == 3 && ax[0] == ax[1])) {
            delete h;
            return LDG_ERR_MESH;
          }
        }
        int mt[2], nt = 0, tt[2], ntt = 0;
        for (int b = 0; b < D; ++b) {
          if (b != d) mt[nt++] = b;
          if (b != dn) tt[ntt++] = b;
        }
        for (int l = 0; l < nl; ++l) {
          const int a = line_node(D, p, d, l, end * p);
          int idx[3] = {a % n, (a / n) % n, (a / (n * n)) % n};
          int nidx[3] = {0, 0, 0};
          nidx[dn] = endn * p;
          for (int k = 0; k < D - 1; ++k) {
            const int v = idx[mt[k]];
            nidx[tt[ax[k]]] = flip[k] ? p - v : v;
          }
          const int an = nidx[0] + n * nidx[1] + n * n * nidx[2];
          const int64_t g = en * npe + an;
          if (g > INT32_MAX) {
            delete h;
            return LDG_ERR_ARG;
          }
          h->nbr_h[((e * D + d) * nl + l) * 2 + end] = (int32_t)g;
        }
      }
  h->nbf_h.assign(E * 2 * D, -1);
  for (int64_t k = 0; k < E * 2 * D; ++k) h->nbf_h[k] = (int8_t)nb_f[k];
  // ---- switch function -------------------------------------------------------
  h->sw_h.assign(E * D * 2, 0);
  for (int64_t e0 = 0; e0 < E; ++e0)
    for (int d0 = 0; d0 < D; ++d0) {
      if (h->sw_h[(e0 * D + d0) * 2]) continue;
      h->sw_h[(e0 * D + d0) * 2 + 1] = 1;
      h->sw_h[(e0 * D + d0) * 2 + 0] = -1;
      for (int start = 1; start >= 0; --start) {
        int64_t e = e0;
        int d = d0, end = start;
        for (;;) {
          const int f = 2 * d + end;
          const int64_t en = nb_e[e * 2 * D + f];
          if (en < 0) break;
          const int fn = nb_f[e * 2 * D + f], dn = fn / 2, endn = fn % 2;
          const int8_t want = (int8_t)-h->sw_h[(e * D + d) * 2 + end];
          int8_t* sn = &h->sw_h[(en * D + dn) * 2];
          if (sn[0] != 0) {
            if (sn[endn] != want) {
              delete h;
              return LDG_ERR_MESH;
            }
            break;
          }
          sn[endn] = want;
          sn[1 - endn] = (int8_t)-want;
          e = en;
          d = dn;
          end = 1 - endn;
        }
      }
    }
  if (mesh->switches) {  // the caller's switch function (a part of a partitioned mesh)
    for (int64_t k = 0; k < E * D; ++k) {
      const int8_t sm = mesh->switches[2 * k], sp = mesh->switches[2 * k + 1];
      if ((sp != 1 && sp != -1) || sm != -sp) {
        delete h;
        return LDG_ERR_MESH;
      }
    }
    for (int64_t e = 0; e < E; ++e)
      for (int f = 0; f < 2 * D; ++f) {
        const int64_t en = nb_e[e * 2 * D + f];
        if (en < 0) continue;
        const int fn = nb_f[e * 2 * D + f];
        if (mesh->switches[(e * D + f / 2) * 2 + f % 2] != -mesh->switches[(en * D + fn / 2) * 2 + fn % 2]) {
          delete h;
          return LDG_ERR_MESH;
        }
      }
    std::memcpy(h->sw_h.data(), mesh->switches, h->sw_h.size());
  }
  // ---- metric terms ------------------------------------------------------------
  linemet.assign((size_t)E * nl * D * D, 0.0f);
  ng.assign((size_t)E * D * nl * nq * D, 0.0);
  nend.assign((size_t)E * D * nl * 2 * D, 0.0);
  invJ.assign((size_t)E * npe, 0.0);
  // All metric arithmetic runs in long double and is rounded once: the
  // residual cancels large flux values against each other, so rounding of
  // the metric terms (coordinates of size L against spacings h) is amplified
  // by about L/h times the flux-to-residual ratio.
  auto cof_col = [D](const ld* G, int d, ld* nd) {
    // column d of J G^-T; G[a*3+b] = dx_a/dX_b
    if (D == 2) {
      if (d == 0) {
        nd[0] = G[1 * 3 + 1];
        nd[1] = -G[0 * 3 + 1];
      } else {
        nd[0] = -G[1 * 3 + 0];
        nd[1] = G[0 * 3 + 0];
      }
    } else {
      const int b1 = (d + 1) % 3, b2 = (d + 2) % 3;
      const ld u[3] = {G[0 * 3 + b1], G[1 * 3 + b1], G[2 * 3 + b1]};
      const ld v[3] = {G[0 * 3 + b2], G[1 * 3 + b2], G[2 * 3 + b2]};
      nd[0] = u[1] * v[2] - u[2] * v[1];
      nd[1] = u[2] * v[0] - u[0] * v[2];
      nd[2] = u[0] * v[1] - u[1] * v[0];
    }
  };
  std::vector<ld> xq, wq, phi, dphi;
  gauss01(nq, xq, wq);
  barycentric(s, xq, phi, dphi);
  // elements are independent: the loop runs on the host's cores (long double
  // is emulated in software on some hosts), every element computed the same way
  std::atomic<bool> bad{false};
  auto metric_range = [&](int64_t e_begin, int64_t e_end) {
  std::vector<ld> Gn((size_t)npe * 9);
  for (int64_t e = e_begin; e < e_end && !bad.load(std::memory_order_relaxed); ++e) {
    const double* X = mesh->nodes + e * npe * D;
    // G at the nodes: dx_x/dX_b by the nodal derivative matrix along b
    std::fill(Gn.begin(), Gn.end(), (ld)0);
    for (int b = 0; b < D; ++b)
      for (int l = 0; l < nl; ++l)
        for (int t = 0; t < n; ++t) {
          const int a = line_node(D, p, b, l, t);
          for (int x = 0; x < D; ++x) {
            ld acc = 0;
            for (int j = 0; j < n; ++j) acc += Dnode[t * n + j] * (ld)X[line_node(D, p, b, l, j) * D + x];
            Gn[a * 9 + x * 3 + b] = acc;
          }
        }
    // predictor features: G averaged over each direction-1 line, over the
    // line average of h = J^(1/D)
    for (int l = 0; l < nl; ++l) {
      ld gs[9] = {0}, hs = 0;
      for (int t2 = 0; t2 < n; ++t2) {
        const int a = line_node(D, p, 0, l, t2);
        const ld* G = &Gn[a * 9];
        const ld J = (D == 2) ? G[0] * G[4] - G[1] * G[3]
                              : G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
                                    G[2] * (G[3] * G[7] - G[4] * G[6]);
        hs += std::pow(J > 0 ? J : (ld)0, (ld)1 / D);
        for (int x = 0; x < D; ++x)
          for (int b = 0; b < D; ++b) gs[x * D + b] += G[x * 3 + b];
      }
      for (int k = 0; k < D * D; ++k) linemet[((size_t)e * nl + l) * D * D + k] = (float)(gs[k] / hs);
    }
    for (int a = 0; a < npe; ++a) {
      const ld* G = &Gn[a * 9];
      ld J;
      if (D == 2)
        J = G[0] * G[4] - G[1] * G[3];
      else
        J = G[0] * (G[4] * G[8] - G[5] * G[7]) - G[1] * (G[3] * G[8] - G[5] * G[6]) +
            G[2] * (G[3] * G[7] - G[4] * G[6]);
      if (!(J > 0)) {
        bad = true;
        return;
      }
      invJ[e * npe + a] = (double)(1 / J);
    }
    for (int d = 0; d < D; ++d)
      for (int l = 0; l < nl; ++l) {
        const size_t L = (size_t)(e * D + d) * nl + l;
        // at (xi_q, other nodes): dx/dX_d from the derivative of the line
        // interpolant, the other columns by interpolating nodal derivatives
        for (int q = 0; q < nq; ++q) {
          ld G[9] = {0};
          for (int x = 0; x < D; ++x)
            for (int b = 0; b < D; ++b) {
              ld acc = 0;
              for (int t = 0; t < n; ++t) {
                const int a = line_node(D, p, d, l, t);
                if (b == d)
                  acc += dphi[q * n + t] * (ld)X[a * D + x];
                else
                  acc += phi[q * n + t] * Gn[a * 9 + x * 3 + b];
              }
              G[x * 3 + b] = acc;
            }
          ld nd[3] = {0, 0, 0};
          cof_col(G, d, nd);
          for (int x = 0; x < D; ++x) ng[(L * nq + q) * D + x] = (double)nd[x];
        }
        // N^- at xi = 0 and N^+ at xi = 1 (Eqs. 4 and 6)
        for (int end = 0; end < 2; ++end) {
          const int a = line_node(D, p, d, l, end * p);
          ld nd[3] = {0, 0, 0};
          cof_col(&Gn[a * 9], d, nd);
          for (int x = 0; x < D; ++x) nend[(L * 2 + end) * D + x] = (double)(end ? nd[x] : -nd[x]);
        }
      }
  }
  };
  {
    unsigned nth = std::thread::hardware_concurrency();
    nth = nth < 1 ? 1 : (nth > 64 ? 64 : nth);
    if ((int64_t)nth > E) nth = (unsigned)(E > 0 ? E : 1);
    const int64_t chunk = (E + nth - 1) / nth;
    std::vector<std::thread> pool;
    for (unsigned k = 0; k < nth; ++k) {
      const int64_t e0 = (int64_t)k * chunk, e1 = e0 + chunk < E ? e0 + chunk : E;
      if (e0 < e1) pool.emplace_back(metric_range, e0, e1);
    }
    for (auto& th : pool) th.join();
  }
  if (bad) {
    delete h;
    return LDG_ERR_MESH;
  }
  *hp = h;
  return LDG_OK;
}

extern "C" int ldg_setup(const ldg_mesh_t* mesh, const ldg_equations_t* eq, ldg_handle_t** out) {
  if (!mesh || !eq || !out) return LDG_ERR_ARG;
  *out = nullptr;
  std::vector<double> ng, nend, invJ;
  std::vector<float> linemet;
  ldg_handle_t* h = nullptr;
  int rc = host_setup(mesh, eq, &h, ng, nend, invJ, linemet);
  if (rc != LDG_OK) return rc;
  const int D = h->D;
  // ---- upload ---------------------------------------------------------------
  auto up = [](void** dst, const void* src, size_t bytes) -> cudaError_t {
    cudaError_t err = cudaMalloc(dst, bytes);
    if (err != cudaSuccess) return err;
    return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cudaError_t err = cudaSuccess;
  err = up((void**)&h->nbr, h->nbr_h.data(), h->nbr_h.size() * sizeof(int32_t));
  if (err == cudaSuccess) err = up((void**)&h->sw, h->sw_h.data(), h->sw_h.size());
  if (err == cudaSuccess) err = up((void**)&h->ng, ng.data(), ng.size() * sizeof(double));
  if (err == cudaSuccess) err = up((void**)&h->nend, nend.data(), nend.size() * sizeof(double));
  if (err == cudaSuccess) err = up((void**)&h->invJ, invJ.data(), invJ.size() * sizeof(double));
  if (err == cudaSuccess && eq->g_D)
    err = up((void**)&h->gD, eq->g_D, (size_t)h->ndof * sizeof(double));
  if (err == cudaSuccess && eq->source)
    err = up((void**)&h->src, eq->source, (size_t)h->ndof * sizeof(double));
  if (err == cudaSuccess && eq->g_N)
    err = up((void**)&h->gN, eq->g_N, (size_t)h->ndof * D * sizeof(double));
  if (err == cudaSuccess) err = up((void**)&h->nbf, h->nbf_h.data(), h->nbf_h.size());
  if (err == cudaSuccess) err = up((void**)&h->linemet, linemet.data(), linemet.size() * sizeof(float));
  if (err == cudaSuccess && h->viscous())
    err = cudaMalloc((void**)&h->Qbuf, (size_t)h->ndof * D * sizeof(double));
  if (err == cudaSuccess) {
    // element Line-DG pattern (Sec. 2.3): row i couples to the D p + 1 nodes
    // of its lines; wavefront levels i + j + k order the triangular solves
    const int n = h->p + 1, npe = h->npe, W = h->pat_w();
    std::vector<int16_t> pat((size_t)npe * W), lvl(npe);
    std::vector<int8_t> slot((size_t)npe * npe, -1);
    std::vector<int32_t> lptr(D * h->p + 2, 0);
    for (int i = 0; i < npe; ++i) {
      const int ii[3] = {i % n, (i / n) % n, (i / (n * n)) % n};
      std::vector<int> cols;
      for (int j = 0; j < npe; ++j) {
        const int jj[3] = {j % n, (j / n) % n, (j / (n * n)) % n};
        int diff = 0;
        for (int b = 0; b < D; ++b) diff += (ii[b] != jj[b]);
        if (diff <= 1) cols.push_back(j);
      }
      for (int s = 0; s < W; ++s) {
        pat[(size_t)i * W + s] = (int16_t)cols[s];
        slot[(size_t)i * npe + cols[s]] = (int8_t)s;
      }
      lptr[ii[0] + ii[1] + ii[2] + 1]++;
    }
    for (int k = 1; k < (int)lptr.size(); ++k) lptr[k] += lptr[k - 1];
    std::vector<int32_t> fill(lptr.begin(), lptr.end());
    for (int i = 0; i < npe; ++i) {
      const int lv = (i % n) + ((i / n) % n) + ((i / (n * n)) % n);
      lvl[fill[lv]++] = (int16_t)i;
    }
    err = up((void**)&h->pat, pat.data(), pat.size() * sizeof(int16_t));
    if (err == cudaSuccess) err = up((void**)&h->slot, slot.data(), slot.size());
    if (err == cudaSuccess) err = up((void**)&h->lvl, lvl.data(), lvl.size() * sizeof(int16_t));
    if (err == cudaSuccess) err = up((void**)&h->lvl_ptr, lptr.data(), lptr.size() * sizeof(int32_t));
  }
  if (err == cudaSuccess) {
    h->red_len = 4096;
    err = cudaMalloc((void**)&h->red, h->red_len * sizeof(double));
  }
  if (err != cudaSuccess) {
    ldg_destroy(h);
    return LDG_ERR_CUDA;
  }
  *out = h;
  return LDG_OK;
}

extern "C" int ldg_setup_host(const ldg_mesh_t* mesh, const ldg_equations_t* eq, int64_t* nbr,
                              int8_t* sw, double* ng, double* nend, double* invJ, double* tables) {
  if (!mesh || !eq) return LDG_ERR_ARG;
  std::vector<double> vng, vnend, vinvJ;
  std::vector<float> vlm;
  ldg_handle_t* h = nullptr;
  int rc = host_setup(mesh, eq, &h, vng, vnend, vinvJ, vlm);
  if (rc != LDG_OK) return rc;
  if (nbr)
    for (size_t i = 0; i < h->nbr_h.size(); ++i) nbr[i] = h->nbr_h[i];
  if (sw) std::memcpy(sw, h->sw_h.data(), h->sw_h.size());
  if (ng) std::memcpy(ng, vng.data(), vng.size() * sizeof(double));
  if (nend) std::memcpy(nend, vnend.data(), vnend.size() * sizeof(double));
  if (invJ) std::memcpy(invJ, vinvJ.data(), vinvJ.size() * sizeof(double));
  if (tables) {
    // Phi [nq][p+1], Kd [p+1][nq], L0 [p+1], L1 [p+1]
    const int n = h->p + 1, nq = h->nq;
    double* o = tables;
    for (int q = 0; q < nq; ++q)
      for (int j = 0; j < n; ++j) *o++ = h->tab.Phi[q][j];
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < nq; ++q) *o++ = h->tab.Kd[i][q];
    for (int i = 0; i < n; ++i) *o++ = h->tab.L0[i];
    for (int i = 0; i < n; ++i) *o++ = h->tab.L1[i];
  }
  delete h;
  return LDG_OK;
}

extern "C" int ldg_destroy(ldg_handle_t* h) {
  if (!h) return LDG_OK;
  if (h->gs_pin) cudaFreeHost(h->gs_pin);
  if (h->gs_ev) cudaEventDestroy(h->gs_ev);
  ldg_jac_destroy(h->Jn);
  ldg_pc_destroy(h->Pn);
  cudaFree(h->ws);
  cudaFree(h->nbr);
  cudaFree(h->sw);
  cudaFree(h->ng);
  cudaFree(h->nend);
  cudaFree(h->invJ);
  cudaFree(h->gD);
  cudaFree(h->gN);
  free_coupled(h->cpl);
  cudaFree(h->src);
  cudaFree(h->Qbuf);
  cudaFree(h->dirk);
  cudaFree(h->red);
  cudaFree(h->nbf);
  cudaFree(h->linemet);
  cudaFree(h->pat);
  cudaFree(h->slot);
  cudaFree(h->lvl);
  cudaFree(h->lvl_ptr);
  delete h;
  return LDG_OK;
}

extern "C" int ldg_info(const ldg_handle_t* h, int64_t info[10]) {
  if (!h || !info) return LDG_ERR_ARG;
  const int64_t NL = h->nlines();
  int64_t v[10] = {h->D,  h->p,  h->nc,   h->E, h->npe, h->nl, h->nq, h->ndof, (int64_t)h->nk11() * NL,
                   (int64_t)h->nk12() * NL};
  for (int i = 0; i < 10; ++i) info[i] = v[i];
  return LDG_OK;
}

extern "C" int ldg_export_tables(const ldg_handle_t* h, int64_t* nbr, int8_t* sw) {
  if (!h) return LDG_ERR_ARG;
  if (nbr)
    for (size_t i = 0; i < h->nbr_h.size(); ++i) nbr[i] = h->nbr_h[i];
  if (sw) std::memcpy(sw, h->sw_h.data(), h->sw_h.size());
  return LDG_OK;
}
