/*
 * ldg.h -- C ABI of the GB300 Line-DG library (libldg.so).
 *
 * Line-based discontinuous Galerkin discretisation of Persson, "A sparse and
 * high-order accurate line-based discontinuous Galerkin method for
 * unstructured meshes": residual evaluation, the line-sparse Jacobian, its
 * split Jacobian-vector product, the element-block ILU(0) preconditioner and
 * a BDF2 Newton-GMRES step.
 *
 * Conventions for every call
 *   - returns LDG_OK (0) or a negative LDG_ERR_* code; on error nothing the
 *     caller owns has been freed, and outputs may be partially written;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); work is enqueued on it and the call returns without waiting
 *     unless stated otherwise;
 *   - pointers named U, R, Q, x, y, r, z are DEVICE pointers owned by the
 *     caller; the library never frees them;
 *   - the library owns the handle and every object it returns (tables,
 *     metrics, Jacobians, factors, Krylov bases) until the matching destroy
 *     call;
 *   - nodal arrays use the layout [n_elem][n_c][(p+1)^D] (row-major) with
 *     local node a = i + (p+1) j + (p+1)^2 k, i running along reference
 *     direction 1 (Sec. 2.1); the flat DOF index is (e n_c + c) (p+1)^D + a.
 */
#ifndef LDG_H
#define LDG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LDG_OK 0
#define LDG_ERR_ARG (-1)              /* invalid argument or size           */
#define LDG_ERR_CUDA (-2)             /* a CUDA runtime call failed         */
#define LDG_ERR_MESH (-3)             /* non-conforming mesh, bad face
                                         orientation, non-symmetric node set,
                                         inconsistent switch, J <= 0       */
#define LDG_ERR_NONFINITE (-4)        /* NaN/Inf in a residual or norm      */
#define LDG_ERR_GMRES_BREAKDOWN (-5)  /* Krylov basis lost rank             */
#define LDG_ERR_NEWTON_MAXIT (-6)     /* Newton iteration cap reached       */
#define LDG_ERR_NOT_BUILT (-7)        /* object used before it was built    */
#define LDG_ERR_UNSUPPORTED (-8)      /* (D, p, equation) not compiled in   */
#define LDG_ERR_TOO_LARGE (-9)        /* problem exceeds a fixed-size buffer  */

/* ---- equations (Sec. 2.1 Eq. 1, Sec. 3 Eq. 14, Sec. 5 Eqs. 42-48) ------- */
#define LDG_EQ_POISSON 0        /* -div(grad u) = f, F = -q, n_c = 1         */
#define LDG_EQ_EULER 1          /* compressible Euler, n_c = D + 2           */
#define LDG_EQ_NAVIER_STOKES 2  /* compressible NS, constant mu, n_c = D + 2 */
#define LDG_EQ_ADVECTION 3      /* scalar u_t + div(a u) = 0, n_c = 1        */

#define LDG_FLUX_ROE 0  /* Roe averages, Harten entropy fix delta = 0.1 c   */
#define LDG_FLUX_LF 1   /* local Lax-Friedrichs (Rusanov)                  */

#define LDG_BC_DIRICHLET 0  /* Eqs. 27-28: u^ = g_D, penalty C11_b        */
#define LDG_BC_WALL 1       /* no-slip adiabatic wall (NS; builder-defined) */
#define LDG_BC_NEUMANN 2    /* Eqs. 29-30 (C22 = 0): F^.n = G.n from the
                               prescribed flux G (g_N below), u^ = u_inside */

#define LDG_PREC_FP32 0
#define LDG_PREC_FP64 1

/*
 * Mesh (host memory, copied by ldg_setup). Sec. 2.1: each element carries
 * a Cartesian grid of (p+1)^D nodes x_ijk = x(X_ijk), X_ijk = (s_i, s_j, s_k).
 *   s        [p+1]                    increasing node set on [0,1], s_0 = 0,
 *                                     s_p = 1, symmetric (s_{p-i} = 1 - s_i)
 *   nodes    [n_elem][(p+1)^D][D]     node coordinates
 *   vertices [n_elem][2^D]            global vertex ids; local corner c sits at
 *                                     reference corner (c&1, (c>>1)&1, (c>>2)&1);
 *                                     periodic images share ids
 *   btag     [n_elem][2D]             face f = 2d + end (end 0: X_d = 0, end 1:
 *                                     X_d = 1); -1 = interior (matched through
 *                                     vertex ids), >= 0 = boundary tag
 *   switches [n_elem][D][2] or NULL  the switch function S^-_d, S^+_d (Sec. 3)
 *                                     to use instead of deriving it: one part of a
 *                                     partitioned mesh passes the global function
 *                                     restricted to its elements. Checked: values
 *                                     +-1, S^- = -S^+, opposite signs across
 *                                     every matched face (else LDG_ERR_MESH)
 */
typedef struct {
  int32_t D;
  int32_t p;
  int64_t n_elem;
  const double* s;
  const double* nodes;
  const int64_t* vertices;
  const int32_t* btag;
  const int8_t* switches;
} ldg_mesh_t;

/*
 * Equations and fluxes (host memory, copied).
 *   kind, flux        LDG_EQ_*, LDG_FLUX_*
 *   gamma, mu, Pr     ideal gas ratio, constant viscosity, Prandtl number
 *   C11, C11_b        LDG penalty at interior faces (0 = minimal dissipation)
 *                     and at Dirichlet/wall boundaries (> 0), Eqs. 25, 27:
 *                     an interior line end's F^.n (non-unit n of Eq. 7) gains
 *                     C11 (u_in - u_out), a penalty per unit reference length
 *                     (C11 / h physically); a boundary end gains
 *                     C11_b |n| (u_in - g_D)
 *   adv[3]            advection velocity (LDG_EQ_ADVECTION)
 *   n_bc, bc_kind     bc_kind[tag] = LDG_BC_* for boundary tags 0..n_bc-1
 *   g_D               [n_elem][n_c][(p+1)^D] Dirichlet data (read at boundary
 *                     face nodes) or NULL
 *   source            [n_elem][n_c][(p+1)^D] source S(x) added to R, or NULL
 *   g_N               [n_elem][n_c][D][(p+1)^D] prescribed flux vector G at
 *                     the nodes of Neumann faces, or NULL (zero flux). A line
 *                     end on a Neumann face takes F^.n = G.n with its
 *                     non-unit normal n (a scalar normal flux g_N is
 *                     G = g_N n/|n|); a corner node shared by two Neumann
 *                     faces carries one vector for both. The flux does not
 *                     depend on the state, so its Jacobian entries are zero;
 *                     the gradient's trace there is the inside value.
 *   C22               LDG penalty on the jump of the normal viscous flux in
 *                     the trace u^ (Eq. 26; >= 0, Poisson only). 0 is the
 *                     minimal-dissipation scheme every other call computes;
 *                     with C22 > 0 the gradient depends on itself, and only
 *                     ldg_gradient_uq, ldg_residual_uq and ldg_coupled_solve
 *                     accept the handle (others return LDG_ERR_UNSUPPORTED).
 */
typedef struct {
  int32_t kind;
  int32_t flux;
  double gamma;
  double mu;
  double Pr;
  double C11;
  double C11_b;
  double adv[3];
  int32_t n_bc;
  const int32_t* bc_kind;
  const double* g_D;
  const double* source;
  const double* g_N;
  double C22;
} ldg_equations_t;

typedef struct ldg_handle ldg_handle_t;
typedef struct ldg_jac ldg_jac_t;
typedef struct ldg_pc ldg_pc_t;

/*
 * Build a handle: 1-D rules (Gauss-Legendre with ceil((3p+1)/2) points,
 * Lagrange basis, mass matrix, Cholesky, Sec. 2.2), face matching and
 * neighbour-node tables (Sec. 2.1), the switch function (Sec. 3) and the
 * metric terms J, n_d at Gauss points and n^+- at line ends (Eqs. 2, 4-6,
 * Sec. 2.2), uploaded to the current device. Synchronous. *out receives the
 * handle (freed by ldg_destroy).
 * Errors: LDG_ERR_ARG (sizes), LDG_ERR_MESH, LDG_ERR_UNSUPPORTED, LDG_ERR_CUDA.
 */
int ldg_setup(const ldg_mesh_t* mesh, const ldg_equations_t* eq, ldg_handle_t** out);

/*
 * The host half of ldg_setup alone, for checks without a GPU: writes the
 * integer tables and metric terms the device would receive to any non-NULL
 * host buffer (sizes as for ldg_export_tables, plus ng [n_elem][D][nl][n_q][D],
 * nend [n_elem][D][nl][2][D] (n^- at end 0, n^+ at end 1), invJ
 * [n_elem][(p+1)^D], and tables = Phi [n_q][p+1], Kd [p+1][n_q], L0 [p+1],
 * L1 [p+1] of Sec. 2.2). Touches no device. Errors as ldg_setup.
 */
int ldg_setup_host(const ldg_mesh_t* mesh, const ldg_equations_t* eq, int64_t* nbr, int8_t* sw,
                   double* ng, double* nend, double* invJ, double* tables);

/* Free the handle and everything it owns. NULL is accepted. */
int ldg_destroy(ldg_handle_t* h);

/*
 * Sizes: info[0..9] = {D, p, n_c, n_elem, (p+1)^D, (p+1)^(D-1) lines per
 * direction, n_q Gauss points, ndof, K11 floats, K12 floats}.
 */
int ldg_info(const ldg_handle_t* h, int64_t info[10]);

/*
 * Copy the integer tables to host memory (for bit-exact checks):
 *   nbr [n_elem][D][(p+1)^(D-1)][2]  global id e (p+1)^D + a of the outside
 *                                    node of each line end, or -1 - tag
 *   sw  [n_elem][D][2]               switch S^-_d (end 0), S^+_d (end 1)
 * Either pointer may be NULL.
 */
int ldg_export_tables(const ldg_handle_t* h, int64_t* nbr, int8_t* sw);

/*
 * Residual of the semi-discrete system, dU/dt = R(U) (Eqs. 10, 31, 36):
 * R = -(1/J) sum_d r^(d) + S, r^(d) from Eq. 7 per line. For second-order
 * equations the LDG gradient Q = D(U) (Eqs. 19-20, 32) is evaluated first
 * into a library-owned buffer. FP64 throughout. U, R: device [n_elem][n_c][(p+1)^D].
 */
int ldg_residual(ldg_handle_t* h, const double* U, double* R, void* stream);

/*
 * The same residual as ldg_residual, computed without allocating anything,
 * for callers that must not call cudaMalloc after start-up (their device
 * memory is owned by another allocator, or their run loop may not
 * allocate). The paper has no counterpart: this is an interface variant.
 * The LDG gradient scratch of second-order equations lives in a fixed
 * device array of LDG_NOALLOC_MAX_Q doubles (8 MiB, held by every GPU that
 * loads the library until the process exits) instead of the handle's
 * buffer. Returns LDG_ERR_TOO_LARGE when n_elem n_c D (p+1)^D exceeds
 * LDG_NOALLOC_MAX_Q. The first call on a device looks up the array's device
 * address; make that first call before any stream capture. All calls share
 * the array, so calls that overlap on the GPU race on it; each call
 * overwrites what it reads, so nothing carries over between calls.
 * First-order equations need no scratch and never touch the array. For the
 * stabilised scheme (C22 != 0) the call returns LDG_ERR_UNSUPPORTED, as
 * ldg_residual does.
 * U, R: device [n_elem][n_c][(p+1)^D], FP64.
 */
#define LDG_NOALLOC_MAX_Q 1048576
int ldg_residual_noalloc(ldg_handle_t* h, const double* U, double* R, void* stream);

/* The LDG gradient alone: Q = D(U), device [n_elem][n_c][D][(p+1)^D], FP64. */
int ldg_gradient(ldg_handle_t* h, const double* U, double* Q, void* stream);

/* R(U, Q) for a given Q (the split form of Eq. 33), FP64. */
int ldg_residual_uq(ldg_handle_t* h, const double* U, const double* Q, double* R, void* stream);

/*
 * Jacobian matrices in the line-block format (Sec. 4.1 Eq. 35, Sec. 2.3):
 * K11 = dR/dU and, for second-order equations, K12 = dR/dQ and the constant
 * K21 = dD/dU. If *J is NULL a new object is allocated, otherwise its
 * buffers are reused. prec = LDG_PREC_FP32 (values computed in FP32 from the
 * FP64 state) or LDG_PREC_FP64. Storage, per element e, direction d, line l,
 * with L = (e D + d) nl + l and NL = n_elem D nl lines:
 *   K11 in-line : K11[((i (p+1) + j) n_c + c) n_c + c'][L]   dR_(i,c)/dU_(j,c')
 *   K11 faces   : K11[OFF + ((end (p+1) + i) n_c + c) n_c + c'][L]
 *                 dR_(i,c)/dU_out(end,c'),  OFF = (p+1)^2 n_c^2
 *   K12         : same with n_c x (n_c D) blocks, index c' -> c' D + b,
 *                 one face block per line (the end whose switch takes the
 *                 viscous flux from outside), end index dropped
 *   K21         : scalar, in-line [(i (p+1) + j) D + b][L], face
 *                 [KOFF + i D + b][L] for the end whose u^ comes from outside
 * (entry-major, line-minor: a thread per line reads coalesced).
 * On meshes with no-slip walls (LDG_BC_WALL; Euler and Navier-Stokes) K11
 * and K12 include the wall flux, and the gradient's wall trace (the wall
 * state of the inside trace, a nonlinear function of it) adds a
 * state-dependent part to K21: for each wall line end the energy row
 * w = (|m|^2 / (2 rho^2), -m / rho, 1) of the wall state's derivative is
 * stored with the Jacobian (identity on rho, zero on momentum); the split
 * matvec and the preconditioner apply it. It is not part of the export.
 */
int ldg_jacobian(ldg_handle_t* h, const double* U, int prec, ldg_jac_t** J, void* stream);

/* Free a Jacobian object. NULL is accepted. */
int ldg_jac_destroy(ldg_jac_t* J);

/*
 * Copy the Jacobian arrays to host memory in the layout above (FP32 or FP64
 * as built). Any pointer may be NULL. Synchronous.
 */
int ldg_jac_export(const ldg_jac_t* J, void* K11, void* K12, void* K21);

/*
 * Split Jacobian-vector product (Eq. 41):
 *   y = shift x + scale (K11 x + K12 (K21 x)).
 * With shift = 1, scale = -alpha dt this is the Newton matrix of Eq. 39.
 * x, y: device [ndof] of type float (prec = LDG_PREC_FP32) or double
 * (LDG_PREC_FP64; matrix values are used at the precision they were built).
 */
int ldg_jacvec(ldg_handle_t* h, const ldg_jac_t* J, double shift, double scale, const void* x,
               void* y, int prec, void* stream);

/*
 * The two halves of the split product of Eq. 41, for runs on a partitioned
 * mesh (one part per process or GPU) that exchange the face-node traces of
 * the discrete gradient between them: a part's K12 reaches K21 x at the
 * outside node of its lines' ends, which another part owns.
 *   ldg_k21_apply: g = K21 x (second-order equations; LDG_ERR_UNSUPPORTED
 *     otherwise), g device [n_elem][n_c][D][(p+1)^D] in the vector precision.
 *   ldg_jacvec_g: y = shift x + scale (K11 x + K12 g) with the given g (g may
 *     be NULL for first-order equations).
 * Precisions and errors as ldg_jacvec. ldg_k21_apply followed by
 * ldg_jacvec_g on the same g equals ldg_jacvec.
 */
int ldg_k21_apply(ldg_handle_t* h, const ldg_jac_t* J, const void* x, void* g, int prec, void* stream);
int ldg_jacvec_g(ldg_handle_t* h, const ldg_jac_t* J, double shift, double scale, const void* x,
                 const void* g, void* y, int prec, void* stream);

/*
 * ldg_jacobian at a given gradient Q (device FP64 [n_elem][n_c][D][(p+1)^D],
 * required for second-order equations, ignored for first-order ones)
 * instead of Q = D(U): a part of a partitioned mesh passes the gradient whose
 * face-node traces at its cut faces came from the parts that own them.
 * Otherwise as ldg_jacobian.
 */
int ldg_jacobian_uq(ldg_handle_t* h, const double* U, const double* Q, int prec, ldg_jac_t** J,
                    void* stream);

/*
 * Block-Jacobi preconditioner (Sec. 4.2): per element, A~_e = shift I +
 * scale mask(K11 + K12 K21) on the element-local Line-DG pattern (node i
 * couples to the Dp+1 nodes of its D lines), inter-element couplings and
 * out-of-pattern fill dropped, then block ILU(0) in that pattern with n_c x
 * n_c blocks in node order i + (p+1) j + (p+1)^2 k. Factors are kept at
 * the Jacobian's precision. *P allocated if NULL, else reused.
 */
int ldg_precond(ldg_handle_t* h, const ldg_jac_t* J, double shift, double scale, ldg_pc_t** P,
                void* stream);

/* z = (L U)^{-1} r per element; r, z device [ndof] float or double (prec). */
int ldg_precond_apply(ldg_handle_t* h, const ldg_pc_t* P, const void* r, void* z, int prec,
                      void* stream);

/* Free a preconditioner. NULL is accepted. */
int ldg_pc_destroy(ldg_pc_t* P);

/*
 * Copy the ILU(0) factors to host: [n_elem][(p+1)^D][Dp+1][n_c][n_c] in the
 * precision they were built; column order of each row = sorted local node
 * ids of its pattern. Strictly-lower blocks hold L (unit diagonal implied),
 * the rest hold U. Synchronous.
 */
int ldg_pc_export(const ldg_pc_t* P, void* factors);

/* ---- implicit step ----------------------------------------------------- */
#define LDG_MODE_FP64 0   /* FP64 Jacobian, ILU, Krylov basis              */
#define LDG_MODE_MIXED 1  /* FP32 Jacobian/ILU/Krylov, FP64 refinement      */

#define LDG_PRED_EXTRAP 0  /* U0 = 2 U^n - U^{n-1} (U^n on the first step)   */
#define LDG_PRED_GIVEN 1   /* U0 = the caller's U_next on entry             */
#define LDG_PRED_CHECKED 2 /* the caller's guess U1 judged by the BDF residual:
                              U0 = extrapolation, the guess is U0 + b (U1 - U0)
                              with b in [0,1] minimising the linearised
                              ||G||; b = 0 falls back to extrapolation       */

typedef struct {
  int32_t mode;          /* LDG_MODE_*                                        */
  int32_t predictor;     /* LDG_PRED_*                                        */
  int32_t first_step;    /* 1: BDF1 (U_nm1 unused)                            */
  int32_t restart;       /* GMRES restart length (<= 64)                      */
  int32_t max_newton;    /* iteration cap                                      */
  int32_t reuse;         /* rebuild K, P when Newton its since rebuild > reuse */
  int32_t max_refine;    /* GMRES cycles per linear solve, each restarted from
                            the true FP64 residual (the FP64 refinement of the
                            mixed mode; restarted GMRES in the FP64 mode)     */
  int32_t force_rebuild; /* 1: build K, P at the first Newton iteration       */
  double rtol;           /* ||G(U)||_2 <= rtol ||G(U^n)||_2                  */
  double gmres_tol;      /* relative tolerance of each linear solve           */
  int32_t stall_rebuild; /* 1: also rebuild K, P when a Newton step fails to
                            halve ||G|| (an addition to the paper's policy)   */
  int32_t forcing;       /* LDG_FORCING_*: relative tolerance of each linear
                            solve (not in the paper)                          */
  int32_t ortho;         /* LDG_ORTHO_*: Gram-Schmidt of the Arnoldi columns
                            (the paper does not name one)                     */
  double reorth_factor;  /* LDG_ORTHO_SELECTIVE: a second pass when the first
                            shrinks the column by more than this factor
                            (<= 0: 10, Rutishauser's value; 1: always)        */
} ldg_solver_opts_t;

#define LDG_ORTHO_CGS2 0      /* classical Gram-Schmidt, always twice          */
#define LDG_ORTHO_SELECTIVE 1 /* FP64 basis: classical Gram-Schmidt, a second
                                 pass only where the first shrank the column
                                 by more than a factor 10 (Rutishauser's
                                 criterion); an FP32 basis (LDG_MODE_MIXED)
                                 always takes CGS2                            */

#define LDG_FORCING_FIXED 0  /* every linear solve to gmres_tol ||G||          */
#define LDG_FORCING_TARGET 1 /* to max(gmres_tol, 0.5 target / ||G||) ||G||
                                (target = rtol ||G(U^n)||): no solve reduces
                                ||G|| further than the stopping rule needs, so
                                the linear work follows the decades between
                                the start and the target                      */

typedef struct {
  int32_t newton_its;
  int32_t gmres_its;
  int32_t jac_builds;
  int32_t refine_sweeps;
  double res0;           /* ||G(U^n)||_2                                      */
  double res_final;      /* ||G(U_next)||_2                                   */
  double res_pred;       /* ||G(U0)||_2 of the predictor                      */
  double t_residual_ms;  /* host-timed phases (events)                        */
  double t_jacobian_ms;
  double t_precond_ms;
  double t_linear_ms;
  double res_extrap;     /* ||G|| of the extrapolation (LDG_PRED_CHECKED)     */
  double pred_weight;    /* weight b of the caller's guess (LDG_PRED_CHECKED) */
  int32_t reorth_its;    /* GMRES iterations whose Arnoldi column took a
                            second Gram-Schmidt pass                          */
} ldg_step_stats_t;

/*
 * One BDF2 time level (BDF1 when opts->first_step) solved by Newton's
 * method on G(U) = U - 4/3 U^n + 1/3 U^{n-1} - 2/3 dt R(U) with
 * (I - 2/3 dt A) delta = -G(U) (Eqs. 39-41) by right-preconditioned
 * GMRES(restart) with the block-Jacobi ILU(0) preconditioner, Jacobian
 * re-use (Sec. 4.3), and in LDG_MODE_MIXED FP64 iterative refinement of each
 * linear solve. U_next: device FP64 [ndof], in/out. U_nm2 is accepted for
 * interface symmetry and may be NULL. Synchronises on stream (reads norms).
 * Errors: LDG_ERR_NEWTON_MAXIT, LDG_ERR_NONFINITE, LDG_ERR_GMRES_BREAKDOWN.
 */
int ldg_newton_step(ldg_handle_t* h, double* U_next, const double* U_n, const double* U_nm1,
                    const double* U_nm2, double dt, const ldg_solver_opts_t* opts,
                    ldg_step_stats_t* stats, void* stream);

/*
 * One step of the paper's own integrator, Alexander's L-stable three-stage
 * third-order DIRK (Sec. 4.1, Eqs. dirk1-dirk2 and their tableau, diagonal
 * alpha = 0.435866521508459): stage i solves
 *   U_i - alpha dt R(U_i) = B_i,   B_i = U^n + dt sum_{j<i} a_ij K_j,
 * by the Newton-GMRES solver of ldg_newton_step (its BDF1 form with U^n
 * replaced by B_i and dt by alpha dt, started from B_i), K_i = R(U_i), and
 * U^{n+1} = U^n + dt sum_j b_j K_j. All stages share (I - alpha dt A), so
 * the Jacobian and preconditioner are re-used across stages and steps under
 * opts->reuse (the paper's policy); opts->force_rebuild applies to the first
 * stage only, opts->first_step and opts->predictor are ignored. U_next and
 * U_n: device FP64 [ndof], distinct. stats: counts and phase times summed
 * over the three stages; res0 / res_final / res_pred of the last stage.
 * Work buffers (5 ndof doubles) are allocated on first use and kept with
 * the handle. Synchronises on stream. Errors as ldg_newton_step.
 */
int ldg_dirk3_step(ldg_handle_t* h, double* U_next, const double* U_n, double dt,
                   const ldg_solver_opts_t* opts, ldg_step_stats_t* stats, void* stream);

/*
 * One step of the classical explicit fourth-order Runge-Kutta method, the
 * paper's explicit time-stepping of dU/dt = R(U, D(U)) (Sec. 4.1):
 * K1 = R(U^n), K2 = R(U^n + dt/2 K1), K3 = R(U^n + dt/2 K2),
 * K4 = R(U^n + dt K3), U_next = U^n + dt/6 (K1 + 2 K2 + 2 K3 + K4).
 * U_next and U_n: device FP64 [ndof] (may be the same array). Four
 * residual evaluations, enqueued on stream without synchronising; work
 * buffers (5 ndof doubles, shared with ldg_dirk3_step) are allocated on
 * first use and kept with the handle. No stability check: dt is the
 * caller's.
 */
int ldg_rk4_step(ldg_handle_t* h, double* U_next, const double* U_n, double dt, void* stream);

/*
 * Steady state by pseudo-time continuation (Sec. 4.1): up to n_steps
 * backward Euler steps with increasing time steps dt_k = dt0 growth^k, each
 * solved by the Newton-GMRES solver of ldg_newton_step, then a final step
 * without the time derivative (R(U) = 0, solved as a backward Euler step
 * with dt = 1e15, for which (I - dt A) is dt A up to rounding), stopping as
 * soon as ||R(U)||_2 <= opts->rtol ||R(U_initial)||_2. U: device FP64
 * [ndof], in: the initial state, out: the steady state. opts as in
 * ldg_newton_step (first_step and predictor are ignored; every step starts
 * from the previous level); stats: counts and phase times summed over the
 * steps, res0 = ||R(U_initial)||_2, res_final = ||R(U)||_2 at return.
 * Work buffers shared with ldg_dirk3_step. Synchronises on stream. Errors
 * as ldg_newton_step; LDG_ERR_ARG for dt0 <= 0, growth < 1 or n_steps < 0.
 */
int ldg_steady_solve(ldg_handle_t* h, double* U, double dt0, double growth, int32_t n_steps,
                     const ldg_solver_opts_t* opts, ldg_step_stats_t* stats, void* stream);

/*
 * The stabilised LDG scheme (C22 > 0 in ldg_equations_t; scalar Poisson,
 * Sec. 3 Eqs. 25-26 and 30, Table 2's lower half). The trace u^ carries
 * C22 (F.n(inside) - F.n(outside)) with F = -q and the unit normal (the sign
 * that penalises the jump of the normal flux), so the gradient depends on
 * itself and the steady problem is the coupled split system of Eq. 36,
 *   Phi(U, Q) = (R(U, Q), Q - D(U, Q)) = 0.
 *
 * ldg_gradient_uq: Qout = D(U, Q) (also valid with C22 = 0, where Q may be
 * NULL and the result is ldg_gradient's). U [n_elem][1][(p+1)^D], Q and Qout
 * [n_elem][1][D][(p+1)^D], device FP64; Q and Qout may not alias.
 * Errors: LDG_ERR_ARG (NULL U/Qout, Q NULL with C22 > 0, Q == Qout),
 * LDG_ERR_UNSUPPORTED (first-order equations; Q with n_c > 1).
 */
int ldg_gradient_uq(ldg_handle_t* h, const double* U, const double* Q, double* Qout, void* stream);

/*
 * ldg_coupled_solve: solves Phi(U, Q) = 0 (Poisson, any C22 >= 0) by
 * right-preconditioned restarted GMRES(restart) on its Jacobian
 * [[K11, K12], [-K21, I - K22]] (Sec. 4.1), applied matrix-free by the
 * gradient and residual kernels without boundary data and source. The
 * preconditioner is the element block-Jacobi of that Jacobian (each
 * element's U and Q rows against its own U and Q columns, couplings between
 * elements dropped, as in Sec. 4.2), probed once per handle column by column
 * on a colouring of the elements and inverted on the device; it needs
 * (1 + D)(p+1)^D <= 128. Each cycle restarts from the true residual
 * Phi(U, Q); the solve stops when ||Phi||_2 <= rtol ||Phi(U_in, Q_in)||_2.
 * U, Q: device FP64, in: the initial guess (zeros are fine), out: the
 * solution. stats: newton_its = GMRES cycles, gmres_its = iterations,
 * res0 / res_final = ||Phi||_2 at entry / return, t_precond_ms = the
 * preconditioner build (first call), t_linear_ms = the iterations. The
 * handle keeps the preconditioner and the Krylov basis ((restart + 6) vectors
 * of (1 + D) ndof doubles) until ldg_destroy. Synchronises on stream.
 * Errors: LDG_ERR_ARG (rtol <= 0, restart outside 1..64, max_cycles < 1),
 * LDG_ERR_UNSUPPORTED (not Poisson; block too large), LDG_ERR_NEWTON_MAXIT
 * (target not met in max_cycles cycles; U, Q hold the last iterate),
 * LDG_ERR_NONFINITE, LDG_ERR_GMRES_BREAKDOWN, LDG_ERR_CUDA.
 */
int ldg_coupled_solve(ldg_handle_t* h, double* U, double* Q, double rtol, int32_t restart, int32_t max_cycles,
                      ldg_step_stats_t* stats, void* stream);

/* ---- learned Newton predictor (not in the paper) ------------------------
 * A line-local MLP n_in -> 128 -> 128 -> 128 -> n_out with GELU (tanh form)
 * predicts, for every line of reference direction 1, the correction to the
 * linear extrapolation 2 U^n - U^{n-1} of the next BDF level. Features per
 * line: [u^n, u^n - u^{n-1}, u^{n-1} - u^{n-2}] over the line's nodes
 * (index (level (p+1) + t) n_c + c) and the D x D deformation gradient
 * averaged over the line divided by the line average of J^(1/D), each
 * standardised; n_in = 3 (p+1) n_c + D^2 <= 96, n_out = (p+1) n_c <= 32.
 * Weights are FP32 masters with BF16 copies; products run on BF16 tensor
 * cores with FP32 accumulation. Parameters are exchanged as one flat vector
 * W1 [n_in][128], b1, W2 [128][128], b2, W3 [128][128], b3, W4 [128][n_out],
 * b4. Feature rows X are BF16 [M][96] (device), targets and outputs FP32
 * [M][n_out] (device), in units of the per-output scale.
 */
typedef struct ldg_mlp ldg_mlp_t;

/* Create a network with zero weights (set them with ldg_mlp_params). */
int ldg_mlp_create(int32_t n_in, int32_t n_out, ldg_mlp_t** out);
int ldg_mlp_destroy(ldg_mlp_t* m);

/* Get (set = 0) or set (set = 1) the FP32 master parameters through a host
 * FP64 array; setting resets the Adam state. Synchronous. */
int ldg_mlp_params(ldg_mlp_t* m, double* theta, int32_t set);

/* Standardisation of the features (mean, std; host [n_in]) and the output
 * scale (host [n_out]). */
int ldg_mlp_set_scaling(ldg_mlp_t* m, const double* in_mean, const double* in_std,
                        const double* out_scale);

/* Y = MLP(X) for M rows. */
int ldg_mlp_forward(ldg_mlp_t* m, const void* X, int64_t M, float* Y, void* stream);

/* Gradient of the mean squared error mean((Y - T)^2) over all M n_out
 * outputs: grad device [n_params], loss device scalar (may be NULL). */
int ldg_mlp_grad(ldg_mlp_t* m, const void* X, const float* T, int64_t M, float* grad, float* loss,
                 void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the gradient of
 * ldg_mlp_grad's loss; loss device scalar or NULL. */
int ldg_mlp_train_step(ldg_mlp_t* m, const void* X, const float* T, int64_t M, double lr, float* loss,
                       void* stream);

/* Standardised features of every direction-1 line of U^n, U^{n-1}, U^{n-2}
 * (device FP64 nodal arrays) into X (device BF16 [n_elem (p+1)^(D-1)][96]). */
int ldg_line_features(ldg_handle_t* h, const ldg_mlp_t* m, const double* Un, const double* Unm1,
                      const double* Unm2, void* X, void* stream);

/* Scaled targets (U^{n+1} - 2 U^n + U^{n-1}) / scale per line, FP32 [lines][n_out]. */
int ldg_line_targets(ldg_handle_t* h, const ldg_mlp_t* m, const double* Unext, const double* Un,
                     const double* Unm1, float* T, void* stream);

/* U0 = 2 U^n - U^{n-1} + scale * MLP(features), device FP64 nodal array. */
int ldg_mlp_predict(ldg_handle_t* h, ldg_mlp_t* m, const double* Un, const double* Unm1,
                    const double* Unm2, double* U0, void* stream);

/* Number of kernels the library has launched since it was loaded (a host
 * counter; for benchmarks that report launches per step). */
int ldg_launch_count(long long* out);

/* Benchmark instrumentation; the paper has no counterpart. While enabled
 * (enable != 0; each call also clears what was recorded), every launch of
 * the timed kernels is bracketed by two CUDA events recorded on the stream
 * it is launched on, and carries its algorithmic work. Timed kernels:
 *   LDG_KT_APPLY  (0) the ILU(0) apply (ldg_precond_apply, inside
 *                     ldg_newton_step): bytes = factors read
 *                     E (p+1)^D (Dp+1) n_c^2 + r read + z written;
 *   LDG_KT_JACVEC (1) the split matvec: bytes = K11 + K12 values + x + y;
 *   LDG_KT_ORTHO  (2) each GMRES Gram-Schmidt sweep: bytes = basis vectors
 *                     read + w read (+ written), FLOPs = 2 per multiply-add.
 * Events are created on first use and kept for reuse. */
#define LDG_KT_APPLY 0
#define LDG_KT_JACVEC 1
#define LDG_KT_ORTHO 2
int ldg_kernel_timer(int enable);

/* Launches of `kernel` with vectors of precision `prec` (LDG_PREC_FP32 /
 * LDG_PREC_FP64) recorded since the last ldg_kernel_timer call, their summed
 * device time in ms and summed algorithmic bytes and FLOPs (either pointer
 * may be null). Synchronizes on the recorded events. LDG_ERR_ARG for an
 * unknown kernel or precision or null launches/ms. */
int ldg_kernel_timer_read(int kernel, int prec, long long* launches, double* ms, double* bytes,
                          double* flops);

/* Benchmark instrumentation; the paper has no counterpart. Enqueues one
 * kernel of FP64 fused multiply-adds with no memory traffic in its loop
 * (16 independent chains per thread, 256 threads, 4 blocks per SM of the
 * current device, `iters` steps per chain) so that a caller timing it with
 * CUDA events on `stream` gets the FP64 FMA rate the device sustains, the
 * denominator of the FP64-bound kernels' roofline. sink: device buffer of at
 * least 4 x (number of SMs) doubles owned by the caller (one value per block
 * lands there). *fmas (host) receives the number of FMAs enqueued
 * (2 FLOPs each). LDG_ERR_ARG for iters < 1, a null pointer or a short sink. */
int ldg_fp64_fma_probe(int32_t iters, double* sink, int64_t sink_len, double* fmas, void* stream);

/* Change the constant viscosity of a Navier-Stokes handle (for sweeps over
 * Reynolds numbers); a retained Jacobian is marked stale. */
int ldg_set_viscosity(ldg_handle_t* h, double mu);

/* ||x||_2 of a device FP64 vector (synchronous; for drivers and tests). */
int ldg_norm2(ldg_handle_t* h, const double* x, int64_t n, double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LDG_H */
