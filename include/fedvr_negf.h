/*
 * fedvr_negf.h -- C ABI of the GB300 (sm_103a) FE-DVR second-Born library.
 *
 * The library computes the equilibrium (Matsubara) second-Born ground state of
 * the FE-DVR method of Balzer, Bauch & Bonitz (arXiv:0911.4348): basis and
 * quadrature setup (Sec. 2.1-2.2), Hartree-Fock (Sec. 2.3, Eqs. sigmahf,
 * hamhf, hfgf), the second-Born self-energy in two-index form (Sec. 2.3,
 * Eq. sigma2ndb), the two tau-convolutions of the Matsubara Dyson equation
 * (Sec. 2.3, Eq. deq) on a uniform power mesh (Sec. 3.1) and the
 * Galitskii-Migdal total energy (Sec. 2.3). Every step runs in CUDA kernels of
 * this library on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point:
 *  - Return value: FEDVR_OK (0) or a negative fedvr_status. Arguments are
 *    validated before any launch; an invalid one returns FEDVR_ERR_ARG and
 *    changes nothing. The library never aborts and never throws. The message
 *    of the last failure is kept per context (fedvr_last_error). A CUDA error
 *    inside a call returns FEDVR_ERR_CUDA, a device wait that gave up
 *    FEDVR_ERR_TIMEOUT; both are sticky: later calls on that context return
 *    FEDVR_ERR_STATE.
 *  - Matrices are dense, row-major, unpadded. A tau-stack of matrices is
 *    [M][n][n] with tau ascending from -beta (index 0) to 0 (index M-1), the
 *    paper's interval tau in [-beta, 0]. All floating point is IEEE double
 *    unless stated.
 *  - Memory: the context owns all its device workspace. Buffers passed in are
 *    caller-owned; the library never frees them. Pointers documented as
 *    "device" must be allocated on the context's device; "host" pointers are
 *    ordinary host memory.
 *  - Streams: all work of a context is enqueued on the stream given to
 *    fedvr_create. Calls that return scalars or write host buffers synchronise
 *    that stream before returning; stage-level calls that only write device
 *    buffers return without synchronising.
 *  - Order: build_fedvr -> set_potential -> solve_hf -> solve_2b. Calling out
 *    of order returns FEDVR_ERR_STATE. A context is not re-entrant; distinct
 *    contexts are independent.
 */
#ifndef FEDVR_NEGF_H
#define FEDVR_NEGF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fedvr_ctx fedvr_ctx;

typedef enum {
  FEDVR_OK = 0,
  FEDVR_ERR_ARG = -1,      /* invalid argument, nothing was launched */
  FEDVR_ERR_CUDA = -2,     /* a CUDA call failed; the context is now unusable */
  FEDVR_ERR_NOCONV = -3,   /* max_iter reached before the tolerance */
  FEDVR_ERR_DIVERGED = -4, /* residual grew for 8 consecutive iterations */
  FEDVR_ERR_TIMEOUT = -5,  /* a bounded device-side wait gave up; the kernel
                              returned with its work unfinished, so the
                              context is now unusable (later calls return
                              FEDVR_ERR_STATE) */
  FEDVR_ERR_NAN = -6,      /* a NaN or Inf reached the iterate */
  FEDVR_ERR_STATE = -7     /* call out of order, or context already failed */
} fedvr_status;

typedef enum {
  FEDVR_FP64 = 0,        /* every contraction in IEEE double */
  FEDVR_SPLIT_TF32 = 1,  /* Sigma^(2) (exchange and V Q V), I^(1) and, for
                            n_b >= 96, the I^(2) products on tensor cores:
                            hi+lo TF32 operands, FP32 accumulation, FP64
                            cross-block sums (I^(2) below n_b = 96 in FP32 on
                            the CUDA cores); tables, update, residual, N and
                            E0 in FP64. Requires n_b <= 304. */
  FEDVR_SPLIT_BF16 = 2,  /* reserved (three-way BF16 splits); rejected */
  FEDVR_SPLIT_F16 = 3    /* as FEDVR_SPLIT_TF32, with the exchange and the
                            I^(1) contractions on kind::f16 tensor cores
                            (V Q V and I^(2) stay split TF32):
                            operands scaled by powers of two into FP16's
                            normal range and split as hi + lo (22 significant
                            bits, as the TF32 split), twice the TF32 rate.
                            Requires |g| < 65504/4096 (just below 16; g's
                            eigenvalues lie in [0, 1]), checked on the
                            device: an entry beyond it (or not finite) makes
                            the call return FEDVR_ERR_ARG (a step whose
                            iterate is not finite returns FEDVR_ERR_NAN).
                            Requires n_b <= 304. */
} fedvr_precision;

/* ---------------------------------------------------------------------- */
/* Context                                                                 */
/* ---------------------------------------------------------------------- */

/* Create a context on the current CUDA device. cuda_stream is a cudaStream_t
 * (NULL = legacy default stream), e.g. torch.cuda.current_stream().cuda_stream.
 * *out receives the handle (NULL on failure). */
int fedvr_create(fedvr_ctx **out, void *cuda_stream);

/* Free the context and all its device workspace. NULL is allowed. */
void fedvr_destroy(fedvr_ctx *ctx);

/* Text of the last failure on ctx ("" if none). Owned by ctx; valid until the
 * next call on ctx. */
const char *fedvr_last_error(const fedvr_ctx *ctx);

/* ---------------------------------------------------------------------- */
/* Basis and operators (Sec. 2.1-2.2)                                      */
/* ---------------------------------------------------------------------- */

/* FE-DVR basis on [xmin, xmax] with n_elem finite elements of pts_per_elem
 * Gauss-Lobatto-Legendre points each (Sec. 2.1, Eqs. xim, wim, basis): the
 * element polynomials have order n_g = pts_per_elem - 1, the paper's n_g in
 * the root and weight formulas. grid_kind 0: equal elements (Sec. 3.1 case
 * I); 1: a central element of width 1 and widths growing linearly outward
 * (case II). The basis excludes both box ends, so
 * *n_b_out = n_elem*(pts_per_elem - 1) - 1 (Eq. basisdim; the paper's
 * n_e = 29, n_g = 7 run is pts_per_elem = 8, n_b = 202). Nodes, weights, the
 * index map and the kinetic matrix T (Eq. tmat) are built on the device
 * bit-identically to a plain IEEE evaluation in a fixed order (no fused
 * multiply-add).
 * Limits: 1 <= n_elem, 2 <= pts_per_elem <= 33, 2 <= n_b <= 1024,
 * xmin < xmax. Resets any potential/HF/2B state of the context. */
int build_fedvr(fedvr_ctx *ctx, int n_elem, int pts_per_elem, double xmin, double xmax,
                int grid_kind, int *n_b_out);

/* Nuclear potential and interaction (Sec. 2.2 Eqs. vmat, umat1; Sec. 3 model
 * potentials): v_a = sum_A -Z_A / sqrt((x_a - R_A)^2 + soft_en),
 * V_ab = 1/sqrt((x_a - x_b)^2 + soft_ee), h = T + diag(v). Z and R are host
 * arrays of n_nuc doubles. n_elec electrons, closed shell (n_elec even).
 * *E_nn_out (may be NULL) receives sum_{A<B} Z_A Z_B / |R_A - R_B|, which is
 * NOT part of any E0 this library returns. */
int set_potential(fedvr_ctx *ctx, int n_nuc, const double *Z, const double *R,
                  double soft_en, double soft_ee, int n_elec, double *E_nn_out);

/* Copy the basis to host buffers of n_b entries each (any may be NULL):
 * node coordinates, quadrature weights W_a (bridge = sum of two element
 * weights), element index and local point index of each basis function (a
 * bridge reports the left element and local index pts_per_elem - 1). */
int fedvr_get_basis(const fedvr_ctx *ctx, double *nodes, double *weights, int *elem,
                    int *local);

/* Copy the GLL reference points and weights (pts_per_elem each) to host. */
int fedvr_get_gll(const fedvr_ctx *ctx, double *xi, double *omega);

/* Copy operators to host [n_b][n_b] buffers (v: [n_b]); any may be NULL.
 * Requires set_potential for v, V, h. */
int fedvr_get_operators(const fedvr_ctx *ctx, double *T, double *v, double *V, double *h);

/* ---------------------------------------------------------------------- */
/* Hartree-Fock (Sec. 2.3, Eqs. sigmahf, hamhf, hfgf)                      */
/* ---------------------------------------------------------------------- */

/* Self-consistent HF at inverse temperature beta: F = h + Sigma^HF[rho],
 * Sigma^HF = sigma diag(V diag rho) - V o rho (sigma = 2), diagonalisation on
 * the GPU (Jacobi), chemical potential from the Fermi normalisation
 * sum_a f(eps_a - mu) = n_elec/2 solved in its balanced holes = particles form,
 * rho' = C diag f C^T, linear mixing 0.5, stop when max|rho' - rho| < tol.
 * Outputs (host, may be NULL): E_hf = 2 Tr[h rho] + Tr[Sigma^HF rho] (no E_nn)
 * and mu. Returns FEDVR_ERR_NOCONV after max_iter steps. */
int solve_hf(fedvr_ctx *ctx, double beta, double tol, int max_iter, double *E_hf, double *mu);

/* Chemical potential of the second-Born run (Sec. 2.3: mu enters g^0 through
 * the Fermi factors of Eq. hfgf; the paper fixes it by the HF normalisation
 * and keeps it during the iteration). Replaces the HF value for the next
 * fedvr_2b_prepare / solve_2b until the next solve_hf; drops a prepared run.
 * Lets a caller re-fix mu between solves (e.g. so that N = n_elec) or show
 * that N does not depend on mu inside the gap. Errors: FEDVR_ERR_STATE before
 * solve_hf, FEDVR_ERR_ARG for a non-finite mu. */
int fedvr_set_mu(fedvr_ctx *ctx, double mu);

/* Copy the HF solution to host (any may be NULL): eps [n_b] ascending, C
 * [n_b][n_b] (column a = orbital a), rho0 = g^0(0^-) [n_b][n_b] and
 * Sigma0 = F - h [n_b][n_b]. */
int fedvr_get_hf(const fedvr_ctx *ctx, double *eps, double *C, double *rho0, double *Sigma0);

/* Sources of fedvr_density. */
typedef enum {
  FEDVR_DENSITY_HF = 0, /* rho0 of the last solve_hf */
  FEDVR_DENSITY_2B = 1  /* g(0^-) of the current second-Born iterate (after
                           solve_2b: its final g; after fedvr_2b_prepare
                           alone: g^0, the HF density) */
} fedvr_density_source;

/* One-electron density at the basis nodes (Sec. 2.3: n(x) sums the products
 * chi chi of basis functions weighted by g(0^-)). A DVR function is
 * 1/sqrt(W_a) at its own node and zero at every other node, so
 * n_out[a] = spin * g_aa(0^-) / W_a, with g the Green's function of one spin
 * (the density integrates to N: sum_a W_a n_out[a] = spin Tr g(0^-)).
 * n_out: host buffer of n_b doubles. Computed on the device from the context's
 * own g and weights; synchronises the context's stream.
 * Errors: FEDVR_ERR_ARG (n_out NULL or unknown source), FEDVR_ERR_STATE (no HF
 * solution, resp. no prepared second-Born run). */
int fedvr_density(const fedvr_ctx *ctx, int source, double *n_out);

/* ---------------------------------------------------------------------- */
/* Second Born (Sec. 2.3 Eqs. sigma2ndb, deq; Sec. 3.1 mesh)               */
/* ---------------------------------------------------------------------- */

/* Second-Born Matsubara self-consistency on the uniform power mesh with
 * M = 2up+1 points. Iteration k: Sigma_k = Sigma^corr[g_k] (Eq. sigma2ndb),
 * I1 = (Sigma^HF[g_k(0^-)] - Sigma^0) g_k + Sigma_k * g_k,
 * I2 = g^0 * I1 (Eq. deq), g_new = sym(g^0 + I2),
 * g_{k+1} = (1 - mixing) g_k + mixing g_new, r_k = max|g_{k+1} - g_k|; stop at
 * r_k < tol. E0_k (Galitskii-Migdal, no E_nn) and N_k = 2 Tr g_k(0^-) are
 * evaluated on (g_k, Sigma_k). precision: fedvr_precision.
 * Outputs: G_out = g_{k+1}, Sigma_out = Sigma_k (each [M][n_b][n_b]), tau_out
 * [M]; any may be NULL; device pointers if out_on_device else host.
 * Scalars (host, may be NULL): E0, N_out, iters. Limits: u, p >= 1,
 * M <= 4097, 0 < mixing <= 1. */
int solve_2b(fedvr_ctx *ctx, double beta, int u, int p, double mixing, double tol,
             int max_iter, int precision, int out_on_device, double *G_out,
             double *Sigma_out, double *tau_out, double *E0, double *N_out, int *iters);

/* Split form of solve_2b for callers that drive the iteration themselves.
 * fedvr_2b_prepare builds the mesh, g^0 on the mesh and the convolution
 * tables for (beta, u, p, precision) and sets g_0 = g^0 (or keeps a warm-start
 * Sigma for the first step). fedvr_2b_step runs exactly one iteration of the
 * solve_2b scheme; if G_in is non-NULL the iterate g_k is first replaced by
 * G_in ([M][n_b][n_b], device if in_on_device else host). Host scalars (may be
 * NULL): res = max|g_{k+1} - g_k|, E0 and N evaluated on (g_k, Sigma_k).
 * fedvr_2b_read copies the current iterate g and the last Sigma out (any may
 * be NULL; device pointers if out_on_device). */
int fedvr_2b_prepare(fedvr_ctx *ctx, double beta, int u, int p, int precision);
int fedvr_2b_step(fedvr_ctx *ctx, double mixing, const double *G_in, int in_on_device,
                  double *res, double *E0, double *N_out);
int fedvr_2b_read(fedvr_ctx *ctx, int out_on_device, double *G_out, double *Sigma_out,
                  double *tau_out);

/* Device durations (milliseconds, CUDA events on the context's stream) of the
 * stages of the last fedvr_2b_step: [0] Sigma^(2) build, [1] HF self-energy
 * change and energy, [2] first convolution I1, [3] second convolution I2,
 * [4] update and residual, [5] whole step. *launches (may be NULL) receives the
 * number of kernels that step launched. ms is a host array of 6 doubles. */
int fedvr_stage_times(const fedvr_ctx *ctx, double *ms, int *launches);

/* Graph replay of the iteration (the driver loop of Sec. 2.3 with its launch
 * overhead removed; the paper has no counterpart). With graphs enabled (the
 * default) the first regular fedvr_2b_step after fedvr_2b_prepare captures
 * its kernels into a CUDA graph and later steps replay it; warm-start inner
 * steps and a change of mixing are handled by re-capture or eager launch.
 * Results are identical either way. enable: 1 on, 0 off, < 0 leave as is.
 * *last_step_graph (may be NULL) receives 1 if the last step ran as a graph
 * replay. If the driver refuses a capture, the context keeps running eagerly
 * and reports 0 there; this is not an error. */
int fedvr_use_graphs(fedvr_ctx *ctx, int enable, int *last_step_graph);

/* Work split of the split-precision first convolution (Eq. deq; the paper
 * has no counterpart): each 128-row tile of the stacked rows (i, a) may be cut
 * into S ranges of mesh points j, computed by different CTAs into separate
 * partial stacks and summed in a fixed order. Each range is a whole number of
 * the fixed FP32 accumulation blocks (whose length depends on n_b and M
 * only), so S changes only the order of the FP64 additions of the block sums.
 * Candidates: {1, 2, 3, 4, 6, 8, 12, 16}, at most the number of blocks.
 * request = 0 (default): fedvr_2b_prepare times the candidates once per
 * (device, n_b, M, precision) in the process and keeps the fastest; request > 0: use the
 * largest candidate <= request (1 = no split; also read by
 * fedvr_conv_sigma_g); request < 0: leave the setting. *in_use (may be NULL)
 * receives S of the currently prepared run (or of the last stage-level
 * convolution). Takes effect at the next prepare. */
int fedvr_conv1_splits(fedvr_ctx *ctx, int request, int *in_use);

/* Quadrature of the two Dyson integrals (Eq. deq; the paper's "direct
 * integration" names no rule). order 2 (default): the split trapezoid with
 * Sigma^corr linearly interpolated at off-mesh lags, second order in the mesh
 * spacing. order 4: each side of the split at tau_i integrated with the
 * exactly integrated cubic of each interval (through the interval's four
 * nearest mesh points of that side), Sigma^corr interpolated by the cubic
 * through four mesh points, and the energy's tau integral with the same
 * rule; fourth order. Order 4 runs on the FP64 path only (a split precision
 * returns FEDVR_ERR_ARG) and needs M >= 4. Applies to the next
 * fedvr_2b_prepare / solve_2b and to the stage-level fedvr_conv_sigma_g and
 * fedvr_conv_g0; drops a prepared run. Errors: FEDVR_ERR_ARG for another
 * order. */
int fedvr_set_quadrature(fedvr_ctx *ctx, int order);

/* Correlation self-energy of the next fedvr_2b_prepare / solve_2b:
 * kind 0 = second Born (Sec. 2.3, Eq. sigma2ndb; default), kind 1 = GW, the
 * approximation Sec. 4 names as the next one the FE-DVR form simplifies. In
 * this basis the interaction is two-index, so the bubble is too: with
 * Q_j = g_j o g_{M-1-j} the correlated screened interaction solves
 *   w = V Q V - sigma V (Q * w)   (Q * w the periodic tau-convolution on the
 *                                  mesh, trapezoid with Q interpolated at the lag),
 * and Sigma^GW = sigma g o w (its lowest order w = V Q V is the direct term of
 * Eq. sigma2ndb; GW has no second-order exchange). Each outer iteration solves
 * for w by the damped fixed-point iteration w <- (1 - w_mixing) w +
 * w_mixing (V Q V - sigma V (Q * w)) until max|w_new - w| < w_tol, starting
 * from the previous outer iteration's w (V Q V at the first). GW runs on the
 * FP64 path with the trapezoid rule (other precisions or quadratures:
 * FEDVR_ERR_ARG at prepare) and eagerly (one host readback per inner
 * iteration, no graph replay). An inner iteration that has not converged in
 * w_max_iter steps ends the step with FEDVR_ERR_NOCONV. Drops a prepared run.
 * kind 2 = T-matrix, the other approximation Sec. 4 names: the
 * particle-particle ladder of the two-index interaction. A pair of particles
 * at the nodes (a, k) scatters through V_ak without changing nodes, so with
 * the pair propagator K(tau) = g(tau) (x) g(tau) and V^ the diagonal pair-space
 * matrix of the V_ak the correlated ladder solves
 *   t = V^ K V^ - V^ (K * t)      (K * t periodic, as Q * w above),
 * and Sigma^T_ab(tau_j) = sum_kl [sigma t_j(ak; bl) - t_j(ak; lb)] g_{M-1-j}(l, k)
 * (its lowest order is Eq. sigma2ndb, direct and exchange terms). Pair space
 * holds n_b^2 x n_b^2 values per mesh point, so kind 2 needs n_b <= 32
 * (FEDVR_ERR_ARG at prepare otherwise) and three such stacks of device
 * memory; the inner iteration, its parameters, warm start and errors are as
 * for GW. Errors: FEDVR_ERR_ARG for a kind outside 0..2 or for w_mixing
 * outside (0, 1], w_tol <= 0 or w_max_iter < 1 (kinds 1 and 2). */
int fedvr_set_self_energy(fedvr_ctx *ctx, int kind, double w_mixing, double w_tol,
                          int w_max_iter);

/* Inner iterations of the last GW screened-interaction or T-matrix ladder
 * solve of the context. */
int fedvr_gw_last_inner(const fedvr_ctx *ctx, int *iters);

/* Stage-level GW on caller device buffers (the context's stream): Sigma^GW
 * [M][n][n] of G [M][n][n] on the power mesh (beta, u, p), V [n][n], spin
 * factor spin. w_io (device [M][n][n] or NULL): with w_valid != 0 the inner
 * iteration starts from it (else from V Q V); the converged w is written back
 * when given. iters (host, may be NULL): inner iterations. Synchronises the
 * stream. Errors: FEDVR_ERR_ARG for invalid sizes, mesh or iteration
 * parameters; FEDVR_ERR_NOCONV if w does not converge in w_max_iter steps;
 * FEDVR_ERR_NAN if it diverges. */
int fedvr_sigma_gw(fedvr_ctx *ctx, int n, double beta, int u, int p, double spin, const double *V,
                   const double *G, double *Sigma, double *w_io, int w_valid, double w_mixing,
                   double w_tol, int w_max_iter, int *iters);

/* Stage-level T-matrix self-energy on caller device buffers (the context's
 * stream): Sigma^T [M][n][n] of G [M][n][n] on the power mesh (beta, u, p),
 * V [n][n], spin factor spin, 1 <= n <= 32 (see fedvr_set_self_energy, kind
 * 2). t_io (device, M n^4 doubles, or NULL) is the ladder in the layout
 * t[j][b][l][a][k] = t_j(ak; bl): with t_valid != 0 the iteration starts from
 * it (else from V^ K V^); the converged ladder is written back when given.
 * iters (host, may be NULL): inner iterations. Synchronises the stream.
 * Errors: FEDVR_ERR_ARG for invalid sizes, mesh or iteration parameters;
 * FEDVR_ERR_NOCONV if the ladder does not converge in t_max_iter steps;
 * FEDVR_ERR_NAN if it diverges. */
int fedvr_sigma_tmatrix(fedvr_ctx *ctx, int n, double beta, int u, int p, double spin,
                        const double *V, const double *G, double *Sigma, double *t_io,
                        int t_valid, double t_mixing, double t_tol, int t_max_iter, int *iters);

/* Start the next solve_2b from this Sigma^corr (warm start). Sigma0 is
 * [M][n_b][n_b] on host or device; M must match the next solve's mesh; copied
 * at once; NULL clears. inner_steps = 0: the first iteration uses Sigma0
 * instead of Sigma^corr[g^0]. inner_steps > 0: the first inner_steps
 * iterations keep Sigma0 fixed and take the full Dyson step (no mixing), so g
 * moves to the Green's function of Sigma0 before the regular iteration
 * starts; no convergence test is made during them. */
int fedvr_set_initial_sigma(fedvr_ctx *ctx, const double *Sigma0, int M, int on_device,
                            int inner_steps);

/* Per-iteration record of the last solve_2b: 5 doubles per iteration
 * (iteration, residual, E0, N, wall milliseconds). Copies min(cap, count)
 * records to buf (host, 5*cap doubles); *len = number of records. */
int fedvr_get_history(const fedvr_ctx *ctx, double *buf, int cap, int *len);

/* Batched solve over n_sys independent prepared contexts (each has run
 * build_fedvr, set_potential and solve_hf at its beta). Arrays have n_sys
 * entries; the per-system results E0, N_out (host doubles) and iters (host
 * ints) may be NULL. All systems advance together on the stream of ctxs[0]:
 * per iteration one tensor-core launch per contraction kernel covers every
 * unconverged system of the batch (a work queue over all systems' tiles), and
 * each system stops updating when its residual is below tol. A system with a
 * warm start set (fedvr_set_initial_sigma, fedvr_warm_start) takes it as in
 * solve_2b: its warm-start steps run inside the batched iterations (no
 * exchange work for them; the fixed-Sigma inner steps use mixing 1 and no
 * convergence test), and the warm start is cleared afterwards. The first
 * convolution's split count is measured once per batch (fedvr_batch_create;
 * results do not depend on it beyond the order of FP64 additions). Requires a
 * split precision (FEDVR_SPLIT_TF32 or FEDVR_SPLIT_F16; FEDVR_FP64 returns
 * FEDVR_ERR_ARG) and distinct contexts on one device. Returns the
 * worst per-system status; each context keeps its history and its last
 * g and Sigma (fedvr_2b_read). */
int solve_2b_batched(fedvr_ctx **ctxs, int n_sys, const double *beta, const int *u,
                     const int *p, double mixing, double tol, int max_iter, int precision,
                     double *E0, double *N_out, int *iters);

/* The batch behind solve_2b_batched, for callers that drive the iteration:
 * fedvr_batch_create prepares every context (fedvr_2b_prepare) and the device
 * work tables; fedvr_batch_step runs one iteration of every active system
 * (active[k] != 0, host int array, updated in place: a system whose residual
 * falls below tol > 0 becomes inactive) and writes per-system res, E0, N (host
 * arrays, may be NULL). The contexts must outlive the batch. */
typedef struct fedvr_batch fedvr_batch;
int fedvr_batch_create(fedvr_batch **out, fedvr_ctx **ctxs, int n_sys, const double *beta,
                       const int *u, const int *p, int precision);
int fedvr_batch_step(fedvr_batch *b, double mixing, double tol, int *active, double *res,
                     double *E0, double *N_out);
void fedvr_batch_destroy(fedvr_batch *b);

/* ---------------------------------------------------------------------- */
/* Learned warm start (no counterpart in the paper)                        */
/* ---------------------------------------------------------------------- */

/* A per-(a, b)-pair network that predicts the converged self-energy of a new
 * system from its one-shot Sigma^(2)[g^0]: input [S1_ab(tau)/s (M values),
 * g^0_ab(tau) (M), V_ab, x_a/L, x_b/L] (s = max|S1|, L = box length), hidden
 * ReLU layers of `hidden` units, output Delta_ab(tau)/s (M) with
 * Sigma_pred = S1 + s * Delta. FP32 master weights (He-normal initialisation
 * from `seed`), Adam training, BF16 inference; all on the GPU. M is fixed
 * per network (the mesh size it serves); n_b may differ between systems. */
typedef struct fedvr_mlp fedvr_mlp;
int fedvr_mlp_create(fedvr_mlp **out, int M, int hidden, unsigned long long seed,
                     void *cuda_stream);
void fedvr_mlp_destroy(fedvr_mlp *m);
const char *fedvr_mlp_last_error(const fedvr_mlp *m);
/* Parameter vector: W1 [2M+3][hidden], b1, W2 [hidden][hidden], b2,
 * W3 [hidden][M], b3, row-major, FP32, host buffers of *count floats. */
int fedvr_mlp_num_params(const fedvr_mlp *m, long *count);
int fedvr_mlp_get_params(fedvr_mlp *m, float *params, long count);
int fedvr_mlp_set_params(fedvr_mlp *m, const float *params, long count);
/* Loss sum (y-t)^2 / (2 rows M) and its gradient (host, num_params floats) for
 * device rows X [rows][2M+3], T [rows][M], FP32 weights. */
int fedvr_mlp_loss_grad(fedvr_mlp *m, const float *X, const float *T, int rows, float *grad,
                        double *loss);
/* y = net(X) for device rows; bf16 != 0 uses the BF16 weights (as updated by
 * the last fedvr_mlp_train or fedvr_mlp_set_params). */
int fedvr_mlp_forward(fedvr_mlp *m, const float *X, int rows, float *Y, int bf16);
/* Run a plain split-TF32 solve_2b on ctx (HF solved, mesh with M points) and
 * add the system's pairs (features, scaled converged correction) to the
 * training set if it converged. *iters (may be NULL) = iterations used. */
int fedvr_mlp_collect(fedvr_mlp *m, fedvr_ctx *ctx, double beta, int u, int p, double mixing,
                      double tol, int max_iter, int *iters);
/* Adam over the training set: `epochs` shuffled passes of `batch` rows at
 * learning rate lr; *final_loss (may be NULL) = mean loss of the last pass;
 * refreshes the BF16 weights. Training rows: fedvr_mlp_rows. */
int fedvr_mlp_train(fedvr_mlp *m, int epochs, int batch, double lr, double *final_loss);
int fedvr_mlp_rows(const fedvr_mlp *m, long *rows);
/* Copy `count` collected training rows starting at `start` to host buffers
 * X [count][2M+3] and T [count][M] (either may be NULL). */
int fedvr_mlp_get_rows(fedvr_mlp *m, long start, long count, float *X, float *T);
/* Predict Sigma for ctx's next solve_2b at (beta, u, p) with the BF16 weights
 * and set it with fedvr_set_initial_sigma(..., inner_steps). */
int fedvr_warm_start(fedvr_ctx *ctx, fedvr_mlp *m, double beta, int u, int p, int inner_steps);

/* ---------------------------------------------------------------------- */
/* Stage-level calls on caller device buffers (the hot-path kernels)       */
/* ---------------------------------------------------------------------- */

/* Uniform power mesh (Sec. 3.1): B_p = beta/2, B_{k-1} = B_k/2, B_0 = 0,
 * segment k cut in u parts, tau_j = -beta + s_j (j <= up), tau_{M-1-m} = -s_m.
 * Trapezoid weights w, left/right half weights wm, wp. Device outputs of M
 * doubles each (any may be NULL); lag_k [M][M] int32 and lag_t [M][M] double
 * (may be NULL): for i != j the bracket k and weight t of the lag
 * tau_i - tau_j mapped to [-beta, 0] (anti-periodic extension); diagonal
 * k = -1, t = 0. Bit-identical to a plain IEEE evaluation. */
int fedvr_power_mesh(fedvr_ctx *ctx, double beta, int u, int p, double *tau, double *w,
                     double *wm, double *wp, int *lag_k, double *lag_t);

/* Second-Born self-energy for a whole tau-stack (Sec. 2.3, Eq. sigma2ndb in
 * two-index form): Sigma_j = spin * g_j o (V (g_j o gb_j) V) - X_j with
 * gb_j = G[M-1-j] and X_j,ab = sum_kl V_ak V_bl g_j,al gb_j,lk g_j,kb.
 * V [n][n] and G [M][n][n] are device inputs; each G_j and V must be symmetric
 * (the lower triangle is used). Sigma [M][n][n] is a device output.
 * spin >= 0 (FEDVR_ERR_ARG otherwise). precision: fedvr_precision. Uses
 * context workspace. */
int fedvr_sigma2(fedvr_ctx *ctx, int n, int M, double spin, const double *V,
                 const double *G, double *Sigma, int precision);

/* Allocation-free Sigma^(2) build. The paper has no counterpart: this is a
 * service for callers that cannot let the library allocate device memory --
 * processes whose device memory belongs to another allocator (a framework's
 * caching allocator that reserves the pool), or loops that cannot accept the
 * device synchronisation cudaMalloc/cudaFree imply. It computes exactly what
 * fedvr_sigma2 computes with precision FEDVR_FP64 (same kernels), needs no
 * context, and calls no cudaMalloc, cudaFree or allocating library routine:
 * its workspace is a fixed 12 MiB device array inside the library, which every
 * GPU that loads the library holds until the process exits.
 *  - Limit: M * n * n <= 524288 (2^19), 1 <= n <= 1024, 1 <= M <= 4097;
 *    larger sizes return FEDVR_ERR_ARG.
 *  - V [n][n], G [M][n][n] (symmetric) and Sigma [M][n][n] are caller-owned
 *    device buffers on the current device; work is enqueued on cuda_stream
 *    (a cudaStream_t, NULL = legacy default stream) without synchronising.
 *  - The first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress, with that device current); make that first
 *    call before any stream capture.
 *  - Every call shares the one array and leaves its contents behind; nothing in
 *    it needs to start at zero (every workspace element is written before it
 *    is read). Calls that overlap on the GPU (concurrent streams or threads)
 *    race on the array and give wrong results; serialise them.
 *  - Errors: FEDVR_ERR_ARG for invalid arguments or sizes beyond the limit,
 *    FEDVR_ERR_CUDA if the address lookup or a launch fails. */
int fedvr_sigma2_noalloc(int n, int M, double spin, const double *V, const double *G,
                         double *Sigma, void *cuda_stream);

/* First Dyson convolution (Eq. deq): I1_i = dHF g_i + int Sigma(tau_i - t) g(t) dt
 * on the power mesh (beta, u, p), split trapezoid at t = tau_i with
 * Sigma(0^+) = -Sigma_0, Sigma(0^-) = Sigma_{M-1}; Sigma at off-mesh lags by
 * linear interpolation, anti-periodic beyond 0. dHF [n][n], Sigma and G
 * [M][n][n] device inputs; I1 [M][n][n] device output. In the split
 * precisions the FP32 accumulation blocks are fixed ranges of mesh points
 * (their length depends on n and M only) and the call cuts the mesh-point
 * range into the split count requested with fedvr_conv1_splits (largest
 * candidate in {1, 2, 3, 4, 6, 8, 12, 16} not above it and not above the
 * number of blocks; no request: 1); results of different split counts
 * differ only in the order of the FP64 additions of the block sums. */
int fedvr_conv_sigma_g(fedvr_ctx *ctx, int n, double beta, int u, int p, const double *dHF,
                       const double *Sigma, const double *G, double *I1, int precision);

/* Second Dyson convolution (Eq. deq): I2_i = int g^0(tau_i - t) I1(t) dt with
 * g^0(x) = C diag(phi(x)) C^T evaluated exactly at every lag (Eq. hfgf), same
 * split trapezoid (g^0(0^+) = -g^0(-beta)); computed as
 * I2_i = C sum_j diag(w_ij phi(tau_i - tau_j)) C^T I1_j, i.e. with the left
 * index in the HF eigenbasis (three products).
 * eps [n] (ascending not required), C [n][n], I1 [M][n][n] device inputs;
 * I2 [M][n][n] device output. precision FEDVR_FP64: all three products in
 * FP64; a split precision: the kernel table K(i, j) rounded to FP32 and the
 * products of the split iteration (split TF32 on tensor cores for n >= 96,
 * FP32 on the CUDA cores below), FP64 I1 in and I2 out. */
int fedvr_conv_g0(fedvr_ctx *ctx, int n, double beta, int u, int p, const double *eps,
                  const double *C, double mu, const double *I1, double *I2, int precision);

/* Self-test of the bounded device-side waits that every tensor-core kernel
 * uses (no counterpart in the paper): one warp waits on a shared-memory
 * mbarrier with the kernels' own wait helper, limited to limit_seconds
 * (1e-6 to 1) of wall time. release != 0: the barrier is released before
 * the wait, which succeeds (FEDVR_OK). release = 0: nothing releases it; the
 * wait gives up at the limit, the kernel records the timeout in a device flag
 * and returns, and the call returns FEDVR_ERR_TIMEOUT and leaves the context
 * failed, as every timeout does (later calls: FEDVR_ERR_STATE). Nothing
 * faults or hangs. Synchronises the context's stream. */
int fedvr_selftest_wait(fedvr_ctx *ctx, int release, double limit_seconds);

/* Real-time two-time Kadanoff-Baym propagation (Sec. 2, Eqs. kbe, skkbe and
 * skkbesigma; the self-energy is the time-local HF part of Eq. sigmahf plus,
 * with second_born != 0, the second-Born part of Eq. sigma2ndb on the Keldysh
 * components; second_born = 0 gives time-dependent HF). The paper states the
 * equations and runs only their equilibrium (Matsubara) problem; this entry
 * starts from an uncorrelated state rho0 at t = 0, so the collision integrals
 * run over [0, t] only.
 *
 * Functions: L(t, t') = -i G^<(t, t') (L(t, t) = rho(t), the density matrix
 * per spin) and Gt = -i G^> (Gt(t, t) = rho(t) - 1) on the grid t_k = k dt,
 * k = 0 .. n_steps, advanced by Heun's predictor-corrector with trapezoid
 * collision integrals (second order in dt), in complex FP64 on the device.
 * Heun's step is explicit: a mode of energy e grows by
 * sqrt(1 + (e dt)^4 / 4) per step, so dt must stay well below 1 / max|e| of
 * h_HF (max|e| grows with the grid's highest kinetic energy, about 27 Ha at
 * n_b = 74 on [-20, 20]); an unstable choice ends in Inf/NaN outputs, not an
 * error code.
 * The Hamiltonian is the context's h (after set_potential) plus
 * diag(dv(t_k)) (a time-dependent potential at the nodes, e.g. x_a E(t_k)).
 *
 * precision: FEDVR_FP64 (everything in complex FP64), or FEDVR_SPLIT_TF32
 * (second Born only): the two collision integrals of each time row run as
 * split-TF32 tensor-core products (three TF32 products per product, FP32
 * accumulation, about 2^-21 relative per product) over FP32 copies of L, Gt
 * and the weighted L - Gt kept beside the FP64 matrices (3 x 8 (T n_b)^2
 * more bytes; needs T n_b <= 32750); for n_b <= 64 the second-Born
 * self-energy's exchange products run the same way and its direct term and
 * exchange k-sum in FP32; the -i h_HF F term, the energy, the HF self-energy
 * and the stepping stay FP64.
 *
 * rho0: host [n_b][n_b] complex (interleaved re, im; 16 bytes per entry), or
 * NULL for the real HF density rho0 of the last solve_hf. dv: host
 * [n_steps+1][n_b] or NULL. Outputs (host, any may be NULL): rho_out
 * [n_steps+1][n_b][n_b] complex interleaved; E_out [n_steps+1], the total
 * energy sigma Tr[h(t) rho] + sigma/2 Tr[Sigma^HF rho] + sigma/2 Re Tr[i K_L(t, t)]
 * (one-body, HF and correlation parts; E_nn excluded; constant without dv);
 * N_out [n_steps+1] = sigma Tr rho.
 *
 * Device memory: the two-time L and Gt are held whole, 2 (T n_b)^2 x 16 bytes
 * with T = n_steps + 1 (about 1.2 GB at n_b = 15, T = 401), kept after the
 * call for fedvr_kbe_get_block until the next call or fedvr_destroy.
 * Errors: FEDVR_ERR_STATE before set_potential (or before solve_hf with
 * rho0 = NULL); FEDVR_ERR_ARG for dt <= 0, n_steps outside [0, 32766],
 * n_b > 80, another precision or storage beyond the free device memory;
 * FEDVR_ERR_TIMEOUT if a tensor-core wait gave up (the context is then
 * failed). Synchronises the stream. */
int fedvr_kbe_propagate(fedvr_ctx *ctx, double dt, int n_steps, int second_born, int precision,
                        const double *rho0, const double *dv, double *rho_out, double *E_out,
                        double *N_out);

/* Copy block (i, j) (time indices of the last fedvr_kbe_propagate) of
 * which = 0: L = -i G^<, 1: Gt = -i G^> to host out [n_b][n_b] complex
 * interleaved. Errors: FEDVR_ERR_STATE without a completed propagation,
 * FEDVR_ERR_ARG for indices outside it. */
int fedvr_kbe_get_block(const fedvr_ctx *ctx, int which, int i, int j, double *out);

/* Timing of the last fedvr_kbe_propagate (CUDA events on the context's
 * stream), out[8]: out[0] total ms, out[1] ms in the collision-integral
 * kernels, out[2] ms in the self-energy kernels, out[3] their algorithmic
 * flops (8 per complex multiply-add of the collision integrals), out[4] the
 * self-energy's, out[5] kernel launches, out[6] ms in the split-TF32
 * collision products alone (0 in FP64 mode), out[7] the shadow bytes those
 * products read once (L and Gt over the row's contraction, the triangle of
 * the weighted L - Gt). */
int fedvr_kbe_stats(const fedvr_ctx *ctx, double *out);

#ifdef __cplusplus
}
#endif

#endif /* FEDVR_NEGF_H */
