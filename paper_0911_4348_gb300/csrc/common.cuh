// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/fedvr_negf.h"

namespace fedvr {

// Device buffer that only grows; freed with the context.
struct DevBuf {
  void *ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace fedvr

struct fedvr_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  char err[640] = {0};
  bool failed = false;  // sticky after a CUDA error or a timed-out device wait
  int stage = 0;        // 0 none, 1 basis, 2 potential, 3 hf

  // basis (Sec. 2.1)
  int n_elem = 0, order = 0, n = 0, grid_kind = 0;
  double xmin = 0, xmax = 0;
  // potential (Sec. 2.2)
  int n_elec = 0, nocc = 0;
  double soft_en = 1.0, soft_ee = 1.0, spin = 2.0;
  // HF (Sec. 2.3)
  double beta_hf = 0, mu = 0, E_hf = 0;
  int hf_iters = 0;
  // warm start
  int sigma_init_M = 0;
  int warm_inner = 0;
  // prepared second-Born run
  bool prepared = false;
  int u = 0, p = 0, M = 0, precision = 0, step_k = 0;
  double beta = 0;
  // stage timing of the last step
  cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int step_launches = 0;
  int num_sms = 0;
  // CUDA graph of one regular iteration: captured on a private stream at the
  // first step after prepare, replayed on `stream`; dropped when the mixing
  // changes or a workspace buffer moves.
  bool use_graphs = true;
  bool last_step_graph = false;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_graph = nullptr;
  double graph_mixing = 0;
  int graph_launches = 0;
  // splits of the first convolution's mesh-point range (split-TF32 path):
  // requested (0 = measured choice) and in use by the prepared run
  int c1_request = 0;
  int c1_splits = 1;
  // incremented by every fedvr_2b_prepare (batches check it before each step)
  unsigned long long prep_gen = 0;
  // n of the exchange tile table held in w_xrow (0: none)
  int xrow_n = 0;
  // quadrature of the Dyson integrals: 2 = split trapezoid with linear lag
  // interpolation (default), 4 = the fourth-order variant (FP64 path)
  int quad_order = 2;
  // correlation self-energy: 0 second Born, 1 GW, 2 T-matrix (FP64 path); the
  // damped inner iteration (screened interaction or ladder) and its state
  // across outer steps
  int self_energy = 0;
  double gw_mixing = 0.3, gw_tol = 1e-12;
  int gw_max_iter = 500, gw_last_inner = 0;
  bool gw_w_valid = false;
  // history of the last solve_2b: iter, res, E0, N, ms
  std::vector<double> history;
  // last real-time propagation: time points and n (0: none), stage times and
  // algorithmic work (total ms, collision ms, self-energy ms, collision
  // flops, self-energy flops, launches, ms and shadow bytes of the split
  // collision products), events reused across calls
  int kbe_T = 0, kbe_n = 0;
  double kbe_stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::vector<cudaEvent_t> kbe_events;

  // named device buffers
  fedvr::DevBuf b_xi, b_om, b_edges, b_nodes, b_weights, b_elem, b_local, b_tt;
  fedvr::DevBuf b_T, b_v, b_V, b_h;
  fedvr::DevBuf b_eps, b_C, b_rho, b_rho_new, b_rho_mix, b_F, b_Sigma0, b_f, b_A, b_A2,
      b_J, b_scal, b_hf_tmp;
  fedvr::DevBuf b_sigma_init;
  // solve_2b / stage workspace
  fedvr::DevBuf w_tau, w_w, w_wm, w_wp, w_coef, w_K, w_phi, w_G0, w_G, w_S, w_I1, w_I2,
      w_t1, w_t2, w_t3, w_dHF, w_part, w_red, w_tc, w_K32, w_tab, w_btab, w_c1p, w_coef32, w_h16,
      w_xrow, w_dens, w_q4coef, w_q4W, w_q4w;
  // real-time propagation: two-time L and Gt, self-energy row, scratch, outputs
  fedvr::DevBuf k_L, k_G, k_S, k_T1, k_R, k_aux, k_out, k_part, k_sh, k_aop, k_o, k_flag, k_x;
  // GW: screened interaction w, V Q V, convolution and update scratch, periodic table, flag
  fedvr::DevBuf g_w, g_vqv, g_c, g_new, g_coef, g_res;
  // T-matrix: the ladder t, its source V^ K V^ and the convolution (pair-space stacks)
  fedvr::DevBuf m_t, m_src, m_y;
  // partial stacks of the FP64 first convolution's mesh-range splits (small launches)
  fedvr::DevBuf w_c1f;
};

namespace fedvr {

int fail(fedvr_ctx *ctx, int code, const char *fmt, ...);
// Sigma^corr[g] of the current iterate of a prepared context into its Sigma
// workspace (split-TF32 or FP64 per the prepared precision); synchronous.
int sigma_of_current_g(fedvr_ctx *ctx);
int cuda_fail(fedvr_ctx *ctx, cudaError_t e, const char *what, const char *file, int line);
// Ensure buf holds at least `bytes`; returns false (and records the error) on failure.
bool ensure(fedvr_ctx *ctx, DevBuf &buf, size_t bytes, const char *name);
void release(DevBuf &buf);
// Destroy the context's captured iteration graph (if any).
void drop_graph(fedvr_ctx *ctx);

template <typename T>
inline T *P(DevBuf &b) { return reinterpret_cast<T *>(b.ptr); }
template <typename T>
inline const T *CP(const DevBuf &b) { return reinterpret_cast<const T *>(b.ptr); }

// ---- kernels launched across translation units (all enqueue on `s`) ----

// basis.cu (bit-exact IEEE setup; compiled without FMA contraction)
cudaError_t launch_gll(int order, double *xi, double *om, int *status, cudaStream_t s);
cudaError_t launch_basis(int n_elem, int order, double xmin, double xmax, int grid_kind,
                         const double *xi, const double *om, double *edges, double *nodes,
                         double *weights, int *elem, int *local, double *tt, double *T,
                         int *status, cudaStream_t s);
cudaError_t launch_potential(int n, const double *nodes, int n_nuc, const double *Z,
                             const double *R, double soft_en, double soft_ee, const double *T,
                             double *v, double *V, double *h, cudaStream_t s);
cudaError_t launch_mesh(double beta, int u, int p, double *tau, double *w, double *wm,
                        double *wp, int *lag_k, double *lag_t, cudaStream_t s);
// conv1 coefficients: per (i,j) the bracket k and c1 = s w_j (1-t), c2 = s w_j t
struct ConvCoef {
  int k;
  int diag;
  double c1, c2;
};
cudaError_t launch_conv_coef(int M, double beta, const double *tau, const double *w,
                             const double *wm, const double *wp, ConvCoef *coef, cudaStream_t s);
// Fourth-order variant of the Dyson integrals (conv.cu): per (i, j) the rows
// k0 .. k0 + 3 and weights c[] of the cubic lag interpolation times the side
// weight (diagonal: c[0] for Sigma_0, c[1] for Sigma_{M-1}).
struct ConvCoef4 {
  int k0;
  int diag;
  double c[4];
};
// coef [M][M]; W [M][M] side weights (0 on the diagonal); wL, wR [M] the end
// weights of the two sides of the split at tau_i; wE [M] whole-mesh weights.
cudaError_t launch_quad4_tables(int M, double beta, const double *tau, ConvCoef4 *coef,
                                double *W, double *wL, double *wR, double *wE, cudaStream_t s);

// linalg.cu
// C[b] = alpha * op(A[b]) diag(sk[b]) op(B[b]) + beta * C[b]  (row-major, FP64)
cudaError_t dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                  long lda, long sA, const double *B, long ldb, long sB, const double *sk,
                  long sS, double beta, double *C, long ldc, long sC, int batch, cudaStream_t s);
// Symmetric eigen-decomposition by cyclic-by-rounds Jacobi on the device.
// A (n x n, overwritten), V (n x n, in: starting basis or identity, out:
// eigenvectors as columns, unsorted), scratch A2 (n x n), J (rotation scratch,
// >= 2*(n+1) doubles), scal (>= 4 doubles). Returns sweeps used or <0.
int jacobi_eig(int n, double *A, double *A2, double *V, double *J, double *scal, double tol,
               int max_sweeps, cudaStream_t s, cudaError_t *err);
// Sort eigenpairs ascending: eps_out[r] = diag(A)[idx], C_out[:, r] = V[:, idx].
cudaError_t launch_sort_eig(int n, const double *A, const double *V, double *eps_out,
                            double *C_out, cudaStream_t s);
cudaError_t launch_identity(int n, double *I, cudaStream_t s);
cudaError_t launch_copy(size_t count, const double *src, double *dst, cudaStream_t s);
cudaError_t launch_max_abs_diff(size_t count, const double *a, const double *b,
                                unsigned long long *out, cudaStream_t s);

// hf.cu
cudaError_t launch_hf_selfenergy(int n, double spin, const double *rho, const double *V,
                                 const double *add, const double *sub, double *out,
                                 cudaStream_t s);
cudaError_t launch_mu_fermi(int n, int nocc, double beta, const double *eps, double *mu_out,
                            double *f, cudaStream_t s);
cudaError_t launch_phi_table(int n, int M, double beta, const double *eps, const double *mu_dev,
                             double mu_host, const double *tau, double *phi, cudaStream_t s);

// sigma2.cu (FP64 path)
cudaError_t sigma2_fp64(int n, int M, double spin, const double *V, const double *G,
                        double *Sigma, double *Q, double *T1, double *W, cudaStream_t s);
// GW pieces: the bubble Q_j = g_j o g_{M-1-j} and V Q_j V; Sigma = spin g o w.
cudaError_t gw_bubble(int n, int M, const double *V, const double *G, double *Q, double *T1,
                      double *VQV, cudaStream_t s);
cudaError_t launch_gw_sigma(long count, double spin, const double *G, const double *w,
                            double *Sigma, cudaStream_t s);
// tmatrix.cu: the particle-particle ladder on pair-space stacks t[j][b][l][a][k]
// (n <= 32): source V_ak g_ab g_kl V_bl, the periodic convolution of the pair
// propagator g (x) g with t (bosonic table coef), the damped update
// t <- (1 - m) t + m (S - V^ Y) with *res = max|t_new - t| (double bits), and
// Sigma^T = sum_kl [spin t(ak; bl) - t(ak; lb)] g_{M-1-j}(l, k).
cudaError_t tm_source(int n, int M, const double *V, const double *G, double *S, cudaStream_t s);
cudaError_t tm_ladder(int n, int M, const ConvCoef *coef, const double *G, const double *T,
                      double *Y, cudaStream_t s);
cudaError_t tm_update(int n, int M, const double *V, const double *S, const double *Y, double *T,
                      double mixing, unsigned long long *res, cudaStream_t s);
cudaError_t tm_sigma(int n, int M, double spin, const double *G, const double *T, double *Sigma,
                     cudaStream_t s);
// basis.cu: periodic convolution coefficients (every (i, j), no diagonal case)
cudaError_t launch_conv_coef_bose(int M, double beta, const double *tau, const double *w,
                                  ConvCoef *coef, cudaStream_t s);

// tmap.cu: 3-D TMA map over [M][n][ld] floats, box 32 x rows x 1, 128B swizzle,
// rows beyond n read as zero.
cudaError_t make_tmap_rows(CUtensorMap *map, const float *base, int n, int M, int ld, int rows,
                           int box_cols = 32);
cudaError_t make_tmap_rows16(CUtensorMap *map, const void *base, int n, int M, int ld16, int rows);
// 2-D map over FP16 rows [n][pitch] of `cols` used columns, box 64 halves x rows.
cudaError_t make_tmap_tail16(CUtensorMap *map, const void *base, int n, int cols, int pitch,
                             int rows);

// sigma2_tc.cu (tensor cores, split TF32): the split workspace of a system
// holds 4 * M*n*ld + n*ld floats (g32, gh, gl, VQ, V32; ld = n rounded up to 32).
size_t sigma2_tc_smem_bytes(int n);
int sigma2_tc_max_n();

// g32 = (float)G, gh/gl = TF32 hi/lo of G, rows padded to ld = n rounded up to 32.
cudaError_t launch_split_g(int n, int M, const double *G, float *g32, float *gh, float *gl,
                           cudaStream_t s);

// conv_tc.cu (tensor cores, split TF32): S32 = Sigma in FP32 (pitch ld); gh/gl
// are the split copies of G from launch_split_g / sigma2_tc.
cudaError_t launch_sigma_to_f32(int n, int M, const double *S, float *S32, cudaStream_t s,
                                unsigned *smax = nullptr);

// conv.cu
// part (may be NULL: one CTA per row tile and mesh point): scratch of
// (conv1_fp64_splits(n, M) - 1) M n n doubles that lets a small launch split
// the mesh-point range over more CTAs (partial sums added in split order).
int conv1_fp64_splits(int n, int M);
cudaError_t conv1_fp64(int n, int M, const ConvCoef *coef, const double *dHF, const double *A,
                       const double *G, double *I1, cudaStream_t s, double *part = nullptr);
cudaError_t conv1_fp64_q4(int n, int M, const ConvCoef4 *coef, const double *dHF,
                          const double *A, const double *G, double *I1, cudaStream_t s,
                          double *part = nullptr);
// W (may be NULL): per-(i, j) weights replacing w_j (fourth-order variant;
// wm, wp are then its end weights wL, wR).
cudaError_t launch_conv2_kernel(int n, int M, double beta, const double *tau, const double *w,
                                const double *wm, const double *wp, const double *eps,
                                const double *mu_dev, double mu_host, double *K, cudaStream_t s,
                                const double *W = nullptr);
cudaError_t conv2_apply(int n, int M, const double *K, const double *C, const double *I1,
                        double *I2, double *t1, double *t2, cudaStream_t s);

cudaError_t launch_to_f32(size_t count, const double *x, float *y, cudaStream_t s);
cudaError_t conv2_apply_f32(int n, int M, const float *K32, const double *C, const double *I1,
                            double *I2, float *t1, float *t2, int *err, cudaStream_t s);

// selftest.cu: one warp waits (bounded by limit_ns, the tensor-core kernels'
// wait helper) on an mbarrier that is released first (release) or never; a
// wait that gives up sets *flag = 1.
cudaError_t launch_wait_probe(bool release, unsigned long long limit_ns, int *flag,
                              cudaStream_t s);

// update.cu
// n_out[a] = spin g[a][a] / W[a] (density at the nodes from g(0^-)).
cudaError_t launch_density(int n, const double *g, const double *W, double spin, double *n_out,
                           cudaStream_t s);
cudaError_t launch_update(int n, int M, double mixing, const double *G0, const double *I2,
                          double *G, unsigned long long *res_bits, cudaStream_t s);
cudaError_t launch_axpby(size_t count, double a, const double *x, double b, const double *y,
                         double *out, cudaStream_t s);
cudaError_t launch_energy_hf(int n, double spin, const double *h, const double *V,
                             const double *rho, double *out, cudaStream_t s);
cudaError_t launch_energy(int n, int M, double spin, const double *h, const double *V,
                          const double *G, const double *A, const double *w, double *part,
                          double *out, cudaStream_t s);

}  // namespace fedvr

#define FEDVR_CK(ctx, call)                                                   \
  do {                                                                        \
    cudaError_t e__ = (call);                                                 \
    if (e__ != cudaSuccess)                                                   \
      return fedvr::cuda_fail((ctx), e__, #call, __FILE__, __LINE__);         \
  } while (0)
