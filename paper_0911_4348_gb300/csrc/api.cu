// C ABI entry points and the host-side drivers of the FE-DVR second-Born
// library: context and workspace management, the HF self-consistency and the
// second-Born Dyson iteration (Sec. 2.3). Every numerical step is a kernel of
// this library; the host only sequences launches and reads scalars.
#include "common.cuh"
#include "tc_sys.cuh"

#include <math.h>
#include <string.h>

#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

namespace fedvr {

int fail(fedvr_ctx *ctx, int code, const char *fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_fail(fedvr_ctx *ctx, cudaError_t e, const char *what, const char *file, int line) {
  if (ctx) {
    ctx->failed = true;
    snprintf(ctx->err, sizeof(ctx->err), "CUDA error %d (%s) in %s at %s:%d", (int)e,
             cudaGetErrorString(e), what, file, line);
  }
  return FEDVR_ERR_CUDA;
}

bool ensure(fedvr_ctx *ctx, DevBuf &buf, size_t bytes, const char *name) {
  if (bytes == 0) bytes = 16;
  if (buf.bytes >= bytes) return true;
  drop_graph(ctx);  // the captured iteration holds the old address
  if (buf.ptr) cudaFree(buf.ptr);
  buf.ptr = nullptr;
  buf.bytes = 0;
  cudaError_t e = cudaMalloc(&buf.ptr, bytes);
  if (e != cudaSuccess) {
    buf.ptr = nullptr;
    cudaGetLastError();
    fail(ctx, FEDVR_ERR_CUDA, "cudaMalloc of %zu bytes for %s failed: %s", bytes, name,
         cudaGetErrorString(e));
    ctx->failed = true;
    return false;
  }
  buf.bytes = bytes;
  return true;
}

void release(DevBuf &buf) {
  if (buf.ptr) cudaFree(buf.ptr);
  buf.ptr = nullptr;
  buf.bytes = 0;
}

void drop_graph(fedvr_ctx *ctx) {
  if (ctx && ctx->step_graph) {
    cudaGraphExecDestroy(ctx->step_graph);
    ctx->step_graph = nullptr;
  }
}

}  // namespace fedvr

using namespace fedvr;

#define ENSURE(ctx, buf, bytes)                                   \
  do {                                                            \
    if (!ensure((ctx), (ctx)->buf, (bytes), #buf)) return FEDVR_ERR_CUDA; \
  } while (0)

#define CHECK_CTX(ctx)                                                           \
  do {                                                                           \
    if (!(ctx)) return FEDVR_ERR_ARG;                                            \
    if ((ctx)->failed)                                                           \
      return FEDVR_ERR_STATE;                                                    \
  } while (0)

namespace {

inline size_t dsz(size_t n) { return n * sizeof(double); }

inline bool is_fin(double x) { return isfinite(x); }

int sync(fedvr_ctx *ctx) {
  FEDVR_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return FEDVR_OK;
}

int copy_out(fedvr_ctx *ctx, void *dst, const void *src, size_t bytes, bool on_device) {
  FEDVR_CK(ctx, cudaMemcpyAsync(dst, src, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                ctx->stream));
  return FEDVR_OK;
}

// Mesh (tau, w, wm, wp) and, if requested, conv1 coefficients into workspace.
int build_mesh(fedvr_ctx *ctx, double beta, int u, int p, bool coef) {
  int M = 2 * u * p + 1;
  ENSURE(ctx, w_tau, dsz(M));
  ENSURE(ctx, w_w, dsz(M));
  ENSURE(ctx, w_wm, dsz(M));
  ENSURE(ctx, w_wp, dsz(M));
  FEDVR_CK(ctx, launch_mesh(beta, u, p, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                            P<double>(ctx->w_wm), P<double>(ctx->w_wp), nullptr, nullptr,
                            ctx->stream));
  if (coef) {
    ENSURE(ctx, w_coef, (size_t)M * M * sizeof(ConvCoef));
    FEDVR_CK(ctx, launch_conv_coef(M, beta, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                                   P<double>(ctx->w_wm), P<double>(ctx->w_wp),
                                   P<ConvCoef>(ctx->w_coef), ctx->stream));
    ENSURE(ctx, w_coef32, (size_t)M * M * sizeof(int4));
    FEDVR_CK(ctx, launch_coef32(M, P<ConvCoef>(ctx->w_coef), P<int4>(ctx->w_coef32), ctx->stream));
  }
  return FEDVR_OK;
}

// Scratch of the FP64 first convolution's mesh-range splits (small launches).
int ensure_c1f(fedvr_ctx *ctx, int n, int M) {
  const int sp = conv1_fp64_splits(n, M);
  ENSURE(ctx, w_c1f, dsz((size_t)(sp > 1 ? sp - 1 : 1) * M * n * n));
  return FEDVR_OK;
}

// GW screened interaction of g and Sigma^GW = spin g o w: the damped fixed-point
// iteration w <- (1 - a) w + a (V Q V - spin V (Q * w)) from w (V Q V when
// !w_valid) until max|w_new - w| < tol, with Q * w the periodic convolution of
// the table coef (conv1_fp64 with no diagonal entries; dummy is never read).
// One host readback of the residual per inner iteration. Workspace: Q, T1,
// VQV, C, Nw stacks and an 8-byte residual word.
int gw_solve(fedvr_ctx *ctx, int n, int M, const double *V, const double *G, double *Sigma,
             const ConvCoef *coef, double *w, bool w_valid, double *Q, double *T1, double *VQV,
             double *C, double *Nw, unsigned long long *res_d, const double *dummy,
             double mixing, double tol, int max_iter, int *iters) {
  cudaStream_t s = ctx->stream;
  const size_t stack = (size_t)M * n * n;
  const long nn = (long)n * n;
  FEDVR_CK(ctx, gw_bubble(n, M, V, G, Q, T1, VQV, s));
  if (!w_valid) FEDVR_CK(ctx, launch_copy(stack, VQV, w, s));
  double r = 0.0;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    FEDVR_CK(ctx, conv1_fp64(n, M, coef, dummy, Q, w, C, s, P<double>(ctx->w_c1f)));
    FEDVR_CK(ctx, launch_copy(stack, VQV, Nw, s));
    FEDVR_CK(ctx, dgemm(false, false, n, n, n, -ctx->spin, V, n, 0, C, n, nn, nullptr, 0, 1.0, Nw,
                        n, nn, M, s));
    FEDVR_CK(ctx, cudaMemsetAsync(res_d, 0, sizeof(unsigned long long), s));
    FEDVR_CK(ctx, launch_max_abs_diff(stack, Nw, w, res_d, s));
    FEDVR_CK(ctx, launch_axpby(stack, 1.0 - mixing, w, mixing, Nw, w, s));
    unsigned long long bits = 0;
    FEDVR_CK(ctx, cudaMemcpyAsync(&bits, res_d, sizeof(bits), cudaMemcpyDeviceToHost, s));
    if (int rr = sync(ctx)) return rr;
    memcpy(&r, &bits, sizeof(r));
    if (!is_fin(r)) return fail(ctx, FEDVR_ERR_NAN, "GW screened interaction is not finite");
    if (r < tol) break;
  }
  if (it > max_iter)
    return fail(ctx, FEDVR_ERR_NOCONV,
                "GW screened interaction not converged in %d iterations (residual %.3e)",
                max_iter, r);
  FEDVR_CK(ctx, launch_gw_sigma((long)stack, ctx->spin, G, w, Sigma, s));
  *iters = it;
  return FEDVR_OK;
}

// T-matrix ladder of g and Sigma^T: the damped fixed-point iteration
// t <- (1 - a) t + a (V^ K V^ - V^ (K * t)) from t (the source V^ K V^ when
// !t_valid) until max|t_new - t| < tol, with K * t the periodic convolution of
// the pair propagator (bosonic table coef). One host readback of the residual
// per inner iteration.
int tm_solve(fedvr_ctx *ctx, int n, int M, const double *V, const double *G, double *Sigma,
             const ConvCoef *coef, double *t, bool t_valid, double *src, double *Y,
             unsigned long long *res_d, double mixing, double tol, int max_iter, int *iters) {
  cudaStream_t s = ctx->stream;
  const size_t pstack = (size_t)M * n * n * n * n;
  FEDVR_CK(ctx, tm_source(n, M, V, G, src, s));
  if (!t_valid) FEDVR_CK(ctx, launch_copy(pstack, src, t, s));
  double r = 0.0;
  int it = 0;
  for (it = 1; it <= max_iter; ++it) {
    FEDVR_CK(ctx, tm_ladder(n, M, coef, G, t, Y, s));
    FEDVR_CK(ctx, cudaMemsetAsync(res_d, 0, sizeof(unsigned long long), s));
    FEDVR_CK(ctx, tm_update(n, M, V, src, Y, t, mixing, res_d, s));
    unsigned long long bits = 0;
    FEDVR_CK(ctx, cudaMemcpyAsync(&bits, res_d, sizeof(bits), cudaMemcpyDeviceToHost, s));
    if (int rr = sync(ctx)) return rr;
    memcpy(&r, &bits, sizeof(r));
    if (!is_fin(r)) return fail(ctx, FEDVR_ERR_NAN, "T-matrix ladder is not finite");
    if (r < tol) break;
  }
  if (it > max_iter)
    return fail(ctx, FEDVR_ERR_NOCONV, "T-matrix ladder not converged in %d iterations (residual %.3e)",
                max_iter, r);
  FEDVR_CK(ctx, tm_sigma(n, M, ctx->spin, G, t, Sigma, s));
  *iters = it;
  return FEDVR_OK;
}

int tm_workspace(fedvr_ctx *ctx, int n, int M) {
  const size_t pstack = (size_t)M * n * n * n * n;
  ENSURE(ctx, m_t, dsz(pstack));
  ENSURE(ctx, m_src, dsz(pstack));
  ENSURE(ctx, m_y, dsz(pstack));
  ENSURE(ctx, g_coef, (size_t)M * M * sizeof(ConvCoef));
  ENSURE(ctx, g_res, 16);
  return FEDVR_OK;
}

int gw_workspace(fedvr_ctx *ctx, int n, int M) {
  const size_t stack = (size_t)M * n * n;
  ENSURE(ctx, g_w, dsz(stack));
  ENSURE(ctx, g_vqv, dsz(stack));
  ENSURE(ctx, g_c, dsz(stack));
  ENSURE(ctx, g_new, dsz(stack));
  ENSURE(ctx, g_coef, (size_t)M * M * sizeof(ConvCoef));
  ENSURE(ctx, g_res, 16);
  ENSURE(ctx, w_t1, dsz(stack));
  ENSURE(ctx, w_t2, dsz(stack));
  return ensure_c1f(ctx, n, M);
}

// Tables of the fourth-order variant for the mesh in w_tau (M points).
int build_quad4(fedvr_ctx *ctx, int M, double beta) {
  ENSURE(ctx, w_q4coef, (size_t)M * M * sizeof(ConvCoef4));
  ENSURE(ctx, w_q4W, dsz((size_t)M * M));
  ENSURE(ctx, w_q4w, dsz(3 * (size_t)M));
  double *q = P<double>(ctx->w_q4w);
  FEDVR_CK(ctx, launch_quad4_tables(M, beta, P<double>(ctx->w_tau), P<ConvCoef4>(ctx->w_q4coef),
                                    P<double>(ctx->w_q4W), q, q + M, q + 2 * M, ctx->stream));
  return FEDVR_OK;
}

// The per-i end weights and the energy weights in use: the split trapezoid's
// (wm, wp, w) or the fourth-order variant's (wL, wR, wE).
const double *end_weight_left(fedvr_ctx *ctx) {
  return ctx->quad_order == 4 ? P<double>(ctx->w_q4w) : P<double>(ctx->w_wm);
}
const double *end_weight_right(fedvr_ctx *ctx) {
  return ctx->quad_order == 4 ? P<double>(ctx->w_q4w) + ctx->M : P<double>(ctx->w_wp);
}
const double *energy_weights(fedvr_ctx *ctx) {
  return ctx->quad_order == 4 ? P<double>(ctx->w_q4w) + 2 * ctx->M : P<double>(ctx->w_w);
}

int check_quad(fedvr_ctx *ctx, int precision, int M) {
  if (ctx->quad_order != 4) return FEDVR_OK;
  if (precision != FEDVR_FP64)
    return fail(ctx, FEDVR_ERR_ARG, "the fourth-order quadrature runs on the FP64 path only");
  if (M < 4) return fail(ctx, FEDVR_ERR_ARG, "the fourth-order quadrature needs M >= 4");
  return FEDVR_OK;
}

int check_mesh_args(fedvr_ctx *ctx, double beta, int u, int p) {
  if (!(beta > 0.0) || !is_fin(beta)) return fail(ctx, FEDVR_ERR_ARG, "beta must be > 0");
  if (u < 1 || p < 1 || p > 60) return fail(ctx, FEDVR_ERR_ARG, "need u >= 1, 1 <= p <= 60");
  long M = 2L * u * p + 1;
  if (M > 4097) return fail(ctx, FEDVR_ERR_ARG, "mesh too large: M = %ld > 4097", M);
  return FEDVR_OK;
}

// Eigen-decomposition of the symmetric n x n matrix in A (destroyed), starting
// from the orthogonal basis in Vinit (or the identity): eps ascending, C columns.
int eig(fedvr_ctx *ctx, double *A, const double *Vinit, double *eps, double *C) {
  int n = ctx->n;
  double *V = P<double>(ctx->b_hf_tmp);
  if (Vinit) {
    FEDVR_CK(ctx, launch_copy((size_t)n * n, Vinit, V, ctx->stream));
  } else {
    FEDVR_CK(ctx, launch_identity(n, V, ctx->stream));
  }
  cudaError_t err = cudaSuccess;
  int sweeps = jacobi_eig(n, A, P<double>(ctx->b_A2), V, P<double>(ctx->b_J),
                          P<double>(ctx->b_scal), 1e-14, 60, ctx->stream, &err);
  if (err != cudaSuccess) return cuda_fail(ctx, err, "jacobi_eig", __FILE__, __LINE__);
  if (sweeps < 0) return fail(ctx, FEDVR_ERR_NOCONV, "Jacobi did not converge in 60 sweeps");
  FEDVR_CK(ctx, launch_sort_eig(n, A, V, eps, C, ctx->stream));
  return FEDVR_OK;
}

// Workspace of the tensor-core Sigma^(2) build: split operands, VQ, V32, an
// FP32 copy of Sigma followed by the diagonal operands B_ii of the first
// convolution (both read by the tensor-core convolution), V Q V and the error
// flag (offsets in tc_sys.cuh).
int tc_workspace(fedvr_ctx *ctx, int n, int M, float **ws, float **S32, int **err) {
  ENSURE(ctx, w_tc, tc_ws_floats(n, M) * sizeof(float));
  float *base = P<float>(ctx->w_tc);
  *ws = base;
  *S32 = base + tc_ws_s32(n, M);
  *err = reinterpret_cast<int *>(base + tc_ws_w(n, M) + tc_ws_stack(n, M));
  return FEDVR_OK;
}

int tc_err_ptr(fedvr_ctx *ctx, int **err) {
  float *ws, *S32;
  return tc_workspace(ctx, ctx->n, ctx->M, &ws, &S32, err);
}

// Decode the tensor-core path's device error flag (read back after a
// synchronisation). Bit 0 (value 1): a bounded mbarrier wait gave up; the
// kernel left its work unfinished, so the workspace is undefined and the
// context is marked failed (later calls return FEDVR_ERR_STATE). Bit 1
// (value 2): an entry of g outside the FP16 split's range; nothing is
// corrupted, the flag is cleared and the call reports FEDVR_ERR_ARG.
int flag_status(fedvr_ctx *ctx, int h_err, int *dflag) {
  if (h_err & 1) {
    ctx->failed = true;
    return fail(ctx, FEDVR_ERR_TIMEOUT, "a tensor-core kernel's bounded wait gave up");
  }
  if (h_err & 2) {
    if (dflag) {
      FEDVR_CK(ctx, cudaMemsetAsync(dflag, 0, sizeof(int), ctx->stream));
      FEDVR_CK(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return fail(ctx, FEDVR_ERR_ARG,
                "an entry of g has |g| >= 16 or is not finite: outside the FP16 split's range "
                "(FEDVR_SPLIT_TF32 and FEDVR_FP64 have no such limit)");
  }
  return FEDVR_OK;
}

bool is_split(int precision) {
  return precision == FEDVR_SPLIT_TF32 || precision == FEDVR_SPLIT_F16;
}

int check_precision(fedvr_ctx *ctx, int precision, int n) {
  if (precision == FEDVR_FP64) return FEDVR_OK;
  if (is_split(precision)) {
    if (n > sigma2_tc_max_n())
      return fail(ctx, FEDVR_ERR_ARG, "split precision supports n_b <= %d", sigma2_tc_max_n());
    return FEDVR_OK;
  }
  return fail(ctx, FEDVR_ERR_ARG, "precision %d is not available in this build", precision);
}

// FP16-split workspace: the hi and lo FP16 stacks of g ([M][n][ld16] each) and
// the first convolution's packed tail, then the operand scales. NULL pointers
// when the context is not in that mode.
int f16_workspace(fedvr_ctx *ctx, int n, int M, void **h16, TcScale **scale) {
  const size_t halves = f16_split_halves(n, M);
  const size_t off = (halves * 2 + 255) / 256 * 256;
  ENSURE(ctx, w_h16, off + 256);
  *h16 = ctx->w_h16.ptr;
  *scale = reinterpret_cast<TcScale *>(P<uint8_t>(ctx->w_h16) + off);
  return FEDVR_OK;
}

// The exchange tile table for basis size n in w_xrow (built on the host once per n).
int ensure_xrows(fedvr_ctx *ctx, int n) {
  if (ctx->xrow_n == n) return FEDVR_OK;
  std::vector<uint32_t> tiles;
  exchange_tile_table(n, tiles);
  ENSURE(ctx, w_xrow, tiles.size() * sizeof(uint32_t));
  FEDVR_CK(ctx, cudaMemcpyAsync(ctx->w_xrow.ptr, tiles.data(), tiles.size() * sizeof(uint32_t),
                                cudaMemcpyHostToDevice, ctx->stream));
  if (int r = sync(ctx)) return r;  // the host vector goes out of scope
  ctx->xrow_n = n;
  return FEDVR_OK;
}

// Device tables of the tensor-core kernels for one system: XSys, C1Sys and
// the two work-queue prefixes {0, items}, at 256-byte aligned offsets.
constexpr size_t kTabX = 0;
constexpr size_t kTabC = (sizeof(XSys) + 255) / 256 * 256;
constexpr size_t kTabPX = kTabC + (sizeof(C1Sys) + 255) / 256 * 256;
constexpr size_t kTabPC = kTabPX + 256;
constexpr size_t kTabBytes = kTabPC + 256;

int upload_single_tables(fedvr_ctx *ctx, int n, int M, const float *ws, double *Sigma,
                         float *S32, const double *dHF, const ConvCoef *coef, double *I1,
                         int splits = 1, double *part = nullptr, double spin = -1.0) {
  ENSURE(ctx, w_tab, kTabBytes);
  XSys x;
  C1Sys c;
  memset(&x, 0, sizeof(x));
  memset(&c, 0, sizeof(c));
  void *h16 = nullptr;
  TcScale *scale = nullptr;
  if (ctx->precision == FEDVR_SPLIT_F16) {
    if (int r = f16_workspace(ctx, n, M, &h16, &scale)) return r;
  }
  if (int r = ensure_xrows(ctx, n)) return r;
  // spin < 0: the context's own spin factor (a stage-level call passes its own)
  FEDVR_CK(ctx, xsys_fill(&x, n, M, spin >= 0.0 ? spin : ctx->spin, ws, Sigma, S32,
                          P<uint32_t>(ctx->w_xrow), scale ? &scale->maxS : nullptr, h16, scale));
  (void)coef;
  FEDVR_CK(ctx, c1sys_fill(&c, n, M, splits, ws, S32, dHF, P<int4>(ctx->w_coef32), I1, part, h16,
                           scale));
  long px[2] = {0, exchange_items(n, M)}, pc[2] = {0, conv1_items(n, M, splits)};
  uint8_t *base = P<uint8_t>(ctx->w_tab);
  FEDVR_CK(ctx, cudaMemcpyAsync(base + kTabX, &x, sizeof(x), cudaMemcpyHostToDevice, ctx->stream));
  FEDVR_CK(ctx, cudaMemcpyAsync(base + kTabC, &c, sizeof(c), cudaMemcpyHostToDevice, ctx->stream));
  FEDVR_CK(ctx, cudaMemcpyAsync(base + kTabPX, px, sizeof(px), cudaMemcpyHostToDevice, ctx->stream));
  FEDVR_CK(ctx, cudaMemcpyAsync(base + kTabPC, pc, sizeof(pc), cudaMemcpyHostToDevice, ctx->stream));
  return sync(ctx);  // host descriptors go out of scope
}

// First convolution of the prepared single system (tables at w_tab) with its
// splits summed into I1.
int launch_conv1_single(fedvr_ctx *ctx, int splits, int *err, cudaStream_t s, int *launches) {
  const int n = ctx->n, M = ctx->M;
  const TcGeom g = tc_geom(n, M);
  uint8_t *tab = P<uint8_t>(ctx->w_tab);
  FEDVR_CK(ctx, conv1_tc_launch(reinterpret_cast<const C1Sys *>(tab + kTabC),
                                reinterpret_cast<const long *>(tab + kTabPC), 1,
                                conv1_items(n, M, splits), g.Np, err, ctx->num_sms, s,
                                ctx->precision == FEDVR_SPLIT_F16));
  *launches += 1;
  if (splits > 1) {
    FEDVR_CK(ctx, conv1_sum_splits((long)M * n * n, splits - 1, P<double>(ctx->w_c1p),
                                   P<double>(ctx->w_I1), s));
    *launches += 1;
  }
  return FEDVR_OK;
}

// Measured choice of the first convolution's splits, once per (device, n, M,
// precision) in this process: every candidate's persistent launch (and split sum) is
// timed on the prepared buffers and the fastest kept. A candidate takes whole
// accumulation blocks (S <= the block count), so every choice gives the same
// block sums and the results differ only in the order in which the FP64
// partial sums are added; candidates also keep at most 16 work items per SM.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_conv1_splits;

int choose_conv1_splits(fedvr_ctx *ctx, float *ws, float *S32, int *err) {
  const int n = ctx->n, M = ctx->M;
  const size_t stack = (size_t)M * n * n;
  const long RT = ((long)M * n + 127) / 128;
  const int NB = conv1_blocks(n, M, ctx->precision == FEDVR_SPLIT_F16);
  std::vector<int> cand;
  for (int S : {1, 2, 3, 4, 6, 8, 12, 16}) {
    if (S > 1 && (S > NB || RT * S > 16L * ctx->num_sms || (S - 1) * stack * 8 > (2ull << 30)))
      continue;
    cand.push_back(S);
  }
  int best = 1;
  if (ctx->c1_request > 0) {
    best = 1;
    for (int S : cand)
      if (S <= ctx->c1_request) best = S;
  } else {
    // the block count, hence the candidate set, depends on the precision
    const auto key = std::make_tuple(ctx->device, n, M, ctx->precision);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_conv1_splits.find(key);
      if (it != g_conv1_splits.end()) best = it->second;
    }
    if (cand.size() > 1 && best == 1 && !g_conv1_splits.count(key)) {
      ENSURE(ctx, w_c1p, dsz((size_t)(cand.back() - 1) * stack));
      float best_ms = 0.f;
      cudaStream_t s = ctx->stream;
      for (int S : cand) {
        if (int r = upload_single_tables(ctx, n, M, ws, P<double>(ctx->w_S), S32,
                                         P<double>(ctx->w_dHF), P<ConvCoef>(ctx->w_coef),
                                         P<double>(ctx->w_I1), S, P<double>(ctx->w_c1p)))
          return r;
        int launches = 0;
        if (int r = launch_conv1_single(ctx, S, err, s, &launches)) return r;  // warm-up
        FEDVR_CK(ctx, cudaEventRecord(ctx->ev[0], s));
        if (int r = launch_conv1_single(ctx, S, err, s, &launches)) return r;
        FEDVR_CK(ctx, cudaEventRecord(ctx->ev[6], s));
        int h_err = 0;
        FEDVR_CK(ctx, cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (int r = sync(ctx)) return r;
        if (int r = flag_status(ctx, h_err, err)) return r;
        float ms = 0.f;
        FEDVR_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[6]));
        if (S == cand.front() || ms < 0.97f * best_ms) {  // more splits must win clearly
          best = S;
          best_ms = ms;
        }
      }
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_conv1_splits[key] = best;
    }
  }
  if (best > 1) ENSURE(ctx, w_c1p, dsz((size_t)(best - 1) * stack));
  ctx->c1_splits = best;
  return FEDVR_OK;
}

// The pieces of one iteration for one system, enqueued on stream s.
// (1) Sigma^(2): operand preparation (split path) or the whole FP64 build.
// err: device flag that the split path's tensor-core kernels raise on a timeout.
int phase_sigma_pre(fedvr_ctx *ctx, bool warm, cudaStream_t s, int *launches, int *err) {
  const int n = ctx->n, M = ctx->M;
  const size_t stack = (size_t)M * n * n;
  double *G = P<double>(ctx->w_G), *S = P<double>(ctx->w_S);
  const double *V = P<double>(ctx->b_V);
  void *h16 = nullptr;
  TcScale *scale = nullptr;
  if (is_split(ctx->precision) && !err) {
    if (int r = tc_err_ptr(ctx, &err)) return r;
  }
  if (ctx->precision == FEDVR_SPLIT_F16) {  // FP16 operands of g; the Sigma bound restarts
    if (int r = f16_workspace(ctx, n, M, &h16, &scale)) return r;
    float *ws, *S32;
    int *own;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &own)) return r;
    // with the FP32 copy of g for the exchange's producers and V Q V (ws offset 0)
    FEDVR_CK(ctx, launch_split_f16(n, M, G, h16, s, err, warm ? nullptr : ws));
    FEDVR_CK(ctx, cudaMemsetAsync(&scale->maxS, 0, sizeof(unsigned), s));
    *launches += 1;
  }
  if (warm) {
    FEDVR_CK(ctx, launch_copy(stack, P<double>(ctx->b_sigma_init), S, s));
    *launches += 1;
    if (is_split(ctx->precision)) {  // operands for the tensor-core convolution
      float *ws, *S32;
      int *err;
      if (int r = tc_workspace(ctx, n, M, &ws, &S32, &err)) return r;
      if (!scale) {  // the FP16 path reads g through its FP16 split, made above
        const size_t tstack = (size_t)M * n * ((n + 31) / 32 * 32);
        FEDVR_CK(ctx, launch_split_g(n, M, G, ws, ws + tstack, ws + 2 * tstack, s));
        *launches += 1;
      }
      FEDVR_CK(ctx, launch_sigma_to_f32(n, M, S, S32, s, scale ? &scale->maxS : nullptr));
      *launches += 1;
    }
  } else if (is_split(ctx->precision)) {
    float *ws, *S32;
    int *own_err;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &own_err)) return r;
    FEDVR_CK(ctx, sigma2_tc_pre(n, M, V, G, ws, s, !scale, err, scale != nullptr));
    *launches += scale ? 3 : 4;  // splits of g (TF32 path) and V, VQ, W = (VQ) V
  } else if (ctx->self_energy == 1) {
    int it = 0;
    if (int r = gw_solve(ctx, n, M, V, G, S, P<ConvCoef>(ctx->g_coef), P<double>(ctx->g_w),
                         ctx->gw_w_valid, P<double>(ctx->w_t1), P<double>(ctx->w_t2),
                         P<double>(ctx->g_vqv), P<double>(ctx->g_c), P<double>(ctx->g_new),
                         P<unsigned long long>(ctx->g_res), P<double>(ctx->w_dHF), ctx->gw_mixing,
                         ctx->gw_tol, ctx->gw_max_iter, &it))
      return r;
    ctx->gw_w_valid = true;
    ctx->gw_last_inner = it;
    *launches += 3 + 6 * it;
  } else if (ctx->self_energy == 2) {
    int it = 0;
    if (int r = tm_solve(ctx, n, M, V, G, S, P<ConvCoef>(ctx->g_coef), P<double>(ctx->m_t),
                         ctx->gw_w_valid, P<double>(ctx->m_src), P<double>(ctx->m_y),
                         P<unsigned long long>(ctx->g_res), ctx->gw_mixing, ctx->gw_tol,
                         ctx->gw_max_iter, &it))
      return r;
    ctx->gw_w_valid = true;
    ctx->gw_last_inner = it;
    *launches += 2 + 2 * it;
  } else {
    FEDVR_CK(ctx, sigma2_fp64(n, M, ctx->spin, V, G, S, P<double>(ctx->w_t1), P<double>(ctx->w_t2),
                              P<double>(ctx->w_t3), s));
    *launches += 4;
  }
  return FEDVR_OK;
}

// (2) HF self-energy change and the energy/particle number of (g_k, Sigma_k).
int phase_mid(fedvr_ctx *ctx, cudaStream_t s, int *launches) {
  const int n = ctx->n, M = ctx->M;
  const size_t nn = (size_t)n * n;
  double *G = P<double>(ctx->w_G), *S = P<double>(ctx->w_S);
  const double *V = P<double>(ctx->b_V);
  FEDVR_CK(ctx, launch_hf_selfenergy(n, ctx->spin, G + (size_t)(M - 1) * nn, V, nullptr,
                                     P<double>(ctx->b_Sigma0), P<double>(ctx->w_dHF), s));
  FEDVR_CK(ctx, launch_energy(n, M, ctx->spin, P<double>(ctx->b_h), V, G, S, energy_weights(ctx),
                              P<double>(ctx->w_part), P<double>(ctx->w_red), s));
  *launches += 4;
  if (is_split(ctx->precision)) {
    float *ws, *S32;
    int *err;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &err)) return r;
    void *h16 = nullptr;
    TcScale *scale = nullptr;
    if (ctx->precision == FEDVR_SPLIT_F16) {
      if (int r = f16_workspace(ctx, n, M, &h16, &scale)) return r;
    }
    FEDVR_CK(ctx, launch_diag_f32(n, M, P<double>(ctx->w_dHF), S, P<double>(ctx->w_wm),
                                  P<double>(ctx->w_wp), S32, s, scale ? &scale->maxS : nullptr));
    *launches += 1;
  }
  return FEDVR_OK;
}

// (3) FP64 first convolution (the split path launches its tensor-core kernel instead).
int phase_conv1_fp64(fedvr_ctx *ctx, cudaStream_t s, int *launches) {
  const int extra = conv1_fp64_splits(ctx->n, ctx->M) > 1 ? 1 : 0;  // the split sum
  if (ctx->quad_order == 4) {
    FEDVR_CK(ctx, conv1_fp64_q4(ctx->n, ctx->M, P<ConvCoef4>(ctx->w_q4coef), P<double>(ctx->w_dHF),
                                P<double>(ctx->w_S), P<double>(ctx->w_G), P<double>(ctx->w_I1), s,
                                P<double>(ctx->w_c1f)));
    *launches += 1 + extra;
    return FEDVR_OK;
  }
  FEDVR_CK(ctx, conv1_fp64(ctx->n, ctx->M, P<ConvCoef>(ctx->w_coef), P<double>(ctx->w_dHF),
                           P<double>(ctx->w_S), P<double>(ctx->w_G), P<double>(ctx->w_I1), s,
                           P<double>(ctx->w_c1f)));
  *launches += 1 + extra;
  return FEDVR_OK;
}


// (4) second convolution.
int phase_conv2(fedvr_ctx *ctx, cudaStream_t s, int *launches, int *err) {
  const int n = ctx->n, M = ctx->M;
  const double *C = P<double>(ctx->b_C);
  double *I1 = P<double>(ctx->w_I1), *I2 = P<double>(ctx->w_I2);
  if (is_split(ctx->precision)) {
    if (!err) {
      if (int r = tc_err_ptr(ctx, &err)) return r;
    }
    FEDVR_CK(ctx, conv2_apply_f32(n, M, P<float>(ctx->w_K32), C, I1, I2, P<float>(ctx->w_t1),
                                  P<float>(ctx->w_t2), err, s));
  } else {
    FEDVR_CK(ctx, conv2_apply(n, M, P<double>(ctx->w_K), C, I1, I2, P<double>(ctx->w_t1),
                              P<double>(ctx->w_t2), s));
  }
  *launches += 3;
  return FEDVR_OK;
}

// (5) mixed update and residual.
int phase_update(fedvr_ctx *ctx, double mixing, cudaStream_t s, int *launches) {
  double *red = P<double>(ctx->w_red);
  FEDVR_CK(ctx, cudaMemsetAsync(red + 2, 0, sizeof(double), s));
  FEDVR_CK(ctx, launch_update(ctx->n, ctx->M, mixing, P<double>(ctx->w_G0), P<double>(ctx->w_I2),
                              P<double>(ctx->w_G), reinterpret_cast<unsigned long long *>(red + 2),
                              s));
  *launches += 1;
  return FEDVR_OK;
}

// Enqueue one iteration on s without host synchronisation, recording the
// stage events with evflags (cudaEventRecordExternal inside a capture).
int enqueue_step(fedvr_ctx *ctx, bool warm, double mixing, cudaStream_t s, unsigned evflags,
                 int *launches) {
  const int n = ctx->n, M = ctx->M;
  const bool split = is_split(ctx->precision);
  int *err = nullptr;
  if (split) {
    if (int r = tc_err_ptr(ctx, &err)) return r;
  }
  FEDVR_CK(ctx, cudaEventRecordWithFlags(ctx->ev[1], s, evflags));
  if (int r = phase_sigma_pre(ctx, warm, s, launches, err)) return r;
  uint8_t *tab = P<uint8_t>(ctx->w_tab);
  if (split && !warm) {
    const TcGeom g = tc_geom(n, M);
    FEDVR_CK(ctx, exchange_tc_launch(reinterpret_cast<const XSys *>(tab + kTabX),
                                     reinterpret_cast<const long *>(tab + kTabPX), 1,
                                     exchange_items(n, M), g.Np, g.ld, err, ctx->num_sms, s,
                                     ctx->precision == FEDVR_SPLIT_F16));
    *launches += 1;
  }
  FEDVR_CK(ctx, cudaEventRecordWithFlags(ctx->ev[2], s, evflags));
  if (int r = phase_mid(ctx, s, launches)) return r;
  FEDVR_CK(ctx, cudaEventRecordWithFlags(ctx->ev[3], s, evflags));
  if (split) {
    if (int r = launch_conv1_single(ctx, ctx->c1_splits, err, s, launches)) return r;
  } else {
    if (int r = phase_conv1_fp64(ctx, s, launches)) return r;
  }
  FEDVR_CK(ctx, cudaEventRecordWithFlags(ctx->ev[4], s, evflags));
  if (int r = phase_conv2(ctx, s, launches, err)) return r;
  FEDVR_CK(ctx, cudaEventRecordWithFlags(ctx->ev[5], s, evflags));
  if (int r = phase_update(ctx, mixing, s, launches)) return r;
  FEDVR_CK(ctx, cudaEventRecordWithFlags(ctx->ev[6], s, evflags));
  return FEDVR_OK;
}

// Capture one regular iteration into ctx->step_graph. Capture happens on a
// private non-blocking stream (the context's stream may be the legacy default
// stream, which cannot be captured). If the driver refuses the capture the
// context carries on without graphs: the refusal is not an error of the run.
int capture_step(fedvr_ctx *ctx, double mixing) {
  if (!ctx->cap_stream) {
    if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ctx->cap_stream = nullptr;
      ctx->use_graphs = false;
      return FEDVR_OK;
    }
  }
  cudaStream_t cs = ctx->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    ctx->use_graphs = false;
    return FEDVR_OK;
  }
  int launches = 0;
  const int r = enqueue_step(ctx, false, mixing, cs, cudaEventRecordExternal, &launches);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaGraphExec_t exec = nullptr;
  if (r == FEDVR_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (r != FEDVR_OK || e != cudaSuccess || !exec) {
    // a launcher that cannot be captured: run this context eagerly from now on
    cudaGetLastError();
    ctx->failed = false;
    ctx->err[0] = 0;
    ctx->use_graphs = false;
    return FEDVR_OK;
  }
  ctx->step_graph = exec;
  ctx->graph_mixing = mixing;
  ctx->graph_launches = launches;
  return FEDVR_OK;
}

}  // namespace

int fedvr::sigma_of_current_g(fedvr_ctx *ctx) {
  if (!ctx->prepared) return fail(ctx, FEDVR_ERR_STATE, "no prepared second-Born run");
  cudaStream_t s = ctx->stream;
  int launches = 0;
  int *err = nullptr;
  if (is_split(ctx->precision)) {
    if (int r = tc_err_ptr(ctx, &err)) return r;
    FEDVR_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
  }
  if (int r = phase_sigma_pre(ctx, false, s, &launches, err)) return r;
  if (is_split(ctx->precision)) {
    const TcGeom g = tc_geom(ctx->n, ctx->M);
    uint8_t *tab = P<uint8_t>(ctx->w_tab);
    FEDVR_CK(ctx, exchange_tc_launch(reinterpret_cast<const XSys *>(tab + kTabX),
                                     reinterpret_cast<const long *>(tab + kTabPX), 1,
                                     exchange_items(ctx->n, ctx->M), g.Np, g.ld, err,
                                     ctx->num_sms, s, ctx->precision == FEDVR_SPLIT_F16));
    int h_err = 0;
    FEDVR_CK(ctx, cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (int r = sync(ctx)) return r;
    return flag_status(ctx, h_err, err);
  }
  return sync(ctx);
}

extern "C" {

int fedvr_create(fedvr_ctx **out, void *cuda_stream) {
  if (!out) return FEDVR_ERR_ARG;
  *out = nullptr;
  fedvr_ctx *ctx = new (std::nothrow) fedvr_ctx();
  if (!ctx) return FEDVR_ERR_ARG;
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaGetDevice(&ctx->device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FEDVR_ERR_CUDA;
  }
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) !=
      cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FEDVR_ERR_CUDA;
  }
  for (int i = 0; i < 7; ++i) {
    if (cudaEventCreate(&ctx->ev[i]) != cudaSuccess) {
      cudaGetLastError();
      for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->ev[j]);
      delete ctx;
      return FEDVR_ERR_CUDA;
    }
  }
  *out = ctx;
  return FEDVR_OK;
}

void fedvr_destroy(fedvr_ctx *ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  DevBuf *bufs[] = {&ctx->b_xi, &ctx->b_om, &ctx->b_edges, &ctx->b_nodes, &ctx->b_weights,
                    &ctx->b_elem, &ctx->b_local, &ctx->b_tt, &ctx->b_T, &ctx->b_v, &ctx->b_V,
                    &ctx->b_h, &ctx->b_eps, &ctx->b_C, &ctx->b_rho, &ctx->b_rho_new,
                    &ctx->b_rho_mix, &ctx->b_F, &ctx->b_Sigma0, &ctx->b_f, &ctx->b_A, &ctx->b_A2,
                    &ctx->b_J, &ctx->b_scal, &ctx->b_hf_tmp, &ctx->b_sigma_init, &ctx->w_tau,
                    &ctx->w_w, &ctx->w_wm, &ctx->w_wp, &ctx->w_coef, &ctx->w_K, &ctx->w_phi,
                    &ctx->w_G0, &ctx->w_G, &ctx->w_S, &ctx->w_I1, &ctx->w_I2, &ctx->w_t1,
                    &ctx->w_t2, &ctx->w_t3, &ctx->w_dHF, &ctx->w_part, &ctx->w_red, &ctx->w_tc,
                    &ctx->w_K32, &ctx->w_tab, &ctx->w_btab, &ctx->w_c1p,
                    &ctx->w_coef32, &ctx->w_h16, &ctx->w_xrow, &ctx->w_dens,
                    &ctx->w_q4coef, &ctx->w_q4W, &ctx->w_q4w, &ctx->k_L, &ctx->k_G,
                    &ctx->k_S, &ctx->k_T1, &ctx->k_R, &ctx->k_aux, &ctx->k_out,
                    &ctx->k_part, &ctx->k_sh, &ctx->k_aop, &ctx->k_o, &ctx->k_flag, &ctx->k_x,
                    &ctx->g_w, &ctx->g_vqv, &ctx->g_c, &ctx->g_new, &ctx->g_coef, &ctx->g_res,
                    &ctx->m_t, &ctx->m_src, &ctx->m_y, &ctx->w_c1f};
  drop_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  for (DevBuf *b : bufs) release(*b);
  for (int i = 0; i < 7; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (cudaEvent_t e : ctx->kbe_events) cudaEventDestroy(e);
  delete ctx;
}

const char *fedvr_last_error(const fedvr_ctx *ctx) { return ctx ? ctx->err : "null context"; }

int build_fedvr(fedvr_ctx *ctx, int n_elem, int pts_per_elem, double xmin, double xmax,
                int grid_kind, int *n_b_out) {
  CHECK_CTX(ctx);
  if (n_elem < 1 || pts_per_elem < 2 || pts_per_elem > 33)
    return fail(ctx, FEDVR_ERR_ARG, "need n_elem >= 1 and 2 <= pts_per_elem <= 33");
  const int order = pts_per_elem - 1;  // polynomial order n_g of the Lobatto rule
  long n = (long)n_elem * order - 1;
  if (n < 2 || n > 1024) return fail(ctx, FEDVR_ERR_ARG, "n_b = %ld outside [2, 1024]", n);
  if (!is_fin(xmin) || !is_fin(xmax) || !(xmin < xmax))
    return fail(ctx, FEDVR_ERR_ARG, "need finite xmin < xmax");
  if (grid_kind != 0 && grid_kind != 1) return fail(ctx, FEDVR_ERR_ARG, "grid_kind must be 0 or 1");
  ctx->stage = 0;
  ctx->n_elem = n_elem;
  ctx->order = order;
  ctx->n = (int)n;
  ctx->xmin = xmin;
  ctx->xmax = xmax;
  ctx->grid_kind = grid_kind;
  ctx->sigma_init_M = 0;
  ENSURE(ctx, b_xi, dsz(order + 1));
  ENSURE(ctx, b_om, dsz(order + 1));
  ENSURE(ctx, b_edges, dsz(n_elem + 1));
  ENSURE(ctx, b_nodes, dsz(n));
  ENSURE(ctx, b_weights, dsz(n));
  ENSURE(ctx, b_elem, n * sizeof(int));
  ENSURE(ctx, b_local, n * sizeof(int));
  ENSURE(ctx, b_tt, dsz((size_t)n_elem * (order + 1) * (order + 1)));
  ENSURE(ctx, b_T, dsz(n * n));
  ENSURE(ctx, b_scal, dsz(16));
  int *status = reinterpret_cast<int *>(P<double>(ctx->b_scal) + 8);
  FEDVR_CK(ctx, cudaMemsetAsync(status, 0, 2 * sizeof(int), ctx->stream));
  FEDVR_CK(ctx, launch_gll(order, P<double>(ctx->b_xi), P<double>(ctx->b_om), status, ctx->stream));
  FEDVR_CK(ctx, launch_basis(n_elem, order, xmin, xmax, grid_kind, P<double>(ctx->b_xi),
                             P<double>(ctx->b_om), P<double>(ctx->b_edges), P<double>(ctx->b_nodes),
                             P<double>(ctx->b_weights), P<int>(ctx->b_elem), P<int>(ctx->b_local),
                             P<double>(ctx->b_tt), P<double>(ctx->b_T), status + 1, ctx->stream));
  int st[2];
  FEDVR_CK(ctx, cudaMemcpyAsync(st, status, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream));
  if (int r = sync(ctx)) return r;
  if (st[0] != 0) return fail(ctx, FEDVR_ERR_ARG, "GLL root scan failed for order %d", order);
  if (st[1] != 0) return fail(ctx, FEDVR_ERR_ARG, "graded grid: non-positive element width");
  ctx->stage = 1;
  if (n_b_out) *n_b_out = (int)n;
  return FEDVR_OK;
}

int set_potential(fedvr_ctx *ctx, int n_nuc, const double *Z, const double *R, double soft_en,
                  double soft_ee, int n_elec, double *E_nn_out) {
  CHECK_CTX(ctx);
  if (ctx->stage < 1) return fail(ctx, FEDVR_ERR_STATE, "set_potential before build_fedvr");
  if (n_nuc < 0 || n_nuc > 256 || (n_nuc > 0 && (!Z || !R)))
    return fail(ctx, FEDVR_ERR_ARG, "need 0 <= n_nuc <= 256 and Z, R arrays");
  if (!(soft_en > 0.0) || !(soft_ee > 0.0) || !is_fin(soft_en) || !is_fin(soft_ee))
    return fail(ctx, FEDVR_ERR_ARG, "soft-Coulomb parameters must be > 0");
  if (n_elec < 2 || (n_elec & 1) || n_elec / 2 >= ctx->n)
    return fail(ctx, FEDVR_ERR_ARG, "need even n_elec >= 2 with n_elec/2 < n_b");
  for (int A = 0; A < n_nuc; ++A)
    if (!is_fin(Z[A]) || !is_fin(R[A])) return fail(ctx, FEDVR_ERR_ARG, "non-finite nucleus");
  int n = ctx->n;
  ctx->stage = 1;
  ctx->n_elec = n_elec;
  ctx->nocc = n_elec / 2;
  ctx->soft_en = soft_en;
  ctx->soft_ee = soft_ee;
  ENSURE(ctx, b_v, dsz(n));
  ENSURE(ctx, b_V, dsz((size_t)n * n));
  ENSURE(ctx, b_h, dsz((size_t)n * n));
  ENSURE(ctx, b_hf_tmp, dsz((size_t)n * n > 512 ? (size_t)n * n : 512));
  double *dZ = P<double>(ctx->b_hf_tmp), *dR = dZ + 256;
  if (n_nuc > 0) {
    FEDVR_CK(ctx, cudaMemcpyAsync(dZ, Z, dsz(n_nuc), cudaMemcpyHostToDevice, ctx->stream));
    FEDVR_CK(ctx, cudaMemcpyAsync(dR, R, dsz(n_nuc), cudaMemcpyHostToDevice, ctx->stream));
  }
  FEDVR_CK(ctx, launch_potential(n, P<double>(ctx->b_nodes), n_nuc, dZ, dR, soft_en, soft_ee,
                                 P<double>(ctx->b_T), P<double>(ctx->b_v), P<double>(ctx->b_V),
                                 P<double>(ctx->b_h), ctx->stream));
  if (int r = sync(ctx)) return r;  // host Z/R copies complete before returning
  double enn = 0.0;
  for (int A = 0; A < n_nuc; ++A)
    for (int B = A + 1; B < n_nuc; ++B) {
      double d = fabs(R[A] - R[B]);
      if (d > 0.0) enn += Z[A] * Z[B] / d;
    }
  if (E_nn_out) *E_nn_out = enn;
  ctx->stage = 2;
  return FEDVR_OK;
}

int fedvr_get_basis(const fedvr_ctx *cctx, double *nodes, double *weights, int *elem, int *local) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  CHECK_CTX(ctx);
  if (ctx->stage < 1) return fail(ctx, FEDVR_ERR_STATE, "no basis");
  int n = ctx->n;
  if (nodes) { if (int r = copy_out(ctx, nodes, ctx->b_nodes.ptr, dsz(n), false)) return r; }
  if (weights) { if (int r = copy_out(ctx, weights, ctx->b_weights.ptr, dsz(n), false)) return r; }
  if (elem) { if (int r = copy_out(ctx, elem, ctx->b_elem.ptr, n * sizeof(int), false)) return r; }
  if (local) { if (int r = copy_out(ctx, local, ctx->b_local.ptr, n * sizeof(int), false)) return r; }
  return sync(ctx);
}

int fedvr_get_gll(const fedvr_ctx *cctx, double *xi, double *omega) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  CHECK_CTX(ctx);
  if (ctx->stage < 1) return fail(ctx, FEDVR_ERR_STATE, "no basis");
  if (xi) { if (int r = copy_out(ctx, xi, ctx->b_xi.ptr, dsz(ctx->order + 1), false)) return r; }
  if (omega) { if (int r = copy_out(ctx, omega, ctx->b_om.ptr, dsz(ctx->order + 1), false)) return r; }
  return sync(ctx);
}

int fedvr_get_operators(const fedvr_ctx *cctx, double *T, double *v, double *V, double *h) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  CHECK_CTX(ctx);
  if (ctx->stage < 1) return fail(ctx, FEDVR_ERR_STATE, "no basis");
  if ((v || V || h) && ctx->stage < 2) return fail(ctx, FEDVR_ERR_STATE, "no potential");
  size_t nn = (size_t)ctx->n * ctx->n;
  if (T) { if (int r = copy_out(ctx, T, ctx->b_T.ptr, dsz(nn), false)) return r; }
  if (v) { if (int r = copy_out(ctx, v, ctx->b_v.ptr, dsz(ctx->n), false)) return r; }
  if (V) { if (int r = copy_out(ctx, V, ctx->b_V.ptr, dsz(nn), false)) return r; }
  if (h) { if (int r = copy_out(ctx, h, ctx->b_h.ptr, dsz(nn), false)) return r; }
  return sync(ctx);
}

int solve_hf(fedvr_ctx *ctx, double beta, double tol, int max_iter, double *E_hf, double *mu) {
  CHECK_CTX(ctx);
  if (ctx->stage < 2) return fail(ctx, FEDVR_ERR_STATE, "solve_hf before set_potential");
  if (!(beta > 0.0) || !is_fin(beta)) return fail(ctx, FEDVR_ERR_ARG, "beta must be > 0");
  if (!(tol > 0.0) || max_iter < 1) return fail(ctx, FEDVR_ERR_ARG, "need tol > 0, max_iter >= 1");
  const int n = ctx->n, nocc = ctx->nocc;
  const size_t nn = (size_t)n * n;
  const double spin = ctx->spin;
  cudaStream_t s = ctx->stream;
  ctx->stage = 2;
  ENSURE(ctx, b_eps, dsz(n));
  ENSURE(ctx, b_C, dsz(nn));
  ENSURE(ctx, b_rho, dsz(nn));
  ENSURE(ctx, b_rho_new, dsz(nn));
  ENSURE(ctx, b_rho_mix, dsz(nn));
  ENSURE(ctx, b_F, dsz(nn));
  ENSURE(ctx, b_Sigma0, dsz(nn));
  ENSURE(ctx, b_f, dsz(n));
  ENSURE(ctx, b_A, dsz(nn));
  ENSURE(ctx, b_A2, dsz(nn));
  ENSURE(ctx, b_J, dsz(4 * (n / 2 + 2)));
  ENSURE(ctx, b_hf_tmp, dsz(nn > 512 ? nn : 512));
  double *eps = P<double>(ctx->b_eps), *C = P<double>(ctx->b_C), *rho = P<double>(ctx->b_rho);
  double *rho_new = P<double>(ctx->b_rho_new), *rho_mix = P<double>(ctx->b_rho_mix);
  double *F = P<double>(ctx->b_F), *A = P<double>(ctx->b_A), *f = P<double>(ctx->b_f);
  double *scal = P<double>(ctx->b_scal);
  double *mu_dev = scal + 4;
  const double *h = P<double>(ctx->b_h), *V = P<double>(ctx->b_V);

  // start: projector on the nocc lowest eigenvectors of h
  FEDVR_CK(ctx, launch_copy(nn, h, A, s));
  if (int r = eig(ctx, A, nullptr, eps, C)) return r;
  FEDVR_CK(ctx, dgemm(false, true, n, n, nocc, 1.0, C, n, 0, C, n, 0, nullptr, 0, 0.0, rho, n, 0, 1, s));
  int it = 0;
  bool conv = false;
  for (it = 1; it <= max_iter; ++it) {
    FEDVR_CK(ctx, launch_hf_selfenergy(n, spin, rho, V, h, nullptr, F, s));
    // A = C^T F C in the previous eigenbasis, Jacobi from there (warm start)
    double *t = rho_mix;
    FEDVR_CK(ctx, dgemm(false, false, n, n, n, 1.0, F, n, 0, C, n, 0, nullptr, 0, 0.0, t, n, 0, 1, s));
    FEDVR_CK(ctx, dgemm(true, false, n, n, n, 1.0, C, n, 0, t, n, 0, nullptr, 0, 0.0, A, n, 0, 1, s));
    FEDVR_CK(ctx, launch_copy(nn, C, rho_new, s));  // starting basis (rho_new is free here)
    if (int r = eig(ctx, A, rho_new, eps, C)) return r;
    FEDVR_CK(ctx, launch_mu_fermi(n, nocc, beta, eps, mu_dev, f, s));
    FEDVR_CK(ctx, dgemm(false, true, n, n, n, 1.0, C, n, 0, C, n, 0, f, 0, 0.0, rho_new, n, 0, 1, s));
    unsigned long long *bits = reinterpret_cast<unsigned long long *>(scal + 5);
    FEDVR_CK(ctx, cudaMemsetAsync(bits, 0, sizeof(unsigned long long), s));
    FEDVR_CK(ctx, launch_max_abs_diff(nn, rho_new, rho, bits, s));
    double r_host;
    FEDVR_CK(ctx, cudaMemcpyAsync(&r_host, scal + 5, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (int r = sync(ctx)) return r;
    if (r_host != r_host) return fail(ctx, FEDVR_ERR_NAN, "NaN in the HF density");
    if (r_host < tol) { conv = true; break; }
    FEDVR_CK(ctx, launch_axpby(nn, 0.5, rho, 0.5, rho_new, rho_mix, s));
    double *tmp = P<double>(ctx->b_rho);
    ctx->b_rho.ptr = ctx->b_rho_mix.ptr;
    ctx->b_rho_mix.ptr = tmp;
    rho = P<double>(ctx->b_rho);
    rho_mix = P<double>(ctx->b_rho_mix);
  }
  if (!conv) return fail(ctx, FEDVR_ERR_NOCONV, "HF not converged after %d iterations", max_iter);
  // Sigma0 = F - h; E_hf on rho0 = C f C^T
  FEDVR_CK(ctx, launch_axpby(nn, 1.0, F, -1.0, h, P<double>(ctx->b_Sigma0), s));
  FEDVR_CK(ctx, launch_energy_hf(n, spin, h, V, rho_new, scal + 6, s));
  double out[3];
  FEDVR_CK(ctx, cudaMemcpyAsync(out, scal + 4, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (int r = sync(ctx)) return r;
  ctx->mu = out[0];
  ctx->E_hf = out[2];
  ctx->beta_hf = beta;
  ctx->hf_iters = it;
  ctx->stage = 3;
  if (E_hf) *E_hf = ctx->E_hf;
  if (mu) *mu = ctx->mu;
  return FEDVR_OK;
}

int fedvr_get_hf(const fedvr_ctx *cctx, double *eps, double *C, double *rho0, double *Sigma0) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  CHECK_CTX(ctx);
  if (ctx->stage < 3) return fail(ctx, FEDVR_ERR_STATE, "no HF solution");
  size_t nn = (size_t)ctx->n * ctx->n;
  if (eps) { if (int r = copy_out(ctx, eps, ctx->b_eps.ptr, dsz(ctx->n), false)) return r; }
  if (C) { if (int r = copy_out(ctx, C, ctx->b_C.ptr, dsz(nn), false)) return r; }
  if (rho0) { if (int r = copy_out(ctx, rho0, ctx->b_rho_new.ptr, dsz(nn), false)) return r; }
  if (Sigma0) { if (int r = copy_out(ctx, Sigma0, ctx->b_Sigma0.ptr, dsz(nn), false)) return r; }
  return sync(ctx);
}

int fedvr_density(const fedvr_ctx *cctx, int source, double *n_out) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  CHECK_CTX(ctx);
  if (!n_out) return fail(ctx, FEDVR_ERR_ARG, "n_out must not be NULL");
  const double *g = nullptr;
  if (source == FEDVR_DENSITY_HF) {
    if (ctx->stage < 3) return fail(ctx, FEDVR_ERR_STATE, "no HF solution");
    g = P<double>(ctx->b_rho_new);
  } else if (source == FEDVR_DENSITY_2B) {
    if (!ctx->prepared) return fail(ctx, FEDVR_ERR_STATE, "no prepared second-Born run");
    g = P<double>(ctx->w_G) + (size_t)(ctx->M - 1) * ctx->n * ctx->n;  // g(0^-)
  } else {
    return fail(ctx, FEDVR_ERR_ARG, "source must be FEDVR_DENSITY_HF or FEDVR_DENSITY_2B");
  }
  ENSURE(ctx, w_dens, dsz(ctx->n));
  FEDVR_CK(ctx, launch_density(ctx->n, g, P<double>(ctx->b_weights), ctx->spin,
                               P<double>(ctx->w_dens), ctx->stream));
  if (int r = copy_out(ctx, n_out, ctx->w_dens.ptr, dsz(ctx->n), false)) return r;
  return sync(ctx);
}

int fedvr_set_initial_sigma(fedvr_ctx *ctx, const double *Sigma0, int M, int on_device,
                            int inner_steps) {
  CHECK_CTX(ctx);
  if (ctx->stage < 1) return fail(ctx, FEDVR_ERR_STATE, "no basis");
  if (!Sigma0) {
    ctx->sigma_init_M = 0;
    ctx->warm_inner = 0;
    return FEDVR_OK;
  }
  if (M < 3 || M > 4097) return fail(ctx, FEDVR_ERR_ARG, "M outside [3, 4097]");
  if (inner_steps < 0 || inner_steps > 64) return fail(ctx, FEDVR_ERR_ARG, "inner_steps outside [0, 64]");
  size_t cnt = (size_t)M * ctx->n * ctx->n;
  ENSURE(ctx, b_sigma_init, dsz(cnt));
  FEDVR_CK(ctx, cudaMemcpyAsync(ctx->b_sigma_init.ptr, Sigma0, dsz(cnt),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                ctx->stream));
  if (int r = sync(ctx)) return r;
  ctx->sigma_init_M = M;
  ctx->warm_inner = inner_steps;
  return FEDVR_OK;
}

int fedvr_2b_prepare(fedvr_ctx *ctx, double beta, int u, int p, int precision) {
  CHECK_CTX(ctx);
  if (ctx->stage < 3) return fail(ctx, FEDVR_ERR_STATE, "second Born before solve_hf");
  if (int r = check_mesh_args(ctx, beta, u, p)) return r;
  if (beta != ctx->beta_hf)
    return fail(ctx, FEDVR_ERR_ARG, "beta differs from the HF solution's beta");
  if (int r = check_precision(ctx, precision, ctx->n)) return r;
  const int n = ctx->n, M = 2 * u * p + 1;
  if (int r = check_quad(ctx, precision, M)) return r;
  if (ctx->sigma_init_M && ctx->sigma_init_M != M)
    return fail(ctx, FEDVR_ERR_ARG, "initial Sigma has M = %d, mesh has %d", ctx->sigma_init_M, M);
  if (ctx->self_energy != 0 && (precision != FEDVR_FP64 || ctx->quad_order != 2))
    return fail(ctx, FEDVR_ERR_ARG, "GW and the T-matrix run on the FP64 path with the trapezoid rule");
  if (ctx->self_energy == 2 && ctx->n > 32)
    return fail(ctx, FEDVR_ERR_ARG, "the T-matrix ladder needs n_b <= 32 (pair space n_b^2)");
  ctx->prepared = false;
  drop_graph(ctx);
  const size_t nn = (size_t)n * n, stack = (size_t)M * nn;
  cudaStream_t s = ctx->stream;
  ENSURE(ctx, w_K, dsz((size_t)n * M * M));
  ENSURE(ctx, w_phi, dsz((size_t)M * n));
  ENSURE(ctx, w_G0, dsz(stack));
  ENSURE(ctx, w_G, dsz(stack));
  ENSURE(ctx, w_S, dsz(stack));
  ENSURE(ctx, w_I1, dsz(stack));
  ENSURE(ctx, w_I2, dsz(stack));
  ENSURE(ctx, w_t1, dsz(stack));
  ENSURE(ctx, w_t2, dsz(stack));
  ENSURE(ctx, w_t3, dsz(stack));
  ENSURE(ctx, w_dHF, dsz(nn));
  ENSURE(ctx, w_part, dsz(4 * (size_t)M + 3 * (size_t)n));  // launch_energy's partials
  ENSURE(ctx, w_red, dsz(8));
  if (!is_split(precision)) {
    if (int r = ensure_c1f(ctx, n, M)) return r;
  }
  if (is_split(precision)) {
    float *ws, *S32;
    int *err;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &err)) return r;
    FEDVR_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
    // the Sigma^(2) epilogue writes columns < n of the FP32 source stack only;
    // its padding (read as zeros by the convolution) is cleared once here
    FEDVR_CK(ctx, cudaMemsetAsync(S32, 0, 2 * (size_t)M * n * ((n + 31) / 32 * 32) * sizeof(float),
                                  s));
  }
  if (int r = build_mesh(ctx, beta, u, p, true)) return r;
  ctx->M = M;  // the weight accessors below read it
  if (ctx->quad_order == 4) {
    if (int r = build_quad4(ctx, M, beta)) return r;
  }
  if (ctx->self_energy != 0) {
    if (int r = ctx->self_energy == 1 ? gw_workspace(ctx, n, M) : tm_workspace(ctx, n, M))
      return r;
    FEDVR_CK(ctx, launch_conv_coef_bose(M, beta, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                                        P<ConvCoef>(ctx->g_coef), s));
    // the first outer step starts the inner iteration from its lowest order
    // (V Q V, or the ladder's V^ K V^)
    ctx->gw_w_valid = false;
  }
  double *tau = P<double>(ctx->w_tau), *w = P<double>(ctx->w_w);
  const double *eps = P<double>(ctx->b_eps), *C = P<double>(ctx->b_C);
  // g^0 on the mesh (Eq. hfgf) and the conv2 eigen-kernel, fixed for the run
  FEDVR_CK(ctx, launch_phi_table(n, M, beta, eps, nullptr, ctx->mu, tau, P<double>(ctx->w_phi), s));
  FEDVR_CK(ctx, dgemm(false, true, n, n, n, 1.0, C, n, 0, C, n, 0, P<double>(ctx->w_phi), n, 0.0,
                      P<double>(ctx->w_G0), n, nn, M, s));
  FEDVR_CK(ctx, launch_conv2_kernel(n, M, beta, tau, w, end_weight_left(ctx), end_weight_right(ctx),
                                    eps, nullptr, ctx->mu, P<double>(ctx->w_K), s,
                                    ctx->quad_order == 4 ? P<double>(ctx->w_q4W) : nullptr));
  if (is_split(precision)) {
    ENSURE(ctx, w_K32, (size_t)n * M * M * sizeof(float));
    FEDVR_CK(ctx, launch_to_f32((size_t)n * M * M, P<double>(ctx->w_K), P<float>(ctx->w_K32), s));
    float *ws, *S32;
    int *err;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &err)) return r;
    ctx->n = n;
    ctx->M = M;
    ctx->precision = precision;  // the tables and the split timing below depend on it
    if (precision == FEDVR_SPLIT_F16) {
      void *h16;
      TcScale *scale;
      if (int r = f16_workspace(ctx, n, M, &h16, &scale)) return r;
      FEDVR_CK(ctx, launch_scale_init(M, P<int4>(ctx->w_coef32), n, P<double>(ctx->b_V), scale,
                                      s));
    }
    if (int r = choose_conv1_splits(ctx, ws, S32, err)) return r;
    if (int r = upload_single_tables(ctx, n, M, ws, P<double>(ctx->w_S), S32, P<double>(ctx->w_dHF),
                                     P<ConvCoef>(ctx->w_coef), P<double>(ctx->w_I1),
                                     ctx->c1_splits, P<double>(ctx->w_c1p)))
      return r;
  } else {
    ctx->c1_splits = 1;
  }
  FEDVR_CK(ctx, launch_copy(stack, P<double>(ctx->w_G0), P<double>(ctx->w_G), s));
  if (int r = sync(ctx)) return r;
  ctx->history.clear();
  ctx->beta = beta;
  ctx->u = u;
  ctx->p = p;
  ctx->M = M;
  ctx->precision = precision;
  ctx->step_k = 0;
  ctx->prepared = true;
  ctx->prep_gen++;
  return FEDVR_OK;
}

int fedvr_2b_step(fedvr_ctx *ctx, double mixing, const double *G_in, int in_on_device,
                  double *res_out, double *E0, double *N_out) {
  CHECK_CTX(ctx);
  if (!ctx->prepared) return fail(ctx, FEDVR_ERR_STATE, "fedvr_2b_step before fedvr_2b_prepare");
  if (!(mixing > 0.0 && mixing <= 1.0)) return fail(ctx, FEDVR_ERR_ARG, "need 0 < mixing <= 1");
  const size_t stack = (size_t)ctx->M * ctx->n * ctx->n;
  cudaStream_t s = ctx->stream;
  auto t0 = std::chrono::steady_clock::now();
  const bool split = is_split(ctx->precision);
  int *err = nullptr;
  if (split) {
    if (int r = tc_err_ptr(ctx, &err)) return r;
  }
  FEDVR_CK(ctx, cudaEventRecord(ctx->ev[0], s));
  if (G_in)
    FEDVR_CK(ctx, cudaMemcpyAsync(P<double>(ctx->w_G), G_in, dsz(stack),
                                  in_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  const bool warm = ctx->sigma_init_M &&
                    ctx->step_k < (ctx->warm_inner > 0 ? ctx->warm_inner : 1);
  if (warm && ctx->warm_inner > 0) mixing = 1.0;  // full Dyson step at the fixed warm-start Sigma
  int launches = 0;
  ctx->last_step_graph = false;
  // the GW inner iteration reads its residual on the host: no graph capture
  if (ctx->use_graphs && !warm && ctx->self_energy == 0) {
    if (ctx->step_graph && ctx->graph_mixing != mixing) drop_graph(ctx);
    if (!ctx->step_graph) {
      if (int r = capture_step(ctx, mixing)) return r;
    }
  }
  if (ctx->step_graph && !warm && ctx->self_energy == 0) {
    FEDVR_CK(ctx, cudaGraphLaunch(ctx->step_graph, s));
    launches = ctx->graph_launches;
    ctx->last_step_graph = true;
  } else {
    if (int r = enqueue_step(ctx, warm, mixing, s, cudaEventRecordDefault, &launches)) return r;
  }
  ctx->step_launches = launches;
  double hr[3];
  int tc_err = 0;
  FEDVR_CK(ctx, cudaMemcpyAsync(hr, P<double>(ctx->w_red), sizeof(hr), cudaMemcpyDeviceToHost, s));
  if (split) FEDVR_CK(ctx, cudaMemcpyAsync(&tc_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (int r = sync(ctx)) return r;
  if ((tc_err & 1) || ((tc_err & 2) && hr[2] == hr[2] && is_fin(hr[0])))
    return flag_status(ctx, tc_err, err);
  if (tc_err) {  // a non-finite iterate also trips the FP16 range check: reported as NaN below
    FEDVR_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
  }
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  double rec[5] = {(double)ctx->step_k, hr[2], hr[0], hr[1], ms};
  ctx->history.insert(ctx->history.end(), rec, rec + 5);
  ctx->step_k++;
  if (res_out) *res_out = hr[2];
  if (E0) *E0 = hr[0];
  if (N_out) *N_out = hr[1];
  if (hr[2] != hr[2] || !is_fin(hr[0]))
    return fail(ctx, FEDVR_ERR_NAN, "NaN/Inf at iteration %d", ctx->step_k - 1);
  return FEDVR_OK;
}

int fedvr_conv1_splits(fedvr_ctx *ctx, int request, int *in_use) {
  CHECK_CTX(ctx);
  if (request > 64) return fail(ctx, FEDVR_ERR_ARG, "at most 64 splits");
  if (request >= 0) ctx->c1_request = request;
  if (in_use) *in_use = ctx->c1_splits;
  return FEDVR_OK;
}

int fedvr_set_mu(fedvr_ctx *ctx, double mu) {
  CHECK_CTX(ctx);
  if (ctx->stage < 3) return fail(ctx, FEDVR_ERR_STATE, "fedvr_set_mu before solve_hf");
  if (!is_fin(mu)) return fail(ctx, FEDVR_ERR_ARG, "mu must be finite");
  ctx->mu = mu;
  ctx->prepared = false;  // g^0 and the second convolution's table depend on mu
  drop_graph(ctx);
  return FEDVR_OK;
}

int fedvr_set_self_energy(fedvr_ctx *ctx, int kind, double w_mixing, double w_tol,
                          int w_max_iter) {
  CHECK_CTX(ctx);
  if (kind < 0 || kind > 2) return fail(ctx, FEDVR_ERR_ARG, "self-energy kind must be 0, 1 or 2");
  if (kind != 0 && (!(w_mixing > 0.0 && w_mixing <= 1.0) || !(w_tol > 0.0) || !is_fin(w_tol) ||
                    w_max_iter < 1))
    return fail(ctx, FEDVR_ERR_ARG,
                "GW and the T-matrix need 0 < w_mixing <= 1, w_tol > 0, w_max_iter >= 1");
  ctx->self_energy = kind;
  if (kind != 0) {
    ctx->gw_mixing = w_mixing;
    ctx->gw_tol = w_tol;
    ctx->gw_max_iter = w_max_iter;
  }
  ctx->prepared = false;  // a prepared run's tables belong to the old self-energy
  drop_graph(ctx);
  return FEDVR_OK;
}

int fedvr_gw_last_inner(const fedvr_ctx *ctx, int *iters) {
  if (!ctx || !iters) return FEDVR_ERR_ARG;
  *iters = ctx->gw_last_inner;
  return FEDVR_OK;
}

int fedvr_sigma_gw(fedvr_ctx *ctx, int n, double beta, int u, int p, double spin, const double *V,
                   const double *G, double *Sigma, double *w_io, int w_valid, double w_mixing,
                   double w_tol, int w_max_iter, int *iters) {
  CHECK_CTX(ctx);
  if (int r = check_mesh_args(ctx, beta, u, p)) return r;
  if (n < 1 || n > 1024 || !V || !G || !Sigma || !is_fin(spin) || spin < 0.0)
    return fail(ctx, FEDVR_ERR_ARG, "need 1 <= n <= 1024, spin >= 0 and device buffers");
  if (!(w_mixing > 0.0 && w_mixing <= 1.0) || !(w_tol > 0.0) || w_max_iter < 1 ||
      (w_valid && !w_io))
    return fail(ctx, FEDVR_ERR_ARG, "GW needs 0 < w_mixing <= 1, w_tol > 0, w_max_iter >= 1");
  ctx->prepared = false;  // the workspace below is shared with a prepared run
  drop_graph(ctx);
  if (int r = build_mesh(ctx, beta, u, p, false)) return r;
  const int M = 2 * u * p + 1;
  const size_t stack = (size_t)M * n * n;
  if (int r = gw_workspace(ctx, n, M)) return r;
  ENSURE(ctx, w_dHF, dsz((size_t)n * n));
  cudaStream_t s = ctx->stream;
  FEDVR_CK(ctx, launch_conv_coef_bose(M, beta, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                                      P<ConvCoef>(ctx->g_coef), s));
  double *w = P<double>(ctx->g_w);
  if (w_valid) FEDVR_CK(ctx, cudaMemcpyAsync(w, w_io, dsz(stack), cudaMemcpyDeviceToDevice, s));
  const double spin0 = ctx->spin;
  ctx->spin = spin;
  int it = 0;
  int r = gw_solve(ctx, n, M, V, G, Sigma, P<ConvCoef>(ctx->g_coef), w, w_valid != 0,
                   P<double>(ctx->w_t1), P<double>(ctx->w_t2), P<double>(ctx->g_vqv),
                   P<double>(ctx->g_c), P<double>(ctx->g_new), P<unsigned long long>(ctx->g_res),
                   P<double>(ctx->w_dHF), w_mixing, w_tol, w_max_iter, &it);
  ctx->spin = spin0;
  if (r) return r;
  if (w_io) FEDVR_CK(ctx, cudaMemcpyAsync(w_io, w, dsz(stack), cudaMemcpyDeviceToDevice, s));
  if (iters) *iters = it;
  return sync(ctx);
}

int fedvr_sigma_tmatrix(fedvr_ctx *ctx, int n, double beta, int u, int p, double spin,
                        const double *V, const double *G, double *Sigma, double *t_io,
                        int t_valid, double t_mixing, double t_tol, int t_max_iter, int *iters) {
  CHECK_CTX(ctx);
  if (int r = check_mesh_args(ctx, beta, u, p)) return r;
  if (n < 1 || n > 32 || !V || !G || !Sigma || !is_fin(spin) || spin < 0.0)
    return fail(ctx, FEDVR_ERR_ARG, "need 1 <= n <= 32, spin >= 0 and device buffers");
  if (!(t_mixing > 0.0 && t_mixing <= 1.0) || !(t_tol > 0.0) || t_max_iter < 1 ||
      (t_valid && !t_io))
    return fail(ctx, FEDVR_ERR_ARG,
                "the T-matrix needs 0 < t_mixing <= 1, t_tol > 0, t_max_iter >= 1");
  ctx->prepared = false;  // the workspace below is shared with a prepared run
  drop_graph(ctx);
  if (int r = build_mesh(ctx, beta, u, p, false)) return r;
  const int M = 2 * u * p + 1;
  const size_t pstack = (size_t)M * n * n * n * n;
  if (int r = tm_workspace(ctx, n, M)) return r;
  cudaStream_t s = ctx->stream;
  FEDVR_CK(ctx, launch_conv_coef_bose(M, beta, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                                      P<ConvCoef>(ctx->g_coef), s));
  double *t = P<double>(ctx->m_t);
  if (t_valid) FEDVR_CK(ctx, cudaMemcpyAsync(t, t_io, dsz(pstack), cudaMemcpyDeviceToDevice, s));
  const double spin0 = ctx->spin;
  ctx->spin = spin;
  int it = 0;
  int r = tm_solve(ctx, n, M, V, G, Sigma, P<ConvCoef>(ctx->g_coef), t, t_valid != 0,
                   P<double>(ctx->m_src), P<double>(ctx->m_y), P<unsigned long long>(ctx->g_res),
                   t_mixing, t_tol, t_max_iter, &it);
  ctx->spin = spin0;
  if (r) return r;
  if (t_io) FEDVR_CK(ctx, cudaMemcpyAsync(t_io, t, dsz(pstack), cudaMemcpyDeviceToDevice, s));
  if (iters) *iters = it;
  return sync(ctx);
}

int fedvr_set_quadrature(fedvr_ctx *ctx, int order) {
  CHECK_CTX(ctx);
  if (order != 2 && order != 4) return fail(ctx, FEDVR_ERR_ARG, "quadrature order must be 2 or 4");
  ctx->quad_order = order;
  ctx->prepared = false;  // the tables of a prepared run belong to the old rule
  drop_graph(ctx);
  return FEDVR_OK;
}

int fedvr_use_graphs(fedvr_ctx *ctx, int enable, int *last_step_graph) {
  CHECK_CTX(ctx);
  if (last_step_graph) *last_step_graph = ctx->last_step_graph ? 1 : 0;
  if (enable >= 0) {
    ctx->use_graphs = enable != 0;
    if (!ctx->use_graphs) drop_graph(ctx);
  }
  return FEDVR_OK;
}

int fedvr_2b_read(fedvr_ctx *ctx, int out_on_device, double *G_out, double *Sigma_out,
                  double *tau_out) {
  CHECK_CTX(ctx);
  if (!ctx->prepared) return fail(ctx, FEDVR_ERR_STATE, "no prepared second-Born run");
  size_t stack = (size_t)ctx->M * ctx->n * ctx->n;
  bool dev = out_on_device != 0;
  if (G_out) { if (int r = copy_out(ctx, G_out, ctx->w_G.ptr, dsz(stack), dev)) return r; }
  if (Sigma_out) { if (int r = copy_out(ctx, Sigma_out, ctx->w_S.ptr, dsz(stack), dev)) return r; }
  if (tau_out) { if (int r = copy_out(ctx, tau_out, ctx->w_tau.ptr, dsz(ctx->M), dev)) return r; }
  return sync(ctx);
}

int solve_2b(fedvr_ctx *ctx, double beta, int u, int p, double mixing, double tol, int max_iter,
             int precision, int out_on_device, double *G_out, double *Sigma_out, double *tau_out,
             double *E0, double *N_out, int *iters) {
  CHECK_CTX(ctx);
  if (!(mixing > 0.0 && mixing <= 1.0)) return fail(ctx, FEDVR_ERR_ARG, "need 0 < mixing <= 1");
  if (!(tol > 0.0) || max_iter < 1) return fail(ctx, FEDVR_ERR_ARG, "need tol > 0, max_iter >= 1");
  if (int r = fedvr_2b_prepare(ctx, beta, u, p, precision)) return r;
  double E = 0, Nel = 0, res = INFINITY, best = INFINITY;
  int grow = 0, k = 0, status = FEDVR_OK;
  bool conv = false;
  const int inner = ctx->sigma_init_M ? ctx->warm_inner : 0;
  for (k = 0; k < max_iter; ++k) {
    int r = fedvr_2b_step(ctx, mixing, nullptr, 0, &res, &E, &Nel);
    if (r == FEDVR_ERR_NAN) { status = r; break; }
    if (r) return r;
    if (k < inner) continue;  // fixed-Sigma warm-start steps
    if (res < tol) { conv = true; break; }
    if (res < best) { best = res; grow = 0; } else if (++grow >= 8) {
      status = fail(ctx, FEDVR_ERR_DIVERGED, "residual grew for 8 iterations (at %d)", k);
      break;
    }
  }
  int done = (k < max_iter) ? k + 1 : max_iter;
  if (status == FEDVR_OK && !conv)
    status = fail(ctx, FEDVR_ERR_NOCONV, "not converged after %d iterations (res %.3e)", max_iter, res);
  if (int r = fedvr_2b_read(ctx, out_on_device, G_out, Sigma_out, tau_out)) return r;
  ctx->sigma_init_M = 0;
  ctx->warm_inner = 0;
  if (E0) *E0 = E;
  if (N_out) *N_out = Nel;
  if (iters) *iters = done;
  return status;
}

int fedvr_stage_times(const fedvr_ctx *cctx, double *ms, int *launches) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  CHECK_CTX(ctx);
  if (!ms) return fail(ctx, FEDVR_ERR_ARG, "ms must not be NULL");
  if (!ctx->prepared || ctx->step_k == 0) return fail(ctx, FEDVR_ERR_STATE, "no step has run");
  float t;
  for (int i = 0; i < 5; ++i) {
    FEDVR_CK(ctx, cudaEventElapsedTime(&t, ctx->ev[i + 1], ctx->ev[i + 2]));
    ms[i] = t;
  }
  FEDVR_CK(ctx, cudaEventElapsedTime(&t, ctx->ev[0], ctx->ev[6]));
  ms[5] = t;
  if (launches) *launches = ctx->step_launches;
  return FEDVR_OK;
}

int fedvr_get_history(const fedvr_ctx *ctx, double *buf, int cap, int *len) {
  if (!ctx || (cap > 0 && !buf)) return FEDVR_ERR_ARG;
  int count = (int)(ctx->history.size() / 5);
  int m = count < cap ? count : cap;
  if (m > 0) memcpy(buf, ctx->history.data(), sizeof(double) * 5 * m);
  if (len) *len = count;
  return FEDVR_OK;
}

}  // extern "C"

struct fedvr_batch {
  std::vector<fedvr_ctx *> ctxs;
  std::vector<unsigned long long> gens;  // each context's prepare generation at creation
  int Np_max = 16, ld_max = 32;
  size_t off_c = 0, off_px = 0, off_pc = 0, off_err = 0, off_red = 0;
  std::vector<long> px, pc;
  std::vector<int> S;  // measured split count of each system's first convolution
  std::vector<double> hred;
  std::vector<double> best;
  std::vector<int> grow;
  // CUDA graph of one batched iteration for the active set `g_active`, the
  // systems taking a warm-start step `g_warm` and mixing `g_mix`
  cudaGraphExec_t graph = nullptr;
  std::vector<int> g_active, g_warm;
  double g_mix = 0;
  int g_launches = 0;
  ~fedvr_batch() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};


namespace {

// The next step of a prepared context is a warm-start step: the first step
// from an initial Sigma, or one of its fixed-Sigma inner steps.
bool warm_step(const fedvr_ctx *c) {
  return c->sigma_init_M && c->step_k < (c->warm_inner > 0 ? c->warm_inner : 1);
}

// Enqueue one batched iteration of the active systems on s (no host sync).
// Systems in a warm-start step take their Sigma from the initial one (no
// exchange work items) and, in the fixed-Sigma inner steps, the full Dyson
// step (mixing 1).
int enqueue_batch(fedvr_batch *B, const int *active, const int *warm, double mixing,
                  cudaStream_t s, int *launches) {
  fedvr_ctx *lead = B->ctxs[0];
  const int n_sys = (int)B->ctxs.size();
  uint8_t *bt = P<uint8_t>(lead->w_btab);
  int *d_err = reinterpret_cast<int *>(bt + B->off_err);
  const bool f16 = lead->precision == FEDVR_SPLIT_F16;
  for (int k = 0; k < n_sys; ++k)
    if (active[k]) {
      if (int r = phase_sigma_pre(B->ctxs[k], warm[k] != 0, s, launches, d_err)) return r;
    }
  if (B->px[n_sys] > 0) {
    FEDVR_CK(lead, exchange_tc_launch(reinterpret_cast<const XSys *>(bt),
                                      reinterpret_cast<const long *>(bt + B->off_px), n_sys,
                                      B->px[n_sys], B->Np_max, B->ld_max, d_err, lead->num_sms, s,
                                      f16));
    *launches += 1;
  }
  for (int k = 0; k < n_sys; ++k)
    if (active[k]) {
      if (int r = phase_mid(B->ctxs[k], s, launches)) return r;
    }
  FEDVR_CK(lead, conv1_tc_launch(reinterpret_cast<const C1Sys *>(bt + B->off_c),
                                 reinterpret_cast<const long *>(bt + B->off_pc), n_sys,
                                 B->pc[n_sys], B->Np_max, d_err, lead->num_sms, s, f16));
  *launches += 1;
  for (int k = 0; k < n_sys; ++k)
    if (active[k]) {
      fedvr_ctx *c = B->ctxs[k];
      if (B->S[k] > 1) {  // this system's partial stacks into its I1, in a fixed order
        FEDVR_CK(lead, conv1_sum_splits((long)c->M * c->n * c->n, B->S[k] - 1,
                                        P<double>(c->w_c1p), P<double>(c->w_I1), s));
        *launches += 1;
      }
      if (int r = phase_conv2(c, s, launches, d_err)) return r;
      const double mix = (warm[k] && c->warm_inner > 0) ? 1.0 : mixing;
      if (int r = phase_update(c, mix, s, launches)) return r;
      FEDVR_CK(lead, cudaMemcpyAsync(bt + B->off_red + (size_t)k * 3 * sizeof(double),
                                     c->w_red.ptr, 3 * sizeof(double), cudaMemcpyDeviceToDevice,
                                     s));
    }
  return FEDVR_OK;
}

// Capture enqueue_batch into B->graph on the lead context's private stream;
// a refused capture leaves the batch running eagerly (not an error).
int capture_batch(fedvr_batch *B, const int *active, const int *warm, double mixing) {
  fedvr_ctx *lead = B->ctxs[0];
  const int n_sys = (int)B->ctxs.size();
  if (!lead->cap_stream &&
      cudaStreamCreateWithFlags(&lead->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    lead->cap_stream = nullptr;
    return FEDVR_OK;
  }
  cudaStream_t cs = lead->cap_stream;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return FEDVR_OK;
  }
  int launches = 0;
  const int r = enqueue_batch(B, active, warm, mixing, cs, &launches);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  cudaGraphExec_t exec = nullptr;
  if (r == FEDVR_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (r != FEDVR_OK || e != cudaSuccess || !exec) {
    cudaGetLastError();
    for (fedvr_ctx *c : B->ctxs) {  // clear what the refused capture recorded
      c->failed = false;
      c->err[0] = 0;
    }
    return FEDVR_OK;
  }
  B->graph = exec;
  B->g_active.assign(active, active + n_sys);
  B->g_warm.assign(warm, warm + n_sys);
  B->g_mix = mixing;
  B->g_launches = launches;
  return FEDVR_OK;
}

// Write each system's first-convolution descriptor with split count
// min(S, its block count) (partial stacks in the context's w_c1p) and the
// batch's conv1 work-queue prefix for all systems active.
int batch_c1_tables(fedvr_batch *B, std::vector<C1Sys> &hc, int S) {
  fedvr_ctx *lead = B->ctxs[0];
  const int n_sys = (int)B->ctxs.size();
  const bool f16 = lead->precision == FEDVR_SPLIT_F16;
  uint8_t *bt = P<uint8_t>(lead->w_btab);
  cudaStream_t s = lead->stream;
  B->pc[0] = 0;
  for (int k = 0; k < n_sys; ++k) {
    fedvr_ctx *c = B->ctxs[k];
    const int NB = conv1_blocks(c->n, c->M, f16);
    const int Sk = S < NB ? S : NB;
    const size_t stack = (size_t)c->M * c->n * c->n;
    if (Sk > 1) ENSURE(c, w_c1p, dsz((size_t)(Sk - 1) * stack));
    hc[k].S = Sk;
    hc[k].part = Sk > 1 ? P<double>(c->w_c1p) : nullptr;
    B->S[k] = Sk;
    B->pc[k + 1] = B->pc[k] + conv1_items(c->n, c->M, Sk);
  }
  FEDVR_CK(lead, cudaMemcpyAsync(bt + B->off_c, hc.data(), n_sys * sizeof(C1Sys),
                                 cudaMemcpyHostToDevice, s));
  FEDVR_CK(lead, cudaMemcpyAsync(bt + B->off_pc, B->pc.data(), (n_sys + 1) * sizeof(long),
                                 cudaMemcpyHostToDevice, s));
  return sync(lead);  // the host tables may change right after
}

// Measured split count of the batch's first convolution: the batched launch
// (and the split sums) timed on the prepared buffers for S in {1, 2, 3, 4}
// (each system capped at its own block count; every choice gives the same
// FP32 block sums, see fedvr_conv1_splits), keeping the fastest (a larger S
// must win by 3 %). A batch whose work queue already fills the GPU several
// times over keeps S = 1 without timing; a split request on the lead context
// (fedvr_conv1_splits) is taken as is.
int tune_batch_splits(fedvr_batch *B, std::vector<C1Sys> &hc) {
  fedvr_ctx *lead = B->ctxs[0];
  const int n_sys = (int)B->ctxs.size();
  const bool f16 = lead->precision == FEDVR_SPLIT_F16;
  long items1 = 0;
  for (fedvr_ctx *c : B->ctxs) items1 += conv1_items(c->n, c->M, 1);
  int best = 1;
  if (lead->c1_request > 0) {  // an explicit request on the lead context: no timing
    for (int S : {1, 2, 3, 4})
      if (S <= lead->c1_request) best = S;
  } else if (items1 < 4L * lead->num_sms) {
    uint8_t *bt = P<uint8_t>(lead->w_btab);
    int *d_err = reinterpret_cast<int *>(bt + B->off_err);
    cudaStream_t s = lead->stream;
    float best_ms = 0.f;
    for (int S : {1, 2, 3, 4}) {
      if (int r = batch_c1_tables(B, hc, S)) return r;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // a warm-up launch, then the timed one
        FEDVR_CK(lead, cudaEventRecord(lead->ev[0], s));
        FEDVR_CK(lead, conv1_tc_launch(reinterpret_cast<const C1Sys *>(bt + B->off_c),
                                       reinterpret_cast<const long *>(bt + B->off_pc), n_sys,
                                       B->pc[n_sys], B->Np_max, d_err, lead->num_sms, s, f16));
        for (int k = 0; k < n_sys; ++k) {
          fedvr_ctx *c = B->ctxs[k];
          if (B->S[k] > 1)
            FEDVR_CK(lead, conv1_sum_splits((long)c->M * c->n * c->n, B->S[k] - 1,
                                            P<double>(c->w_c1p), P<double>(c->w_I1), s));
        }
        FEDVR_CK(lead, cudaEventRecord(lead->ev[6], s));
        int h_err = 0;
        FEDVR_CK(lead, cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        if (int r = sync(lead)) return r;
        if (int r = flag_status(lead, h_err, d_err)) return r;
        FEDVR_CK(lead, cudaEventElapsedTime(&ms, lead->ev[0], lead->ev[6]));
      }
      if (S == 1 || ms < 0.97f * best_ms) {
        best = S;
        best_ms = ms;
      }
    }
  }
  return batch_c1_tables(B, hc, best);
}

}  // namespace

extern "C" {

int fedvr_batch_create(fedvr_batch **out, fedvr_ctx **ctxs, int n_sys, const double *beta,
                       const int *u, const int *p, int precision) {
  if (!out) return FEDVR_ERR_ARG;
  *out = nullptr;
  if (!ctxs || n_sys < 1 || n_sys > 4096 || !beta || !u || !p) return FEDVR_ERR_ARG;
  for (int k = 0; k < n_sys; ++k) {
    if (!ctxs[k]) return FEDVR_ERR_ARG;
    if (ctxs[k]->failed) return FEDVR_ERR_STATE;
  }
  fedvr_ctx *lead = ctxs[0];
  if (!is_split(precision))
    return fail(lead, FEDVR_ERR_ARG, "the batched solve runs a split-precision tensor-core path");
  for (int k = 0; k < n_sys; ++k) {
    if (ctxs[k]->device != lead->device)
      return fail(lead, FEDVR_ERR_ARG, "all systems must be on one device");
    for (int q = 0; q < k; ++q)
      if (ctxs[q] == ctxs[k]) return fail(lead, FEDVR_ERR_ARG, "a context appears twice");
  }
  fedvr_batch *B = new (std::nothrow) fedvr_batch();
  if (!B) return fail(lead, FEDVR_ERR_ARG, "out of host memory");
  B->ctxs.assign(ctxs, ctxs + n_sys);
  cudaStream_t s = lead->stream;
  for (int k = 0; k < n_sys; ++k) {
    if (int r = fedvr_2b_prepare(ctxs[k], beta[k], u[k], p[k], precision)) {
      fail(lead, r, "system %d: %s", k, ctxs[k]->err);
      delete B;
      return r;
    }
    const TcGeom g = tc_geom(ctxs[k]->n, ctxs[k]->M);
    B->Np_max = g.Np > B->Np_max ? g.Np : B->Np_max;
    B->ld_max = g.ld > B->ld_max ? g.ld : B->ld_max;
  }
  for (int k = 0; k < n_sys; ++k) B->gens.push_back(ctxs[k]->prep_gen);
  if (tc_smem_bytes(B->Np_max, B->ld_max, true) > 232448) {
    delete B;
    return fail(lead, FEDVR_ERR_ARG, "batch too wide for one shared-memory stage layout");
  }
  const size_t xs = (size_t)n_sys * sizeof(XSys), cs = (size_t)n_sys * sizeof(C1Sys);
  const size_t pfx = ((size_t)(n_sys + 1) * sizeof(long) + 255) / 256 * 256;
  B->off_c = (xs + 255) / 256 * 256;
  B->off_px = B->off_c + (cs + 255) / 256 * 256;
  B->off_pc = B->off_px + pfx;
  B->off_err = B->off_pc + pfx;
  B->off_red = B->off_err + 256;
  if (!ensure(lead, lead->w_btab, B->off_red + (size_t)n_sys * 3 * sizeof(double), "w_btab")) {
    delete B;
    return FEDVR_ERR_CUDA;
  }
  uint8_t *bt = P<uint8_t>(lead->w_btab);
  std::vector<XSys> hx(n_sys);
  std::vector<C1Sys> hc(n_sys);
  for (int k = 0; k < n_sys; ++k) {
    fedvr_ctx *c = ctxs[k];
    float *ws, *S32;
    int *err;
    if (int r = tc_workspace(c, c->n, c->M, &ws, &S32, &err)) {
      delete B;
      return r;
    }
    memset(&hx[k], 0, sizeof(XSys));
    memset(&hc[k], 0, sizeof(C1Sys));
    void *h16 = nullptr;
    TcScale *scale = nullptr;
    if (precision == FEDVR_SPLIT_F16) {
      if (int r = f16_workspace(c, c->n, c->M, &h16, &scale)) {
        delete B;
        return r;
      }
    }
    if (int r = ensure_xrows(c, c->n)) {
      delete B;
      return r;
    }
    cudaError_t e = xsys_fill(&hx[k], c->n, c->M, c->spin, ws, P<double>(c->w_S), S32,
                              P<uint32_t>(c->w_xrow), scale ? &scale->maxS : nullptr, h16, scale);
    if (e == cudaSuccess)
      e = c1sys_fill(&hc[k], c->n, c->M, 1, ws, S32, P<double>(c->w_dHF),
                     P<int4>(c->w_coef32), P<double>(c->w_I1), nullptr, h16, scale);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt + k * sizeof(XSys), &hx[k], sizeof(XSys),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bt + B->off_c + k * sizeof(C1Sys), &hc[k],
                                              sizeof(C1Sys), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      delete B;
      return cuda_fail(lead, e, "batch tables", __FILE__, __LINE__);
    }
  }
  if (cudaMemsetAsync(bt + B->off_err, 0, sizeof(int), s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    delete B;
    return cuda_fail(lead, cudaGetLastError(), "batch tables", __FILE__, __LINE__);
  }
  B->px.assign(n_sys + 1, 0);
  B->pc.assign(n_sys + 1, 0);
  B->S.assign(n_sys, 1);
  B->hred.assign(3 * (size_t)n_sys, 0.0);
  B->best.assign(n_sys, INFINITY);
  B->grow.assign(n_sys, 0);
  if (int r = tune_batch_splits(B, hc)) {
    delete B;
    return r;
  }
  *out = B;
  return FEDVR_OK;
}

void fedvr_batch_destroy(fedvr_batch *b) { delete b; }

int fedvr_batch_step(fedvr_batch *B, double mixing, double tol, int *active, double *res_out,
                     double *E0, double *N_out) {
  if (!B || !active) return FEDVR_ERR_ARG;
  fedvr_ctx *lead = B->ctxs[0];
  CHECK_CTX(lead);
  if (!(mixing > 0.0 && mixing <= 1.0)) return fail(lead, FEDVR_ERR_ARG, "need 0 < mixing <= 1");
  const int n_sys = (int)B->ctxs.size();
  cudaStream_t s = lead->stream;
  uint8_t *bt = P<uint8_t>(lead->w_btab);
  auto t0 = std::chrono::steady_clock::now();
  B->px[0] = B->pc[0] = 0;
  std::vector<int> warm(n_sys, 0);
  for (int k = 0; k < n_sys; ++k) {
    const fedvr_ctx *c = B->ctxs[k];
    if (!c->prepared || c->prep_gen != B->gens[k])
      return fail(lead, FEDVR_ERR_STATE, "system %d was re-prepared or released after the batch was made",
                  k);
    warm[k] = active[k] && warm_step(c);
    B->px[k + 1] = B->px[k] + ((active[k] && !warm[k]) ? exchange_items(c->n, c->M) : 0);
    B->pc[k + 1] = B->pc[k] + (active[k] ? conv1_items(c->n, c->M, B->S[k]) : 0);
  }
  if (B->pc[n_sys] == 0) return FEDVR_OK;
  FEDVR_CK(lead, cudaMemcpyAsync(bt + B->off_px, B->px.data(), (n_sys + 1) * sizeof(long),
                                 cudaMemcpyHostToDevice, s));
  FEDVR_CK(lead, cudaMemcpyAsync(bt + B->off_pc, B->pc.data(), (n_sys + 1) * sizeof(long),
                                 cudaMemcpyHostToDevice, s));
  int *d_err = reinterpret_cast<int *>(bt + B->off_err);
  int launches = 0;
  // one iteration of the whole batch: replayed from a CUDA graph captured for
  // this active set and mixing, or launched eagerly
  const std::vector<int> act(active, active + n_sys);
  if (lead->use_graphs &&
      (!B->graph || B->g_active != act || B->g_warm != warm || B->g_mix != mixing)) {
    if (B->graph) {
      cudaGraphExecDestroy(B->graph);
      B->graph = nullptr;
    }
    if (int r = capture_batch(B, active, warm.data(), mixing)) return r;
  }
  if (B->graph && lead->use_graphs) {
    FEDVR_CK(lead, cudaGraphLaunch(B->graph, s));
    launches = B->g_launches;
    lead->last_step_graph = true;
  } else {
    if (int r = enqueue_batch(B, active, warm.data(), mixing, s, &launches)) return r;
    lead->last_step_graph = false;
  }
  FEDVR_CK(lead, cudaMemcpyAsync(B->hred.data(), bt + B->off_red, B->hred.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, s));
  int h_err = 0;
  FEDVR_CK(lead, cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (int r = sync(lead)) return r;
  if (h_err & 2) {  // a non-finite iterate also trips the FP16 range check
    bool nonfinite = false;
    for (int k = 0; k < n_sys; ++k) {
      const double E = B->hred[3 * k], r = B->hred[3 * k + 2];
      if (active[k] && (r != r || !is_fin(E))) nonfinite = true;
    }
    if (nonfinite && !(h_err & 1)) {
      FEDVR_CK(lead, cudaMemsetAsync(d_err, 0, sizeof(int), s));
      h_err = 0;
    }
  }
  if (int r = flag_status(lead, h_err, d_err)) return r;
  const double ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  lead->step_launches = launches;
  int worst = FEDVR_OK;
  for (int k = 0; k < n_sys; ++k) {
    if (!active[k]) continue;
    fedvr_ctx *c = B->ctxs[k];
    const double E = B->hred[3 * k], Nel = B->hred[3 * k + 1], r = B->hred[3 * k + 2];
    double rec[5] = {(double)c->step_k, r, E, Nel, ms};
    c->history.insert(c->history.end(), rec, rec + 5);
    c->step_k++;
    if (res_out) res_out[k] = r;
    if (E0) E0[k] = E;
    if (N_out) N_out[k] = Nel;
    if (r != r || !is_fin(E)) {
      worst = fail(c, FEDVR_ERR_NAN, "NaN/Inf at iteration %d", c->step_k - 1);
      active[k] = 0;
    } else if (tol > 0.0 && r < tol && !(warm[k] && c->warm_inner > 0)) {
      active[k] = 0;  // no convergence test in the fixed-Sigma warm-start steps
    }
  }
  return worst;
}

int solve_2b_batched(fedvr_ctx **ctxs, int n_sys, const double *beta, const int *u, const int *p,
                     double mixing, double tol, int max_iter, int precision, double *E0,
                     double *N_out, int *iters) {
  if (!ctxs || n_sys < 1) return FEDVR_ERR_ARG;
  if (!(mixing > 0.0 && mixing <= 1.0) || !(tol > 0.0) || max_iter < 1)
    return ctxs[0] ? fail(ctxs[0], FEDVR_ERR_ARG, "need 0 < mixing <= 1, tol > 0, max_iter >= 1")
                   : FEDVR_ERR_ARG;
  fedvr_batch *B = nullptr;
  if (int r = fedvr_batch_create(&B, ctxs, n_sys, beta, u, p, precision)) return r;
  std::vector<int> active(n_sys, 1), status(n_sys, FEDVR_OK), done(n_sys, 0);
  std::vector<double> res(n_sys, INFINITY), best(n_sys, INFINITY), e(n_sys, 0.0), nn(n_sys, 0.0);
  std::vector<int> grow(n_sys, 0);
  for (int it = 0; it < max_iter; ++it) {
    int remaining = 0;
    for (int k = 0; k < n_sys; ++k) remaining += active[k] != 0;
    if (!remaining) break;
    std::vector<int> was(active), inner(n_sys, 0);
    for (int k = 0; k < n_sys; ++k)  // fixed-Sigma warm-start steps: no divergence watch
      inner[k] = ctxs[k]->sigma_init_M && ctxs[k]->warm_inner > 0 &&
                 ctxs[k]->step_k < ctxs[k]->warm_inner;
    int r = fedvr_batch_step(B, mixing, tol, active.data(), res.data(), e.data(), nn.data());
    if (r != FEDVR_OK && r != FEDVR_ERR_NAN) {
      fedvr_batch_destroy(B);
      return r;
    }
    for (int k = 0; k < n_sys; ++k) {
      if (!was[k]) continue;
      done[k] = it + 1;
      if (E0) E0[k] = e[k];
      if (N_out) N_out[k] = nn[k];
      if (res[k] != res[k]) {
        status[k] = FEDVR_ERR_NAN;
      } else if (active[k] && !inner[k]) {  // still running: watch for a growing residual
        if (res[k] < best[k]) {
          best[k] = res[k];
          grow[k] = 0;
        } else if (++grow[k] >= 8) {
          status[k] = fail(ctxs[k], FEDVR_ERR_DIVERGED, "residual grew for 8 iterations (at %d)",
                           it);
          active[k] = 0;
        }
      }
    }
  }
  fedvr_batch_destroy(B);
  int worst = FEDVR_OK;
  for (int k = 0; k < n_sys; ++k) {
    ctxs[k]->sigma_init_M = 0;  // a warm start serves one solve, as in solve_2b
    ctxs[k]->warm_inner = 0;
    if (active[k])
      status[k] = fail(ctxs[k], FEDVR_ERR_NOCONV, "not converged after %d iterations", max_iter);
    if (iters) iters[k] = done[k];
    if (status[k] < worst) worst = status[k];
  }
  return worst;
}

int fedvr_power_mesh(fedvr_ctx *ctx, double beta, int u, int p, double *tau, double *w,
                     double *wm, double *wp, int *lag_k, double *lag_t) {
  CHECK_CTX(ctx);
  if (int r = check_mesh_args(ctx, beta, u, p)) return r;
  if ((lag_k == nullptr) != (lag_t == nullptr))
    return fail(ctx, FEDVR_ERR_ARG, "lag_k and lag_t go together");
  ctx->prepared = false;
  if (int r = build_mesh(ctx, beta, u, p, false)) return r;
  int M = 2 * u * p + 1;
  cudaStream_t s = ctx->stream;
  if (lag_k)
    FEDVR_CK(ctx, launch_mesh(beta, u, p, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                              P<double>(ctx->w_wm), P<double>(ctx->w_wp), lag_k, lag_t, s));
  if (tau) FEDVR_CK(ctx, cudaMemcpyAsync(tau, ctx->w_tau.ptr, dsz(M), cudaMemcpyDeviceToDevice, s));
  if (w) FEDVR_CK(ctx, cudaMemcpyAsync(w, ctx->w_w.ptr, dsz(M), cudaMemcpyDeviceToDevice, s));
  if (wm) FEDVR_CK(ctx, cudaMemcpyAsync(wm, ctx->w_wm.ptr, dsz(M), cudaMemcpyDeviceToDevice, s));
  if (wp) FEDVR_CK(ctx, cudaMemcpyAsync(wp, ctx->w_wp.ptr, dsz(M), cudaMemcpyDeviceToDevice, s));
  return FEDVR_OK;
}

int fedvr_sigma2(fedvr_ctx *ctx, int n, int M, double spin, const double *V, const double *G,
                 double *Sigma, int precision) {
  CHECK_CTX(ctx);
  if (n < 1 || n > 1024 || M < 1 || M > 4097 || !V || !G || !Sigma)
    return fail(ctx, FEDVR_ERR_ARG, "need 1 <= n <= 1024, 1 <= M <= 4097 and device buffers");
  if (!is_fin(spin) || spin < 0.0)
    return fail(ctx, FEDVR_ERR_ARG, "spin factor must be finite and non-negative");
  if (int r = check_precision(ctx, precision, n)) return r;
  ctx->prepared = false;  // the workspace below is shared with a prepared run
  if (is_split(precision)) {
    ctx->precision = precision;
    const bool f16 = precision == FEDVR_SPLIT_F16;
    float *ws, *S32;
    int *err;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &err)) return r;
    cudaStream_t s = ctx->stream;
    FEDVR_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
    if (f16) {  // operand scales from this V, and the FP16 split of G for the gb operand
      void *h16;
      TcScale *scale;
      if (int r = f16_workspace(ctx, n, M, &h16, &scale)) return r;
      FEDVR_CK(ctx, launch_scale_init(0, nullptr, n, V, scale, s));
      FEDVR_CK(ctx, launch_split_f16(n, M, G, h16, s, err, ws));
    }
    if (int r = upload_single_tables(ctx, n, M, ws, Sigma, nullptr, nullptr, nullptr, nullptr, 1,
                                     nullptr, spin))
      return r;
    FEDVR_CK(ctx, sigma2_tc_pre(n, M, V, G, ws, s, !f16, err, f16));
    const TcGeom g = tc_geom(n, M);
    uint8_t *tab = P<uint8_t>(ctx->w_tab);
    FEDVR_CK(ctx, exchange_tc_launch(reinterpret_cast<const XSys *>(tab + kTabX),
                                     reinterpret_cast<const long *>(tab + kTabPX), 1,
                                     exchange_items(n, M), g.Np, g.ld, err, ctx->num_sms, s,
                                     f16));
    int h_err = 0;
    FEDVR_CK(ctx, cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (int r = sync(ctx)) return r;
    return flag_status(ctx, h_err, err);
  }
  size_t stack = (size_t)M * n * n;
  ENSURE(ctx, w_t1, dsz(stack));
  ENSURE(ctx, w_t2, dsz(stack));
  ENSURE(ctx, w_t3, dsz(stack));
  FEDVR_CK(ctx, sigma2_fp64(n, M, spin, V, G, Sigma, P<double>(ctx->w_t1), P<double>(ctx->w_t2),
                            P<double>(ctx->w_t3), ctx->stream));
  return FEDVR_OK;
}

int fedvr_conv_sigma_g(fedvr_ctx *ctx, int n, double beta, int u, int p, const double *dHF,
                       const double *Sigma, const double *G, double *I1, int precision) {
  CHECK_CTX(ctx);
  if (int r = check_mesh_args(ctx, beta, u, p)) return r;
  if (n < 1 || n > 1024 || !dHF || !Sigma || !G || !I1)
    return fail(ctx, FEDVR_ERR_ARG, "need 1 <= n <= 1024 and device buffers");
  if (int r = check_precision(ctx, precision, n)) return r;
  if (int r = check_quad(ctx, precision, 2 * u * p + 1)) return r;
  ctx->prepared = false;  // the workspace below is shared with a prepared run
  if (int r = build_mesh(ctx, beta, u, p, true)) return r;
  int M = 2 * u * p + 1;
  if (is_split(precision)) {
    ctx->precision = precision;
    float *ws, *S32;
    int *err;
    if (int r = tc_workspace(ctx, n, M, &ws, &S32, &err)) return r;
    const size_t tstack = (size_t)M * n * ((n + 31) / 32 * 32);
    cudaStream_t s = ctx->stream;
    FEDVR_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
    void *h16 = nullptr;
    TcScale *scale = nullptr;
    const bool f16 = precision == FEDVR_SPLIT_F16;
    // work split of the mesh-point range: the request of fedvr_conv1_splits
    // (largest candidate not above it, whole accumulation blocks), else none
    int S = 1;
    if (ctx->c1_request > 1) {
      const int NB = conv1_blocks(n, M, f16);
      for (int c : {2, 3, 4, 6, 8, 12, 16})
        if (c <= ctx->c1_request && c <= NB) S = c;
    }
    const size_t stack = (size_t)M * n * n;
    if (S > 1) ENSURE(ctx, w_c1p, dsz((size_t)(S - 1) * stack));
    if (f16) {
      if (int r = f16_workspace(ctx, n, M, &h16, &scale)) return r;
      FEDVR_CK(ctx, launch_scale_init(M, P<int4>(ctx->w_coef32), 0, nullptr, scale, s));
      FEDVR_CK(ctx, launch_split_f16(n, M, G, h16, s, err));
    }
    if (int r = upload_single_tables(ctx, n, M, ws, nullptr, S32, dHF, P<ConvCoef>(ctx->w_coef), I1,
                                     S, S > 1 ? P<double>(ctx->w_c1p) : nullptr))
      return r;
    if (!f16) FEDVR_CK(ctx, launch_split_g(n, M, G, ws, ws + tstack, ws + 2 * tstack, s));
    FEDVR_CK(ctx, launch_sigma_to_f32(n, M, Sigma, S32, s, f16 ? &scale->maxS : nullptr));
    FEDVR_CK(ctx, launch_diag_f32(n, M, dHF, Sigma, P<double>(ctx->w_wm), P<double>(ctx->w_wp),
                                  S32, s, f16 ? &scale->maxS : nullptr));
    const TcGeom g = tc_geom(n, M);
    uint8_t *tab = P<uint8_t>(ctx->w_tab);
    FEDVR_CK(ctx, conv1_tc_launch(reinterpret_cast<const C1Sys *>(tab + kTabC),
                                  reinterpret_cast<const long *>(tab + kTabPC), 1,
                                  conv1_items(n, M, S), g.Np, err, ctx->num_sms, s, f16));
    if (S > 1) FEDVR_CK(ctx, conv1_sum_splits((long)stack, S - 1, P<double>(ctx->w_c1p), I1, s));
    ctx->c1_splits = S;
    int h_err = 0;
    FEDVR_CK(ctx, cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (int r = sync(ctx)) return r;
    return flag_status(ctx, h_err, err);
  }
  if (ctx->quad_order == 4) {
    if (int r = check_quad(ctx, precision, M)) return r;
    if (int r = build_quad4(ctx, M, beta)) return r;
    if (int r = ensure_c1f(ctx, n, M)) return r;
    FEDVR_CK(ctx, conv1_fp64_q4(n, M, P<ConvCoef4>(ctx->w_q4coef), dHF, Sigma, G, I1, ctx->stream,
                                P<double>(ctx->w_c1f)));
    return FEDVR_OK;
  }
  if (int r = ensure_c1f(ctx, n, M)) return r;
  FEDVR_CK(ctx, conv1_fp64(n, M, P<ConvCoef>(ctx->w_coef), dHF, Sigma, G, I1, ctx->stream,
                           P<double>(ctx->w_c1f)));
  return FEDVR_OK;
}

int fedvr_conv_g0(fedvr_ctx *ctx, int n, double beta, int u, int p, const double *eps,
                  const double *C, double mu, const double *I1, double *I2, int precision) {
  CHECK_CTX(ctx);
  if (int r = check_mesh_args(ctx, beta, u, p)) return r;
  if (n < 1 || n > 1024 || !eps || !C || !I1 || !I2 || !is_fin(mu))
    return fail(ctx, FEDVR_ERR_ARG, "need 1 <= n <= 1024, finite mu and device buffers");
  if (int r = check_precision(ctx, precision, n)) return r;
  ctx->prepared = false;
  if (int r = build_mesh(ctx, beta, u, p, false)) return r;
  int M = 2 * u * p + 1;
  size_t stack = (size_t)M * n * n;
  ENSURE(ctx, w_K, dsz((size_t)n * M * M));
  ENSURE(ctx, w_t1, dsz(stack));
  ENSURE(ctx, w_t2, dsz(stack));
  cudaStream_t s = ctx->stream;
  if (int r = check_quad(ctx, precision, M)) return r;
  const bool q4 = ctx->quad_order == 4;
  if (q4) {
    if (int r = build_quad4(ctx, M, beta)) return r;
  }
  const double *qw = q4 ? P<double>(ctx->w_q4w) : nullptr;
  FEDVR_CK(ctx, launch_conv2_kernel(n, M, beta, P<double>(ctx->w_tau), P<double>(ctx->w_w),
                                    q4 ? qw : P<double>(ctx->w_wm), q4 ? qw + M : P<double>(ctx->w_wp),
                                    eps, nullptr, mu, P<double>(ctx->w_K), s,
                                    q4 ? P<double>(ctx->w_q4W) : nullptr));
  if (is_split(precision)) {  // the split path's products: FP32 table, split TF32 / FP32 GEMMs
    ENSURE(ctx, w_K32, (size_t)n * M * M * sizeof(float));
    ENSURE(ctx, w_red, dsz(8));
    int *err = reinterpret_cast<int *>(P<double>(ctx->w_red) + 7);
    FEDVR_CK(ctx, cudaMemsetAsync(err, 0, sizeof(int), s));
    FEDVR_CK(ctx, launch_to_f32((size_t)n * M * M, P<double>(ctx->w_K), P<float>(ctx->w_K32), s));
    FEDVR_CK(ctx, conv2_apply_f32(n, M, P<float>(ctx->w_K32), C, I1, I2, P<float>(ctx->w_t1),
                                  P<float>(ctx->w_t2), err, s));
    int h_err = 0;
    FEDVR_CK(ctx, cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (int r = sync(ctx)) return r;
    return flag_status(ctx, h_err, err);
  }
  FEDVR_CK(ctx, conv2_apply(n, M, P<double>(ctx->w_K), C, I1, I2, P<double>(ctx->w_t1),
                            P<double>(ctx->w_t2), s));
  return FEDVR_OK;
}

int fedvr_selftest_wait(fedvr_ctx *ctx, int release, double limit_seconds) {
  CHECK_CTX(ctx);
  if (!(limit_seconds >= 1e-6 && limit_seconds <= 1.0))
    return fail(ctx, FEDVR_ERR_ARG, "limit_seconds must lie in [1e-6, 1]");
  ENSURE(ctx, b_scal, dsz(16));
  int *flag = reinterpret_cast<int *>(P<double>(ctx->b_scal) + 10);
  cudaStream_t s = ctx->stream;
  FEDVR_CK(ctx, cudaMemsetAsync(flag, 0, sizeof(int), s));
  FEDVR_CK(ctx, launch_wait_probe(release != 0, (unsigned long long)(limit_seconds * 1e9), flag, s));
  int h_err = 0;
  FEDVR_CK(ctx, cudaMemcpyAsync(&h_err, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (int r = sync(ctx)) return r;
  return flag_status(ctx, h_err, flag);
}

}  // extern "C"
