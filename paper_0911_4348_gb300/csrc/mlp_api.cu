// C ABI of the learned warm start (network object, data collection,
// training, prediction). The paper has no learned component; see mlp.cu.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "mlp.cuh"

struct fedvr_mlp {
  int M = 0, H = 0;
  fedvr::MlpNet L;
  cudaStream_t stream = nullptr;
  int device = 0;
  char err[640] = {0};
  bool failed = false;
  int adam_t = 0;
  long rows = 0, cap = 0;  // training rows held / capacity
  unsigned long long seed = 0;
  fedvr::DevBuf W, m, v, g, Wbf, act, Y, dbuf, part, X, T, idx, bX, bT, sdev, F, S1;
};

namespace {

using fedvr::DevBuf;
using fedvr::P;

int mfail(fedvr_mlp *m, int code, const char *what) {
  if (m) snprintf(m->err, sizeof(m->err), "%s", what);
  return code;
}

int mcuda(fedvr_mlp *m, cudaError_t e, const char *what, int line) {
  if (m) {
    m->failed = true;
    snprintf(m->err, sizeof(m->err), "CUDA error %d (%s) in %s at mlp_api.cu:%d", (int)e,
             cudaGetErrorString(e), what, line);
  }
  return FEDVR_ERR_CUDA;
}

#define MCK(m, call)                                       \
  do {                                                     \
    cudaError_t e__ = (call);                              \
    if (e__ != cudaSuccess) return mcuda((m), e__, #call, __LINE__); \
  } while (0)

bool mensure(fedvr_mlp *m, DevBuf &b, size_t bytes) {
  if (b.bytes >= bytes) return true;
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.ptr, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    b.ptr = nullptr;
    mfail(m, FEDVR_ERR_CUDA, "cudaMalloc failed");
    m->failed = true;
    return false;
  }
  b.bytes = bytes;
  return true;
}

// Grow a device buffer keeping its first `keep` bytes.
bool mgrow(fedvr_mlp *m, DevBuf &b, size_t bytes, size_t keep) {
  if (b.bytes >= bytes) return true;
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    mfail(m, FEDVR_ERR_CUDA, "cudaMalloc failed");
    m->failed = true;
    return false;
  }
  if (keep && b.ptr) cudaMemcpy(p, b.ptr, keep, cudaMemcpyDeviceToDevice);
  if (b.ptr) cudaFree(b.ptr);
  b.ptr = p;
  b.bytes = bytes;
  return true;
}

#define MENSURE(m, buf, bytes)                                      \
  do {                                                              \
    if (!mensure((m), (m)->buf, (bytes))) return FEDVR_ERR_CUDA;    \
  } while (0)

uint64_t splitmix(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double uniform01(uint64_t &x) { return ((splitmix(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

// scratch for `rows` rows
int ensure_rows(fedvr_mlp *m, int rows) {
  const fedvr::MlpNet &L = m->L;
  const int wide = L.H > L.dout ? L.H : L.dout;
  MENSURE(m, act, (size_t)4 * rows * L.H * sizeof(float));
  MENSURE(m, Y, (size_t)rows * L.dout * sizeof(float));
  MENSURE(m, dbuf, (size_t)2 * rows * wide * sizeof(float));
  MENSURE(m, part, 256 * sizeof(double));
  return FEDVR_OK;
}

double read_loss(fedvr_mlp *m, int *status) {
  double h[256];
  if (cudaMemcpyAsync(h, m->part.ptr, sizeof(h), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    *status = mcuda(m, cudaGetLastError(), "loss readback", __LINE__);
    return 0.0;
  }
  double s = 0.0;
  for (int i = 0; i < 256; ++i) s += h[i];
  *status = FEDVR_OK;
  return s;
}

}  // namespace

extern "C" {

int fedvr_mlp_create(fedvr_mlp **out, int M, int hidden, unsigned long long seed, void *stream) {
  if (!out) return FEDVR_ERR_ARG;
  *out = nullptr;
  if (M < 3 || M > 4097 || hidden < 8 || hidden > 4096) return FEDVR_ERR_ARG;
  fedvr_mlp *m = new (std::nothrow) fedvr_mlp();
  if (!m) return FEDVR_ERR_ARG;
  m->M = M;
  m->H = hidden;
  m->L = fedvr::mlp_layout(M, hidden);
  m->stream = reinterpret_cast<cudaStream_t>(stream);
  m->seed = seed;
  cudaGetDevice(&m->device);
  const fedvr::MlpNet &L = m->L;
  const size_t pb = (size_t)L.nparam * sizeof(float);
  if (!mensure(m, m->W, pb) || !mensure(m, m->m, pb) || !mensure(m, m->v, pb) ||
      !mensure(m, m->g, pb) || !mensure(m, m->Wbf, (size_t)L.nparam * 2) ||
      !mensure(m, m->sdev, 64)) {
    fedvr_mlp_destroy(m);
    return FEDVR_ERR_CUDA;
  }
  // He-normal weights (Box-Muller on splitmix64), zero biases
  std::vector<float> w((size_t)L.nparam, 0.f);
  uint64_t st = seed;
  auto fill = [&](long off, long count, int fan_in) {
    const double sd = sqrt(2.0 / fan_in);
    for (long i = 0; i < count; ++i) {
      const double u1 = uniform01(st), u2 = uniform01(st);
      w[off + i] = (float)(sd * sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
  };
  fill(L.o_W1, (long)L.din * L.H, L.din);
  fill(L.o_W2, (long)L.H * L.H, L.H);
  fill(L.o_W3, (long)L.H * L.dout, L.H);
  if (cudaMemcpy(m->W.ptr, w.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m.ptr, 0, pb) != cudaSuccess || cudaMemset(m->v.ptr, 0, pb) != cudaSuccess ||
      fedvr::mlp_to_bf16(L.nparam, P<float>(m->W), m->Wbf.ptr, m->stream) != cudaSuccess ||
      cudaStreamSynchronize(m->stream) != cudaSuccess) {
    cudaGetLastError();
    fedvr_mlp_destroy(m);
    return FEDVR_ERR_CUDA;
  }
  *out = m;
  return FEDVR_OK;
}

void fedvr_mlp_destroy(fedvr_mlp *m) {
  if (!m) return;
  cudaStreamSynchronize(m->stream);
  DevBuf *bufs[] = {&m->W, &m->m, &m->v, &m->g, &m->Wbf, &m->act, &m->Y, &m->dbuf, &m->part,
                    &m->X, &m->T, &m->idx, &m->bX, &m->bT, &m->sdev, &m->F, &m->S1};
  for (DevBuf *b : bufs) fedvr::release(*b);
  delete m;
}

const char *fedvr_mlp_last_error(const fedvr_mlp *m) { return m ? m->err : "null network"; }

int fedvr_mlp_num_params(const fedvr_mlp *m, long *count) {
  if (!m || !count) return FEDVR_ERR_ARG;
  *count = m->L.nparam;
  return FEDVR_OK;
}

int fedvr_mlp_rows(const fedvr_mlp *m, long *rows) {
  if (!m || !rows) return FEDVR_ERR_ARG;
  *rows = m->rows;
  return FEDVR_OK;
}

int fedvr_mlp_get_rows(fedvr_mlp *m, long start, long count, float *X, float *T) {
  if (!m || start < 0 || count < 0 || start + count > m->rows) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  const fedvr::MlpNet &L = m->L;
  if (X && count)
    MCK(m, cudaMemcpy(X, P<float>(m->X) + (size_t)start * L.din, (size_t)count * L.din * sizeof(float),
                      cudaMemcpyDeviceToHost));
  if (T && count)
    MCK(m, cudaMemcpy(T, P<float>(m->T) + (size_t)start * L.dout,
                      (size_t)count * L.dout * sizeof(float), cudaMemcpyDeviceToHost));
  return FEDVR_OK;
}

int fedvr_mlp_get_params(fedvr_mlp *m, float *params, long count) {
  if (!m || !params || count != m->L.nparam) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  MCK(m, cudaMemcpyAsync(params, m->W.ptr, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost,
                         m->stream));
  MCK(m, cudaStreamSynchronize(m->stream));
  return FEDVR_OK;
}

int fedvr_mlp_set_params(fedvr_mlp *m, const float *params, long count) {
  if (!m || !params || count != m->L.nparam) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  MCK(m, cudaMemcpyAsync(m->W.ptr, params, (size_t)count * sizeof(float), cudaMemcpyHostToDevice,
                         m->stream));
  MCK(m, fedvr::mlp_to_bf16(count, P<float>(m->W), m->Wbf.ptr, m->stream));
  MCK(m, cudaStreamSynchronize(m->stream));
  return FEDVR_OK;
}

int fedvr_mlp_loss_grad(fedvr_mlp *m, const float *X, const float *T, int rows, float *grad,
                        double *loss) {
  if (!m || !X || !T || rows < 1 || rows > (1 << 20)) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  if (int r = ensure_rows(m, rows)) return r;
  MCK(m, fedvr::mlp_loss_grad(m->L, P<float>(m->W), rows, X, T, P<float>(m->act), P<float>(m->Y),
                              P<float>(m->dbuf), P<float>(m->g), P<double>(m->part), m->stream));
  int st;
  const double l = read_loss(m, &st);
  if (st) return st;
  if (loss) *loss = l;
  if (grad) {
    MCK(m, cudaMemcpy(grad, m->g.ptr, (size_t)m->L.nparam * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return FEDVR_OK;
}

int fedvr_mlp_forward(fedvr_mlp *m, const float *X, int rows, float *Y, int bf16) {
  if (!m || !X || !Y || rows < 1 || rows > (1 << 22)) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  MENSURE(m, act, (size_t)4 * rows * m->L.H * sizeof(float));
  if (bf16) {
    MCK(m, fedvr::mlp_forward_bf16(m->L, m->Wbf.ptr, P<float>(m->W), rows, X, P<float>(m->act), Y,
                                   m->stream));
  } else {
    MCK(m, fedvr::mlp_forward_f32(m->L, P<float>(m->W), rows, X, P<float>(m->act), Y, m->stream));
  }
  return FEDVR_OK;
}

// Features of ctx's current system from its one-shot Sigma (placed in m->S1);
// *pairs receives the row count, m->sdev the scale s.
static int system_features(fedvr_mlp *m, fedvr_ctx *ctx, const double *Sstar, float *F, float *T,
                           long *pairs) {
  const int n = ctx->n, M = ctx->M;
  *pairs = (long)n * (n + 1) / 2;
  MCK(m, fedvr::mlp_features(n, M, ctx->xmax - ctx->xmin, P<double>(m->S1), P<double>(ctx->w_G0),
                             P<double>(ctx->b_V), P<double>(ctx->b_nodes), P<double>(m->sdev),
                             Sstar, F, T, m->stream));
  return FEDVR_OK;
}

// One-shot Sigma^(2)[g0] of a freshly prepared ctx into m->S1.
static int one_shot_sigma(fedvr_mlp *m, fedvr_ctx *ctx) {
  if (int r = fedvr::sigma_of_current_g(ctx)) return mfail(m, r, ctx->err);
  const size_t bytes = (size_t)ctx->M * ctx->n * ctx->n * sizeof(double);
  MENSURE(m, S1, bytes);
  MCK(m, cudaMemcpyAsync(m->S1.ptr, ctx->w_S.ptr, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  MCK(m, cudaStreamSynchronize(ctx->stream));
  return FEDVR_OK;
}

int fedvr_mlp_collect(fedvr_mlp *m, fedvr_ctx *ctx, double beta, int u, int p, double mixing,
                      double tol, int max_iter, int *iters) {
  if (!m || !ctx) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  if (2 * u * p + 1 != m->M) return mfail(m, FEDVR_ERR_ARG, "mesh size differs from the network's M");
  if (int r = fedvr_2b_prepare(ctx, beta, u, p, FEDVR_SPLIT_TF32)) return mfail(m, r, ctx->err);
  if (int r = one_shot_sigma(m, ctx)) return r;
  int it = 0;
  double E0, N;
  int r = solve_2b(ctx, beta, u, p, mixing, tol, max_iter, FEDVR_SPLIT_TF32, 0, nullptr, nullptr,
                   nullptr, &E0, &N, &it);
  if (iters) *iters = it;
  if (r != FEDVR_OK) return mfail(m, r, ctx->err);
  const int n = ctx->n, M = ctx->M;
  const long pairs = (long)n * (n + 1) / 2;
  const fedvr::MlpNet &L = m->L;
  const size_t need = (size_t)(m->rows + pairs);
  if (need > (size_t)m->cap) {
    size_t cap = m->cap ? (size_t)m->cap : 65536;
    while (cap < need) cap *= 2;
    if (!mgrow(m, m->X, cap * L.din * sizeof(float), (size_t)m->rows * L.din * sizeof(float)) ||
        !mgrow(m, m->T, cap * L.dout * sizeof(float), (size_t)m->rows * L.dout * sizeof(float)))
      return FEDVR_ERR_CUDA;
    m->cap = (long)cap;
  }
  float *F = P<float>(m->X) + (size_t)m->rows * L.din;
  float *T = P<float>(m->T) + (size_t)m->rows * L.dout;
  long got = 0;
  if (int rr = system_features(m, ctx, P<double>(ctx->w_S), F, T, &got)) return rr;
  MCK(m, cudaStreamSynchronize(m->stream));
  m->rows += got;
  (void)M;
  return FEDVR_OK;
}

int fedvr_mlp_train(fedvr_mlp *m, int epochs, int batch, double lr, double *final_loss) {
  if (!m || epochs < 1 || batch < 1 || batch > (1 << 16) || !(lr > 0.0)) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  if (m->rows < 1) return mfail(m, FEDVR_ERR_STATE, "no training rows collected");
  const fedvr::MlpNet &L = m->L;
  if (int r = ensure_rows(m, batch)) return r;
  MENSURE(m, idx, (size_t)m->rows * sizeof(int));
  MENSURE(m, bX, (size_t)batch * L.din * sizeof(float));
  MENSURE(m, bT, (size_t)batch * L.dout * sizeof(float));
  std::vector<int> perm((size_t)m->rows);
  uint64_t st = m->seed ^ 0x5DEECE66Dull;
  double last = 0.0;
  for (int e = 0; e < epochs; ++e) {
    for (long i = 0; i < m->rows; ++i) perm[i] = (int)i;
    for (long i = m->rows - 1; i > 0; --i) {
      long j = (long)(splitmix(st) % (uint64_t)(i + 1));
      int t = perm[i];
      perm[i] = perm[j];
      perm[j] = t;
    }
    MCK(m, cudaMemcpyAsync(m->idx.ptr, perm.data(), perm.size() * sizeof(int),
                           cudaMemcpyHostToDevice, m->stream));
    double sum = 0.0;
    long nb = 0;
    for (long r0 = 0; r0 < m->rows; r0 += batch) {
      const int rows = (int)((m->rows - r0) < batch ? (m->rows - r0) : batch);
      const int *ix = P<int>(m->idx) + r0;
      MCK(m, fedvr::mlp_gather(rows, L.din, ix, P<float>(m->X), P<float>(m->bX), m->stream));
      MCK(m, fedvr::mlp_gather(rows, L.dout, ix, P<float>(m->T), P<float>(m->bT), m->stream));
      MCK(m, fedvr::mlp_loss_grad(L, P<float>(m->W), rows, P<float>(m->bX), P<float>(m->bT),
                                  P<float>(m->act), P<float>(m->Y), P<float>(m->dbuf),
                                  P<float>(m->g), P<double>(m->part), m->stream));
      MCK(m, fedvr::mlp_adam(L.nparam, (float)lr, ++m->adam_t, P<float>(m->g), P<float>(m->m),
                             P<float>(m->v), P<float>(m->W), m->stream));
      if (e == epochs - 1) {
        int s2;
        sum += read_loss(m, &s2);
        if (s2) return s2;
        ++nb;
      }
    }
    if (e == epochs - 1) last = sum / (double)(nb ? nb : 1);
  }
  MCK(m, fedvr::mlp_to_bf16(L.nparam, P<float>(m->W), m->Wbf.ptr, m->stream));
  MCK(m, cudaStreamSynchronize(m->stream));
  if (final_loss) *final_loss = last;
  return FEDVR_OK;
}

int fedvr_warm_start(fedvr_ctx *ctx, fedvr_mlp *m, double beta, int u, int p, int inner_steps) {
  if (!m || !ctx) return FEDVR_ERR_ARG;
  if (m->failed) return FEDVR_ERR_STATE;
  if (2 * u * p + 1 != m->M) return mfail(m, FEDVR_ERR_ARG, "mesh size differs from the network's M");
  if (int r = fedvr_2b_prepare(ctx, beta, u, p, FEDVR_SPLIT_TF32)) return mfail(m, r, ctx->err);
  if (int r = one_shot_sigma(m, ctx)) return r;
  const int n = ctx->n, M = ctx->M;
  const long pairs = (long)n * (n + 1) / 2;
  const fedvr::MlpNet &L = m->L;
  MENSURE(m, F, (size_t)pairs * L.din * sizeof(float));
  MENSURE(m, Y, (size_t)pairs * L.dout * sizeof(float));
  MENSURE(m, act, (size_t)4 * pairs * L.H * sizeof(float));
  long got = 0;
  if (int r = system_features(m, ctx, nullptr, P<float>(m->F), nullptr, &got)) return r;
  MCK(m, fedvr::mlp_forward_bf16(L, m->Wbf.ptr, P<float>(m->W), (int)pairs, P<float>(m->F),
                                 P<float>(m->act), P<float>(m->Y), m->stream));
  // Sigma_pred = S1 + s * Delta lands in ctx's Sigma workspace, then becomes the warm start
  MCK(m, fedvr::mlp_scatter(n, M, P<double>(m->S1), P<double>(m->sdev), P<float>(m->Y),
                            P<double>(ctx->w_S), m->stream));
  MCK(m, cudaStreamSynchronize(m->stream));
  if (int r = fedvr_set_initial_sigma(ctx, P<double>(ctx->w_S), M, 1, inner_steps))
    return mfail(m, r, ctx->err);
  return FEDVR_OK;
}

}  // extern "C"
