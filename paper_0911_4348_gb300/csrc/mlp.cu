// Learned warm start for the second-Born iteration. The paper has no learned
// component: this is a service of the library that predicts the converged
// self-energy of a new system from its one-shot Sigma^(2)[g^0], so that the
// iteration starts close to its fixed point.
//
// A per-(a, b)-pair MLP maps x = [Sigma1_ab(tau)/s (M), g0_ab(tau) (M), V_ab,
// X_a/L, X_b/L] (s = max|Sigma1|, L = box length) to Delta_ab(tau)/s (M), the
// correction Sigma*_ab - Sigma1_ab of the converged self-energy:
//   h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3.
// Training (FP32 master weights, MSE, Adam) and inference (BF16 weights, FP32
// accumulation) are CUDA-core kernels of this file: the layers are small
// dense products (rows x 517 x 512) far from the tensor-core regime of the
// self-energy contractions.
#include <cuda_bf16.h>

#include <vector>

#include "mlp.cuh"

namespace fedvr {
namespace {

enum Epi { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_RELU = 2 };

// C[rows x N] = op(A) op(B) (+ bias, relu). A, B row-major float (B may be bf16).
// With EPI_BIAS_RELU the pre-activation goes to Z and relu(Z) to C.
template <bool TA, bool TB, typename Tb, int EPI>
__global__ void __launch_bounds__(256) mlp_gemm(int M, int N, int K, const float *__restrict__ A,
                                                int lda, const Tb *__restrict__ B, int ldb,
                                                const float *__restrict__ bias,
                                                float *__restrict__ Z, float *__restrict__ C,
                                                int ldc) {
  __shared__ float As[16][65], Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int kk, mm;
      if (TA) { mm = e % 64; kk = e / 64; } else { kk = e % 16; mm = e / 16; }
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? (TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk]) : 0.f;
      int nn;
      if (TB) { kk = e % 16; nn = e / 16; } else { nn = e % 64; kk = e / 64; }
      int gn = n0 + nn;
      gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K)
                       ? (float)(TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn])
                       : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(av[r], bv[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int gm = m0 + ty + 16 * r;
    if (gm >= M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gn = n0 + tx + 16 * q;
      if (gn >= N) continue;
      float v = acc[r][q];
      if (EPI != EPI_STORE) v += bias[gn];
      if (EPI == EPI_BIAS_RELU) {
        Z[(long)gm * ldc + gn] = v;
        v = fmaxf(v, 0.f);
      }
      C[(long)gm * ldc + gn] = v;
    }
  }
}

template <bool TA, bool TB, typename Tb, int EPI>
cudaError_t gemm(int M, int N, int K, const float *A, int lda, const Tb *B, int ldb,
                 const float *bias, float *Z, float *C, int ldc, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  mlp_gemm<TA, TB, Tb, EPI><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, bias, Z, C, ldc);
  return cudaGetLastError();
}

// dY = (Y - T) / (rows * N); per-block loss partials sum (Y - T)^2 / (2 rows N).
__global__ void mse_grad_kernel(long count, long denom, const float *__restrict__ Y,
                                const float *__restrict__ T, float *__restrict__ dY,
                                double *__restrict__ part) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d / (float)denom;
    acc += (double)d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0] / (2.0 * (double)denom);
}

// g[c] = sum_r D[r][c] (fixed order), bias gradients.
__global__ void colsum_kernel(int rows, int cols, const float *__restrict__ D, float *__restrict__ g) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float acc = 0.f;
  for (int r = 0; r < rows; ++r) acc += D[(long)r * cols + c];
  g[c] = acc;
}

// D = D o (Z > 0)
__global__ void relu_mask_kernel(long count, const float *__restrict__ Z, float *__restrict__ D) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x)
    if (!(Z[i] > 0.f)) D[i] = 0.f;
}

__global__ void adam_kernel(long count, float lr, float b1, float b2, float eps, float c1,
                            float c2, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float *__restrict__ w) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(long count, const float *__restrict__ x, __nv_bfloat16 *__restrict__ y) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void gather_rows_kernel(int rows, int cols, const int *__restrict__ idx,
                                   const float *__restrict__ src, float *__restrict__ dst) {
  long total = (long)rows * cols;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total;
       i += (long)gridDim.x * blockDim.x) {
    long r = i / cols, c = i % cols;
    dst[i] = src[(long)idx[r] * cols + c];
  }
}

// s = max |S1| over the stack (non-negative bit pattern max).
__global__ void absmax_kernel(long count, const double *__restrict__ x, unsigned long long *out) {
  double m = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count;
       i += (long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// Feature row of pair p = (a, b), a >= b (lower triangle, row-major):
// [S1_ab(tau_j)/s for j; g0_ab(tau_j) for j; V_ab; X_a/L; X_b/L]; optional
// target row (Sstar - S1)_ab(tau_j)/s.
__device__ __forceinline__ void pair_of(long p, int *a, int *b) {
  int aa = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
  while ((long)aa * (aa + 1) / 2 > p) --aa;
  while ((long)(aa + 1) * (aa + 2) / 2 <= p) ++aa;
  *a = aa;
  *b = (int)(p - (long)aa * (aa + 1) / 2);
}

__global__ void features_kernel(int n, int M, double L, const double *__restrict__ S1,
                                const double *__restrict__ G0, const double *__restrict__ V,
                                const double *__restrict__ X, const double *__restrict__ s_ptr,
                                const double *__restrict__ Sstar, float *__restrict__ F,
                                float *__restrict__ T) {
  const long pairs = (long)n * (n + 1) / 2;
  const int din = 2 * M + 3;
  const long nn = (long)n * n;
  const double s = *s_ptr > 0.0 ? *s_ptr : 1.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < pairs * din;
       i += (long)gridDim.x * blockDim.x) {
    const long p = i / din;
    const int c = (int)(i % din);
    int a, b;
    pair_of(p, &a, &b);
    const long ab = (long)a * n + b;
    float v;
    if (c < M) v = (float)(S1[(long)c * nn + ab] / s);
    else if (c < 2 * M) v = (float)G0[(long)(c - M) * nn + ab];
    else if (c == 2 * M) v = (float)V[ab];
    else if (c == 2 * M + 1) v = (float)(X[a] / L);
    else v = (float)(X[b] / L);
    F[i] = v;
  }
  if (T) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < pairs * M;
         i += (long)gridDim.x * blockDim.x) {
      const long p = i / M;
      const int j = (int)(i % M);
      int a, b;
      pair_of(p, &a, &b);
      const long off = (long)j * nn + (long)a * n + b;
      T[i] = (float)((Sstar[off] - S1[off]) / s);
    }
  }
}

// Sigma_pred[j][a][b] = Sigma_pred[j][b][a] = S1 + s * Y[p][j]
__global__ void scatter_kernel(int n, int M, const double *__restrict__ S1,
                               const double *__restrict__ s_ptr, const float *__restrict__ Y,
                               double *__restrict__ out) {
  const long pairs = (long)n * (n + 1) / 2;
  const long nn = (long)n * n;
  const double s = *s_ptr > 0.0 ? *s_ptr : 1.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < pairs * M;
       i += (long)gridDim.x * blockDim.x) {
    const long p = i / M;
    const int j = (int)(i % M);
    int a, b;
    pair_of(p, &a, &b);
    const double v = S1[(long)j * nn + (long)a * n + b] + s * (double)Y[i];
    out[(long)j * nn + (long)a * n + b] = v;
    out[(long)j * nn + (long)b * n + a] = v;
  }
}

}  // namespace

// ---- host-side network ----
MlpNet mlp_layout(int M, int H) {
  MlpNet L;
  L.din = 2 * M + 3;
  L.H = H;
  L.dout = M;
  L.o_W1 = 0;
  L.o_b1 = L.o_W1 + (long)L.din * H;
  L.o_W2 = L.o_b1 + H;
  L.o_b2 = L.o_W2 + (long)H * H;
  L.o_W3 = L.o_b2 + H;
  L.o_b3 = L.o_W3 + (long)H * L.dout;
  L.nparam = L.o_b3 + L.dout;
  return L;
}

// Forward of `rows` rows. W float (training) or bf16 (inference) parameters.
// act holds Z1, H1, Z2, H2 (rows x H each); Y out (rows x dout).
template <typename Tw>
cudaError_t mlp_forward_t(const MlpNet &L, const Tw *W, const float *Wbias, int rows,
                          const float *X, float *act, float *Y, cudaStream_t s) {
  float *Z1 = act, *H1 = act + (long)rows * L.H, *Z2 = H1 + (long)rows * L.H,
        *H2 = Z2 + (long)rows * L.H;
  cudaError_t e = gemm<false, false, Tw, EPI_BIAS_RELU>(rows, L.H, L.din, X, L.din, W + L.o_W1,
                                                        L.H, Wbias + L.o_b1, Z1, H1, L.H, s);
  if (e != cudaSuccess) return e;
  e = gemm<false, false, Tw, EPI_BIAS_RELU>(rows, L.H, L.H, H1, L.H, W + L.o_W2, L.H,
                                            Wbias + L.o_b2, Z2, H2, L.H, s);
  if (e != cudaSuccess) return e;
  return gemm<false, false, Tw, EPI_BIAS>(rows, L.dout, L.H, H2, L.H, W + L.o_W3, L.dout,
                                          Wbias + L.o_b3, nullptr, Y, L.dout, s);
}

cudaError_t mlp_forward_f32(const MlpNet &L, const float *W, int rows, const float *X, float *act,
                            float *Y, cudaStream_t s) {
  return mlp_forward_t<float>(L, W, W, rows, X, act, Y, s);
}

cudaError_t mlp_forward_bf16(const MlpNet &L, const void *Wbf, const float *W, int rows,
                             const float *X, float *act, float *Y, cudaStream_t s) {
  return mlp_forward_t<__nv_bfloat16>(L, reinterpret_cast<const __nv_bfloat16 *>(Wbf), W, rows, X,
                                      act, Y, s);
}

// Loss and gradient of `rows` rows (forward included). grad has nparam floats;
// dbuf holds rows x max(H, dout) x 2 floats; part >= 256 doubles (loss partials).
cudaError_t mlp_loss_grad(const MlpNet &L, const float *W, int rows, const float *X,
                          const float *T, float *act, float *Y, float *dbuf, float *grad,
                          double *part, cudaStream_t s) {
  cudaError_t e = mlp_forward_f32(L, W, rows, X, act, Y, s);
  if (e != cudaSuccess) return e;
  float *Z1 = act, *H1 = act + (long)rows * L.H, *Z2 = H1 + (long)rows * L.H,
        *H2 = Z2 + (long)rows * L.H;
  const int wide = L.H > L.dout ? L.H : L.dout;
  float *dY = dbuf, *dH = dbuf + (long)rows * wide;
  const long ycount = (long)rows * L.dout;
  mse_grad_kernel<<<256, 256, 0, s>>>(ycount, ycount, Y, T, dY, part);
  // layer 3
  e = gemm<true, false, float, EPI_STORE>(L.H, L.dout, rows, H2, L.H, dY, L.dout, nullptr, nullptr,
                                          grad + L.o_W3, L.dout, s);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<(L.dout + 255) / 256, 256, 0, s>>>(rows, L.dout, dY, grad + L.o_b3);
  e = gemm<false, true, float, EPI_STORE>(rows, L.H, L.dout, dY, L.dout, W + L.o_W3, L.dout,
                                          nullptr, nullptr, dH, L.H, s);
  if (e != cudaSuccess) return e;
  relu_mask_kernel<<<512, 256, 0, s>>>((long)rows * L.H, Z2, dH);
  // layer 2
  e = gemm<true, false, float, EPI_STORE>(L.H, L.H, rows, H1, L.H, dH, L.H, nullptr, nullptr,
                                          grad + L.o_W2, L.H, s);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<(L.H + 255) / 256, 256, 0, s>>>(rows, L.H, dH, grad + L.o_b2);
  e = gemm<false, true, float, EPI_STORE>(rows, L.H, L.H, dH, L.H, W + L.o_W2, L.H, nullptr,
                                          nullptr, dY, L.H, s);  // dY reused as dH1
  if (e != cudaSuccess) return e;
  relu_mask_kernel<<<512, 256, 0, s>>>((long)rows * L.H, Z1, dY);
  // layer 1
  e = gemm<true, false, float, EPI_STORE>(L.din, L.H, rows, X, L.din, dY, L.H, nullptr, nullptr,
                                          grad + L.o_W1, L.H, s);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<(L.H + 255) / 256, 256, 0, s>>>(rows, L.H, dY, grad + L.o_b1);
  (void)H2;
  return cudaGetLastError();
}

cudaError_t mlp_adam(long count, float lr, int t, const float *g, float *m, float *v, float *w,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  adam_kernel<<<512, 256, 0, s>>>(count, lr, b1, b2, 1e-8f, c1, c2, g, m, v, w);
  return cudaGetLastError();
}

cudaError_t mlp_to_bf16(long count, const float *w, void *wbf, cudaStream_t s) {
  to_bf16_kernel<<<512, 256, 0, s>>>(count, w, reinterpret_cast<__nv_bfloat16 *>(wbf));
  return cudaGetLastError();
}

cudaError_t mlp_gather(int rows, int cols, const int *idx, const float *src, float *dst,
                       cudaStream_t s) {
  gather_rows_kernel<<<1024, 256, 0, s>>>(rows, cols, idx, src, dst);
  return cudaGetLastError();
}

cudaError_t mlp_features(int n, int M, double L, const double *S1, const double *G0,
                         const double *V, const double *X, double *s_dev, const double *Sstar,
                         float *F, float *T, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(s_dev, 0, sizeof(double), s);
  if (e != cudaSuccess) return e;
  absmax_kernel<<<512, 256, 0, s>>>((long)M * n * n, S1,
                                     reinterpret_cast<unsigned long long *>(s_dev));
  features_kernel<<<2048, 256, 0, s>>>(n, M, L, S1, G0, V, X, s_dev, Sstar, F, T);
  return cudaGetLastError();
}

cudaError_t mlp_scatter(int n, int M, const double *S1, const double *s_dev, const float *Y,
                        double *out, cudaStream_t s) {
  scatter_kernel<<<2048, 256, 0, s>>>(n, M, S1, s_dev, Y, out);
  return cudaGetLastError();
}

}  // namespace fedvr
