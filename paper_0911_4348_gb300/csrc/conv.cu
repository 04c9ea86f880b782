// The two tau-convolutions of the Matsubara Dyson equation (Sec. 2.3, Eq. deq)
// on the power mesh, FP64 path.
//
// I1_i = sum_j B_ij g_j with B_ij = c1 A_k + c2 A_{k+1} (linear interpolation of
// Sigma^corr at the lag tau_i - tau_j, anti-periodic beyond 0, trapezoid weight
// folded into c1, c2) and B_ii = dHF - wm_i A_0 + wp_i A_{M-1} (split trapezoid
// at the jump). One block owns a tile of whole rows of one I1_i and streams over j.
//
// I2 is evaluated with its left index in the HF eigenbasis, where g^0 is
// diagonal (g^0 multiplies I1 from the left, so the right index needs no
// transform): I2~_i,ab = sum_j K_a(i,j) I1~_j,ab with K_a(i,j) the exact g^0
// eigen-factor at the lag times the same split-trapezoid weights,
// I1~ = C^T I1, I2 = C I2~.
#include "common.cuh"
#include "tc_sys.cuh"

#include <math.h>

namespace fedvr {
namespace {


// Rows and weights of the Sigma^corr combination B_ij of one (i, j) entry:
// linear interpolation (ConvCoef: rows k, k + 1) or the cubic of the
// fourth-order variant (ConvCoef4: rows k0 .. k0 + 3); the diagonal entry
// names rows 0 and M - 1 (the jump values) and adds dHF.
struct CoefView {
  int r[4];
  double c[4];
  int np;
  bool diag;
};
__device__ __forceinline__ CoefView coef_view(const ConvCoef &cf, int M) {
  CoefView v;
  v.diag = cf.diag != 0;
  v.np = 2;
  v.r[0] = cf.k;
  v.r[1] = cf.diag ? (M - 1) : (cf.k + 1);
  v.c[0] = cf.c1;
  v.c[1] = cf.c2;
  return v;
}
__device__ __forceinline__ CoefView coef_view(const ConvCoef4 &cf, int M) {
  CoefView v;
  v.diag = cf.diag != 0;
  v.np = cf.diag ? 2 : 4;
  for (int p = 0; p < 4; ++p) {
    v.r[p] = cf.k0 + p;
    v.c[p] = cf.c[p];
  }
  if (cf.diag) {
    v.r[0] = 0;
    v.r[1] = M - 1;
  }
  return v;
}

// First convolution, FP64. CTA (row tile, i, split): its rows x n outputs of
// I1_i are spread over the 256 threads at up to kC1Q per thread (output
// o = tid + 256 q, row a0 + o / n, column o % n), so no output is padded; for
// each j of its share of the mesh-point range and each 16-wide slice of c it
// stages B_ij[a][c] (the interpolated Sigma^corr, built from up to four rows)
// [rows][16] and g_j[c][b] [16][n] in shared memory. Each output adds its terms
// in the order j, c. With splits > 1 (small launches) split k takes
// j in [M k / S, M (k + 1) / S), split 0 writes I1 and split k > 0 the partial
// stack part + (k - 1) M n n, added to I1 in split order afterwards.
constexpr int kC1Q = 8, kC1K = 16;
template <typename Coef>
__global__ void __launch_bounds__(256) conv1_fp64_kernel(int n, int M, int rows, int splits,
                                                         const Coef *__restrict__ coef,
                                                         const double *__restrict__ dHF,
                                                         const double *__restrict__ A,
                                                         const double *__restrict__ G,
                                                         double *__restrict__ I1,
                                                         double *__restrict__ part) {
  extern __shared__ double c1s[];
  double *Xs = c1s, *Ys = c1s + rows * kC1K;
  const int i = blockIdx.y, a0 = blockIdx.x * rows;
  const int nr = min(rows, n - a0), nout = nr * n;
  const long nn = (long)n * n;
  const int tid = threadIdx.x;
  double acc[kC1Q];
  int xo[kC1Q], yo[kC1Q];
  int nq = 0;
#pragma unroll
  for (int q = 0; q < kC1Q; ++q) {
    const int o = tid + 256 * q;
    acc[q] = 0.0;
    xo[q] = o < nout ? (o / n) * kC1K : 0;
    yo[q] = o < nout ? o % n : 0;
    nq += o < nout ? 1 : 0;
  }
  const int sp = blockIdx.z;
  const int j0 = (int)((long)M * sp / splits), j1 = (int)((long)M * (sp + 1) / splits);
  for (int j = j0; j < j1; ++j) {
    const CoefView cv = coef_view(coef[(long)i * M + j], M);
    const double *g = G + (long)j * nn;
    for (int c0 = 0; c0 < n; c0 += kC1K) {
      const int nc = min(kC1K, n - c0);
      for (int e = tid; e < nr * kC1K; e += 256) {
        const int aa = e / kC1K, cc = e % kC1K;
        double v = 0.0;
        if (cc < nc) {
          const long off = (long)(a0 + aa) * n + c0 + cc;
          v = cv.c[0] * A[(long)cv.r[0] * nn + off] + cv.c[1] * A[(long)cv.r[1] * nn + off];
          if (cv.np == 4)
            v += cv.c[2] * A[(long)cv.r[2] * nn + off] + cv.c[3] * A[(long)cv.r[3] * nn + off];
          if (cv.diag) v += dHF[off];
        }
        Xs[e] = v;
      }
      for (int e = tid; e < nc * n; e += 256) Ys[e] = g[(long)c0 * n + e];
      __syncthreads();
#pragma unroll 2
      for (int cc = 0; cc < nc; ++cc) {
#pragma unroll
        for (int q = 0; q < kC1Q; ++q)
          if (q < nq) acc[q] = fma(Xs[xo[q] + cc], Ys[cc * n + yo[q]], acc[q]);
      }
      __syncthreads();
    }
  }
  double *out = sp == 0 ? I1 : part + (long)(sp - 1) * M * nn;
#pragma unroll
  for (int q = 0; q < kC1Q; ++q) {
    if (q >= nq) break;
    const int o = tid + 256 * q;
    out[(long)i * nn + (long)(a0 + o / n) * n + o % n] = acc[q];
  }
}

// I1 += the partial stacks of splits 1 .. parts, in split order.
__global__ void c1_fp64_reduce_kernel(long count, int parts, const double *__restrict__ part,
                                      double *__restrict__ I1) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  double v = I1[e];
  for (int k = 0; k < parts; ++k) v += part[(long)k * count + e];
  I1[e] = v;
}

inline int c1_rows(int n) { return n < 256 * kC1Q / n ? n : 256 * kC1Q / n; }

template <typename Coef>
cudaError_t launch_conv1_fp64(int n, int M, const Coef *coef, const double *dHF, const double *A,
                              const double *G, double *I1, double *part, cudaStream_t s) {
  const int rows = c1_rows(n);
  if (rows < 1) return cudaErrorInvalidValue;
  const size_t sm = (size_t)(rows * kC1K + kC1K * n) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(conv1_fp64_kernel<Coef>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int tiles = (n + rows - 1) / rows;
  const int splits = part ? conv1_fp64_splits(n, M) : 1;
  dim3 grid((unsigned)tiles, (unsigned)M, (unsigned)splits);
  conv1_fp64_kernel<Coef><<<grid, 256, sm, s>>>(n, M, rows, splits, coef, dHF, A, G, I1, part);
  e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const long count = (long)M * n * n;
  c1_fp64_reduce_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, splits - 1, part, I1);
  return cudaGetLastError();
}

__device__ __forceinline__ double phi_eig(double x, double y, double beta) {
  return (y >= 0.0) ? exp(-((beta + x) * y)) / (1.0 + exp(-(beta * y)))
                    : exp(-(x * y)) / (1.0 + exp(beta * y));
}

// K[a][i][j]: j != i: sign * w_j * phi_a(y) with y the lag of tau_i - tau_j in
// [-beta, 0]; j == i: wm_i * (-phi_a(-beta)) + wp_i * phi_a(0).
// W (fourth-order variant, may be NULL): per-(i, j) weights [M][M] replacing
// w_j, with wm, wp then the per-i end weights of the two sides of the split.
__global__ void conv2_kernel_table(int n, int M, double beta, const double *__restrict__ tau,
                                   const double *__restrict__ w, const double *__restrict__ wm,
                                   const double *__restrict__ wp, const double *__restrict__ W,
                                   const double *__restrict__ eps,
                                   const double *mu_dev, double mu_host, double *__restrict__ K) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long MM = (long)M * M;
  if (idx >= (long)n * MM) return;
  int a = (int)(idx / MM);
  long r = idx % MM;
  int i = (int)(r / M), j = (int)(r % M);
  double mu = mu_dev ? *mu_dev : mu_host;
  double y = eps[a] - mu;
  double v;
  if (i == j) {
    v = wm[i] * (-phi_eig(-beta, y, beta)) + wp[i] * phi_eig(0.0, y, beta);
  } else {
    double x = tau[i] - tau[j];
    double sg = 1.0;
    if (j < i) { x = x - beta; sg = -1.0; }
    v = sg * (W ? W[(long)i * M + j] : w[j]) * phi_eig(x, y, beta);
  }
  K[idx] = v;
}

// ---- fourth-order variant of the integrals (the paper names no quadrature) ----

// Weight of local point jl in the rule for the integral over x[0] .. x[m]: on
// each interval the cubic through x[s0] .. x[s0 + 3] (s0 = q - 1 clamped to
// [0, m - 3]; all points when m < 3), integrated by two-point Gauss.
__device__ double q4_side_weight(const double *x, int m, int jl) {
  if (m <= 0) return 0.0;
  const double g = 1.0 / sqrt(3.0);
  const int ns = m < 3 ? m + 1 : 4;
  const int qlo = m < 3 ? 0 : max(0, jl - 3), qhi = m < 3 ? m - 1 : min(m - 1, jl + 2);
  double w = 0.0;
  for (int q = qlo; q <= qhi; ++q) {
    const int s0 = m < 3 ? 0 : min(max(q - 1, 0), m - 3);
    if (jl < s0 || jl >= s0 + ns) continue;
    const double h = x[q + 1] - x[q], mid = 0.5 * (x[q] + x[q + 1]);
    for (int e = 0; e < 2; ++e) {
      const double node = e ? mid + 0.5 * h * g : mid - 0.5 * h * g;
      double l = 1.0;
      for (int r = s0; r < s0 + ns; ++r)
        if (r != jl) l *= (node - x[r]) / (x[jl] - x[r]);
      w += 0.5 * h * l;
    }
  }
  return w;
}

// One thread per (i, j): the fourth-order coefficient entry (side weight of j
// times the cubic's Lagrange coefficients at the lag, anti-periodic sign), the
// side weight alone (W, for the second convolution's table), and on the
// diagonal the end weights wL_i, wR_i; row 0 also writes the whole-mesh
// weights wE (the energy's tau integral).
__global__ void quad4_tables_kernel(int M, double beta, const double *__restrict__ tau,
                                    ConvCoef4 *__restrict__ coef, double *__restrict__ W,
                                    double *__restrict__ wL, double *__restrict__ wR,
                                    double *__restrict__ wE) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  const int i = (int)(idx / M), j = (int)(idx % M);
  if (i == 0) wE[j] = q4_side_weight(tau, M - 1, j);
  ConvCoef4 c;
  if (i == j) {
    const double l = q4_side_weight(tau, i, i), r = q4_side_weight(tau + i, M - 1 - i, 0);
    wL[i] = l;
    wR[i] = r;
    W[idx] = 0.0;
    c.k0 = 0;
    c.diag = 1;
    c.c[0] = -l;  // Sigma(0^+) = -Sigma_0
    c.c[1] = r;   // Sigma(0^-) = Sigma_{M-1}
    c.c[2] = c.c[3] = 0.0;
    coef[idx] = c;
    return;
  }
  double y = tau[i] - tau[j], sg = 1.0;
  if (j < i) {
    y -= beta;
    sg = -1.0;
  }
  const double wij = j < i ? q4_side_weight(tau, i, j) : q4_side_weight(tau + i, M - 1 - i, j - i);
  W[idx] = wij;
  int lo = 0, hi = M - 1;  // bracket: the largest k in [0, M - 2] with tau_k <= y
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (tau[mid] <= y) lo = mid; else hi = mid;
  }
  const int s0 = min(max(lo - 1, 0), M - 4);
  c.k0 = s0;
  c.diag = 0;
  for (int p = 0; p < 4; ++p) {
    double l = 1.0;
    for (int r = 0; r < 4; ++r)
      if (r != p) l *= (y - tau[s0 + r]) / (tau[s0 + p] - tau[s0 + r]);
    c.c[p] = sg * wij * l;
  }
  coef[idx] = c;
}

// FP32 batched GEMM with mixed input/output types (64x64 tiles, 4x4 per thread):
// C = op(A) op(B), operands converted to float on load, result stored as To.
template <bool TA, bool TB, typename Ta, typename Tb, typename To>
__global__ void __launch_bounds__(256) gemm32_kernel(int M, int N, int K,
                                                     const Ta *__restrict__ A, long lda, long sA,
                                                     const Tb *__restrict__ B, long ldb, long sB,
                                                     To *__restrict__ C, long ldc, long sC) {
  const long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  __shared__ float As[16][65];
  __shared__ float Bs[16][65];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int kk, mm;
      if (TA) { mm = e % 64; kk = e / 64; } else { kk = e % 16; mm = e / 16; }
      int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? (float)(TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk])
                                      : 0.f;
      int nn;
      if (TB) { kk = e % 16; nn = e / 16; } else { nn = e % 64; kk = e / 64; }
      int gn = n0 + nn;
      gk = k0 + kk;
      Bs[kk][nn] = (gn < N && gk < K) ? (float)(TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn])
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
      if (gn < N) C[(long)gm * ldc + gn] = (To)acc[r][q];
    }
  }
}

__global__ void to_f32_kernel(size_t count, const double *__restrict__ x, float *__restrict__ y) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

template <bool TA, bool TB, typename Ta, typename Tb, typename To>
cudaError_t gemm32(int M, int N, int K, const Ta *A, long lda, long sA, const Tb *B, long ldb,
                   long sB, To *C, long ldc, long sC, int batch, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
  gemm32_kernel<TA, TB, Ta, Tb, To><<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_to_f32(size_t count, const double *x, float *y, cudaStream_t s) {
  to_f32_kernel<<<1024, 256, 0, s>>>(count, x, y);
  return cudaGetLastError();
}

// FP32 variant of conv2_apply for the split-precision mode: the same three
// products, split TF32 on the tensor cores for n >= 96 (conv2_tc) and FP32 on
// the CUDA cores below (K32 is the eigen-kernel table in FP32, t1/t2 float
// scratch of M*n*n), FP64 I1 in and FP64 I2 out; err is raised if a
// tensor-core wait gives up.
cudaError_t conv2_apply_f32(int n, int M, const float *K32, const double *C, const double *I1,
                            double *I2, float *t1, float *t2, int *err, cudaStream_t s) {
  const long nn = (long)n * n, MM = (long)M * M;
  cudaError_t e;
  if (n < 96) {  // small matrices: 64 x 64 tiles, one GEMM per mesh point
    e = gemm32<true, false>(n, n, n, C, n, 0, I1, n, nn, t2, n, nn, M, s);
    if (e != cudaSuccess) return e;
    e = gemm32<false, false>(M, n, M, K32, M, MM, (const float *)t2, nn, n, t1, nn, n, n, s);
    if (e != cudaSuccess) return e;
    return gemm32<false, false>(n, n, n, C, n, 0, (const float *)t1, n, nn, I2, n, nn, M, s);
  }
  return conv2_tc(n, M, K32, C, I1, I2, t1, t2, err, s);
}

int conv1_fp64_splits(int n, int M) {
  // about four CTAs per SM of a 152-SM GPU, at most 8 splits of the mesh-point range
  const int rows = c1_rows(n);
  const long ctas = (long)((n + rows - 1) / rows) * M;
  long sp = (608 + ctas - 1) / ctas;
  sp = sp < 1 ? 1 : (sp > 8 ? 8 : sp);
  return (int)(sp > M ? M : sp);
}

cudaError_t conv1_fp64(int n, int M, const ConvCoef *coef, const double *dHF, const double *A,
                       const double *G, double *I1, cudaStream_t s, double *part) {
  return launch_conv1_fp64<ConvCoef>(n, M, coef, dHF, A, G, I1, part, s);
}

cudaError_t conv1_fp64_q4(int n, int M, const ConvCoef4 *coef, const double *dHF,
                          const double *A, const double *G, double *I1, cudaStream_t s,
                          double *part) {
  if (M < 4) return cudaErrorInvalidValue;
  return launch_conv1_fp64<ConvCoef4>(n, M, coef, dHF, A, G, I1, part, s);
}

cudaError_t launch_quad4_tables(int M, double beta, const double *tau, ConvCoef4 *coef,
                                double *W, double *wL, double *wR, double *wE, cudaStream_t s) {
  if (M < 4) return cudaErrorInvalidValue;
  const long mm = (long)M * M;
  quad4_tables_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(M, beta, tau, coef, W, wL, wR,
                                                                  wE);
  return cudaGetLastError();
}

cudaError_t launch_conv2_kernel(int n, int M, double beta, const double *tau, const double *w,
                                const double *wm, const double *wp, const double *eps,
                                const double *mu_dev, double mu_host, double *K, cudaStream_t s,
                                const double *W) {
  long cnt = (long)n * M * M;
  conv2_kernel_table<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(n, M, beta, tau, w, wm, wp, W,
                                                                  eps, mu_dev, mu_host, K);
  return cudaGetLastError();
}

cudaError_t conv2_apply(int n, int M, const double *K, const double *C, const double *I1,
                        double *I2, double *t1, double *t2, cudaStream_t s) {
  long nn = (long)n * n, MM = (long)M * M;
  cudaError_t e;
  // g0(x) = C diag(phi(x)) C^T acts on I1 from the left only, so only the left
  // index goes to the HF eigenbasis (the right-hand C C^T = 1 drops out):
  // t1_j = C^T I1_j
  e = dgemm(true, false, n, n, n, 1.0, C, n, 0, I1, n, nn, nullptr, 0, 0.0, t1, n, nn, M, s);
  if (e != cudaSuccess) return e;
  // t2[i][a][:] = sum_j K_a[i][j] t1[j][a][:]   (batched over a)
  e = dgemm(false, false, M, n, M, 1.0, K, M, MM, t1, nn, n, nullptr, 0, 0.0, t2, nn, n, n, s);
  if (e != cudaSuccess) return e;
  // I2_i = C t2_i
  return dgemm(false, false, n, n, n, 1.0, C, n, 0, t2, n, nn, nullptr, 0, 0.0, I2, n, nn, M, s);
}

}  // namespace fedvr
