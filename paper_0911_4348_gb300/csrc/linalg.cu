// Dense FP64 building blocks on the device: batched GEMM with an optional
// diagonal scaling in the contraction index, a symmetric Jacobi eigensolver,
// eigenpair sorting and small elementwise helpers.
#include "common.cuh"

#include <math.h>

namespace fedvr {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

// C = alpha * op(A) diag(sk) op(B) + beta * C, one 64x64 tile per block,
// 256 threads each owning a 4x4 register tile (rows ty+16i, cols tx+16j).
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, double alpha,
                                                    const double *__restrict__ A, long lda, long sA,
                                                    const double *__restrict__ B, long ldb, long sB,
                                                    const double *__restrict__ sk, long sS,
                                                    double beta, double *__restrict__ C, long ldc,
                                                    long sC) {
  const long bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  if (sk) sk += bz * sS;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k0 = 0; k0 < K; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int kk, mm;
      if (TA) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      int gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) {
        v = TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk];
        if (sk) v *= sk[gk];
      }
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int kk, nn;
      if (TB) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      int gn = n0 + nn, gk = k0 + kk;
      double v = 0.0;
      if (gn < N && gk < K) v = TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double *c = C + (long)gm * ldc + gn;
      *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
    }
  }
}

// ---- Jacobi (cyclic by rounds; Golub & Van Loan, Sec. 8.5) ----
// Round-robin schedule on m = n rounded up to even: position 0 fixed, others
// rotate; pair k joins positions k and m-1-k.
__device__ __forceinline__ int rr_member(int pos, int r, int m) {
  return pos == 0 ? 0 : 1 + (pos - 1 + r) % (m - 1);
}

__global__ void jacobi_rot_kernel(int n, int m, int r, const double *__restrict__ A,
                                  double *__restrict__ J, unsigned long long *maxoff) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int npair = m / 2;
  if (k >= npair) return;
  int a = rr_member(k, r, m), b = rr_member(m - 1 - k, r, m);
  int p = min(a, b), q = max(a, b);
  double c = 1.0, s = 0.0;
  if (q < n) {
    double apq = A[(long)p * n + q];
    double app = A[(long)p * n + p], aqq = A[(long)q * n + q];
    double mag = fabs(apq);
    if (mag > 0.0) {
      atomicMax(maxoff, (unsigned long long)__double_as_longlong(mag));
      double tau = (aqq - app) / (2.0 * apq);
      double t;
      if (fabs(tau) > 1e150) t = 0.5 / tau;
      else t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + t * t);
      s = t * c;
    }
  }
  J[4 * k + 0] = c;
  J[4 * k + 1] = s;
  J[4 * k + 2] = (double)p;  // exact: indices < 2^53
  J[4 * k + 3] = (double)q;
}

__global__ void jacobi_apply_kernel(int n, int m, const double *__restrict__ Ain,
                                    double *__restrict__ Aout, double *__restrict__ V,
                                    const double *__restrict__ J) {
  long npair = m / 2;
  long nblk = npair * npair;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < nblk) {
    int k1 = (int)(idx / npair), k2 = (int)(idx % npair);
    double c1 = J[4 * k1], s1 = J[4 * k1 + 1], c2 = J[4 * k2], s2 = J[4 * k2 + 1];
    int p1 = (int)(J[4 * k1 + 2]), q1 = (int)(J[4 * k1 + 3]);
    int p2 = (int)(J[4 * k2 + 2]), q2 = (int)(J[4 * k2 + 3]);
    bool hq1 = q1 < n, hq2 = q2 < n;
    double x_pp = Ain[(long)p1 * n + p2];
    double x_pq = hq2 ? Ain[(long)p1 * n + q2] : 0.0;
    double x_qp = hq1 ? Ain[(long)q1 * n + p2] : 0.0;
    double x_qq = (hq1 && hq2) ? Ain[(long)q1 * n + q2] : 0.0;
    // rows: J1^T X
    double y_pp = c1 * x_pp - s1 * x_qp, y_pq = c1 * x_pq - s1 * x_qq;
    double y_qp = s1 * x_pp + c1 * x_qp, y_qq = s1 * x_pq + c1 * x_qq;
    // cols: (J1^T X) J2
    Aout[(long)p1 * n + p2] = c2 * y_pp - s2 * y_pq;
    if (hq2) Aout[(long)p1 * n + q2] = s2 * y_pp + c2 * y_pq;
    if (hq1) Aout[(long)q1 * n + p2] = c2 * y_qp - s2 * y_qq;
    if (hq1 && hq2) Aout[(long)q1 * n + q2] = s2 * y_qp + c2 * y_qq;
    return;
  }
  idx -= nblk;
  if (idx >= (long)n * npair) return;
  int i = (int)(idx / npair), k2 = (int)(idx % npair);
  int q2 = (int)(J[4 * k2 + 3]);
  if (q2 >= n) return;
  int p2 = (int)(J[4 * k2 + 2]);
  double c2 = J[4 * k2], s2 = J[4 * k2 + 1];
  double vp = V[(long)i * n + p2], vq = V[(long)i * n + q2];
  V[(long)i * n + p2] = c2 * vp - s2 * vq;
  V[(long)i * n + q2] = s2 * vp + c2 * vq;
}

__global__ void max_abs_kernel(size_t count, const double *a, unsigned long long *out) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void max_abs_diff_kernel(size_t count, const double *a, const double *b,
                                    unsigned long long *out) {
  double m = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs(a[i] - b[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void sort_eig_kernel(int n, const double *A, const double *V, double *eps,
                                double *C) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double di = A[(long)i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double dj = A[(long)j * n + j];
      rank += (dj < di) || (dj == di && j < i);
    }
    eps[rank] = di;
    for (int row = 0; row < n; ++row) C[(long)row * n + rank] = V[(long)row * n + i];
  }
}

__global__ void identity_kernel(int n, double *I) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < (long)n * n) I[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

__global__ void copy_kernel(size_t count, const double *src, double *dst) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

cudaError_t dgemm(bool ta, bool tb, int M, int N, int K, double alpha, const double *A,
                  long lda, long sA, const double *B, long ldb, long sB, const double *sk,
                  long sS, double beta, double *C, long ldc, long sC, int batch, cudaStream_t s) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  if (!ta && !tb)
    dgemm_kernel<false, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, sk, sS,
                                                    beta, C, ldc, sC);
  else if (ta && !tb)
    dgemm_kernel<true, false><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, sk, sS,
                                                   beta, C, ldc, sC);
  else if (!ta && tb)
    dgemm_kernel<false, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, sk, sS,
                                                   beta, C, ldc, sC);
  else
    dgemm_kernel<true, true><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, sk, sS,
                                                  beta, C, ldc, sC);
  return cudaGetLastError();
}

int jacobi_eig(int n, double *A, double *A2, double *V, double *J, double *scal, double tol,
               int max_sweeps, cudaStream_t s, cudaError_t *err) {
  // scal[0]: max |A_ij| at start; scal[1]: max pre-rotation |A_pq| within a sweep
  unsigned long long *bits = reinterpret_cast<unsigned long long *>(scal);
  *err = cudaMemsetAsync(scal, 0, 2 * sizeof(double), s);
  if (*err != cudaSuccess) return -1;
  size_t nn = (size_t)n * n;
  max_abs_kernel<<<64, 256, 0, s>>>(nn, A, bits);
  double host[2];
  *err = cudaMemcpyAsync(host, scal, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (*err == cudaSuccess) *err = cudaStreamSynchronize(s);
  if (*err != cudaSuccess) return -1;
  double anorm = host[0];
  if (n == 1 || anorm == 0.0) return 0;
  int m = n + (n & 1);
  int npair = m / 2;
  long work = (long)npair * npair + (long)n * npair;
  unsigned gapply = (unsigned)((work + 255) / 256);
  double *Ain = A, *Aout = A2;
  int sweep = 0;
  for (sweep = 1; sweep <= max_sweeps; ++sweep) {
    *err = cudaMemsetAsync(bits + 1, 0, sizeof(unsigned long long), s);
    if (*err != cudaSuccess) return -1;
    for (int r = 0; r < m - 1; ++r) {
      jacobi_rot_kernel<<<(npair + 127) / 128, 128, 0, s>>>(n, m, r, Ain, J, bits + 1);
      jacobi_apply_kernel<<<gapply, 256, 0, s>>>(n, m, Ain, Aout, V, J);
      double *t = Ain; Ain = Aout; Aout = t;
    }
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return -1;
    *err = cudaMemcpyAsync(host + 1, scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (*err == cudaSuccess) *err = cudaStreamSynchronize(s);
    if (*err != cudaSuccess) return -1;
    if (host[1] <= tol * anorm) break;
  }
  if (Ain != A) {
    copy_kernel<<<256, 256, 0, s>>>(nn, Ain, A);
    *err = cudaGetLastError();
    if (*err != cudaSuccess) return -1;
  }
  return sweep > max_sweeps ? -2 : sweep;
}

cudaError_t launch_sort_eig(int n, const double *A, const double *V, double *eps_out,
                            double *C_out, cudaStream_t s) {
  sort_eig_kernel<<<1, 1024, 0, s>>>(n, A, V, eps_out, C_out);
  return cudaGetLastError();
}

cudaError_t launch_identity(int n, double *I, cudaStream_t s) {
  long nn = (long)n * n;
  identity_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, I);
  return cudaGetLastError();
}

cudaError_t launch_copy(size_t count, const double *src, double *dst, cudaStream_t s) {
  copy_kernel<<<512, 256, 0, s>>>(count, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_max_abs_diff(size_t count, const double *a, const double *b,
                                unsigned long long *out, cudaStream_t s) {
  max_abs_diff_kernel<<<256, 256, 0, s>>>(count, a, b, out);
  return cudaGetLastError();
}

}  // namespace fedvr
