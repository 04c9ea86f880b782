// T-matrix correlation self-energy (the particle-particle ladder; Sec. 4 names
// the T-matrix approximation beside GW as a further use of the FE-DVR form),
// FP64. With the two-index interaction a pair of particles at the nodes
// (a, k) scatters through V_ak without changing nodes, so the ladder lives on
// node pairs: with K(tau) = g(tau) (x) g(tau) the pair propagator and V^ the
// diagonal pair-space matrix of the V_ak, the correlated ladder solves
//
//   t = V^ K V^ - V^ (K * t),
//   Sigma^T_ab(tau_j) = sum_kl [sigma t_j(ak; bl) - t_j(ak; lb)] gb_j(l, k),
//
// gb_j = g_{M-1-j}. K * t is the periodic convolution over one period
// (trapezoid on the mesh, K at the lag linearly interpolated between mesh
// points: the bosonic coefficient table of the GW bubble). The lowest order
// t = V^ K V^ gives the direct and exchange terms of Eq. sigma2ndb.
//
// Layout of a pair-space stack: t[j][b][l][a][k] = t_j(ak; bl), so that each
// column pair (b, l) is a contiguous n x n matrix X_j^{bl}[a][k] and the action
// of g_r (x) g_r on the row pair is the sandwich g_r X g_r^T. n <= 32.
#include "common.cuh"

namespace fedvr {
namespace {

// S[j][b][l][a][k] = V_ak g_j(a, b) g_j(k, l) V_bl.
__global__ void tm_source_kernel(int n, long count, const double *__restrict__ V,
                                 const double *__restrict__ G, double *__restrict__ S) {
  const long n2 = (long)n * n, n4 = n2 * n2;
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < count;
       x += (long)gridDim.x * blockDim.x) {
    const long j = x / n4;
    const int r = (int)(x % n4);
    const int bl = r / (int)n2, ak = r % (int)n2;
    const int b = bl / n, l = bl % n, a = ak / n, k = ak % n;
    const double *g = G + j * n2;
    S[x] = V[ak] * g[a * n + b] * g[k * n + l] * V[bl];
  }
}

// Y_i^{bl} = sum_j [c1 g_k X_j^{bl} g_k^T + c2 g_{k+1} X_j^{bl} g_{k+1}^T] with
// (k, c1, c2) the bosonic table entry (i, j). One block per (i, column pair),
// one thread per row pair (a, k); X, g_r and the half product in shared memory.
__global__ void tm_ladder_kernel(int n, int M, const ConvCoef *__restrict__ coef,
                                 const double *__restrict__ G, const double *__restrict__ T,
                                 double *__restrict__ Y) {
  __shared__ double X[1024], gr[1024], tmp[1024];
  const int n2 = n * n;
  const int i = (int)(blockIdx.x / n2), bl = (int)(blockIdx.x % n2);
  const int tid = threadIdx.x, a = tid / n, k = tid % n;
  double acc = 0.0;
  for (int j = 0; j < M; ++j) {
    const ConvCoef c = coef[(long)i * M + j];
    X[tid] = T[((long)j * n2 + bl) * n2 + tid];
    for (int r = 0; r < 2; ++r) {
      const double cr = r ? c.c2 : c.c1;  // the same for the whole block
      if (cr == 0.0) continue;
      __syncthreads();  // earlier readers of gr and tmp are done; X is loaded
      gr[tid] = G[(long)(c.k + r) * n2 + tid];
      __syncthreads();
      double s = 0.0;  // (X g_r^T)[a][k]
      for (int q = 0; q < n; ++q) s = fma(X[a * n + q], gr[k * n + q], s);
      tmp[tid] = s;
      __syncthreads();
      s = 0.0;  // (g_r X g_r^T)[a][k]
      for (int q = 0; q < n; ++q) s = fma(gr[a * n + q], tmp[q * n + k], s);
      acc = fma(cr, s, acc);
    }
    __syncthreads();  // X is rewritten next
  }
  Y[((long)i * n2 + bl) * n2 + tid] = acc;
}

// t_new = S - V_ak Y; *res = max |t_new - t| (bit pattern of a non-negative
// double, so that a NaN or Inf shows as such); t <- (1 - m) t + m t_new.
__global__ void tm_update_kernel(int n, long count, const double *__restrict__ V,
                                 const double *__restrict__ S, const double *__restrict__ Y,
                                 double *__restrict__ T, double mixing,
                                 unsigned long long *res) {
  const int n2 = n * n;
  unsigned long long m = 0ull;
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < count;
       x += (long)gridDim.x * blockDim.x) {
    const double nw = S[x] - V[(int)(x % n2)] * Y[x];
    const double old = T[x];
    const unsigned long long d = __double_as_longlong(fabs(nw - old));
    m = d > m ? d : m;
    T[x] = fma(mixing, nw, (1.0 - mixing) * old);
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(res, m);
}

// Sigma_j(a, b) = sum_kl [spin t_j(ak; bl) - t_j(ak; lb)] g_{M-1-j}(l, k).
__global__ void tm_sigma_kernel(int n, int M, double spin, const double *__restrict__ G,
                                const double *__restrict__ T, double *__restrict__ Sigma) {
  const long n2 = (long)n * n, count = (long)M * n2;
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < count;
       x += (long)gridDim.x * blockDim.x) {
    const long j = x / n2;
    const int a = (int)((x % n2) / n), b = (int)(x % n);
    const double *t = T + j * n2 * n2;
    const double *gb = G + (long)(M - 1 - j) * n2;
    double s = 0.0;
    for (int k = 0; k < n; ++k)
      for (int l = 0; l < n; ++l) {
        const double d = t[((long)b * n + l) * n2 + a * n + k];  // t_j(ak; bl)
        const double e = t[((long)l * n + b) * n2 + a * n + k];  // t_j(ak; lb)
        s = fma(fma(spin, d, -e), gb[l * n + k], s);
      }
    Sigma[x] = s;
  }
}

int blocks_for(long count) {
  const long b = (count + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t tm_source(int n, int M, const double *V, const double *G, double *S, cudaStream_t s) {
  const long count = (long)M * n * n * n * n;
  tm_source_kernel<<<blocks_for(count), 256, 0, s>>>(n, count, V, G, S);
  return cudaGetLastError();
}

cudaError_t tm_ladder(int n, int M, const ConvCoef *coef, const double *G, const double *T,
                      double *Y, cudaStream_t s) {
  if (n < 1 || n > 32) return cudaErrorInvalidValue;
  tm_ladder_kernel<<<(unsigned)((long)M * n * n), n * n, 0, s>>>(n, M, coef, G, T, Y);
  return cudaGetLastError();
}

cudaError_t tm_update(int n, int M, const double *V, const double *S, const double *Y, double *T,
                      double mixing, unsigned long long *res, cudaStream_t s) {
  const long count = (long)M * n * n * n * n;
  tm_update_kernel<<<blocks_for(count), 256, 0, s>>>(n, count, V, S, Y, T, mixing, res);
  return cudaGetLastError();
}

cudaError_t tm_sigma(int n, int M, double spin, const double *G, const double *T, double *Sigma,
                     cudaStream_t s) {
  tm_sigma_kernel<<<blocks_for((long)M * n * n), 256, 0, s>>>(n, M, spin, G, T, Sigma);
  return cudaGetLastError();
}

}  // namespace fedvr
