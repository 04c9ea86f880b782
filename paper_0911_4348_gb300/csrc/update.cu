// Dyson update, residual and Galitskii-Migdal energy (Sec. 2.3, Eq. deq and
// the total-energy evaluation), with deterministic reductions.
#include "common.cuh"

#include <math.h>

namespace fedvr {
namespace {

// g_new = g^0 + I2; s = 0.5 * (g_new_ab + g_new_ba); g' = (1 - a) * g + a * s;
// res = max |g' - g| (bit pattern of a non-negative double; NaN propagates as
// the largest pattern). Unfused IEEE operations in this order.
__global__ void update_kernel(int n, int M, double mixing, const double *__restrict__ G0,
                              const double *__restrict__ I2, double *__restrict__ G,
                              unsigned long long *res_bits) {
  long nn = (long)n * n;
  double m = 0.0;
  bool bad = false;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long)M * nn;
       idx += (long)gridDim.x * blockDim.x) {
    long j = idx / nn, e = idx % nn;
    int a = (int)(e / n), b = (int)(e % n);
    long t = j * nn + (long)b * n + a;
    double gab = __dadd_rn(G0[idx], I2[idx]);
    double gba = __dadd_rn(G0[t], I2[t]);
    double sym = __dmul_rn(0.5, __dadd_rn(gab, gba));
    double old = G[idx];
    double nw = __dadd_rn(__dmul_rn(__dsub_rn(1.0, mixing), old), __dmul_rn(mixing, sym));
    G[idx] = nw;
    double d = fabs(nw - old);
    if (d != d || d == INFINITY) bad = true; else m = fmax(m, d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad = __shfl_xor_sync(0xffffffffu, (int)bad, o) || bad;
  }
  if (bad) m = __longlong_as_double(0x7ff8000000000000LL);  // NaN: the largest pattern here
  if ((threadIdx.x & 31) == 0) atomicMax(res_bits, (unsigned long long)__double_as_longlong(m));
}

// Fixed-order block sum (blockDim.x = 256).
__device__ double block_sum256(double v) {
  __shared__ double sh[256];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// part[j] = sum_ab A[M-1-j]_ab G[j]_ab  (one block per j)
__global__ void energy_part_kernel(int n, int M, const double *__restrict__ G,
                                   const double *__restrict__ A, double *__restrict__ part) {
  int j = blockIdx.x;
  long nn = (long)n * n;
  const double *g = G + (long)j * nn;
  const double *s = A + (long)(M - 1 - j) * nn;
  double acc = 0.0;
  for (long e = threadIdx.x; e < nn; e += blockDim.x) acc += s[e] * g[e];
  acc = block_sum256(acc);
  if (threadIdx.x == 0) part[j] = acc;
}

// out[0] = E0 = sigma Tr[h rho] + (sigma/2) Tr[Sigma^HF[rho] rho]
//              - (sigma/2) sum_j w_j part[j];  out[1] = N = sigma Tr rho;  rho = G[M-1]
__global__ void energy_final_kernel(int n, int M, double spin, const double *__restrict__ h,
                                    const double *__restrict__ V, const double *__restrict__ G,
                                    const double *__restrict__ w, const double *__restrict__ part,
                                    double *out) {
  long nn = (long)n * n;
  const double *rho = G + (long)(M - 1) * nn;
  double e1 = 0.0, e2 = 0.0, tr = 0.0, ec = 0.0;
  for (long e = threadIdx.x; e < nn; e += blockDim.x) {
    int a = (int)(e / n), b = (int)(e % n);
    double r = rho[e];
    e1 += h[e] * r;
    double shf = -V[e] * r;
    if (a == b) {
      double hart = 0.0;
      for (int k = 0; k < n; ++k) hart += V[(long)a * n + k] * rho[(long)k * n + k];
      shf += spin * hart;
      tr += r;
    }
    e2 += shf * r;
  }
  if (part)
    for (int j = threadIdx.x; j < M; j += blockDim.x) ec += w[j] * part[j];
  e1 = block_sum256(e1);
  e2 = block_sum256(e2);
  tr = block_sum256(tr);
  ec = block_sum256(ec);
  if (threadIdx.x == 0) {
    out[0] = spin * e1 + 0.5 * spin * e2 - 0.5 * spin * ec;
    out[1] = spin * tr;
  }
}

// out = a * x + b * y
__global__ void axpby_kernel(size_t count, double a, const double *__restrict__ x, double b,
                             const double *__restrict__ y, double *__restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

}  // namespace

cudaError_t launch_axpby(size_t count, double a, const double *x, double b, const double *y,
                         double *out, cudaStream_t s) {
  axpby_kernel<<<512, 256, 0, s>>>(count, a, x, b, y, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_hf(int n, double spin, const double *h, const double *V,
                             const double *rho, double *out, cudaStream_t s) {
  // a one-point "stack" whose only member is rho, with no correlation term
  energy_final_kernel<<<1, 256, 0, s>>>(n, 1, spin, h, V, rho, nullptr, nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_update(int n, int M, double mixing, const double *G0, const double *I2,
                          double *G, unsigned long long *res_bits, cudaStream_t s) {
  long tot = (long)M * n * n;
  long blocks = (tot + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  update_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, M, mixing, G0, I2, G, res_bits);
  return cudaGetLastError();
}

cudaError_t launch_energy(int n, int M, double spin, const double *h, const double *V,
                          const double *G, const double *A, const double *w, double *part,
                          double *out, cudaStream_t s) {
  energy_part_kernel<<<M, 256, 0, s>>>(n, M, G, A, part);
  energy_final_kernel<<<1, 256, 0, s>>>(n, M, spin, h, V, G, w, part, out);
  return cudaGetLastError();
}

}  // namespace fedvr
