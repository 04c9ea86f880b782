// Hartree-Fock pieces (Sec. 2.3, Eqs. sigmahf, hamhf, hfgf): HF self-energy,
// chemical potential with Fermi occupations, and the eigenbasis factors of g^0.
#include "common.cuh"

#include <math.h>

namespace fedvr {
namespace {

// out = add + sigma diag(V diag rho) - V o rho - sub   (add/sub may be NULL)
__global__ void hf_selfenergy_kernel(int n, double spin, const double *__restrict__ rho,
                                     const double *__restrict__ V, const double *__restrict__ addm,
                                     const double *__restrict__ subm, double *__restrict__ out) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  int a = (int)(idx / n), b = (int)(idx % n);
  double v = -V[idx] * rho[idx];
  if (a == b) {
    double hart = 0.0;
    for (int k = 0; k < n; ++k) hart += V[(long)a * n + k] * rho[(long)k * n + k];
    v += spin * hart;
  }
  if (addm) v += addm[idx];
  if (subm) v -= subm[idx];
  out[idx] = v;
}

__device__ __forceinline__ double softplus(double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); }

// Block-wide reductions (blockDim.x = 256).
__device__ double block_max(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
  return r;
}
__device__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = sh[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
  return r;
}

// log-sum-exp of -softplus(beta * x_a) over a in [lo, hi), x_a = sgn*(mu - eps_a)
__device__ double lse_group(const double *eps, int lo, int hi, double mu, double beta, double sgn,
                            double *sh) {
  double m = -INFINITY;
  for (int a = lo + threadIdx.x; a < hi; a += blockDim.x)
    m = fmax(m, -softplus(beta * (sgn * (mu - eps[a]))));
  m = block_max(m, sh);
  double s = 0.0;
  for (int a = lo + threadIdx.x; a < hi; a += blockDim.x)
    s += exp(-softplus(beta * (sgn * (mu - eps[a]))) - m);
  s = block_sum(s, sh);
  return m + log(s);
}

// mu from the Fermi normalisation in balanced form: sum_{a<nocc} f(mu - eps_a)
// = sum_{a>=nocc} f(eps_a - mu), compared as log-sum-exps; bisection on
// [eps_0 - 1, eps_{n-1} + 1] until the midpoint stops moving. Then
// f_a = 1/(exp(beta (eps_a - mu)) + 1) in overflow-free form. eps ascending.
__global__ void mu_fermi_kernel(int n, int nocc, double beta, const double *eps, double *mu_out,
                                double *f) {
  __shared__ double sh[32];
  __shared__ double s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = eps[0] - 1.0;
    s_hi = eps[n - 1] + 1.0;
  }
  __syncthreads();
  for (int it = 0; it < 400; ++it) {
    double lo = s_lo, hi = s_hi;
    double mid = 0.5 * (lo + hi);
    if (!(lo < mid && mid < hi)) break;
    double holes = lse_group(eps, 0, nocc, mid, beta, 1.0, sh);
    double parts = lse_group(eps, nocc, n, mid, beta, -1.0, sh);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (holes - parts > 0.0) s_lo = mid; else s_hi = mid;
    }
    __syncthreads();
  }
  double mu = 0.5 * (s_lo + s_hi);
  if (threadIdx.x == 0) *mu_out = mu;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    double y = beta * (eps[a] - mu);
    if (y > 0.0) {
      double e = exp(-y);
      f[a] = e / (1.0 + e);
    } else {
      f[a] = 1.0 / (1.0 + exp(y));
    }
  }
}

// phi[j][a] = f(y_a) exp(-tau_j y_a), y_a = eps_a - mu, overflow-free (Eq. hfgf):
// y >= 0: exp(-(beta + x) y) / (1 + exp(-beta y)); y < 0: exp(-x y) / (1 + exp(beta y)).
__global__ void phi_table_kernel(int n, int M, double beta, const double *eps, const double *mu_dev,
                                 double mu_host, const double *tau, double *phi) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * n) return;
  int j = (int)(idx / n), a = (int)(idx % n);
  double mu = mu_dev ? *mu_dev : mu_host;
  double y = eps[a] - mu, x = tau[j];
  phi[idx] = (y >= 0.0) ? exp(-((beta + x) * y)) / (1.0 + exp(-(beta * y)))
                        : exp(-(x * y)) / (1.0 + exp(beta * y));
}

}  // namespace

cudaError_t launch_hf_selfenergy(int n, double spin, const double *rho, const double *V,
                                 const double *add, const double *sub, double *out,
                                 cudaStream_t s) {
  long nn = (long)n * n;
  hf_selfenergy_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, spin, rho, V, add, sub, out);
  return cudaGetLastError();
}

cudaError_t launch_mu_fermi(int n, int nocc, double beta, const double *eps, double *mu_out,
                            double *f, cudaStream_t s) {
  mu_fermi_kernel<<<1, 256, 0, s>>>(n, nocc, beta, eps, mu_out, f);
  return cudaGetLastError();
}

cudaError_t launch_phi_table(int n, int M, double beta, const double *eps, const double *mu_dev,
                             double mu_host, const double *tau, double *phi, cudaStream_t s) {
  long cnt = (long)M * n;
  phi_table_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(n, M, beta, eps, mu_dev, mu_host,
                                                                tau, phi);
  return cudaGetLastError();
}

}  // namespace fedvr
