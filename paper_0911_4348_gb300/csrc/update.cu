// Dyson update, residual and Galitskii-Migdal energy (Sec. 2.3, Eq. deq and
// the total-energy evaluation), with deterministic reductions.
#include "common.cuh"

#include <math.h>

namespace fedvr {
namespace {

// g_new = g^0 + I2; g' = (1 - a) g + a (g_new_ab + g_new_ba) / 2, evaluated as
// t = (g_new_ab + g_new_ba) / 2 - g (one add per pair, one fused multiply-add
// per element), g' = g + a t (fused), d = g' - g; res = max |d|, kept as the
// integer maximum of |d|'s bit pattern (the sign bit cleared), which orders
// non-negative doubles like their values and puts Inf and NaN above every
// finite value, so the comparison costs no FP64 instruction. An element then
// costs 4.5 FP64 instructions (the g_new add, half the pair add, two fused
// multiply-adds, the difference): at GB300's FP64 issue rate that, not HBM,
// bounds this kernel.
//
// One block per pair of 32 x 32 tiles (P, Q) = (rows ta, cols tb) and its
// mirror (rows tb, cols ta), ta <= tb, of one mesh point: both tiles of g^0 and
// I2 are read row-contiguously into shared memory, so the transposed partner
// of every element comes from shared memory instead of a strided global read.
constexpr int kUT = 32;

__device__ __forceinline__ double upd_one(double s, double old, double mixing,
                                          unsigned long long &m) {
  const double nw = fma(mixing, fma(0.5, s, -old), old);
  const unsigned long long d =
      (unsigned long long)__double_as_longlong(nw - old) & 0x7fffffffffffffffull;
  m = d > m ? d : m;
  return nw;
}

__global__ void __launch_bounds__(256) update_kernel(int n, int M, int nt, double mixing,
                                                     const double *__restrict__ G0,
                                                     const double *__restrict__ I2,
                                                     double *__restrict__ G,
                                                     unsigned long long *res_bits) {
  __shared__ double P[kUT][kUT + 1], Q[kUT][kUT + 1];
  const long nn = (long)n * n;
  const long pairs = (long)nt * (nt + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  unsigned long long m = 0ull;
  for (long w = blockIdx.x; w < (long)M * pairs; w += gridDim.x) {
    const int j = (int)(w / pairs);
    long p = w % pairs;
    int ta = 0;  // pair p -> (ta, tb), ta <= tb, row-major over the upper triangle
    while (p >= nt - ta) {
      p -= nt - ta;
      ++ta;
    }
    const int tb = ta + (int)p;
    const long base = (long)j * nn;
    // g_new of tile (ta, tb) into P and of tile (tb, ta) into Q; the old g of
    // both tiles into registers in the same pass (one memory round trip)
    double oP[4], oQ[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      const int a = ta * kUT + r, b = tb * kUT + tx;
      oP[q] = oQ[q] = 0.0;
      if (a < n && b < n) {
        const long idx = base + (long)a * n + b;
        P[r][tx] = __dadd_rn(G0[idx], I2[idx]);
        oP[q] = G[idx];
      }
      const int a2 = tb * kUT + r, b2 = ta * kUT + tx;
      if (a2 < n && b2 < n) {
        const long idx = base + (long)a2 * n + b2;
        Q[r][tx] = __dadd_rn(G0[idx], I2[idx]);
        oQ[q] = G[idx];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      const int a = ta * kUT + r, b = tb * kUT + tx;
      // element (a, b) pairs with (b, a) = Q[tx][r]; the pair's sum serves both
      const double sab = P[r][tx] + Q[tx][r];
      if (a < n && b < n) G[base + (long)a * n + b] = upd_one(sab, oP[q], mixing, m);
      if (ta != tb) {
        const int a2 = tb * kUT + r, b2 = ta * kUT + tx;
        if (a2 < n && b2 < n)
          G[base + (long)a2 * n + b2] = upd_one(Q[r][tx] + P[tx][r], oQ[q], mixing, m);
      }
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(res_bits, m);
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

// part[j kE + c] = sum over chunk c of the n^2 entries of A[M-1-j] o G[j]
// (kE blocks per mesh point, so that the M kE blocks fill the GPU; the chunks
// are added in a fixed order by energy_final_kernel).
constexpr int kE = 4;
__global__ void energy_part_kernel(int n, int M, const double *__restrict__ G,
                                   const double *__restrict__ A, double *__restrict__ part) {
  const int j = blockIdx.x / kE, c = blockIdx.x % kE;
  const long nn = (long)n * n;
  const long lo = nn * c / kE, hi = nn * (c + 1) / kE;
  const double *g = G + (long)j * nn;
  const double *s = A + (long)(M - 1 - j) * nn;
  double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0, acc3 = 0.0;
  long e = lo + threadIdx.x;
  for (; e + 768 < hi; e += 1024) {  // four independent load pairs in flight per thread
    const double s0 = s[e], s1 = s[e + 256], s2 = s[e + 512], s3 = s[e + 768];
    const double g0 = g[e], g1 = g[e + 256], g2 = g[e + 512], g3 = g[e + 768];
    acc0 = fma(s0, g0, acc0);
    acc1 = fma(s1, g1, acc1);
    acc2 = fma(s2, g2, acc2);
    acc3 = fma(s3, g3, acc3);
  }
  for (; e < hi; e += 256) acc0 = fma(s[e], g[e], acc0);
  const double acc = block_sum256((acc0 + acc1) + (acc2 + acc3));
  if (threadIdx.x == 0) part[(long)j * kE + c] = acc;
}

// Row partials of the one-body energy terms, one block per row a:
// rows[a] = sum_b h_ab rho_ab, rows[n + a] = sum_b Sigma^HF_ab rho_ab with
// Sigma^HF_ab = sigma delta_ab sum_k V_ak rho_kk - V_ab rho_ab, rows[2n + a] = rho_aa.
__global__ void energy_rows_kernel(int n, int M, double spin, const double *__restrict__ h,
                                   const double *__restrict__ V, const double *__restrict__ G,
                                   double *__restrict__ rows) {
  const int a = blockIdx.x;
  const long nn = (long)n * n;
  const double *rho = G + (long)(M - 1) * nn;
  double e1 = 0.0, e2 = 0.0, hart = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    const long e = (long)a * n + b;
    const double r = rho[e];
    e1 += h[e] * r;
    e2 += (-V[e] * r) * r;
    hart += V[e] * rho[(long)b * n + b];
  }
  e1 = block_sum256(e1);
  e2 = block_sum256(e2);
  hart = block_sum256(hart);
  if (threadIdx.x == 0) {
    const double raa = rho[(long)a * n + a];
    rows[a] = e1;
    rows[n + a] = e2 + spin * hart * raa;
    rows[2 * n + a] = raa;
  }
}

// out[0] = E0 = sigma Tr[h rho] + (sigma/2) Tr[Sigma^HF[rho] rho]
//              - (sigma/2) sum_j w_j part[j];  out[1] = N = sigma Tr rho;  rho = G[M-1].
// With rows (from energy_rows_kernel) the one-body sums are taken over its row
// partials in a fixed order; without, directly (single-matrix use by the HF loop).
__global__ void energy_final_kernel(int n, int M, double spin, const double *__restrict__ h,
                                    const double *__restrict__ V, const double *__restrict__ G,
                                    const double *__restrict__ w, const double *__restrict__ part,
                                    const double *__restrict__ rows, double *out) {
  long nn = (long)n * n;
  const double *rho = G + (long)(M - 1) * nn;
  double e1 = 0.0, e2 = 0.0, tr = 0.0, ec = 0.0;
  if (rows) {
    for (int a = threadIdx.x; a < n; a += blockDim.x) {
      e1 += rows[a];
      e2 += rows[n + a];
      tr += rows[2 * n + a];
    }
  } else {
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
  }
  if (part)
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
      double pj = 0.0;
      for (int c = 0; c < kE; ++c) pj += part[(long)j * kE + c];
      ec += w[j] * pj;
    }
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

// One-electron density at the nodes (Sec. 2.3): n(x) sums chi chi g(0^-) over
// basis pairs, and a DVR function is 1/sqrt(W_a) at its own node and zero at the
// others, so n(x_a) = spin g_aa(0^-) / W_a (g per spin, N = spin Tr g(0^-)).
__global__ void density_kernel(int n, const double *__restrict__ g, const double *__restrict__ W,
                               double spin, double *__restrict__ out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < n) out[a] = spin * g[(size_t)a * n + a] / W[a];
}

}  // namespace

cudaError_t launch_density(int n, const double *g, const double *W, double spin, double *out,
                           cudaStream_t s) {
  density_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, g, W, spin, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(size_t count, double a, const double *x, double b, const double *y,
                         double *out, cudaStream_t s) {
  axpby_kernel<<<512, 256, 0, s>>>(count, a, x, b, y, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_hf(int n, double spin, const double *h, const double *V,
                             const double *rho, double *out, cudaStream_t s) {
  // a one-point "stack" whose only member is rho, with no correlation term
  energy_final_kernel<<<1, 256, 0, s>>>(n, 1, spin, h, V, rho, nullptr, nullptr, nullptr, out);
  return cudaGetLastError();
}

cudaError_t launch_update(int n, int M, double mixing, const double *G0, const double *I2,
                          double *G, unsigned long long *res_bits, cudaStream_t s) {
  const int nt = (n + kUT - 1) / kUT;
  const long work = (long)M * nt * (nt + 1) / 2;
  const long blocks = work < 152 * 16 ? work : 152 * 16;
  update_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, M, nt, mixing, G0, I2, G, res_bits);
  return cudaGetLastError();
}

// part holds kE M + 3 n doubles: the per-mesh-point correlation sums in kE
// chunks, then the row partials.
cudaError_t launch_energy(int n, int M, double spin, const double *h, const double *V,
                          const double *G, const double *A, const double *w, double *part,
                          double *out, cudaStream_t s) {
  energy_part_kernel<<<M * kE, 256, 0, s>>>(n, M, G, A, part);
  energy_rows_kernel<<<n, 256, 0, s>>>(n, M, spin, h, V, G, part + (long)kE * M);
  energy_final_kernel<<<1, 256, 0, s>>>(n, M, spin, h, V, G, w, part, part + (long)kE * M, out);
  return cudaGetLastError();
}

}  // namespace fedvr
