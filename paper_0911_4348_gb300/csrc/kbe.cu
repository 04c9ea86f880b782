// Real-time two-time Kadanoff-Baym propagation (Sec. 2, Eqs. kbe, skkbe,
// skkbesigma with the HF part of Eq. sigmahf and the second-Born part of Eq.
// sigma2ndb), from an uncorrelated initial state: complex FP64, or with the
// dense contractions as split-TF32 tensor-core products (precision 1, below).
//
// Functions and layout. L = -i G^< and Gt = -i G^> (so L(t, t) = rho(t),
// Gt(t, t) = rho(t) - 1, F(t', t) = F(t, t')^H) on the uniform grid
// t_k = k dt, k = 0 .. T-1, stored as two full square matrices of T x T
// blocks: block (s, j) of F is n x n at F + (s n) ld + j n with ld = T n
// complex elements (interleaved double2). Both triangles are kept (the upper
// one written as the mirror of each new time row), so every contraction reads
// whole blocks along rows. Self-energies are needed only on the current time
// row: S[w][k] (w = 0: s^< = -i Sigma^<, w = 1: s^> = -i Sigma^>) at
// S + (w T + k) n n.
//
// One step N -> N+1 (Heun predictor-corrector, trapezoid collision integrals):
//   R0 = rhs(N, j = 0..N); predictor row N+1; HF and self-energy row N+1;
//   R1 = rhs(N+1, j = 0..N+1); corrector row N+1; HF and self-energy row N+1;
//   observables at N+1 (K_L(t, t) from one more collision block).
// with rhs(i, j) = -i h_HF(t_i) F(i, j) + K_F(i, j),
//   K_L = sum_{s<=i} w^i_s [s^> - s^<](i, s) L(s, j) + sum_{s<=j} w^j_s s^<(i, s) [L - Gt](s, j),
//   K_G = sum_{s<=i} w^i_s [s^> - s^<](i, s) Gt(s, j) + sum_{s<=j} w^j_s s^>(i, s) [L - Gt](s, j),
// w^m_s the trapezoid weights on [0, t_m] (dt, halved at both ends; zero for m = 0).
//
// Every FP64 kernel here is bound by GB300's FP64 pipe (2 DFMA per clock per
// SM): operands come from shared memory or L1, and the work per launch is
// counted in complex multiply-adds (4 DFMA each).
//
// Split-TF32 mode (precision 1): the two collision integrals of a time row run
// as split-TF32 tensor-core products (gemm_tc.cu) over FP32 planar shadows of
// L, Gt and the trapezoid-weighted L - Gt, written beside the FP64 matrices by
// every advance: shadow w (0 L, 1 Gt, 2 Dw) holds at row j n + c, column
// (2 s + p) n + b (rows of 2 T n values padded to a multiple of 32, so the
// contraction index is contiguous and every row starts 128-byte aligned)
// part p (re, im) of F(s, j)[b][c], and Dw(s, j) = w^j_s (L - Gt)(s, j)
// for s <= j, zero below (so the second integral is a plain product over
// s <= j, block-triangular in (s, j)). The left factors of both integrals are
// laid out as real [2n][2 T n] matrices (rows re/im of the output, columns
// (s, p, b)) that turn each complex product into one real product. The
// -i h_HF F term, the energy's K_L(t, t), the HF self-energy and the stepping
// stay in FP64. For n_b <= 64 the mode also runs the second-Born self-energy
// row on cheaper arithmetic: the exchange products P^(b)_ak = sum_l g_al V_bl
// gb_lk of all entries as one batched split-TF32 product, the exchange's k-sum
// and the direct term V Q V in FP32 on the CUDA cores (their inputs carry the
// products' precision); for n_b > 64 the self-energy stays FP64.
#include <algorithm>

#include "common.cuh"
#include "tc_sys.cuh"

namespace fedvr {
namespace {

constexpr int kKbeMaxN = 80;  // exchange operands (2 n^2 + 1024 complex) fit one CTA's shared memory

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ void cmla(double2 &acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 conjz(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 addz(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 subz(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 scalez(double s, double2 a) {
  return make_double2(s * a.x, s * a.y);
}
__host__ __device__ __forceinline__ long blk(int s, int j, int n, long ld) {
  return (long)s * n * ld + (long)j * n;
}
// element (s, j)[b][c], part p, of a planar two-time shadow (row j n + c of pitch
// shld, column (2 s + p) n + b)
__device__ __forceinline__ long shi(int s, int j, int b, int c, int p, int n, long shld) {
  return ((long)j * n + c) * shld + ((long)2 * s + p) * n + b;
}
// trapezoid weight of point s on [0, t_m]
__device__ __forceinline__ double trap_w(int s, int m, double dt) {
  if (m == 0) return 0.0;
  return (s == 0 || s == m) ? 0.5 * dt : dt;
}

// Block (0, 0): L = rho0 (complex, already in place), Gt = L - 1.
__global__ void g_from_l_kernel(int n, long ld, long off, const double2 *L, double2 *G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int b = idx / n, c = idx % n;
  double2 v = L[off + b * ld + c];
  if (b == c) v.x -= 1.0;
  G[off + b * ld + c] = v;
}

// Real n x n density -> complex block of L (imaginary part zero).
__global__ void rho_real_kernel(int n, long ld, const double *rho, double2 *L) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int b = idx / n, c = idx % n;
  L[b * ld + c] = make_double2(rho[idx], 0.0);
}

// h_HF = h + diag(dv) + Sigma^HF[rho], Sigma^HF = spin diag(V diag rho) - V o rho
// (Eq. sigmahf with rho = L(t, t)).
__global__ void hf_kernel(int n, double spin, const double *h, const double *dv, const double *V,
                          const double2 *L, long off, long ld, double2 *out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int a = idx / n, b = idx % n;
  const double2 r = L[off + a * ld + b];
  const double vab = V[idx];
  double2 s = make_double2(-vab * r.x, -vab * r.y);
  if (a == b) {
    double2 H = make_double2(0.0, 0.0);
    for (int c = 0; c < n; ++c) {
      const double2 rc = L[off + (long)c * ld + c];
      H.x = fma(V[a * n + c], rc.x, H.x);
      H.y = fma(V[a * n + c], rc.y, H.y);
    }
    s.x = spin * H.x + s.x;
    s.y = spin * H.y + s.y;
  }
  const double hd = h[idx] + ((a == b && dv) ? dv[a] : 0.0);
  out[idx] = make_double2(hd + s.x, s.y);
}

// Second-Born self-energy of row i, entry e = 2k + w (w = 0: s^< from
// g = L(i, k), H = Gt(i, k); w = 1: s^> from g = Gt(i, k), H = L(i, k)), with
// the reversed line gb = -H^H:
//   S = spin g o (V Q V) - X,  Q_kl = g_kl gb_lk = -g_kl conj(H_kl),
//   X_ab = sum_kl V_ak V_bl g_al gb_lk g_kb.
// First V Q into T1 [e][n][n].
__global__ void vq_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                          const double *V, double2 *T1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int e = blockIdx.y, kt = e >> 1, w = e & 1;
  const int a = idx / n, l = idx % n;
  const long off = blk(i, kt, n, ld);
  const double2 *g = (w ? G : L) + off, *H = (w ? L : G) + off;
  double2 acc = make_double2(0.0, 0.0);
  for (int k = 0; k < n; ++k) {
    const double2 q = cmul(g[k * ld + l], conjz(H[k * ld + l]));  // -Q_kl
    const double v = V[a * n + k];
    acc.x = fma(-v, q.x, acc.x);
    acc.y = fma(-v, q.y, acc.y);
  }
  T1[(long)e * n * n + idx] = acc;
}

// Direct term S_e = spin g o (T1 V), written to the row's S[w][k].
__global__ void direct_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                              const double *V, const double2 *T1, double spin, int Tcap,
                              double2 *S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int e = blockIdx.y, kt = e >> 1, w = e & 1;
  const int a = idx / n, b = idx % n;
  const double2 *t1 = T1 + (long)e * n * n + (long)a * n;
  double2 W = make_double2(0.0, 0.0);
  for (int l = 0; l < n; ++l) {
    const double v = V[l * n + b];
    W.x = fma(t1[l].x, v, W.x);
    W.y = fma(t1[l].y, v, W.y);
  }
  const double2 g = (w ? G : L)[blk(i, kt, n, ld) + a * ld + b];
  S[((long)w * Tcap + kt) * n * n + idx] = cmul(scalez(spin, g), W);
}

// Exchange term (n > 16), one CTA per (column b, entry e): with g and
// Hb_lk = V_bl gb_lk in shared memory, the (a, k) pairs of a chunk of rows
// are spread over the threads (four per thread), each computing
// P_ak = sum_l g_al Hb_lk and v_ak = V_ak P_ak g_kb into shared memory; then
// one thread per row adds X_ab = sum_k v_ak in k order and S_ab -= X_ab.
// Small n (<= 16): one warp per row a, lanes over k, warp-shuffle sum over k
// (fewer FP64 instructions in the k-sum than the pair layout below).
__global__ void __launch_bounds__(256) exchange_rows_kernel(int n, int i, long ld,
                                                            const double2 *L, const double2 *G,
                                                            const double *V, int Tcap,
                                                            double2 *S) {
  extern __shared__ double2 xs[];
  double2 *gs = xs, *hb = xs + n * n;
  const int b = blockIdx.x, e = blockIdx.y, kt = e >> 1, w = e & 1;
  const long off = blk(i, kt, n, ld);
  const double2 *g = (w ? G : L) + off, *H = (w ? L : G) + off;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int r = q / n, c = q % n;
    gs[q] = g[r * ld + c];
    const double2 h = H[r * ld + c];
    const double v = V[b * n + c];
    hb[c * n + r] = make_double2(-v * h.x, v * h.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double2 *Sout = S + ((long)w * Tcap + kt) * n * n;
  for (int a = warp; a < n; a += 8) {
    double2 part = make_double2(0.0, 0.0);
    for (int k = lane; k < n; k += 32) {
      double2 P = make_double2(0.0, 0.0);
      for (int l = 0; l < n; ++l) cmla(P, gs[a * n + l], hb[l * n + k]);
      cmla(part, scalez(V[a * n + k], P), gs[k * n + b]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
      part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
    }
    if (lane == 0) Sout[a * n + b] = subz(Sout[a * n + b], part);
  }
}

constexpr int kXPairs = 4;  // (a, k) pairs per thread and chunk
inline int xchg_rows(int n) { return n < 256 * kXPairs / n ? n : 256 * kXPairs / n; }

__global__ void __launch_bounds__(256) exchange_kernel(int n, int i, long ld, const double2 *L,
                                                       const double2 *G, const double *V,
                                                       int Tcap, double2 *S) {
  extern __shared__ double2 xs[];
  const int rows = n < 256 * kXPairs / n ? n : 256 * kXPairs / n;
  double2 *gs = xs, *hb = xs + n * n, *vs = xs + 2 * n * n;
  const int b = blockIdx.x, e = blockIdx.y, kt = e >> 1, w = e & 1;
  const long off = blk(i, kt, n, ld);
  const double2 *g = (w ? G : L) + off, *H = (w ? L : G) + off;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int r = q / n, c = q % n;
    gs[q] = g[r * ld + c];
    // H_rc enters as gb_cr = -conj(H_rc), so Hb[c][r] = -V_bc conj(H_rc)
    const double2 h = H[r * ld + c];
    const double v = V[b * n + c];
    hb[c * n + r] = make_double2(-v * h.x, v * h.y);
  }
  __syncthreads();
  double2 *Sout = S + ((long)w * Tcap + kt) * n * n;
  for (int a0 = 0; a0 < n; a0 += rows) {
    const int nr = min(rows, n - a0), np = nr * n;
    int pa[kXPairs], pk[kXPairs];
    double2 P[kXPairs];
#pragma unroll
    for (int q = 0; q < kXPairs; ++q) {
      const int pp = threadIdx.x + 256 * q;
      pa[q] = pp < np ? a0 + pp / n : a0;
      pk[q] = pp < np ? pp % n : 0;
      P[q] = make_double2(0.0, 0.0);
    }
    for (int l = 0; l < n; ++l) {
#pragma unroll
      for (int q = 0; q < kXPairs; ++q) cmla(P[q], gs[pa[q] * n + l], hb[l * n + pk[q]]);
    }
#pragma unroll
    for (int q = 0; q < kXPairs; ++q) {
      const int pp = threadIdx.x + 256 * q;
      if (pp < np) {
        double2 v = make_double2(0.0, 0.0);
        cmla(v, scalez(V[pa[q] * n + pk[q]], P[q]), gs[pk[q] * n + b]);
        vs[pp] = v;
      }
    }
    __syncthreads();
    if (threadIdx.x < nr) {
      double2 x = make_double2(0.0, 0.0);
      const double2 *vr = vs + threadIdx.x * n;
      for (int k = 0; k < n; ++k) x = addz(x, vr[k]);
      const int a = a0 + threadIdx.x;
      Sout[a * n + b] = subz(Sout[a * n + b], x);
    }
    __syncthreads();
  }
}

// Split mode's direct term and exchange k-sum in FP32 (their inputs carry the
// split products' precision): T1 = V Q as float2, then S = spin g o (T1 V).
__global__ void vq32_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                            const double *V, float2 *T1) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int e = blockIdx.y, kt = e >> 1, w = e & 1;
  const int a = idx / n, l = idx % n;
  const long off = blk(i, kt, n, ld);
  const double2 *g = (w ? G : L) + off, *H = (w ? L : G) + off;
  float2 acc = make_float2(0.f, 0.f);
  for (int k = 0; k < n; ++k) {
    const double2 gg = g[k * ld + l], hh = H[k * ld + l];
    const float gr = (float)gg.x, gi = (float)gg.y, hr = (float)hh.x, hi = (float)hh.y;
    const float qr = gr * hr + gi * hi, qi = gi * hr - gr * hi;  // g conj(H) = -Q_kl
    const float v = (float)V[a * n + k];
    acc.x = fmaf(-v, qr, acc.x);
    acc.y = fmaf(-v, qi, acc.y);
  }
  T1[(long)e * n * n + idx] = acc;
}
__global__ void direct32_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                                const double *V, const float2 *T1, double spin, int Tcap,
                                double2 *S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int e = blockIdx.y, kt = e >> 1, w = e & 1;
  const int a = idx / n, b = idx % n;
  const float2 *t1 = T1 + (long)e * n * n + (long)a * n;
  float2 W = make_float2(0.f, 0.f);
  for (int l = 0; l < n; ++l) {
    const float v = (float)V[l * n + b];
    W.x = fmaf(t1[l].x, v, W.x);
    W.y = fmaf(t1[l].y, v, W.y);
  }
  const double2 g = (w ? G : L)[blk(i, kt, n, ld) + a * ld + b];
  S[((long)w * Tcap + kt) * n * n + idx] = cmul(scalez(spin, g), make_double2(W.x, W.y));
}

// Operands of the batched exchange product of row i, entry e = 2k + w:
// Ap_e[(p, a)][(q, l)] the real form of g (rows re/im of the output, columns
// re/im parts of the contraction), Bp_e[(b, k)][(q, l)] = part q of
// V_bl gb_lk = -V_bl conj(H_kl).
__global__ void xop_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                           const double *V, int xld, float *Ap, float *Bp) {
  const int e = blockIdx.y, kt = e >> 1, w = e & 1;
  const long off = blk(i, kt, n, ld), n2 = (long)n * n;
  const double2 *g = (w ? G : L) + off, *H = (w ? L : G) + off;
  float *A = Ap + (long)e * 2 * n * xld, *B = Bp + (long)e * n2 * xld;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n2 * n; q += (long)gridDim.x * blockDim.x) {
    const int b = (int)(q / n2), k = (int)((q / n) % n), l = (int)(q % n);
    const double2 h = H[k * ld + l];
    const double v = V[b * n + l];
    float *row = B + ((long)b * n + k) * xld;
    row[l] = (float)(-v * h.x);
    row[n + l] = (float)(v * h.y);
    if (q < n2) {  // Ap from g: element (a, l) = (k, l) here
      const int a = (int)(q / n), ll = (int)(q % n);
      const double2 x = g[a * ld + ll];
      A[(long)a * xld + ll] = (float)x.x;
      A[(long)a * xld + n + ll] = (float)(-x.y);
      A[(long)(n + a) * xld + ll] = (float)x.y;
      A[(long)(n + a) * xld + n + ll] = (float)x.x;
    }
  }
}

// k-sum of the exchange from the product (FP32, like the product): S_e[a][b] -=
// sum_k V_ak P_ak g_kb with P_ak = P_e[(b, k)][(0, a)] + i P_e[(b, k)][(1, a)];
// thread per (a, b).
__global__ void xsum_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                            const double *V, const float *P, int Tcap, double2 *S) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int e = blockIdx.y, kt = e >> 1, w = e & 1, a = idx % n, b = idx / n;
  const long off = blk(i, kt, n, ld), n2 = (long)n * n;
  const double2 *g = (w ? G : L) + off;
  const float *Pe = P + (long)e * 2 * n2 * n;
  float xr = 0.f, xi = 0.f;
  for (int k = 0; k < n; ++k) {
    const float *pr = Pe + ((long)b * n + k) * 2 * n;
    const double2 gk = g[k * ld + b];
    const float v = (float)V[a * n + k], pre = v * pr[a], pim = v * pr[n + a];
    const float gr = (float)gk.x, gi = (float)gk.y;
    xr = fmaf(pre, gr, xr);
    xr = fmaf(-pim, gi, xr);
    xi = fmaf(pre, gi, xi);
    xi = fmaf(pim, gr, xi);
  }
  double2 *Se = S + ((long)w * Tcap + kt) * n2;
  Se[a * n + b] = subz(Se[a * n + b], make_double2(xr, xi));
}

struct CollArgs {
  int n, i, j0, Tcap;
  long ld;
  double dt;
  const double2 *L, *G, *S, *hHF;
  double2 *RL, *RG;
  int mode;    // 0: rhs of L and Gt for columns j0 .. j0 + ncols - 1; 1: K_L(i, j0) only
  int corr;    // 0: no collision integrals (time-dependent HF)
  int ncols;   // output column blocks j
  int splits;  // CTAs sharing one column's contraction (partial sums in part)
  int rows;    // output rows a per CTA (rows * n <= 256 * kCollQ)
  double2 *part;  // [splits][ncols][2][n n] partial sums (splits > 1)
};

constexpr int kCollQ = 8;   // outputs per thread
constexpr int kCollKC = 16; // contraction index b per staged slice

// Collision integrals (and with mode 0 the -i h_HF F term) for one time row i.
// CTA (column j, split, row tile): its rows x n outputs of block j are spread
// over the 256 threads (output o = tid + 256 q, q < kCollQ), so no output is
// padded. The terms of column j,
//   kind 0: -i h_HF(i) x [L(i, j), Gt(i, j)]                       (mode 0)
//   kind 1: w^i_s (s^> - s^<)(i, s) x [L(s, j), Gt(s, j)],  s = 0..i
//   kind 2: [w^j_s s^<(i, s), w^j_s s^>(i, s)] x (L - Gt)(s, j), s = 0..j
// times the 16-wide slices of b form a list of units; split k of S takes
// units [U k / S, U (k+1) / S) (an empty range writes zeros). Each unit stages its left factors X [rows][16]
// and right factors Y [16][n] in shared memory.
__global__ void __launch_bounds__(256, 2) collision_kernel(CollArgs p) {
  extern __shared__ double2 cs[];
  const int n = p.n, i = p.i, rows = p.rows;
  double2 *X0 = cs, *X1 = X0 + rows * kCollKC, *Y0 = X1 + rows * kCollKC, *Y1 = Y0 + kCollKC * n;
  const int split = blockIdx.x % p.splits, jj = blockIdx.x / p.splits, j = p.j0 + jj;
  const long ld = p.ld, nn = (long)n * n;
  const int a0 = blockIdx.y * rows, nr = min(rows, n - a0), nout = nr * n;
  const int tid = threadIdx.x;
  const double2 *SL = p.S, *SG = p.S + (long)p.Tcap * nn;
  double2 accL[kCollQ], accG[kCollQ];
  int xo[kCollQ], yo[kCollQ];
  int nq = 0;
#pragma unroll
  for (int q = 0; q < kCollQ; ++q) {
    accL[q] = accG[q] = make_double2(0.0, 0.0);
    const int o = tid + 256 * q;
    xo[q] = (o < nout) ? (o / n) * kCollKC : 0;
    yo[q] = (o < nout) ? o % n : 0;
    nq += (o < nout) ? 1 : 0;
  }
  const int n0 = p.mode == 0 ? 1 : 0;
  const int n1 = (p.corr && i > 0) ? i + 1 : 0;
  const int n2 = (p.corr && j > 0) ? j + 1 : 0;
  const int nch = (n + kCollKC - 1) / kCollKC;
  const long units = (long)(n0 + n1 + n2) * nch;
  const long u0 = units * split / p.splits, u1 = units * (split + 1) / p.splits;
  for (long u = u0; u < u1; ++u) {
    const int t = (int)(u / nch), bc = (int)(u % nch) * kCollKC;
    const int kind = t < n0 ? 0 : (t < n0 + n1 ? 1 : 2);
    const int s = kind == 0 ? i : (kind == 1 ? t - n0 : t - n0 - n1);
    const double w = kind == 1 ? trap_w(s, i, p.dt) : (kind == 2 ? trap_w(s, j, p.dt) : 0.0);
    const long fb = blk(s, j, n, ld);
    const int nb = min(kCollKC, n - bc);
    for (int q = tid; q < nr * kCollKC; q += 256) {
      const int r = q / kCollKC, bb = q % kCollKC, a = a0 + r, b = bc + bb;
      double2 x0 = make_double2(0.0, 0.0), x1 = x0;
      if (bb < nb) {
        if (kind == 0) {
          const double2 hv = p.hHF[a * n + b];
          x0 = make_double2(hv.y, -hv.x);  // -i h
        } else {
          const double2 sl = SL[(long)s * nn + a * n + b], sg = SG[(long)s * nn + a * n + b];
          if (kind == 1) {
            x0 = scalez(w, subz(sg, sl));
          } else {
            x0 = scalez(w, sl);
            x1 = scalez(w, sg);
          }
        }
      }
      X0[q] = x0;
      X1[q] = x1;
    }
    for (int q = tid; q < nb * n; q += 256) {
      const int bb = q / n, c = q % n, b = bc + bb;
      const double2 l = p.L[fb + b * ld + c], g = p.G[fb + b * ld + c];
      if (kind == 2) {
        Y0[q] = subz(l, g);
      } else {
        Y0[q] = l;
        Y1[q] = g;
      }
    }
    __syncthreads();
    if (kind == 2) {
#pragma unroll 2
      for (int bb = 0; bb < nb; ++bb) {
#pragma unroll
        for (int q = 0; q < kCollQ; ++q)
          if (q < nq) {
            const double2 yd = Y0[bb * n + yo[q]];
            cmla(accL[q], X0[xo[q] + bb], yd);
            cmla(accG[q], X1[xo[q] + bb], yd);
          }
      }
    } else {
#pragma unroll 2
      for (int bb = 0; bb < nb; ++bb) {
#pragma unroll
        for (int q = 0; q < kCollQ; ++q)
          if (q < nq) {
            const double2 xa = X0[xo[q] + bb];
            cmla(accL[q], xa, Y0[bb * n + yo[q]]);
            cmla(accG[q], xa, Y1[bb * n + yo[q]]);
          }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kCollQ; ++q) {
    if (q >= nq) break;
    const int o = tid + 256 * q, a = a0 + o / n, c = o % n;
    const long e = (long)a * n + c;
    if (p.splits > 1) {
      double2 *P = p.part + ((long)(split * p.ncols + jj) * 2) * nn;
      P[e] = accL[q];
      P[nn + e] = accG[q];
    } else if (p.mode == 0) {
      p.RL[(long)j * nn + e] = accL[q];
      p.RG[(long)j * nn + e] = accG[q];
    } else {
      p.RL[e] = accL[q];
    }
  }
}

// Sum of the splits' partial results in split order (deterministic).
__global__ void coll_reduce_kernel(int n, int j0, int ncols, int splits, int mode,
                                   const double2 *part, double2 *RL, double2 *RG) {
  const long nn = (long)n * n;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  const int jj = blockIdx.y;
  double2 sl = make_double2(0.0, 0.0), sg = sl;
  for (int k = 0; k < splits; ++k) {
    const double2 *P = part + ((long)(k * ncols + jj) * 2) * nn;
    sl = addz(sl, P[e]);
    sg = addz(sg, P[nn + e]);
  }
  if (mode == 0) {
    RL[(long)(j0 + jj) * nn + e] = sl;
    RG[(long)(j0 + jj) * nn + e] = sg;
  } else {
    RL[e] = sl;
  }
}

// Predictor (R1 == nullptr) or corrector of time row N+1 and its mirror column.
__global__ void advance_kernel(int n, int N, long ld, double2 *L, double2 *G, const double2 *R0L,
                               const double2 *R0G, const double2 *R1L, const double2 *R1G,
                               double dt, float *sh, long shz, long shld) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int j = blockIdx.y, b = idx / n, c = idx % n;
  const long nn = (long)n * n;
  if (j <= N) {
    double2 dl = R0L[(long)j * nn + idx], dg = R0G[(long)j * nn + idx];
    double f = dt;
    if (R1L) {
      dl = addz(dl, R1L[(long)j * nn + idx]);
      dg = addz(dg, R1G[(long)j * nn + idx]);
      f = 0.5 * dt;
    }
    const double2 vl = addz(L[blk(N, j, n, ld) + b * ld + c], scalez(f, dl));
    const double2 vg = addz(G[blk(N, j, n, ld) + b * ld + c], scalez(f, dg));
    L[blk(N + 1, j, n, ld) + b * ld + c] = vl;
    G[blk(N + 1, j, n, ld) + b * ld + c] = vg;
    L[blk(j, N + 1, n, ld) + c * ld + b] = conjz(vl);
    G[blk(j, N + 1, n, ld) + c * ld + b] = conjz(vg);
    if (sh) {
      const long pim = n;  // from part re to part im
      const long r0 = shi(N + 1, j, b, c, 0, n, shld);  // (N+1, j)[b][c]
      const long m0 = shi(j, N + 1, c, b, 0, n, shld);  // (j, N+1)[c][b]
      sh[r0] = (float)vl.x;
      sh[r0 + pim] = (float)vl.y;
      sh[shz + r0] = (float)vg.x;
      sh[shz + r0 + pim] = (float)vg.y;
      sh[m0] = (float)vl.x;
      sh[m0 + pim] = (float)(-vl.y);
      sh[shz + m0] = (float)vg.x;
      sh[shz + m0 + pim] = (float)(-vg.y);
      // Dw(j, N+1) = w^{N+1}_j (L - Gt)(j, N+1), the conjugate transpose of row N+1's
      const double wt = j == 0 ? 0.5 * dt : dt;
      sh[2 * shz + m0] = (float)(wt * (vl.x - vg.x));
      sh[2 * shz + m0 + pim] = (float)(-(wt * (vl.y - vg.y)));
    }
  } else {
    // equal times: d rho/dt = X + X^H with X = rhs_L(t, t)
    double2 d = addz(R0L[(long)N * nn + b * n + c], conjz(R0L[(long)N * nn + c * n + b]));
    double f = dt;
    if (R1L) {
      const double2 d1 =
          addz(R1L[(long)(N + 1) * nn + b * n + c], conjz(R1L[(long)(N + 1) * nn + c * n + b]));
      d = addz(d, d1);
      f = 0.5 * dt;
    }
    const double2 v = addz(L[blk(N, N, n, ld) + b * ld + c], scalez(f, d));
    const double2 vg = make_double2(v.x - (b == c ? 1.0 : 0.0), v.y);
    L[blk(N + 1, N + 1, n, ld) + b * ld + c] = v;
    G[blk(N + 1, N + 1, n, ld) + b * ld + c] = vg;
    if (sh) {
      const long pim = n;
      const long r0 = shi(N + 1, N + 1, b, c, 0, n, shld);
      sh[r0] = (float)v.x;
      sh[r0 + pim] = (float)v.y;
      sh[shz + r0] = (float)vg.x;
      sh[shz + r0 + pim] = (float)vg.y;
      sh[2 * shz + r0] = (float)(0.5 * dt * (v.x - vg.x));
      sh[2 * shz + r0 + pim] = (float)(0.5 * dt * (v.y - vg.y));
    }
  }
}

// E(t) = spin Tr[h(t) rho] + spin/2 Tr[Sigma^HF rho] + spin/2 Re Tr[i K_L(t, t)]
// and N(t) = spin Tr rho; one CTA, fixed-order reduction.
__global__ void observe_kernel(int n, double spin, const double *h, const double *dv,
                               const double *V, const double2 *L, long off, long ld,
                               const double2 *K, double *E_out, double *N_out) {
  __shared__ double red[4][256];
  const int tid = threadIdx.x;
  double e1 = 0.0, e2 = 0.0, ek = 0.0, nn_ = 0.0;
  for (int idx = tid; idx < n * n; idx += 256) {
    const int a = idx / n, b = idx % n;
    const double2 rab = L[off + a * ld + b], rba = L[off + b * ld + a];
    e1 += h[idx] * rba.x;                         // Re h_ab rho_ba (h real)
    e2 -= V[idx] * cmul(rab, rba).x;              // exchange: -V_ab rho_ab rho_ba
    if (a == b) {
      const double2 raa = rab;
      double2 H = make_double2(0.0, 0.0);
      for (int c = 0; c < n; ++c) {
        const double2 rc = L[off + (long)c * ld + c];
        H.x = fma(V[a * n + c], rc.x, H.x);
        H.y = fma(V[a * n + c], rc.y, H.y);
      }
      e2 += spin * cmul(H, raa).x;                // Hartree
      if (dv) e1 += dv[a] * raa.x;
      ek -= K[idx].y;                             // Re(i K_aa)
      nn_ += raa.x;
    }
  }
  red[0][tid] = e1;
  red[1][tid] = e2;
  red[2][tid] = ek;
  red[3][tid] = nn_;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st)
      for (int q = 0; q < 4; ++q) red[q][tid] += red[q][tid + st];
    __syncthreads();
  }
  if (tid == 0) {
    *E_out = spin * red[0][0] + 0.5 * spin * red[1][0] + 0.5 * spin * red[2][0];
    *N_out = spin * red[3][0];
  }
}

// Shadows of block (0, 0) (Dw(0, 0) = w^0_0 (L - Gt) = 0 stays zero).
__global__ void shadow00_kernel(int n, long ld, const double2 *L, const double2 *G, float *sh,
                                long shz, long shld) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int b = idx / n, c = idx % n;
  const double2 l = L[b * ld + c], g = G[b * ld + c];
  const long r0 = shi(0, 0, b, c, 0, n, shld), pim = n;
  sh[r0] = (float)l.x;
  sh[r0 + pim] = (float)l.y;
  sh[shz + r0] = (float)g.x;
  sh[shz + r0 + pim] = (float)g.y;
}

// Left factors of row i as real [2n][lda] matrices (column (2 s + p) n + b):
// A1 from w^i_s (s^> - s^<)(i, s), A2 from s^<(i, s) and A2 + a_z from
// s^>(i, s); row a holds the real part of the product (x.re, -x.im), row n + a
// the imaginary part (x.im, x.re).
__device__ __forceinline__ void put_cplx(float *A, int n, int lda, int a, long k0, double2 x) {
  A[(long)a * lda + k0] = (float)x.x;
  A[(long)a * lda + k0 + n] = (float)(-x.y);
  A[(long)(n + a) * lda + k0] = (float)x.y;
  A[(long)(n + a) * lda + k0 + n] = (float)x.x;
}
__global__ void aop_kernel(int n, int i, int Tcap, double dt, const double2 *S, int lda, float *A1,
                           float *A2, long a_z) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int s = blockIdx.y, a = idx / n, b = idx % n;
  const long nn = (long)n * n;
  const double2 sl = S[(long)s * nn + idx], sg = S[((long)Tcap + s) * nn + idx];
  const long k0 = (long)2 * s * n + b;
  put_cplx(A1, n, lda, a, k0, scalez(trap_w(s, i, dt), subz(sg, sl)));
  put_cplx(A2, n, lda, a, k0, sl);
  put_cplx(A2 + a_z, n, lda, a, k0, sg);
}

// rhs of row i from the product slices: R_F(i, j) = -i h_HF F(i, j) + (sum of the
// slices of both integrals), F = L (z = 0) and Gt (z = 1); O[k][z][j][p][a][c].
__global__ void rhs_finish_kernel(int n, int i, long ld, const double2 *L, const double2 *G,
                                  const double2 *hHF, const double *O1, int ns1, const double *O2,
                                  int ns2, int Tcap, double2 *RL, double2 *RG) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int j = blockIdx.y, a = idx / n, c = idx % n;
  const long nn = (long)n * n, fb = blk(i, j, n, ld);
  double2 hl = make_double2(0.0, 0.0), hg = hl;
  for (int b = 0; b < n; ++b) {
    const double2 hv = hHF[a * n + b];
    cmla(hl, hv, L[fb + b * ld + c]);
    cmla(hg, hv, G[fb + b * ld + c]);
  }
  const long zst = (long)Tcap * 2 * nn, kst = 2 * zst, e = (long)j * 2 * nn + idx;
  double kr[2] = {0.0, 0.0}, ki[2] = {0.0, 0.0};
  for (int z = 0; z < 2; ++z) {
    for (int k = 0; k < ns1; ++k) {
      kr[z] += O1[k * kst + z * zst + e];
      ki[z] += O1[k * kst + z * zst + e + nn];
    }
    for (int k = 0; k < ns2; ++k) {
      kr[z] += O2[k * kst + z * zst + e];
      ki[z] += O2[k * kst + z * zst + e + nn];
    }
  }
  RL[(long)j * nn + idx] = make_double2(hl.y + kr[0], -hl.x + ki[0]);
  RG[(long)j * nn + idx] = make_double2(hg.y + kr[1], -hg.x + ki[1]);
}

__global__ void gather_diag_kernel(int n, long ld, const double2 *L, double2 *out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int t = blockIdx.y, b = idx / n, c = idx % n;
  out[(long)t * n * n + idx] = L[blk(t, t, n, ld) + b * ld + c];
}

// Output rows per CTA and the CTAs' shared memory for n.
int coll_rows(int n) { return std::min(n, 256 * kCollQ / n); }
size_t coll_smem(int n) {
  return (size_t)(2 * coll_rows(n) * kCollKC + 2 * kCollKC * n) * sizeof(double2);
}
// Partial-sum slots (splits x columns) a launch may use: the split count is
// chosen so that a launch has about 4 CTAs per SM of a 152-SM GPU, at most 128
// (a single column, the energy's K_L(t, t), then still spreads over 128 CTAs).
constexpr int kCollTargetCtas = 608;
inline long coll_part_slots(int T) { return (long)kCollTargetCtas + T; }

cudaError_t launch_collision(CollArgs a, cudaStream_t s, long *launches) {
  a.rows = coll_rows(a.n);
  const int tiles = (a.n + a.rows - 1) / a.rows;
  const long ctas = (long)a.ncols * tiles;
  a.splits = (int)std::max(1L, std::min(128L, (kCollTargetCtas + ctas - 1) / ctas));
  dim3 grid((unsigned)(a.ncols * a.splits), (unsigned)tiles);
  collision_kernel<<<grid, 256, coll_smem(a.n), s>>>(a);
  ++*launches;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || a.splits == 1) return e;
  ++*launches;
  dim3 rg((unsigned)(((long)a.n * a.n + 255) / 256), (unsigned)a.ncols);
  coll_reduce_kernel<<<rg, 256, 0, s>>>(a.n, a.j0, a.ncols, a.splits, a.mode, a.part, a.RL, a.RG);
  return cudaGetLastError();
}

#define KBE_CK(ctx, call)                                                   \
  do {                                                                      \
    cudaError_t e__ = (call);                                               \
    if (e__ != cudaSuccess) return cuda_fail((ctx), e__, #call, __FILE__, __LINE__); \
  } while (0)
#define KBE_ENSURE(ctx, buf, bytes)                                         \
  do {                                                                      \
    if (!ensure((ctx), (ctx)->buf, (bytes), #buf)) return FEDVR_ERR_CUDA;   \
  } while (0)

// Algorithmic complex multiply-adds of one rhs call on row i (columns j0 ..
// j0 + ncols - 1; mode 1: K_L only).
double coll_cmacs(int n, int i, int j0, int ncols, int mode, bool corr) {
  const double n3 = (double)n * n * n;
  double c = 0;
  for (int j = j0; j < j0 + ncols; ++j) {
    const double f = mode == 0 ? 2.0 : 1.0;
    if (mode == 0) c += f * n3;
    if (corr && i > 0) c += f * (i + 1) * n3;
    if (corr && j > 0) c += f * (j + 1) * n3;
  }
  return c;
}

struct KbeRun {
  fedvr_ctx *ctx;
  int n, Tcap;
  long ld;
  double dt, spin;
  bool corr;
  double2 *L, *G, *S, *T1, *R0L, *R0G, *R1L, *R1G, *hHF, *K, *part;
  // split-TF32 collision integrals: shadows (null in FP64 mode), left factors, product slices
  float *sh = nullptr, *aop = nullptr;
  // split-TF32 exchange products (null: FP64 exchange kernel)
  float *xa = nullptr, *xb = nullptr, *xp = nullptr;
  double *o1 = nullptr, *o2 = nullptr;
  long shz = 0, Tn = 0, shld = 0, a_z = 0;
  int lda = 0, xld = 0;
  int *err = nullptr;
  const double *h, *V, *dv;
  double *E, *Nn;
  cudaStream_t s;
  std::vector<cudaEvent_t> *ev;
  size_t ev_used = 0;
  double cmac_coll = 0, cmac_sigma = 0, bytes_tc = 0;
  long launches = 0;
  std::vector<std::pair<size_t, int>> marks;  // (event index, stage: 0 collision, 1 sigma)

  cudaError_t mark(int stage_open) {
    if (ev_used >= ev->size()) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      ev->push_back(e);
    }
    if (stage_open >= 0) marks.push_back({ev_used, stage_open});
    return cudaEventRecord((*ev)[ev_used++], s);
  }
  const double *dv_at(int t) const { return dv ? dv + (long)t * n : nullptr; }

  int hf(int t) {
    const int nn = n * n;
    hf_kernel<<<(nn + 255) / 256, 256, 0, s>>>(n, spin, h, dv_at(t), V, L, blk(t, t, n, ld), ld,
                                               hHF);
    KBE_CK(ctx, cudaGetLastError());
    ++launches;
    return FEDVR_OK;
  }
  int sigma(int i) {
    if (!corr) return FEDVR_OK;
    const int nn = n * n, ne = 2 * (i + 1);
    KBE_CK(ctx, mark(1));
    if (xp) {
      float2 *T132 = reinterpret_cast<float2 *>(T1);
      vq32_kernel<<<dim3((nn + 255) / 256, ne), 256, 0, s>>>(n, i, ld, L, G, V, T132);
      KBE_CK(ctx, cudaGetLastError());
      direct32_kernel<<<dim3((nn + 255) / 256, ne), 256, 0, s>>>(n, i, ld, L, G, V, T132, spin,
                                                                 Tcap, S);
    } else {
      vq_kernel<<<dim3((nn + 255) / 256, ne), 256, 0, s>>>(n, i, ld, L, G, V, T1);
      KBE_CK(ctx, cudaGetLastError());
      direct_kernel<<<dim3((nn + 255) / 256, ne), 256, 0, s>>>(n, i, ld, L, G, V, T1, spin, Tcap,
                                                               S);
    }
    KBE_CK(ctx, cudaGetLastError());
    if (xp) {
      const long work = (long)nn * n;
      const unsigned gx = (unsigned)std::min(64L, (work + 255) / 256);
      xop_kernel<<<dim3(gx, ne), 256, 0, s>>>(n, i, ld, L, G, V, xld, xa, xb);
      KBE_CK(ctx, cudaGetLastError());
      KBE_CK(ctx, kbe_exchange_tc(n, ne, xld, xa, xb, xp, err, s));
      xsum_kernel<<<dim3((nn + 255) / 256, ne), 256, 0, s>>>(n, i, ld, L, G, V, xp, Tcap, S);
      launches += 2;
    } else if (n <= 16) {
      exchange_rows_kernel<<<dim3(n, ne), 256, (size_t)2 * nn * sizeof(double2), s>>>(
          n, i, ld, L, G, V, Tcap, S);
    } else {
      const size_t sm = (size_t)(2 * nn + xchg_rows(n) * n) * sizeof(double2);
      exchange_kernel<<<dim3(n, ne), 256, sm, s>>>(n, i, ld, L, G, V, Tcap, S);
    }
    KBE_CK(ctx, cudaGetLastError());
    KBE_CK(ctx, mark(-1));
    const double n3 = (double)n * n * n;
    cmac_sigma += ne * (n3 * n + 2.0 * n3);  // exchange n^4 + n^3, V Q V two half-real n^3
    launches += 3;
    return FEDVR_OK;
  }
  int rhs_tc(int i, double2 *RL, double2 *RG) {
    const int nn = n * n, K = 2 * (i + 1) * n;
    KBE_CK(ctx, mark(0));
    float *A1 = aop, *A2 = aop + a_z;
    aop_kernel<<<dim3((nn + 255) / 256, i + 1), 256, 0, s>>>(n, i, Tcap, dt, S, lda, A1, A2, a_z);
    KBE_CK(ctx, cudaGetLastError());
    // contraction slices: about two CTAs per SM, slices of at least 256 values
    const long rt = ((long)(i + 1) * n + 127) / 128;
    int nkz = (int)std::min(16L, std::max(1L, (304 + 2 * rt - 1) / (2 * rt)));
    nkz = std::max(1, std::min(nkz, K / 256));
    const int kz = ((K + nkz - 1) / nkz + 31) / 32 * 32, ns = (K + kz - 1) / kz;
    const long oz = (long)Tcap * 2 * nn, okz = 2 * oz;
    KBE_CK(ctx, mark(2));
    KBE_CK(ctx, kbe_rows_tc(n, i + 1, K, (int)Tn, (int)shld, sh, shz, A1, lda, 0, nkz, false, o1,
                            oz, okz, err, s));
    KBE_CK(ctx, kbe_rows_tc(n, i + 1, K, (int)Tn, (int)shld, sh + 2 * shz, 0, A2, lda, a_z, nkz,
                            true, o2, oz, okz, err, s));
    KBE_CK(ctx, mark(0));
    // shadow bytes the two products read once: L and Gt rows j <= i over k < K, and the
    // triangle s <= j of Dw
    const double rows = (double)(i + 1) * n;
    bytes_tc += 4.0 * (2.0 * rows * K + 0.5 * rows * K);
    rhs_finish_kernel<<<dim3((nn + 255) / 256, i + 1), 256, 0, s>>>(n, i, ld, L, G, hHF, o1, ns,
                                                                   o2, ns, Tcap, RL, RG);
    KBE_CK(ctx, cudaGetLastError());
    KBE_CK(ctx, mark(-1));
    launches += 4;
    cmac_coll += coll_cmacs(n, i, 0, i + 1, 0, corr);
    return FEDVR_OK;
  }
  int rhs(int i, double2 *RL, double2 *RG) {
    if (sh && corr) return rhs_tc(i, RL, RG);
    CollArgs a{n, i, 0, Tcap, ld, dt, L, G, S, hHF, RL, RG, 0, corr ? 1 : 0, i + 1, 1, 0, part};
    KBE_CK(ctx, mark(0));
    KBE_CK(ctx, launch_collision(a, s, &launches));
    KBE_CK(ctx, mark(-1));
    cmac_coll += coll_cmacs(n, i, 0, i + 1, 0, corr);
    return FEDVR_OK;
  }
  int observe(int t) {
    CollArgs a{n, t, t, Tcap, ld, dt, L, G, S, hHF, K, nullptr, 1, corr ? 1 : 0, 1, 1, 0, part};
    KBE_CK(ctx, mark(0));
    KBE_CK(ctx, launch_collision(a, s, &launches));
    KBE_CK(ctx, mark(-1));
    cmac_coll += coll_cmacs(n, t, t, 1, 1, corr);
    observe_kernel<<<1, 256, 0, s>>>(n, spin, h, dv_at(t), V, L, blk(t, t, n, ld), ld, K, E + t,
                                     Nn + t);
    KBE_CK(ctx, cudaGetLastError());
    ++launches;
    return FEDVR_OK;
  }
  int advance(int N, bool corrector) {
    const int nn = n * n;
    advance_kernel<<<dim3((nn + 255) / 256, N + 2), 256, 0, s>>>(
        n, N, ld, L, G, R0L, R0G, corrector ? R1L : nullptr, corrector ? R1G : nullptr, dt, sh,
        shz, shld);
    KBE_CK(ctx, cudaGetLastError());
    ++launches;
    return FEDVR_OK;
  }
};

}  // namespace
}  // namespace fedvr

using namespace fedvr;

int fedvr_kbe_propagate(fedvr_ctx *ctx, double dt, int n_steps, int second_born, int precision,
                        const double *rho0, const double *dv, double *rho_out, double *E_out,
                        double *N_out) {
  if (!ctx) return FEDVR_ERR_ARG;
  if (ctx->failed) return FEDVR_ERR_STATE;
  if (ctx->stage < 2) return fail(ctx, FEDVR_ERR_STATE, "fedvr_kbe_propagate before set_potential");
  if (!rho0 && ctx->stage < 3)
    return fail(ctx, FEDVR_ERR_STATE, "no initial density: pass rho0 or call solve_hf first");
  if (!(dt > 0.0) || !(dt < 1e300)) return fail(ctx, FEDVR_ERR_ARG, "dt must be finite and > 0");
  // 2 T self-energy entries index one grid dimension (at most 65535)
  if (n_steps < 0 || n_steps > 32766) return fail(ctx, FEDVR_ERR_ARG, "n_steps must be in [0, 32766]");
  const int n = ctx->n;
  if (n > kKbeMaxN)
    return fail(ctx, FEDVR_ERR_ARG, "fedvr_kbe_propagate supports n_b <= %d (got %d)", kKbeMaxN, n);
  if (precision != FEDVR_FP64 && precision != FEDVR_SPLIT_TF32)
    return fail(ctx, FEDVR_ERR_ARG, "precision must be FEDVR_FP64 or FEDVR_SPLIT_TF32");
  const bool split = precision == FEDVR_SPLIT_TF32 && second_born != 0;
  const int T = n_steps + 1;
  const long ld = (long)T * n;
  const long shld = (2 * ld + 31) / 32 * 32;  // shadow row pitch (floats)
  if (split && ld * shld + shld >= (1L << 31))
    return fail(ctx, FEDVR_ERR_ARG, "split-TF32 propagation needs T n_b <= 32750 (got %ld)", ld);
  const size_t nn = (size_t)n * n, cz = sizeof(double2);
  const size_t two = (size_t)ld * (size_t)ld * cz;
  const size_t shz = split ? (size_t)ld * (size_t)shld : 0;  // floats per shadow
  const int lda = (int)shld;
  const int xld = (2 * n + 3) / 4 * 4;  // exchange operand row pitch (floats)
  const size_t aop_floats = split ? 3 * (size_t)2 * n * lda : 0;
  const size_t o_doubles = split ? (size_t)16 * 2 * T * 2 * nn : 0;
  const bool split_x = split && n <= 64;  // exchange products on the tensor cores
  const size_t x_floats =
      split_x ? (size_t)2 * T * ((size_t)2 * n * xld + nn * xld + 2 * nn * n) : 0;
  {
    size_t fre = 0, tot = 0;
    KBE_CK(ctx, cudaMemGetInfo(&fre, &tot));
    const size_t held = ctx->k_L.bytes + ctx->k_G.bytes + ctx->k_sh.bytes;
    const size_t need = 2 * two + 3 * shz * sizeof(float) + aop_floats * sizeof(float) +
                        2 * o_doubles * sizeof(double) + x_floats * sizeof(float) +
                        (size_t)(16 * T + 8) * nn * cz;
    if (need > fre + held)
      return fail(ctx, FEDVR_ERR_ARG,
                  "two-time storage of %.2f GB (T = %d, n_b = %d) exceeds free device memory",
                  need / 1e9, T, n);
  }
  cudaStream_t s = ctx->stream;
  ctx->kbe_T = 0;
  KBE_ENSURE(ctx, k_L, two);
  KBE_ENSURE(ctx, k_G, two);
  KBE_ENSURE(ctx, k_S, 2 * (size_t)T * nn * cz);
  KBE_ENSURE(ctx, k_T1, 2 * (size_t)T * nn * cz);
  KBE_ENSURE(ctx, k_R, 4 * (size_t)T * nn * cz);
  KBE_ENSURE(ctx, k_aux, (2 * nn + 2 * (size_t)T) * cz);
  KBE_ENSURE(ctx, k_out, (size_t)T * nn * cz + (size_t)T * n * sizeof(double));
  KBE_ENSURE(ctx, k_part, (size_t)coll_part_slots(T) * 2 * nn * cz);
  if (split) {
    KBE_ENSURE(ctx, k_sh, 3 * shz * sizeof(float));
    KBE_ENSURE(ctx, k_aop, aop_floats * sizeof(float));
    KBE_ENSURE(ctx, k_o, 2 * o_doubles * sizeof(double));
    KBE_ENSURE(ctx, k_flag, sizeof(int));
    if (split_x) KBE_ENSURE(ctx, k_x, x_floats * sizeof(float));
  }
  double2 *L = P<double2>(ctx->k_L), *G = P<double2>(ctx->k_G);
  double2 *R = P<double2>(ctx->k_R);
  double2 *aux = P<double2>(ctx->k_aux);
  double *obs = reinterpret_cast<double *>(aux + 2 * nn);
  double2 *rho_all = P<double2>(ctx->k_out);
  double *dv_d = reinterpret_cast<double *>(rho_all + (size_t)T * nn);
  KBE_CK(ctx, cudaMemsetAsync(L, 0, two, s));
  KBE_CK(ctx, cudaMemsetAsync(G, 0, two, s));
  KBE_CK(ctx, cudaMemsetAsync(ctx->k_S.ptr, 0, 2 * (size_t)T * nn * cz, s));
  if (split) {
    KBE_CK(ctx, cudaMemsetAsync(ctx->k_sh.ptr, 0, 3 * shz * sizeof(float), s));
    KBE_CK(ctx, cudaMemsetAsync(ctx->k_aop.ptr, 0, aop_floats * sizeof(float), s));
    KBE_CK(ctx, cudaMemsetAsync(ctx->k_flag.ptr, 0, sizeof(int), s));
  }
  if (dv)
    KBE_CK(ctx, cudaMemcpyAsync(dv_d, dv, (size_t)T * n * sizeof(double), cudaMemcpyHostToDevice, s));
  if (rho0) {
    KBE_CK(ctx, cudaMemcpy2DAsync(L, (size_t)ld * cz, rho0, (size_t)n * cz, (size_t)n * cz, n,
                                  cudaMemcpyHostToDevice, s));
  } else {
    rho_real_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, ld, CP<double>(ctx->b_rho_new), L);
    KBE_CK(ctx, cudaGetLastError());
  }
  g_from_l_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, ld, 0, L, G);
  KBE_CK(ctx, cudaGetLastError());
  if (split) {
    shadow00_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, ld, L, G, P<float>(ctx->k_sh),
                                                                 (long)shz, shld);
    KBE_CK(ctx, cudaGetLastError());
  }

  KbeRun run;
  run.ctx = ctx;
  run.n = n;
  run.Tcap = T;
  run.ld = ld;
  run.dt = dt;
  run.spin = ctx->spin;
  run.corr = second_born != 0;
  run.L = L;
  run.G = G;
  run.S = P<double2>(ctx->k_S);
  run.T1 = P<double2>(ctx->k_T1);
  run.R0L = R;
  run.R0G = R + (size_t)T * nn;
  run.R1L = R + 2 * (size_t)T * nn;
  run.R1G = R + 3 * (size_t)T * nn;
  run.hHF = aux;
  run.K = aux + nn;
  run.part = P<double2>(ctx->k_part);
  if (split) {
    run.sh = P<float>(ctx->k_sh);
    run.shz = (long)shz;
    run.Tn = ld;
    run.shld = shld;
    run.lda = lda;
    run.xld = xld;
    run.aop = P<float>(ctx->k_aop);
    run.a_z = (long)2 * n * lda;
    run.o1 = P<double>(ctx->k_o);
    run.o2 = run.o1 + o_doubles;
    run.err = P<int>(ctx->k_flag);
    if (split_x) {
      run.xa = P<float>(ctx->k_x);
      run.xb = run.xa + (size_t)2 * T * 2 * n * xld;
      run.xp = run.xb + (size_t)2 * T * nn * xld;
    }
  }
  run.h = CP<double>(ctx->b_h);
  run.V = CP<double>(ctx->b_V);
  run.dv = dv ? dv_d : nullptr;
  run.E = obs;
  run.Nn = obs + T;
  run.s = s;
  run.ev = &ctx->kbe_events;
  {
    const size_t sm = (2 * nn + (size_t)xchg_rows(n) * n) * cz;
    KBE_CK(ctx, cudaFuncSetAttribute(exchange_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sm));
    KBE_CK(ctx, cudaFuncSetAttribute(collision_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)coll_smem(n)));
  }
  KBE_CK(ctx, run.mark(-1));
  if (int r = run.hf(0)) return r;
  if (int r = run.sigma(0)) return r;
  if (int r = run.observe(0)) return r;
  for (int N = 0; N < n_steps; ++N) {
    if (int r = run.rhs(N, run.R0L, run.R0G)) return r;
    if (int r = run.advance(N, false)) return r;
    if (int r = run.hf(N + 1)) return r;
    if (int r = run.sigma(N + 1)) return r;
    if (int r = run.rhs(N + 1, run.R1L, run.R1G)) return r;
    if (int r = run.advance(N, true)) return r;
    if (int r = run.hf(N + 1)) return r;
    if (int r = run.sigma(N + 1)) return r;
    if (int r = run.observe(N + 1)) return r;
  }
  KBE_CK(ctx, run.mark(-1));
  if (rho_out) {
    gather_diag_kernel<<<dim3((unsigned)((nn + 255) / 256), T), 256, 0, s>>>(n, ld, L, rho_all);
    KBE_CK(ctx, cudaGetLastError());
    KBE_CK(ctx, cudaMemcpyAsync(rho_out, rho_all, (size_t)T * nn * cz, cudaMemcpyDeviceToHost, s));
  }
  if (E_out) KBE_CK(ctx, cudaMemcpyAsync(E_out, obs, T * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (N_out)
    KBE_CK(ctx, cudaMemcpyAsync(N_out, obs + T, T * sizeof(double), cudaMemcpyDeviceToHost, s));
  KBE_CK(ctx, cudaStreamSynchronize(s));
  if (split) {
    int flag = 0;
    KBE_CK(ctx, cudaMemcpy(&flag, ctx->k_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
      ctx->failed = true;
      return fail(ctx, FEDVR_ERR_TIMEOUT, "a tensor-core wait of the collision products timed out");
    }
  }
  // stage times from the recorded events
  double ms[3] = {0, 0, 0};
  for (auto &m : run.marks) {
    float f = 0.f;
    KBE_CK(ctx, cudaEventElapsedTime(&f, (*run.ev)[m.first], (*run.ev)[m.first + 1]));
    ms[m.second] += f;
  }
  float tot = 0.f;
  KBE_CK(ctx, cudaEventElapsedTime(&tot, (*run.ev)[0], (*run.ev)[run.ev_used - 1]));
  ctx->kbe_stats[0] = tot;
  ctx->kbe_stats[1] = ms[0] + ms[2];
  ctx->kbe_stats[2] = ms[1];
  ctx->kbe_stats[6] = ms[2];
  ctx->kbe_stats[7] = run.bytes_tc;
  ctx->kbe_stats[3] = 8.0 * run.cmac_coll;
  ctx->kbe_stats[4] = 8.0 * run.cmac_sigma;
  ctx->kbe_stats[5] = (double)run.launches;
  ctx->kbe_T = T;
  ctx->kbe_n = n;
  return FEDVR_OK;
}

int fedvr_kbe_get_block(const fedvr_ctx *cctx, int which, int i, int j, double *out) {
  fedvr_ctx *ctx = const_cast<fedvr_ctx *>(cctx);
  if (!ctx) return FEDVR_ERR_ARG;
  if (ctx->failed) return FEDVR_ERR_STATE;
  if (ctx->kbe_T == 0) return fail(ctx, FEDVR_ERR_STATE, "no completed fedvr_kbe_propagate");
  if (which != 0 && which != 1) return fail(ctx, FEDVR_ERR_ARG, "which must be 0 (L) or 1 (Gt)");
  const int T = ctx->kbe_T, n = ctx->kbe_n;
  if (i < 0 || j < 0 || i >= T || j >= T || !out)
    return fail(ctx, FEDVR_ERR_ARG, "block (%d, %d) outside the %d time points", i, j, T);
  const long ld = (long)T * n;
  const double2 *F = CP<double2>(which ? ctx->k_G : ctx->k_L);
  KBE_CK(ctx, cudaMemcpy2DAsync(out, (size_t)n * sizeof(double2), F + blk(i, j, n, ld),
                                (size_t)ld * sizeof(double2), (size_t)n * sizeof(double2), n,
                                cudaMemcpyDeviceToHost, ctx->stream));
  KBE_CK(ctx, cudaStreamSynchronize(ctx->stream));
  return FEDVR_OK;
}

int fedvr_kbe_stats(const fedvr_ctx *cctx, double *out) {
  if (!cctx || !out) return FEDVR_ERR_ARG;
  if (cctx->kbe_T == 0)
    return fail(const_cast<fedvr_ctx *>(cctx), FEDVR_ERR_STATE, "no completed fedvr_kbe_propagate");
  for (int q = 0; q < 8; ++q) out[q] = cctx->kbe_stats[q];
  return FEDVR_OK;
}
