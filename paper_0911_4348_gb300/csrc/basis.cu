// Basis, operators and mesh (Sec. 2.1-2.2, Sec. 3.1) built bit-identically to
// a plain IEEE evaluation: only +, -, *, / and sqrt, each correctly rounded
// (the __d*_rn intrinsics are never contracted into fused multiply-adds), in
// the operation order stated beside each formula. This translation unit is
// also compiled with -fmad=false.
#include "common.cuh"

namespace fedvr {
namespace {

constexpr int kScanCells = 4096;  // uniform scan of [-1, 1] bracketing the roots of P'_N

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dv(double a, double b) { return __ddiv_rn(a, b); }

// (P_N(x), P_{N-1}(x)): a = (2k+1)*x; b = a*P_k; c = k*P_{k-1}; P_{k+1} = (b-c)/(k+1)
__device__ void legendre(int N, double x, double *pN, double *pNm1) {
  if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
  double pm1 = 1.0, p = x;
  for (int k = 1; k < N; ++k) {
    double a = mul((double)(2 * k + 1), x);
    double b = mul(a, p);
    double c = mul((double)k, pm1);
    double pn = dv(sub(b, c), (double)(k + 1));
    pm1 = p;
    p = pn;
  }
  *pN = p;
  *pNm1 = pm1;
}

// P'_N(x) = (N * (P_{N-1} - x*P_N)) / (1 - x*x), |x| < 1
__device__ double dlegendre(int N, double x) {
  double p, pm1;
  legendre(N, x, &p, &pm1);
  double num = mul((double)N, sub(pm1, mul(x, p)));
  double den = sub(1.0, mul(x, x));
  return dv(num, den);
}

// Bisection of a sign change of P'_N in (lo, hi) until the midpoint stops moving.
__device__ double bisect_root(int N, double lo, double hi, double dlo) {
  double mid = mul(0.5, add(lo, hi));
  for (int it = 0; it < 400; ++it) {
    mid = mul(0.5, add(lo, hi));
    if (!(lo < mid && mid < hi)) break;
    double dm = dlegendre(N, mid);
    if (dm == 0.0) break;
    if ((dm > 0.0) == (dlo > 0.0)) lo = mid; else hi = mid;
  }
  return mid;
}

// GLL points and weights of order N (Sec. 2.1): scan P'_N on 4095 interior cell
// boundaries, record exact zeros and bracket strict sign changes, bisect each.
// omega_m = 2 / ((N(N+1)) * (P_N(xi_m)^2)).
__global__ void gll_kernel(int N, double *xi, double *om, int *status) {
  __shared__ double dval[kScanCells];
  __shared__ double lo_s[64], hi_s[64], dlo_s[64];
  __shared__ int exact_s[64];
  __shared__ int nroot;
  for (int c = 1 + threadIdx.x; c < kScanCells; c += blockDim.x) {
    double x = add(-1.0, dv(mul(2.0, (double)c), (double)kScanCells));
    dval[c] = dlegendre(N, x);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = 0;
    bool have_prev = false;
    double prev_x = 0, prev_d = 0;
    for (int c = 1; c < kScanCells; ++c) {
      double x = add(-1.0, dv(mul(2.0, (double)c), (double)kScanCells));
      double d = dval[c];
      if (d == 0.0) {
        if (r < 64) { lo_s[r] = x; exact_s[r] = 1; }
        ++r;
      } else if (have_prev && prev_d != 0.0 && ((d > 0.0) != (prev_d > 0.0))) {
        if (r < 64) { lo_s[r] = prev_x; hi_s[r] = x; dlo_s[r] = prev_d; exact_s[r] = 0; }
        ++r;
      }
      have_prev = true;
      prev_x = x;
      prev_d = d;
    }
    nroot = r;
    *status = (r == N - 1) ? 0 : 1;
  }
  __syncthreads();
  int r = nroot;
  if (r != N - 1) return;
  for (int k = threadIdx.x; k < r; k += blockDim.x) {
    double root = exact_s[k] ? lo_s[k] : bisect_root(N, lo_s[k], hi_s[k], dlo_s[k]);
    xi[k + 1] = root;
  }
  if (threadIdx.x == 0) { xi[0] = -1.0; xi[N] = 1.0; }
  __syncthreads();
  double nn1 = (double)(N * (N + 1));
  for (int m = threadIdx.x; m <= N; m += blockDim.x) {
    double p, pm1;
    legendre(N, xi[m], &p, &pm1);
    om[m] = dv(2.0, mul(nn1, mul(p, p)));
  }
}

// Element edges (Sec. 2.1, Sec. 3.1 case I/II). One thread; sequential sums.
__device__ void edges_serial(int ne, double xmin, double xmax, int kind, double *e, int *bad) {
  double L = sub(xmax, xmin);
  if (kind == 0) {
    for (int i = 0; i < ne; ++i) e[i] = add(xmin, dv(mul((double)i, L), (double)ne));
  } else {
    // graded: centre width 1, widths 1 + k*delta (odd n_e) or 1 + (k-1)*delta (even n_e)
    e[0] = xmin;
    for (int i = 0; i + 1 < ne; ++i) {
      double wdt;
      if (ne % 2 == 1) {
        int K = (ne - 1) / 2;
        double delta = dv(sub(sub(L, 1.0), mul(2.0, (double)K)), (double)(K * (K + 1)));
        int k = (i < K) ? (K - i) : (i == K ? 0 : i - K);
        wdt = (k == 0) ? 1.0 : add(1.0, mul((double)k, delta));
      } else {
        int K = ne / 2;
        if (K == 1) {
          wdt = mul(0.5, L);
        } else {
          double delta = dv(sub(mul(0.5, L), (double)K), (double)((K * (K - 1)) / 2));
          int k = (i < K) ? (K - i) : (i - K + 1);
          wdt = add(1.0, mul((double)(k - 1), delta));
        }
      }
      if (!(wdt > 0.0)) *bad = 1;
      e[i + 1] = add(e[i], wdt);
    }
  }
  e[ne] = xmax;
}

__global__ void edges_kernel(int ne, double xmin, double xmax, int kind, double *e, int *status) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int bad = 0;
    edges_serial(ne, xmin, xmax, kind, e, &bad);
    for (int i = 0; i < ne; ++i)
      if (!(e[i + 1] > e[i])) bad = 1;
    *status = bad ? 2 : 0;
  }
}

// Nodes x = e_i + ((xi_m + 1) * h_i) * 0.5, bridge = edge; weights
// w^i_m = (omega_m * h_i) * 0.5, bridge W = w^{i-1}_N + w^i_0 (Eqs. xim, wim, basis).
__global__ void nodes_kernel(int ne, int N, const double *xi, const double *om, const double *e,
                             double *nodes, double *weights, int *elem, int *local) {
  int n = ne * N - 1;
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= n) return;
  int q = a + 1;
  int i = q / N, m = q % N;
  if (m == 0) {
    nodes[a] = e[i];
    double hl = sub(e[i], e[i - 1]);
    double hr = sub(e[i + 1], e[i]);
    double wl = mul(mul(om[N], hl), 0.5);
    double wr = mul(mul(om[0], hr), 0.5);
    weights[a] = add(wl, wr);
    elem[a] = i - 1;
    local[a] = N;
  } else {
    double h = sub(e[i + 1], e[i]);
    nodes[a] = add(e[i], mul(mul(add(xi[m], 1.0), h), 0.5));
    weights[a] = mul(mul(om[m], h), 0.5);
    elem[a] = i;
    local[a] = m;
  }
}

// Lagrange derivative d[m][k] = f'_m(xi_k), then element kinetic matrices
// t~^i_{m1 m2} = sum_k ((D_{m1 k} * D_{m2 k}) * w^i_k), D = (2/h_i) * d (Eq. tmat).
__device__ double lag_deriv(const double *xi, int N1, int m, int k) {
  if (k == m) {
    double s = 0.0;
    for (int l = 0; l < N1; ++l)
      if (l != m) s = add(s, dv(1.0, sub(xi[m], xi[l])));
    return s;
  }
  double prod = dv(1.0, sub(xi[m], xi[k]));
  for (int l = 0; l < N1; ++l)
    if (l != m && l != k) prod = mul(prod, dv(sub(xi[k], xi[l]), sub(xi[m], xi[l])));
  return prod;
}

__global__ void elem_kinetic_kernel(int ne, int N, const double *xi, const double *om,
                                    const double *e, double *tt) {
  int N1 = N + 1;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ne * N1 * N1) return;
  int i = idx / (N1 * N1), r = idx % (N1 * N1);
  int m1 = r / N1, m2 = r % N1;
  double h = sub(e[i + 1], e[i]);
  double sc = dv(2.0, h);
  double acc = 0.0;
  for (int k = 0; k < N1; ++k) {
    double D1 = mul(sc, lag_deriv(xi, N1, m1, k));
    double D2 = mul(sc, lag_deriv(xi, N1, m2, k));
    double wk = mul(mul(om[k], h), 0.5);
    acc = add(acc, mul(mul(D1, D2), wk));
  }
  tt[idx] = acc;
}

// T_ab = (0.5 * S_ab) / sqrt(W_a * W_b), S_ab = sum over elements containing both
// nodes (ascending) of t~, starting from 0.0; T_ab = 0 where S_ab == 0.
__global__ void assemble_T_kernel(int ne, int N, const double *tt, const double *W, double *T) {
  int n = ne * N - 1;
  int N1 = N + 1;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  int a = (int)(idx / n), b = (int)(idx % n);
  int qa = a + 1, qb = b + 1;
  int ilo = (qa % N == 0) ? qa / N - 1 : qa / N;
  int ihi = qa / N;
  if (ihi > ne - 1) ihi = ne - 1;
  double S = 0.0;
  for (int i = ilo; i <= ihi; ++i) {
    if (qb >= i * N && qb <= (i + 1) * N && qa >= i * N && qa <= (i + 1) * N) {
      S = add(S, tt[((long)i * N1 + (qa - i * N)) * N1 + (qb - i * N)]);
    }
  }
  T[idx] = (S != 0.0) ? dv(mul(0.5, S), __dsqrt_rn(mul(W[a], W[b]))) : 0.0;
}

// v_a = sum_A ((-Z_A) / sqrt((x_a - R_A)^2 + soft_en)); V_ab = 1/sqrt((x_a-x_b)^2 + soft_ee);
// h = T + diag(v) (Eqs. vmat, umat1).
__global__ void potential_kernel(int n, const double *x, int n_nuc, const double *Z,
                                 const double *R, double soft_en, double soft_ee,
                                 const double *T, double *v, double *V, double *h) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)n * n) return;
  int a = (int)(idx / n), b = (int)(idx % n);
  double dx = sub(x[a], x[b]);
  V[idx] = dv(1.0, __dsqrt_rn(add(mul(dx, dx), soft_ee)));
  if (a == b) {
    double acc = 0.0;
    for (int A = 0; A < n_nuc; ++A) {
      double d = sub(x[a], R[A]);
      acc = add(acc, dv(-Z[A], __dsqrt_rn(add(mul(d, d), soft_en))));
    }
    v[a] = acc;
    h[idx] = add(T[idx], acc);
  } else {
    h[idx] = T[idx];
  }
}

// Power mesh (Sec. 3.1): B_p = beta/2, B_{k-1} = 0.5*B_k, B_0 = 0; offset
// s_{(k-1)u + r} = B_{k-1} + (width * r) / u with width = B_1 (k = 1) or B_{k-1};
// tau_j = (-beta) + s_j for j = 0..up, then tau_{M-1-m} = -s_m for m = 0..up
// (so tau_{M-1} = -0.0); w_j = (tau_{j+1} - tau_{j-1}) * 0.5 (one-sided at the
// ends), wm_j = (tau_j - tau_{j-1}) * 0.5, wp_j = (tau_{j+1} - tau_j) * 0.5.
__device__ double mesh_offset(const double *B, int u, int idx) {
  if (idx == 0) return 0.0;
  int k = (idx - 1) / u + 1, r = (idx - 1) % u + 1;
  double width = (k == 1) ? B[1] : B[k - 1];
  return add(B[k - 1], dv(mul(width, (double)r), (double)u));
}

__global__ void mesh_kernel(double beta, int u, int p, double *tau, double *w, double *wm,
                            double *wp) {
  int up = u * p, M = 2 * up + 1;
  __shared__ double B[66];
  if (threadIdx.x == 0) {
    B[p] = mul(0.5, beta);
    for (int k = p; k > 1; --k) B[k - 1] = mul(0.5, B[k]);
    B[0] = 0.0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= up; j += blockDim.x) tau[j] = add(-beta, mesh_offset(B, u, j));
  __syncthreads();
  for (int m = threadIdx.x; m <= up; m += blockDim.x) tau[M - 1 - m] = -mesh_offset(B, u, m);
  __syncthreads();
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    wm[j] = (j > 0) ? mul(sub(tau[j], tau[j - 1]), 0.5) : 0.0;
    wp[j] = (j < M - 1) ? mul(sub(tau[j + 1], tau[j]), 0.5) : 0.0;
    if (j == 0) w[j] = mul(sub(tau[1], tau[0]), 0.5);
    else if (j == M - 1) w[j] = mul(sub(tau[M - 1], tau[M - 2]), 0.5);
    else w[j] = mul(sub(tau[j + 1], tau[j - 1]), 0.5);
  }
}

// Lag of tau_i - tau_j mapped to [-beta, 0]: j > i: y = tau_i - tau_j, sign +1;
// j < i: y = (tau_i - tau_j) - beta, sign -1. Bracket: largest k in [0, M-2]
// with tau_k <= y (binary search); t = (y - tau_k) / (tau_{k+1} - tau_k).
__device__ __forceinline__ void lag_bracket(const double *tau, int M, double beta, int i, int j,
                                            int *k_out, double *t_out, double *sgn) {
  double x = sub(tau[i], tau[j]);
  double y;
  if (j > i) { y = x; *sgn = 1.0; } else { y = sub(x, beta); *sgn = -1.0; }
  int lo = 0, hi = M - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (tau[mid] <= y) lo = mid; else hi = mid;
  }
  *k_out = lo;
  *t_out = dv(sub(y, tau[lo]), sub(tau[lo + 1], tau[lo]));
}

__global__ void lag_kernel(int M, double beta, const double *tau, int *lag_k, double *lag_t) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  int i = (int)(idx / M), j = (int)(idx % M);
  if (i == j) { lag_k[idx] = -1; lag_t[idx] = 0.0; return; }
  int k; double t, sg;
  lag_bracket(tau, M, beta, i, j, &k, &t, &sg);
  lag_k[idx] = k;
  lag_t[idx] = t;
}

// conv1 coefficients: c1 = (sign * w_j) * (1 - t), c2 = (sign * w_j) * t for j != i;
// the diagonal carries -wm_i on A_0 and +wp_i on A_{M-1} (split trapezoid, Eq. deq).
__global__ void coef_kernel(int M, double beta, const double *tau, const double *w,
                            const double *wm, const double *wp, ConvCoef *coef) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  int i = (int)(idx / M), j = (int)(idx % M);
  ConvCoef c;
  if (i == j) {
    c.k = 0; c.diag = 1; c.c1 = -wm[i]; c.c2 = wp[i];
  } else {
    int k; double t, sg;
    lag_bracket(tau, M, beta, i, j, &k, &t, &sg);
    double sw = mul(sg, w[j]);
    c.k = k; c.diag = 0; c.c1 = mul(sw, sub(1.0, t)); c.c2 = mul(sw, t);
  }
  coef[idx] = c;
}

// Periodic (bosonic) convolution coefficients for every (i, j), the lag
// tau_i - tau_j taken as is for j >= i (lag 0 at i = j: the last mesh point)
// and shifted by -beta for j < i; c1 = w_j (1 - t), c2 = w_j t, no diagonal
// special case (a periodic function has no jump at lag 0).
__global__ void coef_bose_kernel(int M, double beta, const double *tau, const double *w,
                                 ConvCoef *coef) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  int i = (int)(idx / M), j = (int)(idx % M);
  double x = sub(tau[i], tau[j]);
  double y = (j >= i) ? x : sub(x, beta);
  int lo = 0, hi = M - 1;
  while (hi - lo > 1) {
    int mid = (lo + hi) / 2;
    if (tau[mid] <= y) lo = mid; else hi = mid;
  }
  double t = dv(sub(y, tau[lo]), sub(tau[lo + 1], tau[lo]));
  ConvCoef c;
  c.k = lo; c.diag = 0; c.c1 = mul(w[j], sub(1.0, t)); c.c2 = mul(w[j], t);
  coef[idx] = c;
}

}  // namespace

cudaError_t launch_conv_coef_bose(int M, double beta, const double *tau, const double *w,
                                  ConvCoef *coef, cudaStream_t s) {
  long mm = (long)M * M;
  coef_bose_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(M, beta, tau, w, coef);
  return cudaGetLastError();
}

cudaError_t launch_gll(int order, double *xi, double *om, int *status, cudaStream_t s) {
  gll_kernel<<<1, 256, 0, s>>>(order, xi, om, status);
  return cudaGetLastError();
}

cudaError_t launch_basis(int n_elem, int order, double xmin, double xmax, int grid_kind,
                         const double *xi, const double *om, double *edges, double *nodes,
                         double *weights, int *elem, int *local, double *tt, double *T,
                         int *status, cudaStream_t s) {
  int n = n_elem * order - 1;
  edges_kernel<<<1, 32, 0, s>>>(n_elem, xmin, xmax, grid_kind, edges, status);
  nodes_kernel<<<(n + 127) / 128, 128, 0, s>>>(n_elem, order, xi, om, edges, nodes, weights,
                                                elem, local);
  int ntt = n_elem * (order + 1) * (order + 1);
  elem_kinetic_kernel<<<(ntt + 127) / 128, 128, 0, s>>>(n_elem, order, xi, om, edges, tt);
  long nn = (long)n * n;
  assemble_T_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n_elem, order, tt, weights, T);
  return cudaGetLastError();
}

cudaError_t launch_potential(int n, const double *nodes, int n_nuc, const double *Z,
                             const double *R, double soft_en, double soft_ee, const double *T,
                             double *v, double *V, double *h, cudaStream_t s) {
  long nn = (long)n * n;
  potential_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(n, nodes, n_nuc, Z, R, soft_en,
                                                                 soft_ee, T, v, V, h);
  return cudaGetLastError();
}

cudaError_t launch_mesh(double beta, int u, int p, double *tau, double *w, double *wm,
                        double *wp, int *lag_k, double *lag_t, cudaStream_t s) {
  mesh_kernel<<<1, 256, 0, s>>>(beta, u, p, tau, w, wm, wp);
  if (lag_k && lag_t) {
    int M = 2 * u * p + 1;
    long mm = (long)M * M;
    lag_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(M, beta, tau, lag_k, lag_t);
  }
  return cudaGetLastError();
}

cudaError_t launch_conv_coef(int M, double beta, const double *tau, const double *w,
                             const double *wm, const double *wp, ConvCoef *coef, cudaStream_t s) {
  long mm = (long)M * M;
  coef_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(M, beta, tau, w, wm, wp, coef);
  return cudaGetLastError();
}

}  // namespace fedvr
