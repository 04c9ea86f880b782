// Per-system descriptors of the tensor-core kernels. One persistent launch
// walks a work queue that concatenates the items of every system in a table
// (a batch of systems with different n_b and mesh sizes); a single system is a
// table of one. Descriptors live in device memory and are written before the
// launch; each holds its own TMA maps (CUtensorMap carries its own alignment).
#pragma once

#include <cuda.h>

#include <vector>

#include "common.cuh"

namespace fedvr {

// Shared tile geometry of one system for the split-TF32 kernels.
struct TcGeom {
  int n, M, ld;     // basis size, mesh points, padded row pitch (n rounded up to 32)
  int MT, NT, Np;   // 128-row M tiles, N tiles (1 or 2), N rounded up to 16
  int KC;           // 32-wide contraction chunks per matrix
  int NBUF;         // TMEM accumulator buffers (2 if Np <= 256)
  int n0[2], nsz[2];
};

// Operand scales of the FP16-split path, one per system (device memory).
// Values of g enter FP16 as x * 2^kScaleG (|g| < 16 keeps them below 65504);
// the convolution's interpolated Sigma enters as x * 2^sA with sA from the
// bound maxC * max|Sigma| chosen per launch, the exchange's g V as x * 2^eX
// with eX from max|V|.
constexpr int kScaleG = 12;
struct TcScale {
  unsigned maxS;  // bit pattern of max |x| over the FP32 source stack (Sigma and B_ii rows)
  float maxC;     // max over (i, j) of |c1| + |c2|
  float maxV;     // max |V_ab| (the exchange's A operand g V enters as x 2^(11 - e), |V| < 2^e)
  unsigned pad;
};

// Sigma^(2) exchange kernel: one system.
struct XSys {
  CUtensorMap th[2], tl[2];   // gb = G[M-1-j] split, per N tile
  CUtensorMap hh[2], hl[2];   // FP16 path: the FP16 split of g (scaled by 2^kScaleG), per N tile
  const TcScale *scale;       // FP16 path: operand scales
  const uint32_t *tiles;      // tile t of a mesh point -> (b0 << 16) | a0 (exchange_tile_table)
  int tiles_per_j;
  TcGeom g;
  float spin;
  const float *g32, *V32;
  const float *W;             // V Q V per mesh point (the direct term's matrix), rows of ld
  double *Sigma;
  float *S32;
  unsigned *smax;             // if set: atomic max of |Sigma| (FP32 bits)
};

// First convolution kernel: one system.
struct C1Sys {
  CUtensorMap th[2], tl[2];   // g_j split, per N tile
  CUtensorMap hh[2], hl[2];   // g_j FP16 split (scaled by 2^kScaleG), per N tile
  CUtensorMap th16[2], tl16[2];  // FP16 path, packed tail (c1_tail_units > 0): per N tile
  const TcScale *scale;       // FP16 path: operand scales
  TcGeom g;
  int TU;                     // FP16 path: 16-byte units per mesh point in the packed tail (0: off)
  int JB;                     // mesh points per FP32 accumulation block
  int S;                      // splits of the mesh-point range per row tile
  int RT;                     // 128-row tiles of the stacked (i, a) rows
  const float *S32;
  const double *dHF;
  const int4 *coef32;         // per (i, j): {k1, k2, c1, c2 (float bits)}
  double *I1;                 // output (split 0 and the final sum)
  double *part;               // splits 1..S-1: [S-1][M][n][n]
};

TcGeom tc_geom(int n, int M);
// Largest tile footprint over a table (smem bytes of the shared stage layout).
size_t tc_smem_bytes(int Np_max, int ld_max, bool with_columns);

// Host-side descriptor fill (tensor maps included); the caller copies the
// descriptors to device memory.
cudaError_t xsys_fill(XSys *d, int n, int M, double spin, const float *ws, double *Sigma,
                      float *S32, const uint32_t *tiles, unsigned *smax = nullptr,
                      const void *h16 = nullptr, const TcScale *scale = nullptr);
// The exchange kernel's tiles of one mesh point: every block of 16 values of b
// (b0 a multiple of 16) x 8 values of a (a0 a multiple of 8, a0 >= b0) that
// holds a pair a >= b, b-block-major; entry t = (b0 << 16) | a0.
void exchange_tile_table(int n, std::vector<uint32_t> &tiles);
inline long exchange_tiles(int n) {
  long t = 0;
  for (int b0 = 0; b0 < n; b0 += 16) t += (n - b0 + 7) / 8;
  return t;
}
cudaError_t c1sys_fill(C1Sys *d, int n, int M, int splits, const float *ws, const float *S32,
                       const double *dHF, const int4 *coef32, double *I1, double *part,
                       const void *h16 = nullptr, const TcScale *scale = nullptr);
// Pitch (elements) of the FP16 split rows: n rounded up to 64 (128-byte rows).
inline int ld16_of(int n) { return (n + 63) / 64 * 64; }
// Packed tail of the FP16 first convolution. The last 64-wide column slice of
// g_j holds r = n - ld16 + 64 values; when r <= 32 the slices of 8 / TU
// consecutive mesh points (TU = ceil(r / 8) 16-byte units each) share one
// 64-wide contraction chunk instead of taking one mostly-zero chunk each. The
// split writes those columns a second time into tail arrays [n][pitch] (hi,
// then lo), column j * 8 TU + t holding g_j(a, ld16 - 64 + t) (zero past n).
inline int c1_tail_units(int n) {
  const int r = n - (ld16_of(n) - 64);
  const int u = (r + 7) / 8;
  return u <= 4 ? u : 0;
}
inline int c1_tail_pitch(int n, int M) {
  const int u = c1_tail_units(n);
  return u ? (M * 8 * u + 63) / 64 * 64 : 0;
}
// Halves of the FP16 split of g: the hi and lo stacks [M][n][ld16], then the
// packed tail's hi and lo arrays [n][c1_tail_pitch].
inline size_t f16_split_halves(int n, int M) {
  return 2 * (size_t)M * n * ld16_of(n) + 2 * (size_t)n * c1_tail_pitch(n, M);
}
// FP16 split of g (scaled by 2^kScaleG) into h16 = [hi stack][lo stack],
// [M][n][ld16] halves each, padding zero, followed by the packed tail's hi and
// lo arrays when c1_tail_units(n) > 0. An entry the split cannot hold
// (|g| >= 65504 / 2^kScaleG or not finite) raises bit 1 (value 2) of *flag
// (the tensor-core error flag; may be NULL). With g32 (may be NULL) the same
// pass writes the FP32 copy of g ([M][n][ld], ld = n rounded up to 32).
cudaError_t launch_split_f16(int n, int M, const double *G, void *h16, cudaStream_t s,
                             int *flag, float *g32 = nullptr);
// scale->maxC = max |c1| + |c2| over the coefficient table, scale->maxV =
// max |V| over the n x n interaction matrix, scale->maxS = 0.
cudaError_t launch_scale_init(int M, const int4 *coef32, int n, const double *V, TcScale *scale,
                              cudaStream_t s);
// Compact FP32 convolution coefficients {k1, k2, (float)c1, (float)c2} per
// (i, j) over the extended FP32 source stack [2M][n][ld]: rows k < M are
// Sigma_k, row M + i is the diagonal operand B_ii, taken with weight 1.
cudaError_t launch_coef32(int M, const ConvCoef *coef, int4 *out, cudaStream_t s);
// Diagonal operands B_ii = dHF - wm_i Sigma_0 + wp_i Sigma_{M-1} (FP32, from
// the FP32 copy of Sigma in rows 0..M-1 of S32) into rows M..2M-1 of S32.
cudaError_t launch_diag_f32(int n, int M, const double *dHF, const double *Sigma,
                            const double *wm, const double *wp, float *S32, cudaStream_t s,
                            unsigned *smax = nullptr);
// I1 += part[0] + ... + part[nparts-1] (count doubles each), fixed order.
cudaError_t conv1_sum_splits(long count, int nparts, const double *part, double *I1,
                             cudaStream_t s);

// Float offsets in the tensor-core workspace of one system (ld = n rounded up
// to 32, stack = M n ld): g32 | gh | gl | VQ | V32 (n x ld) | S32 (2 stacks:
// Sigma, then the diagonal operands B_ii) | W | error flag.
inline size_t tc_ws_stack(int n, int M) { return (size_t)M * n * ((n + 31) / 32 * 32); }
inline size_t tc_ws_s32(int n, int M) {
  return 4 * tc_ws_stack(n, M) + (size_t)n * ((n + 31) / 32 * 32);
}
inline size_t tc_ws_w(int n, int M) { return tc_ws_s32(n, M) + 2 * tc_ws_stack(n, M); }
inline size_t tc_ws_floats(int n, int M) { return tc_ws_w(n, M) + tc_ws_stack(n, M) + 64; }

// Per-system preparation of the exchange operands (FP32 copies of G and V,
// VQ and W = (VQ) V, and with tf32_operands the TF32 split of G for the gb
// operand); g32_ready: the FP32 copy of G is already in ws (made by the FP16
// split). err is raised if a tensor-core wait gives up.
cudaError_t sigma2_tc_pre(int n, int M, const double *V, const double *G, float *ws,
                          cudaStream_t s, bool tf32_operands, int *err, bool g32_ready = false);
// Split-TF32 tensor-core products (gemm_tc.cu). vqv_tc: VQ_j = V (g_j o
// g_{M-1-j}) and W_j = VQ_j V for all j (FP32 stacks of row pitch ld).
// conv2_tc: I2_i = C sum_j diag(K(i, j)) C^T I1_j as three products (K32 the
// FP32 eigen-kernel table [n][M][M], t1/t2 FP32 scratch of M n n).
cudaError_t vqv_tc(int n, int M, int ld, const float *V32, const float *g32, float *VQ, float *W,
                   int *err, cudaStream_t s);
cudaError_t conv2_tc(int n, int M, const float *K32, const double *C, const double *I1,
                     double *I2, float *t1, float *t2, int *err, cudaStream_t s);
// Real-time collision integrals of one time row (kbe.cu), two batched products
// (z = 0, 1): O[k][z][j][p][a][c] = sum over the contraction slice k of
// Sh_z[j n + c][k'] Aop_z[p n + a][k'] for j < ncols, k' < K; Sh_z at
// Sh + z sh_z ([T n][sh_ld] FP32 planar two-time shadow, Tn = T n, row pitch
// sh_ld >= 2 T n), Aop_z at
// Aop + z a_z ([2n][lda]); tri: block-triangular shadow (rows of column j
// need k' < 2n (j + 1)). The number of slices actually used is
// ceil(K / kz) with kz = ceil(K / nkz) rounded up to 32.
// Real-time exchange products of ne self-energy entries (kbe.cu), one batch
// entry each: P_e[(b, k)][(p, a)] = sum over (q, l) of Ap_e[(p, a)][(q, l)]
// Bp_e[(b, k)][(q, l)], Ap_e [2n][xld], Bp_e [n n][xld] (rows of pitch
// xld >= 2n), P_e [n n][2n] (FP32); needs 2n <= 128.
cudaError_t kbe_exchange_tc(int n, int ne, int xld, const float *Ap, const float *Bp, float *P,
                            int *err, cudaStream_t s);
cudaError_t kbe_rows_tc(int n, int ncols, int K, int Tn, int sh_ld, const float *Sh, long sh_z,
                        const float *Aop, int lda, long a_z, int nkz, bool tri, double *O,
                        long o_z, long o_kz, int *err, cudaStream_t s);
// Persistent launches over a device table of n_sys systems; prefix[n_sys + 1]
// (device) holds the cumulative work items; Np_max/ld_max size the stages.
cudaError_t exchange_tc_launch(const XSys *sys, const long *prefix, int n_sys, long items,
                               int Np_max, int ld_max, int *err, int num_sms, cudaStream_t s,
                               bool f16 = false);
cudaError_t conv1_tc_launch(const C1Sys *sys, const long *prefix, int n_sys, long items,
                            int Np_max, int *err, int num_sms, cudaStream_t s, bool f16 = false);

// Work items per system: exchange (j, tile) pairs over the 16 x 8 blocks of
// each mesh point; convolution (row tile, split) pairs over the M*n stacked
// rows.
inline long exchange_items(int n, int M) { return (long)M * exchange_tiles(n); }
inline long conv1_items(int n, int M, int splits) {
  return ((long)M * n + 127) / 128 * (long)splits;
}

// Mesh points JB per FP32 accumulation block of the first convolution, a
// function of (n, M) and the mode only: blocks of 512 MMA steps (4096
// contraction terms in TF32, K = 8 per MMA; 8192 in FP16, K = 16), shortened
// when the M n / 128 row tiles are too few to give two work items per SM of a
// 152-SM GPU, so that the mesh-point range can be split over up to 16 CTAs.
inline int conv1_block_points(int n, int M, bool f16) {
  const int terms = f16 ? 8192 : 4096;
  const long RT = ((long)M * n + 127) / 128;
  long smax = (304 + RT - 1) / RT;
  smax = smax < 1 ? 1 : (smax > 16 ? 16 : smax);
  int jb = terms / n;
  const int cap = (int)((M + smax - 1) / smax);
  if (jb > cap) jb = cap;
  return jb > 1 ? jb : 1;
}
// Accumulation blocks of the mesh-point range: the largest split count.
inline int conv1_blocks(int n, int M, bool f16) {
  const int jb = conv1_block_points(n, M, f16);
  return (M + jb - 1) / jb;
}

}  // namespace fedvr
