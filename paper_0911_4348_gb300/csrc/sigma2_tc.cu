// Second-Born self-energy on the tensor cores (Sec. 2.3, Eq. sigma2ndb in
// two-index form), split-TF32 precision:
//
//   Sigma_ab = sum_k V_ak [ sigma g_ab (Q V)_kb - g_kb P^(b)_ak ],
//   P^(b) = g diag(V_b,:) gb,  Q = g o gb,  g = G[j], gb = G[M-1-j].
//
// The first bracket term is the direct term sigma g o (V Q V), the second the
// second-order exchange X. P^(b) is the only O(n^3)-per-column contraction
// (O(n^4) per mesh point): it runs as tcgen05.mma kind::tf32 over the rows
// (b, a), a >= b, of one mesh point, tiled in blocks of 16 values of b x 8
// values of a (128 rows per tile; the rows a < b of the diagonal blocks are
// computed and dropped, so that a tile touches exactly 8 rows of V and 16 rows
// of g), all k in one or two N tiles and the
// contraction over l in 32-wide chunks, each operand split as x = hi + lo
// (TF32) and the product taken as hi*hi + hi*lo + lo*hi with FP32
// accumulation in TMEM. The A operand g_al V_bl of each row is formed by the
// CUDA cores while the previous chunk multiplies; B = gb is the same for every
// row of the mesh point. The direct term's matrix W = V Q V comes from two
// FP32 GEMMs beforehand, so the epilogue reads row (b, a) of P^(b) from TMEM
// and folds sum_k V_ak g_kb P_ak in FP32 (two warps per row, one per half of
// k), with the tile's rows of V and g staged in shared memory; the symmetric
// result is mirrored.
#include "common.cuh"
#include "tc.cuh"
#include "tc_sys.cuh"

namespace fedvr {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;   // bound on every mbarrier wait (2 s)
constexpr uint32_t kTileA = 128 * 128;        // bytes of one 128-row x 32-col fp32 operand half

// g32 = (float)g; gh, gl = TF32 split of g32 (hi = tf32(g32), lo = tf32(g32 - hi));
// rows padded to ld floats with zeros. One warp per row: row-contiguous reads
// of the FP64 source and writes of the FP32 rows.
__global__ void split_kernel(int n, long rows, int ld, const double *__restrict__ G,
                             float *__restrict__ g32, float *__restrict__ gh,
                             float *__restrict__ gl) {
  const int lane = threadIdx.x & 31;
  const long wpb = blockDim.x >> 5, nw = (long)gridDim.x * wpb;
  for (long row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += nw) {
    const double *src = G + row * n;
    const long o = row * ld;
    for (int c0 = 0; c0 < ld; c0 += 128) {
      double x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {  // all loads of the slice in flight before any store
        const int c = c0 + 32 * u + lane;
        x[u] = (c < n) ? src[c] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + 32 * u + lane;
        if (c >= ld) break;
        // one FP64 operation per element (the conversion): the low part is the
        // exact FP32 residual a - hi, which carries all that survives the split
        const float a = (float)x[u];
        const float h = tc::tf32_rna(a);
        const float l = tc::tf32_rna(a - h);
        if (g32) g32[o + c] = a;
        if (gh) gh[o + c] = h;
        if (gl) gl[o + c] = l;
      }
    }
  }
}

// Warp roles: 0-7 epilogue (two warps per TMEM lane quarter, one per half of
// the columns), 8-15 A-operand producers, 16 TMA loads of the gb operand, 17
// MMA issue. Stages handed over with mbarriers: full[s] (producer arrivals +
// TMA bytes), empty[s] (MMA commit); accumulators double-buffered with
// accf/acce; the two column halves of a row meet through a small shared
// buffer handed over with pfull/pempty. Every wait is bounded. The work queue
// is the concatenation of the (j, tile) items of every system in the table
// (mesh-point-major, so that concurrent CTAs share gb in L2); every role walks
// it in the same order. The stage layout uses the table's largest N.
//
// A tile is one block of 16 values of b x 8 values of a (row r of the tile:
// b = b0 + r / 8, a = a0 + r % 8), every block that holds a pair a >= b; the
// rows with a < b of the blocks on the diagonal are computed and dropped. The
// epilogue needs row a of V and row b of g for each row: with `stg` > 0 the
// epilogue warps first copy the tile's 8 rows of V and 16 rows of g into
// shared memory (pitch stg floats, stg = 4 mod 32, so that the eight values
// of a read by a quarter-warp fall into distinct banks and the values of b
// are broadcasts), double-buffered by tile parity and handed over with the
// bounded sfull barrier; with stg = 0 (shared memory too small for large n)
// each lane reads its rows from global memory.
//
// FP16 variant: 128-byte operand rows hold 64 FP16 values, so a chunk covers
// 64 contraction terms and the three products run as kind::f16 at twice the
// TF32 rate. A = g_al V_bl enters as x 2^eX (eX from max|V|, |g| < 16 keeps
// it below 2^15), gb as x 2^kScaleG (the FP16 split of g that the first
// convolution uses as well), and the epilogue scales P^(b) back exactly.
template <bool F16>
struct XRoles {
  static constexpr int kEpi = 8, kProd = 8;       // epilogue and producer warps
  static constexpr int kTma = kEpi + kProd, kMma = kTma + 1;
  static constexpr int kThreads = (kMma + 1) * 32;
  static constexpr int kCols = F16 ? 64 : 32;     // contraction terms per chunk
};

// Bytes after the stages: barriers (256) and the column-half buffer (2 x 128 floats).
constexpr uint32_t kXBarBytes = 256, kXPartBytes = 2 * 128 * 4;

// Exponent eX of the FP16 A operand g V: max|V| < 2^e, |g| < 16.
__device__ __forceinline__ int x_scale_exp(const TcScale *sc) {
  const float vmax = sc->maxV;
  if (!(vmax > 0.f) || !(vmax < 3.0e38f)) return 0;
  int e;
  frexpf(vmax, &e);
  e = 11 - e;
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Tile t of mesh point j of a system: (j, b0, a0); tiles ascend within a mesh point.
struct XTile {
  int j, b0, a0;
};
__device__ __forceinline__ XTile x_tile(const XSys &S, long q) {
  XTile x;
  x.j = (int)(q / S.tiles_per_j);
  const uint32_t e = S.tiles[q % S.tiles_per_j];
  x.b0 = (int)(e >> 16);
  x.a0 = (int)(e & 0xffffu);
  return x;
}

template <bool F16>
__global__ void __launch_bounds__(XRoles<F16>::kThreads, 1)
    exchange_tc_kernel(const XSys *__restrict__ sys, const long *__restrict__ prefix, int n_sys,
                       long items, int Np_max, int nbuf, int stg, int *err) {
  using R = XRoles<F16>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const uint32_t tileB = (uint32_t)Np_max * 128;
  const uint32_t stage_bytes = 2 * kTileA + 2 * tileB;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);
  uint64_t *full = bars, *empty = bars + 2, *accf = bars + 4, *acce = bars + 6, *drain = bars + 8;
  uint64_t *pfull = bars + 9, *pempty = bars + 11, *sfull = bars + 13;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 15);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  float *part = reinterpret_cast<float *>(smem + 2 * stage_bytes + kXBarBytes);  // [2][128]
  float *stage_rows = part + 2 * 128;  // [2][24][stg]: V rows a0.., then g rows b0..
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&full[0], R::kProd + 1);  // one arrival per producer warp + the TMA's
    tc::mbar_init(&full[1], R::kProd + 1);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    tc::mbar_init(&accf[0], 1);
    tc::mbar_init(&accf[1], 1);
    tc::mbar_init(&acce[0], R::kEpi);  // one arrival per epilogue warp
    tc::mbar_init(&acce[1], R::kEpi);
    tc::mbar_init(drain, 1);
    for (int q = 0; q < 2; ++q) {
      tc::mbar_init(&pfull[q], 4);  // the four warps of one column half
      tc::mbar_init(&pempty[q], 4);
      tc::mbar_init(&sfull[q], R::kEpi);  // every epilogue warp copied its staged rows
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool issued = false;
  int cur = 0;  // system of the current item (items ascend within a CTA)

  if (warp >= R::kEpi && warp < R::kTma) {
    // ---- A producers: row (b, a): A(l) = g_al * V_bl, split hi/lo; rows r0 + 32 k
    // (k < 4), 16-byte unit c of each chunk row (TF32: 4 values of a 32-wide chunk,
    // FP16: 8 values of a 64-wide chunk) ----
    const int pt = tid - R::kEpi * 32, c = pt & 7, r0 = pt >> 3;
    uint32_t cc = 0;
    for (long w = blockIdx.x; w < items && !tc::warp_flag(abort_flag); w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const XSys &S = sys[cur];
      const int n = S.g.n, ld = S.g.ld, KC = (n + R::kCols - 1) / R::kCols;
      const XTile xt = x_tile(S, w - prefix[cur]);
      const float *const gA = S.g32 + (long)xt.j * n * ld;
      const float *const V32 = S.V32;  // in a register across the memory-clobbering asm
      const float fX = F16 ? ldexpf(1.f, x_scale_exp(S.scale)) : 1.f;
      const int u = F16 ? 8 * c : 4 * c;  // first column of this thread's unit in a chunk
      uint32_t og[4], ov[4];  // element offsets of row a of g_j and row b of V
      bool live[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int r = r0 + 32 * k;
        const int b = xt.b0 + (r >> 3), a = xt.a0 + (r & 7);
        live[k] = a < n && b <= a;  // rows a < b of a diagonal block: computed as zeros
        og[k] = live[k] ? (uint32_t)(a * ld + u) : 0u;
        ov[k] = live[k] ? (uint32_t)(b * ld + u) : 0u;
      }
      for (int kc = 0; kc < KC; ++kc, ++cc) {
        const int l0 = kc * R::kCols;
        const bool in = l0 + u < n;  // units past n are zero padding: not fetched
        float4 gv[4][F16 ? 2 : 1], vv[4][F16 ? 2 : 1];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
          for (int h = 0; h < (F16 ? 2 : 1); ++h) {
            if (live[k] && in) {
              gv[k][h] = *reinterpret_cast<const float4 *>(gA + og[k] + l0 + 4 * h);
              vv[k][h] = *reinterpret_cast<const float4 *>(V32 + ov[k] + l0 + 4 * h);
            } else {
              gv[k][h] = vv[k][h] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
          }
        }
        const int s = cc & 1;
        const uint32_t use = cc >> 1;
        if (use > 0 && !tc::warp_wait(&empty[s], (use - 1) & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        uint8_t *st = smem + s * stage_bytes;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t off = tc::sw128_offset(r0 + 32 * k, c);
          if constexpr (F16) {
            // (g_al V_bl) 2^eX on pairs of values (packed FP32 pairs, the rounding
            // of the scalar products)
            const uint64_t FX = tc::f2_pack(fX, fX);
            const ulonglong2 ga = *reinterpret_cast<const ulonglong2 *>(&gv[k][0]);
            const ulonglong2 gb = *reinterpret_cast<const ulonglong2 *>(&gv[k][1]);
            const ulonglong2 va = *reinterpret_cast<const ulonglong2 *>(&vv[k][0]);
            const ulonglong2 vb = *reinterpret_cast<const ulonglong2 *>(&vv[k][1]);
            uint4 hi, lo;
            tc::f16_split2p(tc::f2_mul(tc::f2_mul(ga.x, va.x), FX), hi.x, lo.x);
            tc::f16_split2p(tc::f2_mul(tc::f2_mul(ga.y, va.y), FX), hi.y, lo.y);
            tc::f16_split2p(tc::f2_mul(tc::f2_mul(gb.x, vb.x), FX), hi.z, lo.z);
            tc::f16_split2p(tc::f2_mul(tc::f2_mul(gb.y, vb.y), FX), hi.w, lo.w);
            *reinterpret_cast<uint4 *>(st + off) = hi;
            *reinterpret_cast<uint4 *>(st + kTileA + off) = lo;
          } else {
            const float x0 = gv[k][0].x * vv[k][0].x, x1 = gv[k][0].y * vv[k][0].y,
                        x2 = gv[k][0].z * vv[k][0].z, x3 = gv[k][0].w * vv[k][0].w;
            float4 hi, lo;
            tc::tf32_split(x0, hi.x, lo.x);
            tc::tf32_split(x1, hi.y, lo.y);
            tc::tf32_split(x2, hi.z, lo.z);
            tc::tf32_split(x3, hi.w, lo.w);
            *reinterpret_cast<float4 *>(st + off) = hi;
            *reinterpret_cast<float4 *>(st + kTileA + off) = lo;
          }
        }
        tc::fence_smem_to_async();
        tc::warp_arrive(&full[s]);
      }
    }
  } else if (warp == R::kTma) {
    // ---- TMA: gb = G[M-1-j] rows 0..Np-1, one chunk of columns per stage, hi and lo ----
    if (lane == 0) {
      uint32_t cc = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const XSys &S = sys[cur];
        const int n = S.g.n;
        const int j = (int)((w - prefix[cur]) / S.tiles_per_j);
        const uint32_t bytes = 2u * (uint32_t)S.g.Np * 128u;
        const int NT = S.g.NT, KC = (n + R::kCols - 1) / R::kCols, jb = S.g.M - 1 - j;
        const int n00 = S.g.n0[0], n01 = S.g.n0[1];
        const CUtensorMap *th0 = F16 ? &S.hh[0] : &S.th[0], *th1 = F16 ? &S.hh[1] : &S.th[1];
        const CUtensorMap *tl0 = F16 ? &S.hl[0] : &S.tl[0], *tl1 = F16 ? &S.hl[1] : &S.tl[1];
        for (int kc = 0; kc < KC && !*abort_flag; ++kc, ++cc) {
          const int s = cc & 1;
          const uint32_t use = cc >> 1;
          if (use > 0 && !tc::mbar_wait(&empty[s], (use - 1) & 1, kWaitNs)) {
            *abort_flag = 1;
            break;
          }
          uint8_t *st = smem + s * stage_bytes + 2 * kTileA;
          tc::mbar_arrive_expect_tx(&full[s], bytes);
          for (int nt = 0; nt < NT; ++nt) {
            const int r = nt ? n01 : n00;
            tc::tma_load_3d(st + r * 128, nt ? th1 : th0, kc * R::kCols, r, jb, &full[s]);
            tc::tma_load_3d(st + tileB + r * 128, nt ? tl1 : tl0, kc * R::kCols, r, jb,
                            &full[s]);
          }
        }
      }
    }
  } else if (warp == R::kMma) {
    // ---- MMA issue: one accumulator per tile ----
    if (lane == 0) {
      uint32_t cc = 0, tcount = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, ++tcount) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const XSys &S = sys[cur];
        const int n = S.g.n, KC = (n + R::kCols - 1) / R::kCols, NT = S.g.NT;
        const uint32_t n00 = (uint32_t)S.g.n0[0], n01 = (uint32_t)S.g.n0[1];
        const uint32_t id0 = F16 ? tc::idesc_f16(128, S.g.nsz[0]) : tc::idesc_tf32(128, S.g.nsz[0]);
        const uint32_t id1 = F16 ? tc::idesc_f16(128, S.g.nsz[1]) : tc::idesc_tf32(128, S.g.nsz[1]);
        const int buf = tcount & 1;
        const uint32_t tu = tcount >> 1;
        // one TMEM buffer: the previous tile must be drained; two: the one before it
        bool ok = true;
        if (nbuf == 1 && tcount > 0)
          ok = tc::mbar_wait(&acce[(tcount - 1) & 1], ((tcount - 1) >> 1) & 1, kWaitNs);
        else if (nbuf == 2 && tu > 0)
          ok = tc::mbar_wait(&acce[buf], (tu - 1) & 1, kWaitNs);
        if (!ok) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t dbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
        for (int kc = 0; kc < KC; ++kc, ++cc) {
          const int s = cc & 1;
          const uint32_t use = cc >> 1;
          if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
            *abort_flag = 1;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + s * stage_bytes);
          // K per instruction: 8 (tf32) or 16 (f16) values, 32 bytes of the row either way
          constexpr int kK = F16 ? 16 : 8;
          const int ksteps = min(4, (n - kc * R::kCols + kK - 1) / kK);
          for (int kk = 0; kk < ksteps; ++kk) {
            const uint64_t ah = tc::sdesc_k128(sa + kk * 32);
            const uint64_t al = tc::sdesc_k128(sa + kTileA + kk * 32);
            for (int nt = 0; nt < NT; ++nt) {
              const uint32_t r = nt ? n01 : n00;
              const uint32_t boff = 2 * kTileA + r * 128 + kk * 32;
              const uint64_t bh = tc::sdesc_k128(sa + boff);
              const uint64_t bl = tc::sdesc_k128(sa + boff + tileB);
              const uint32_t d = dbase + r;
              const uint32_t idesc = nt ? id1 : id0;
              const uint32_t acc0 = (kc > 0 || kk > 0) ? 1u : 0u;
              if constexpr (F16) {
                tc::mma_f16(d, ah, bh, idesc, acc0);
                tc::mma_f16(d, ah, bl, idesc, 1u);
                tc::mma_f16(d, al, bh, idesc, 1u);
              } else {
                tc::mma_tf32(d, ah, bh, idesc, acc0);
                tc::mma_tf32(d, ah, bl, idesc, 1u);
                tc::mma_tf32(d, al, bh, idesc, 1u);
              }
            }
          }
          tc::mma_commit(&empty[s]);
          issued = true;
        }
        tc::mma_commit(&accf[buf]);
      }
    }
  } else if (warp < R::kEpi) {
    // ---- epilogue, row (b, a) = TMEM lane 32 (warp & 3) + lane, b = b0 + 4 (warp & 3)
    // + lane / 8, a = a0 + lane % 8; warps 0-3 take the first half of the columns k,
    // warps 4-7 the second:
    //   Sigma_ab = sigma g_ab W_ab - sum_k V_ak g_kb P_ak,  W = V Q V ----
    const int quarter = warp & 3, half = warp >> 2, prow = quarter * 32 + lane;
    const int bl = prow >> 3, al = prow & 7;
    uint32_t tcount = 0;
    for (long w = blockIdx.x; w < items && !tc::warp_flag(abort_flag); w += gridDim.x, ++tcount) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const XSys &S = sys[cur];
      const int n = S.g.n, ld = S.g.ld;
      const XTile xt = x_tile(S, w - prefix[cur]);
      const int b = xt.b0 + bl, a = xt.a0 + al;
      const bool live = a < n && b <= a;
      const float *gA = S.g32 + (long)xt.j * n * ld;
      // FP16 operands carry 2^(eX + kScaleG); undo it on P (an exact power of two)
      const float inv = F16 ? ldexpf(1.f, -(x_scale_exp(S.scale) + kScaleG)) : 1.f;
      const int NC = (n + 15) / 16, hc = (NC + 1) / 2;
      const int cb = half ? hc : 0, ce = half ? NC : hc;
      const int buf = tcount & 1;
      const uint32_t tu = tcount >> 1;
      // row a of V (V_ak = V_ka) and row b of g (g_kb = g_bk): staged or global
      const float *Va, *gb_row;
      if (stg > 0) {
        float *sb = stage_rows + (size_t)buf * 24 * stg;
        for (int rr = warp; rr < 24; rr += R::kEpi) {  // rows >= n copy as zeros
          const int src_row = rr < 8 ? xt.a0 + rr : xt.b0 + rr - 8;
          const float *src = rr < 8 ? S.V32 + (long)src_row * ld : gA + (long)src_row * ld;
          for (int c4 = 4 * lane; c4 < ld; c4 += 128) {
            const float4 v = src_row < n ? *reinterpret_cast<const float4 *>(src + c4)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4 *>(sb + rr * stg + c4) = v;
          }
        }
        tc::warp_arrive(&sfull[buf]);
        if (!tc::warp_wait(&sfull[buf], tu & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        Va = sb + al * stg;
        gb_row = sb + (8 + bl) * stg;
      } else {
        Va = S.V32 + (long)(live ? a : 0) * ld;
        gb_row = gA + (long)(live ? b : 0) * ld;
      }
      if (!tc::warp_wait(&accf[buf], tu & 1, kWaitNs)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t tbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
      float acc0 = 0.f, acc1 = 0.f;
      for (int ch = cb; ch < ce; ++ch) {
        // the chunk's operands are requested before the TMEM read, so the two
        // latencies overlap
        float4 vc[4], gc[4];
#pragma unroll
        for (int t4 = 0; t4 < 4; ++t4) {
          vc[t4] = (live || stg > 0) ? *reinterpret_cast<const float4 *>(Va + ch * 16 + 4 * t4)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
          gc[t4] = (live || stg > 0) ? *reinterpret_cast<const float4 *>(gb_row + ch * 16 + 4 * t4)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float pv[16];
        tc::tmem_ld16(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ch * 16), pv);
        // rows are zero beyond n, so padded columns add nothing
#pragma unroll
        for (int t4 = 0; t4 < 4; ++t4) {
          acc0 = fmaf(vc[t4].x * gc[t4].x, pv[4 * t4], acc0);
          acc1 = fmaf(vc[t4].y * gc[t4].y, pv[4 * t4 + 1], acc1);
          acc0 = fmaf(vc[t4].z * gc[t4].z, pv[4 * t4 + 2], acc0);
          acc1 = fmaf(vc[t4].w * gc[t4].w, pv[4 * t4 + 3], acc1);
        }
      }
      tc::fence_before_sync();
      tc::warp_arrive(&acce[buf]);
      const float xh = (acc0 + acc1) * inv;
      float *pb = part + buf * 128;
      if (half) {
        // hand the second half's sum to warp (warp - 4) through the buffer of this
        // tile's parity, once that warp has read the buffer's previous use
        if (tu > 0 && !tc::warp_wait(&pempty[buf], (tu - 1) & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        pb[prow] = xh;
        tc::warp_arrive(&pfull[buf]);
        continue;
      }
      if (!tc::warp_wait(&pfull[buf], tu & 1, kWaitNs)) {
        *abort_flag = 1;
        break;
      }
      const float X = xh + pb[prow];
      tc::warp_arrive(&pempty[buf]);
      float sig = 0.f;
      if (live) sig = S.spin * gA[(long)a * ld + b] * S.W[((long)xt.j * n + b) * ld + a] - X;
      if (S.smax) {  // largest |Sigma| entry, for the FP16 operand scale of the convolution
        float mx = fabsf(sig);
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(S.smax, __float_as_uint(mx));
      }
      if (live) {
        const long nn = (long)n * n;
        const int j = xt.j;
        S.Sigma[(long)j * nn + (long)a * n + b] = (double)sig;
        S.Sigma[(long)j * nn + (long)b * n + a] = (double)sig;
        if (S.S32) {
          S.S32[((long)j * n + a) * ld + b] = sig;
          S.S32[((long)j * n + b) * ld + a] = sig;
        }
      }
    }
  }

  __syncthreads();
  if (*abort_flag) {
    // let MMAs still in flight finish (bounded) before the TMEM goes away
    if (warp == R::kMma && lane == 0) {
      if (issued) tc::mma_commit(drain);
      atomicExch(err, 1);
      if (issued) tc::mbar_wait(drain, 0, kWaitNs);
    }
    __syncthreads();
  }
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

}  // namespace

cudaError_t launch_split_g(int n, int M, const double *G, float *g32, float *gh, float *gl,
                           cudaStream_t s) {
  const int ld = (n + 31) / 32 * 32;
  split_kernel<<<1024, 256, 0, s>>>(n, (long)M * n, ld, G, g32, gh, gl);
  return cudaGetLastError();
}

TcGeom tc_geom(int n, int M) {
  TcGeom g{};
  g.n = n;
  g.M = M;
  g.ld = (n + 31) / 32 * 32;
  g.MT = (n + 127) / 128;
  g.Np = (n + 15) / 16 * 16;
  g.KC = (n + 31) / 32;
  if (g.Np <= 256) {
    g.NT = 1;
    g.n0[0] = 0;
    g.nsz[0] = g.Np;
    g.n0[1] = 0;
    g.nsz[1] = g.Np;
  } else {
    g.NT = 2;
    const int half = ((g.Np / 2) + 15) / 16 * 16;
    g.n0[0] = 0;
    g.nsz[0] = half;
    g.n0[1] = half;
    g.nsz[1] = g.Np - half;
  }
  g.NBUF = (g.Np <= 256) ? 2 : 1;
  return g;
}

size_t tc_smem_bytes(int Np_max, int ld_max, bool with_columns) {
  size_t b = 1024 + 2 * (2 * (size_t)kTileA + 2 * (size_t)Np_max * 128) + 128;
  if (with_columns) b += 2 * (size_t)ld_max * 4;
  return b;
}

size_t sigma2_tc_smem_bytes(int n) {
  const TcGeom g = tc_geom(n, 1);
  return tc_smem_bytes(g.Np, g.ld, true);
}

int sigma2_tc_max_n() {
  int n = 16;
  while (sigma2_tc_smem_bytes(n + 16) <= 232448 && n + 16 <= 512) n += 16;
  return n;
}

cudaError_t sigma2_tc_pre(int n, int M, const double *V, const double *G, float *ws,
                          cudaStream_t s, bool tf32_operands, int *err, bool g32_ready) {
  const int ld = (n + 31) / 32 * 32;
  const long stack = (long)M * n * ld;
  float *g32 = ws, *gh = ws + stack, *gl = ws + 2 * stack, *VQ = ws + 3 * stack;
  float *V32 = ws + 4 * stack;
  // the FP16 path takes gb from the FP16 split of g, which also made g32
  if (tf32_operands || !g32_ready)
    split_kernel<<<1024, 256, 0, s>>>(n, (long)M * n, ld, G, g32, tf32_operands ? gh : nullptr,
                                      tf32_operands ? gl : nullptr);
  split_kernel<<<64, 256, 0, s>>>(n, (long)n, ld, V, V32, nullptr, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // VQ_j = V (g_j o g_{M-1-j}) and W_j = VQ_j V on the tensor cores
  return vqv_tc(n, M, ld, V32, g32, VQ, ws + tc_ws_w(n, M), err, s);
}

void exchange_tile_table(int n, std::vector<uint32_t> &tiles) {
  tiles.clear();
  for (int b0 = 0; b0 < n; b0 += 16)
    for (int a0 = b0; a0 < n; a0 += 8)  // b0 is a multiple of 8: the first a-block on the diagonal
      tiles.push_back((uint32_t)b0 << 16 | (uint32_t)a0);
}

cudaError_t xsys_fill(XSys *d, int n, int M, double spin, const float *ws, double *Sigma,
                      float *S32, const uint32_t *tiles, unsigned *smax, const void *h16,
                      const TcScale *scale) {
  if (!tiles) return cudaErrorInvalidValue;
  d->g = tc_geom(n, M);
  d->tiles = tiles;
  d->tiles_per_j = (int)exchange_tiles(n);
  const long stack = (long)M * n * d->g.ld;
  d->spin = (float)spin;
  d->g32 = ws;
  d->V32 = ws + 4 * stack;
  d->W = ws + tc_ws_w(n, M);
  d->Sigma = Sigma;
  d->S32 = S32;
  d->smax = smax;
  d->scale = scale;
  for (int t = 0; t < 2; ++t) {
    cudaError_t e = make_tmap_rows(&d->th[t], ws + stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e == cudaSuccess) e = make_tmap_rows(&d->tl[t], ws + 2 * stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e != cudaSuccess) return e;
  }
  if (h16) {
    const int ld16 = ld16_of(n);
    const uint16_t *hh = reinterpret_cast<const uint16_t *>(h16);
    const uint16_t *hl = hh + (size_t)M * n * ld16;
    for (int t = 0; t < 2; ++t) {
      cudaError_t e = make_tmap_rows16(&d->hh[t], hh, n, M, ld16, d->g.nsz[t]);
      if (e == cudaSuccess) e = make_tmap_rows16(&d->hl[t], hl, n, M, ld16, d->g.nsz[t]);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

size_t exchange_stage_pitch(int ld_max) { return (size_t)ld_max + 4; }

cudaError_t exchange_tc_launch(const XSys *sys, const long *prefix, int n_sys, long items,
                               int Np_max, int ld_max, int *err, int num_sms, cudaStream_t s,
                               bool f16) {
  size_t smem = 1024 + 2 * (2 * (size_t)kTileA + 2 * (size_t)Np_max * 128) + kXBarBytes +
                kXPartBytes;
  // the epilogue's staged rows of V and g (two buffers of 24 rows), where they fit
  const size_t stg = exchange_stage_pitch(ld_max);
  const size_t staged = smem + 2 * 24 * stg * sizeof(float);
  const int pitch = staged <= 232448 ? (int)stg : 0;
  if (pitch) smem = staged;
  const int grid = (int)(items < num_sms ? items : num_sms);
  const int nbuf = (Np_max <= 256) ? 2 : 1;
  cudaError_t e;
  if (f16) {
    e = cudaFuncSetAttribute(exchange_tc_kernel<true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    exchange_tc_kernel<true><<<grid, XRoles<true>::kThreads, smem, s>>>(sys, prefix, n_sys, items,
                                                                        Np_max, nbuf, pitch, err);
  } else {
    e = cudaFuncSetAttribute(exchange_tc_kernel<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    exchange_tc_kernel<false><<<grid, XRoles<false>::kThreads, smem, s>>>(
        sys, prefix, n_sys, items, Np_max, nbuf, pitch, err);
  }
  return cudaGetLastError();
}

}  // namespace fedvr
