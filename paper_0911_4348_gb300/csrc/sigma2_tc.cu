// Second-Born self-energy on the tensor cores (Sec. 2.3, Eq. sigma2ndb in
// two-index form), split-TF32 precision:
//
//   Sigma_ab = sum_k V_ak [ sigma g_ab (Q V)_kb - g_kb P^(b)_ak ],
//   P^(b) = g diag(V_b,:) gb,  Q = g o gb,  g = G[j], gb = G[M-1-j].
//
// The first bracket term is the direct term sigma g o (V Q V), the second the
// second-order exchange X. P^(b) is the only O(n^3)-per-column contraction
// (O(n^4) per mesh point): it runs as tcgen05.mma kind::tf32 over the rows
// (b, a), a >= b, of one mesh point stacked into n(n+1)/2 rows (128 per tile,
// tiles full except the last), all k in one or two N tiles and the
// contraction over l in 32-wide chunks, each operand split as x = hi + lo
// (TF32) and the product taken as hi*hi + hi*lo + lo*hi with FP32
// accumulation in TMEM. The A operand g_al V_bl of each row is formed by the
// CUDA cores while the previous chunk multiplies; B = gb is the same for every
// row of the mesh point. The epilogue reads row (b, a) of P^(b) from TMEM and
// folds the k-sum in FP32; the symmetric result is mirrored.
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

// Row r of the stacked lower triangle of one mesh point: rows ordered by b,
// then a = b..n-1, so row b starts at off(b) = b n - b (b - 1) / 2.
__device__ __forceinline__ long tri_off(int n, int b) { return (long)b * n - (long)b * (b - 1) / 2; }

__device__ __forceinline__ void tri_row(int n, long r, int *b, int *a) {
  const double h = 2.0 * n + 1.0;
  int bb = (int)((h - sqrt(fmax(h * h - 8.0 * (double)r, 0.0))) * 0.5);
  if (bb < 0) bb = 0;
  if (bb > n - 1) bb = n - 1;
  while (bb > 0 && tri_off(n, bb) > r) --bb;
  while (bb + 1 < n && tri_off(n, bb + 1) <= r) ++bb;
  *b = bb;
  *a = bb + (int)(r - tri_off(n, bb));
}

// Warp roles: 0-3 epilogue (TMEM lanes 0-127), 4-11 A-operand producers,
// 12 TMA loads of the gb operand, 13 MMA issue. Stages handed over with
// mbarriers: full[s] (256 producer arrivals + TMA bytes), empty[s] (MMA
// commit); accumulators double-buffered with accf/acce. The work queue is the
// concatenation of the (j, row tile) items of every system in the table
// (mesh-point-major, so that concurrent CTAs share gb in L2); every role walks
// it in the same order. The stage layout uses the table's largest N.
constexpr int kWarps2 = 14;
constexpr int kThreads2 = kWarps2 * 32;

__global__ void __launch_bounds__(kThreads2, 1)
    exchange_tc_kernel(const XSys *__restrict__ sys, const long *__restrict__ prefix, int n_sys,
                       long items, int Np_max, int nbuf, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const uint32_t tileB = (uint32_t)Np_max * 128;
  const uint32_t stage_bytes = 2 * kTileA + 2 * tileB;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);
  uint64_t *full = bars, *empty = bars + 2, *accf = bars + 4, *acce = bars + 6, *drain = bars + 8;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 10);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&full[0], 257);
    tc::mbar_init(&full[1], 257);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    tc::mbar_init(&accf[0], 1);
    tc::mbar_init(&accf[1], 1);
    tc::mbar_init(&acce[0], 128);
    tc::mbar_init(&acce[1], 128);
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool issued = false;
  int cur = 0;  // system of the current item (items ascend within a CTA)

  if (warp >= 4 && warp < 12) {
    // ---- A producers: row (b, a): A(l) = g_al * V_bl, split hi/lo, 4 rows per thread ----
    const int pt = tid - 128, c = pt & 7, r0 = pt >> 3;
    uint32_t cc = 0;
    for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const XSys &S = sys[cur];
      const int n = S.g.n, ld = S.g.ld, KC = S.g.KC;
      const long T = (long)n * (n + 1) / 2, RT = (T + 127) / 128;
      const long q = w - prefix[cur];
      const int j = (int)(q / RT);
      const long t = q % RT;
      const float *const gA = S.g32 + (long)j * n * ld;
      const float *const V32 = S.V32;  // in a register across the memory-clobbering asm
      uint32_t og[4], ov[4];  // element offsets of row a of g_j and row b of V
      bool live[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long r = t * 128 + r0 + 32 * k;
        live[k] = r < T;
        int b = 0, a = 0;
        if (live[k]) tri_row(n, r, &b, &a);
        og[k] = (uint32_t)(a * ld + 4 * c);
        ov[k] = (uint32_t)(b * ld + 4 * c);
      }
      for (int kc = 0; kc < KC; ++kc, ++cc) {
        const int l0 = kc * 32;
        float4 gv[4], vv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (live[k]) {
            gv[k] = *reinterpret_cast<const float4 *>(gA + og[k] + l0);
            vv[k] = *reinterpret_cast<const float4 *>(V32 + ov[k] + l0);
          } else {
            gv[k] = vv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
        const int s = cc & 1;
        const uint32_t use = cc >> 1;
        if (use > 0 && !tc::mbar_wait(&empty[s], (use - 1) & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        uint8_t *st = smem + s * stage_bytes;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float x0 = gv[k].x * vv[k].x, x1 = gv[k].y * vv[k].y, x2 = gv[k].z * vv[k].z,
                      x3 = gv[k].w * vv[k].w;
          float4 hi, lo;
          tc::tf32_split(x0, hi.x, lo.x);
          tc::tf32_split(x1, hi.y, lo.y);
          tc::tf32_split(x2, hi.z, lo.z);
          tc::tf32_split(x3, hi.w, lo.w);
          const uint32_t off = tc::sw128_offset(r0 + 32 * k, c);
          *reinterpret_cast<float4 *>(st + off) = hi;
          *reinterpret_cast<float4 *>(st + kTileA + off) = lo;
        }
        tc::fence_smem_to_async();
        tc::mbar_arrive(&full[s]);
      }
    }
  } else if (warp == 12) {
    // ---- TMA: gb = G[M-1-j] rows 0..Np-1, 32 columns per chunk, hi and lo ----
    if (lane == 0) {
      uint32_t cc = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const XSys &S = sys[cur];
        const int n = S.g.n;
        const long RT = ((long)n * (n + 1) / 2 + 127) / 128;
        const int j = (int)((w - prefix[cur]) / RT);
        const uint32_t bytes = 2u * (uint32_t)S.g.Np * 128u;
        const int NT = S.g.NT, KC = S.g.KC, jb = S.g.M - 1 - j, n00 = S.g.n0[0], n01 = S.g.n0[1];
        const CUtensorMap *th0 = &S.th[0], *th1 = &S.th[1], *tl0 = &S.tl[0], *tl1 = &S.tl[1];
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
            tc::tma_load_3d(st + r * 128, nt ? th1 : th0, kc * 32, r, jb, &full[s]);
            tc::tma_load_3d(st + tileB + r * 128, nt ? tl1 : tl0, kc * 32, r, jb, &full[s]);
          }
        }
      }
    }
  } else if (warp == 13) {
    // ---- MMA issue: one accumulator per row tile ----
    if (lane == 0) {
      uint32_t cc = 0, tcount = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, ++tcount) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const XSys &S = sys[cur];
        const int n = S.g.n, KC = S.g.KC, NT = S.g.NT;
        const uint32_t n00 = (uint32_t)S.g.n0[0], n01 = (uint32_t)S.g.n0[1];
        const uint32_t id0 = tc::idesc_tf32(128, S.g.nsz[0]), id1 = tc::idesc_tf32(128, S.g.nsz[1]);
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
          const int ksteps = min(4, (n - kc * 32 + 7) / 8);
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
              tc::mma_tf32(d, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
              tc::mma_tf32(d, ah, bl, idesc, 1u);
              tc::mma_tf32(d, al, bh, idesc, 1u);
            }
          }
          tc::mma_commit(&empty[s]);
          issued = true;
        }
        tc::mma_commit(&accf[buf]);
      }
    }
  } else {
    // ---- epilogue, row (b, a): Sigma_ab = sum_k V_ak (sigma g_ab (QV)_kb - g_kb P_ak) ----
    uint32_t tcount = 0;
    for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x, ++tcount) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const XSys &S = sys[cur];
      const int n = S.g.n, ld = S.g.ld;
      const long T = (long)n * (n + 1) / 2, RT = (T + 127) / 128;
      const long q = w - prefix[cur];
      const int j = (int)(q / RT);
      const long r = (q % RT) * 128 + warp * 32 + lane;
      const bool live = r < T;
      int b = 0, a = 0;
      if (live) tri_row(n, r, &b, &a);
      const float *gA = S.g32 + (long)j * n * ld;
      const float *Va = S.V32 + (long)a * ld;              // V_ak = V_ka: row a
      const float *gb_row = gA + (long)b * ld;              // g_kb = g_bk: row b
      const float *qb_row = S.VQ + ((long)j * n + b) * ld;  // (QV)_kb = (VQ)_bk
      const float sg = live ? S.spin * gA[(long)a * ld + b] : 0.f;
      const int buf = tcount & 1;
      const uint32_t tu = tcount >> 1;
      if (!tc::mbar_wait(&accf[buf], tu & 1, kWaitNs)) {
        *abort_flag = 1;
        break;
      }
      tc::fence_after_sync();
      const uint32_t tbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
      float acc = 0.f;
      for (int c0 = 0; c0 < n; c0 += 16) {
        float pv[16];
        tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, pv);
        if (live) {
#pragma unroll
          for (int t4 = 0; t4 < 4; ++t4) {
            const float4 v4 = *reinterpret_cast<const float4 *>(Va + c0 + 4 * t4);
            const float4 g4 = *reinterpret_cast<const float4 *>(gb_row + c0 + 4 * t4);
            const float4 q4 = *reinterpret_cast<const float4 *>(qb_row + c0 + 4 * t4);
            // rows are zero beyond n, so padded columns add nothing
            acc = fmaf(v4.x, sg * q4.x - g4.x * pv[4 * t4], acc);
            acc = fmaf(v4.y, sg * q4.y - g4.y * pv[4 * t4 + 1], acc);
            acc = fmaf(v4.z, sg * q4.z - g4.z * pv[4 * t4 + 2], acc);
            acc = fmaf(v4.w, sg * q4.w - g4.w * pv[4 * t4 + 3], acc);
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&acce[buf]);
      if (S.smax) {  // largest |Sigma| entry, for the FP16 operand scale of the convolution
        float mx = live ? fabsf(acc) : 0.f;
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(S.smax, __float_as_uint(mx));
      }
      if (live) {
        const long nn = (long)n * n;
        S.Sigma[(long)j * nn + (long)a * n + b] = (double)acc;
        S.Sigma[(long)j * nn + (long)b * n + a] = (double)acc;
        if (S.S32) {
          S.S32[((long)j * n + a) * ld + b] = acc;
          S.S32[((long)j * n + b) * ld + a] = acc;
        }
      }
    }
  }

  __syncthreads();
  if (*abort_flag) {
    // let MMAs still in flight finish (bounded) before the TMEM goes away
    if (warp == 13 && lane == 0) {
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
                          cudaStream_t s) {
  const int ld = (n + 31) / 32 * 32;
  const long stack = (long)M * n * ld;
  float *g32 = ws, *gh = ws + stack, *gl = ws + 2 * stack, *VQ = ws + 3 * stack;
  float *V32 = ws + 4 * stack;
  split_kernel<<<1024, 256, 0, s>>>(n, (long)M * n, ld, G, g32, gh, gl);
  split_kernel<<<64, 256, 0, s>>>(n, (long)n, ld, V, V32, nullptr, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_vq(n, M, ld, V32, g32, VQ, s);
}

cudaError_t xsys_fill(XSys *d, int n, int M, double spin, const float *ws, double *Sigma,
                      float *S32, unsigned *smax) {
  d->g = tc_geom(n, M);
  const long stack = (long)M * n * d->g.ld;
  d->spin = (float)spin;
  d->g32 = ws;
  d->VQ = ws + 3 * stack;
  d->V32 = ws + 4 * stack;
  d->Sigma = Sigma;
  d->S32 = S32;
  d->smax = smax;
  for (int t = 0; t < 2; ++t) {
    cudaError_t e = make_tmap_rows(&d->th[t], ws + stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e == cudaSuccess) e = make_tmap_rows(&d->tl[t], ws + 2 * stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t exchange_tc_launch(const XSys *sys, const long *prefix, int n_sys, long items,
                               int Np_max, int ld_max, int *err, int num_sms, cudaStream_t s) {
  (void)ld_max;
  const size_t smem = tc_smem_bytes(Np_max, 0, false);
  cudaError_t e = cudaFuncSetAttribute(exchange_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(items < num_sms ? items : num_sms);
  const int nbuf = (Np_max <= 256) ? 2 : 1;
  exchange_tc_kernel<<<grid, kThreads2, smem, s>>>(sys, prefix, n_sys, items, Np_max, nbuf, err);
  return cudaGetLastError();
}

}  // namespace fedvr
