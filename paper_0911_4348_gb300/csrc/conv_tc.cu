// First Dyson convolution on the tensor cores (Sec. 2.3, Eq. deq), split TF32:
//
//   I1_i = sum_j B_ij g_j,  B_ij = c1 Sigma_k + c2 Sigma_{k+1}   (j != i)
//                           B_ii = dHF - wm_i Sigma_0 + wp_i Sigma_{M-1}
//
// with the lag bracket k and the trapezoid/interpolation weights c1, c2 of the
// FP64 path (FP64 tables, applied here in FP32). The rows (i, a) of all mesh
// points are stacked into one M*n-row matrix, so a 128-row tile is full except
// at the very end of the stack (no padding of n up to a multiple of 128); all
// columns b sit in one or two N tiles. The contraction runs over (j, c) in
// 32-wide chunks: the A operand B_ij(a, c) of each row is formed by the CUDA
// cores and split as hi + lo (TF32); B = g_j(b, c) comes from the split copy of
// g by TMA. Products hi*hi + hi*lo + lo*hi accumulate in FP32 in TMEM over a
// block of JB mesh points (about 4096 contraction terms) and each block is
// then added into the FP64 result, so rounding does not grow with M. Within a
// block the chunks run column slice by column slice, mesh point by mesh point:
// along j the lag bracket of a row moves slowly (on the power mesh a step
// needs 0.6 new bracket rows on average, against 1.8 without reuse), so the
// FP16 kernel's producer threads (two rows each) keep their two bracket rows
// in registers and fetch a row only when the bracket changes. (With four rows
// per thread in the TF32 kernel the cache measured slower than plain loads.)
//
// A work item is (row tile, split s): split s covers the mesh points
// j in [s M / S, (s + 1) M / S). Split 0 writes I1, split s > 0 its own
// partial stack; a fixed-order sum then adds the partials into I1, so results
// do not depend on the schedule. S > 1 only pays when there are too few row
// tiles to fill the GPU (small systems) or to balance the last wave.
#include "common.cuh"
#include "tc.cuh"
#include "tc_sys.cuh"

namespace fedvr {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kTileA = 128 * 128;
constexpr int kWarps = 14;  // 0-3 flush, 4-11 A producers, 12 TMA, 13 MMA
constexpr int kThreads = kWarps * 32;

struct C1Item {
  int t, j_lo, j_hi;
  double *out;  // I1 or the split's partial stack
};

// Item q of a system: split s = q / RT (split-major, so that the CTAs running
// at the same time walk the same mesh points and share g_j in L2), tile t.
// The FP32 accumulation blocks are the fixed mesh-point ranges
// [b JB, (b + 1) JB) of the system (JB depends on n and M only); split s
// takes the whole blocks [s NB / S, (s + 1) NB / S) of the NB blocks, so the
// split count decides which CTA sums a block, never where a block starts or
// ends (the host keeps S <= NB: no split is empty).
__device__ __forceinline__ C1Item c1_item(const C1Sys &S, long q) {
  C1Item it;
  const int s = (int)(q / S.RT);
  it.t = (int)(q % S.RT);
  const int NB = (S.g.M + S.JB - 1) / S.JB;
  it.j_lo = (int)(((long)s * NB) / S.S) * S.JB;
  it.j_hi = min(S.g.M, (int)(((long)(s + 1) * NB) / S.S) * S.JB);
  it.out = (s == 0) ? S.I1 : S.part + (long)(s - 1) * S.g.M * S.g.n * S.g.n;
  return it;
}

__global__ void __launch_bounds__(kThreads, 1)
    conv1_tc_kernel(const C1Sys *__restrict__ sys, const long *__restrict__ prefix, int n_sys,
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
    tc::mbar_init(&full[0], 9);  // one arrival per producer warp + the TMA thread's
    tc::mbar_init(&full[1], 9);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    tc::mbar_init(&accf[0], 1);
    tc::mbar_init(&accf[1], 1);
    tc::mbar_init(&acce[0], 4);  // one arrival per flush warp
    tc::mbar_init(&acce[1], 4);
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool issued = false;
  int cur = 0;

  if (warp >= 4 && warp < 12) {
    // ---- A producers: rows r0 + 32 k of the tile, 16-byte chunk c of each 32-wide slice ----
    const int pt = tid - 128, c = pt & 7, r0 = pt >> 3;
    uint32_t off[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) off[k] = tc::sw128_offset(r0 + 32 * k, c);
    uint32_t cc = 0;
    for (long w = blockIdx.x; w < items && !tc::warp_flag(abort_flag); w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      // fields in registers: the asm statements below clobber memory, which would
      // otherwise make the compiler reload them from the table every chunk
      const int n = S.g.n, ld = S.g.ld, M = S.g.M, KC = S.g.KC;
      const float *const S32 = S.S32;
      const int4 *const coef32 = S.coef32;
      const long R = (long)M * n;
      const C1Item it = c1_item(S, w - prefix[cur]);
      int ia[4], aa[4];
      bool live[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long r = (long)it.t * 128 + r0 + 32 * k;
        live[k] = r < R;
        ia[k] = live[k] ? (int)(r / n) : 0;
        aa[k] = live[k] ? (int)(r % n) : 0;
      }
      const int JB = S.JB;
      // chunks in the order (accumulation block, 32-wide column slice, mesh point),
      // as the MMA and TMA roles walk them
      for (int j0 = it.j_lo; j0 < it.j_hi && !tc::warp_flag(abort_flag); j0 += JB) {
        const int j1 = min(it.j_hi, j0 + JB);
        for (int kc = 0; kc < KC && !tc::warp_flag(abort_flag); ++kc) {
          const int l0 = kc * 32 + 4 * c;
          const bool in = l0 < n;  // units past n are zero padding: not fetched
          float4 s1[4], s2[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) s1[k] = s2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int j = j0; j < j1; ++j, ++cc) {
            float c1[4], c2[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const int4 cf = coef32[(long)ia[k] * M + j];
              c1[k] = __int_as_float(cf.z);
              c2[k] = __int_as_float(cf.w);
              if (live[k] && in) {  // element offsets into S32 ([2M][n][ld]) < 2^31
                s1[k] = *reinterpret_cast<const float4 *>(
                    S32 + (uint32_t)((cf.x * n + aa[k]) * ld + l0));
                s2[k] = *reinterpret_cast<const float4 *>(
                    S32 + (uint32_t)((cf.y * n + aa[k]) * ld + l0));
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
              // rows past n and dead rows stay zero; the diagonal entry j = i reads its
              // precomputed B_ii (row M + i)
              float x[4] = {fmaf(c1[k], s1[k].x, c2[k] * s2[k].x),
                            fmaf(c1[k], s1[k].y, c2[k] * s2[k].y),
                            fmaf(c1[k], s1[k].z, c2[k] * s2[k].z),
                            fmaf(c1[k], s1[k].w, c2[k] * s2[k].w)};
              float4 hi, lo;
              tc::tf32_split(x[0], hi.x, lo.x);
              tc::tf32_split(x[1], hi.y, lo.y);
              tc::tf32_split(x[2], hi.z, lo.z);
              tc::tf32_split(x[3], hi.w, lo.w);
              *reinterpret_cast<float4 *>(st + off[k]) = hi;
              *reinterpret_cast<float4 *>(st + kTileA + off[k]) = lo;
            }
            tc::fence_smem_to_async();
            tc::warp_arrive(&full[s]);
          }
        }
      }
    }
  } else if (warp == 12) {
    // ---- TMA: g_j rows 0..Np-1, 32 columns per chunk, hi and lo ----
    if (lane == 0) {
      uint32_t cc = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const C1Sys &S = sys[cur];
        const C1Item it = c1_item(S, w - prefix[cur]);
        const uint32_t bytes = 2u * (uint32_t)S.g.Np * 128u;
        const int NT = S.g.NT, KC = S.g.KC, n00 = S.g.n0[0], n01 = S.g.n0[1];
        const CUtensorMap *th0 = &S.th[0], *th1 = &S.th[1], *tl0 = &S.tl[0], *tl1 = &S.tl[1];
        const int JB = S.JB;
        for (int j0 = it.j_lo; j0 < it.j_hi && !*abort_flag; j0 += JB) {
          const int j1 = min(it.j_hi, j0 + JB);
          for (int kc = 0; kc < KC && !*abort_flag; ++kc) {
            for (int j = j0; j < j1; ++j, ++cc) {
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
                tc::tma_load_3d(st + r * 128, nt ? th1 : th0, kc * 32, r, j, &full[s]);
                tc::tma_load_3d(st + tileB + r * 128, nt ? tl1 : tl0, kc * 32, r, j, &full[s]);
              }
            }
          }
        }
      }
    }
  } else if (warp == 13) {
    // ---- MMA issue: one accumulator block per JB mesh points ----
    if (lane == 0) {
      uint32_t cc = 0, tcount = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const C1Sys &S = sys[cur];
        const C1Item it = c1_item(S, w - prefix[cur]);
        const int n = S.g.n, KC = S.g.KC, NT = S.g.NT, JB = S.JB;
        const uint32_t n00 = (uint32_t)S.g.n0[0], n01 = (uint32_t)S.g.n0[1];
        const uint32_t id0 = tc::idesc_tf32(128, S.g.nsz[0]), id1 = tc::idesc_tf32(128, S.g.nsz[1]);
        for (int j0 = it.j_lo; j0 < it.j_hi && !*abort_flag; j0 += JB, ++tcount) {
          const int j1 = min(it.j_hi, j0 + JB);
          const int buf = tcount & 1;
          const uint32_t tu = tcount >> 1;
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
          for (int kc = 0; kc < KC && !*abort_flag; ++kc) {
            const int ksteps = min(4, (n - kc * 32 + 7) / 8);
            for (int j = j0; j < j1; ++j, ++cc) {
              const int s = cc & 1;
              const uint32_t use = cc >> 1;
              if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
                *abort_flag = 1;
                break;
              }
              tc::fence_after_sync();
              const uint32_t sa = tc::smem_u32(smem + s * stage_bytes);
              const bool fresh = (j == j0 && kc == 0);
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
                  tc::mma_tf32(d, ah, bh, idesc, (fresh && kk == 0) ? 0u : 1u);
                  tc::mma_tf32(d, ah, bl, idesc, 1u);
                  tc::mma_tf32(d, al, bh, idesc, 1u);
                }
              }
              tc::mma_commit(&empty[s]);
              issued = true;
            }
          }
          tc::mma_commit(&accf[buf]);
        }
      }
    }
  } else {
    // ---- flush: add each FP32 block into the FP64 output rows. TMEM gives each
    // thread one row; a warp-private 32 x 16 staging tile in shared memory turns
    // that into row-contiguous read-modify-writes (16 columns of two rows per
    // instruction) ----
    float *stg = reinterpret_cast<float *>(smem + 2 * stage_bytes + 256) + warp * (32 * 17);
    const int cl = lane & 15, rh = lane >> 4;
    uint32_t tcount = 0;
    for (long w = blockIdx.x; w < items && !tc::warp_flag(abort_flag); w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      const int n = S.g.n, JB = S.JB;
      const long R = (long)S.g.M * n;
      const C1Item it = c1_item(S, w - prefix[cur]);
      const long row0 = (long)it.t * 128 + warp * 32;
      double *const out = it.out;
      for (int j0 = it.j_lo; j0 < it.j_hi; j0 += JB, ++tcount) {
        const int buf = tcount & 1;
        const uint32_t tu = tcount >> 1;
        if (!tc::warp_wait(&accf[buf], tu & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t tbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
        const bool first = j0 == it.j_lo;
        for (int c0 = 0; c0 < n; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
          for (int t = 0; t < 16; ++t) stg[lane * 17 + t] = v[t];
          __syncwarp();
          const int b = c0 + cl;
#pragma unroll 4
          for (int i = 0; i < 16; ++i) {
            const int rr = 2 * i + rh;
            const long grow = row0 + rr;
            if (grow < R && b < n) {
              double *p = out + grow * n + b;
              const double val = (double)stg[rr * 17 + cl];
              *p = first ? val : *p + val;
            }
          }
          __syncwarp();
        }
        tc::fence_before_sync();
        tc::warp_arrive(&acce[buf]);
      }
    }
  }

  __syncthreads();
  if (*abort_flag) {
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

__global__ void coef32_kernel(long mm, int M, const ConvCoef *__restrict__ coef,
                              int4 *__restrict__ out) {
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < mm;
       x += (long)gridDim.x * blockDim.x) {
    const ConvCoef c = coef[x];
    if (c.diag) {
      const int i = (int)(x / M);
      out[x] = make_int4(M + i, M + i, __float_as_int(1.f), __float_as_int(0.f));
    } else {
      // a zero upper weight (the lag falls on a mesh point) names the lower row
      // twice, so that no second row is fetched
      const float c2 = (float)c.c2;
      out[x] = make_int4(c.k, c2 != 0.f ? c.k + 1 : c.k, __float_as_int((float)c.c1),
                         __float_as_int(c2));
    }
  }
}

// D_i = dHF - wm_i Sigma_0 + wp_i Sigma_{M-1} at rows M + i of S32 (zero padded
// to ld), in FP32 from the FP32 copy of Sigma (rows 0 and M-1 of S32): the
// operand is split to TF32 anyway. A thread owns one element (a, c) and writes
// it for every i, so the FP64 matrix dHF is converted once per element.
__global__ void diag_f32_kernel(int n, int M, int ld, const double *__restrict__ dHF,
                                const double *__restrict__ wm, const double *__restrict__ wp,
                                float *__restrict__ S32, unsigned *smax) {
  extern __shared__ float wf[];  // wm, wp in FP32: [2][M]
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    wf[i] = (float)wm[i];
    wf[M + i] = (float)wp[i];
  }
  __syncthreads();
  const long nld = (long)n * ld;
  float *D = S32 + (long)M * nld;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < nld;
       e += (long)gridDim.x * blockDim.x) {
    const int a = (int)(e / ld), c = (int)(e % ld);
    float h = 0.f, s0 = 0.f, s1 = 0.f;
    if (c < n) {
      h = (float)dHF[(long)a * n + c];
      s0 = S32[e];
      s1 = S32[(long)(M - 1) * nld + e];
    }
    float m = 0.f;
    for (int i = 0; i < M; ++i) {
      const float v = (h - wf[i] * s0) + wf[M + i] * s1;
      D[(long)i * nld + e] = v;
      m = fmaxf(m, fabsf(v));
    }
    if (smax) {  // largest |B_ii| entry, for the FP16 operand scale
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if ((threadIdx.x & 31) == 0) atomicMax(smax, __float_as_uint(m));
    }
  }
}

// I1 += part[0] + part[1] + ... (fixed order).
__global__ void conv1_sum_splits_kernel(long count, int nparts, const double *__restrict__ part,
                                        double *__restrict__ I1) {
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < count;
       x += (long)gridDim.x * blockDim.x) {
    double v = I1[x];
    for (int q = 0; q < nparts; ++q) v += part[(long)q * count + x];
    I1[x] = v;
  }
}

// S32 = (float)Sigma with rows padded to ld (zeros beyond n).
__global__ void sigma_to_f32_kernel(int n, long rows, int ld, const double *__restrict__ S,
                                    float *__restrict__ S32, unsigned *smax) {
  const long total = rows * ld;
  float m = 0.f;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const long row = idx / ld;
    const int c = (int)(idx % ld);
    const float v = (c < n) ? (float)S[row * n + c] : 0.f;
    S32[idx] = v;
    m = fmaxf(m, fabsf(v));
  }
  if (smax) {
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(smax, __float_as_uint(m));
  }
}


// ---------------------------------------------------------------------------
// FP16-split variant (precision FEDVR_SPLIT_F16): the same contraction with
// kind::f16 MMAs. A 128-byte operand row holds 64 FP16 values, so a chunk
// covers 64 contraction terms for the same shared-memory stage size, and the
// three products hi*hi + hi*lo + lo*hi run at twice the TF32 rate. Operands are
// scaled by powers of two into FP16's normal range (g by 2^kScaleG, the
// interpolated Sigma by 2^sA with sA from maxC * max|S32|), and the flush
// multiplies the FP32 block sums by 2^-(sA + kScaleG) exactly. 16 producer
// warps, two rows of one 16-byte unit (8 values) per thread and chunk.
constexpr int kWarpsH = 22;  // 0-3 flush, 4-19 A producers, 20 TMA, 21 MMA
constexpr int kThreadsH = kWarpsH * 32;

__device__ __forceinline__ int a_scale_exp(const TcScale *sc) {
  const float amax = __uint_as_float(sc->maxS) * sc->maxC;
  if (!(amax > 0.f) || !(amax < 3.0e38f)) return 0;
  int e;
  frexpf(amax, &e);  // amax < 2^e
  e = 14 - e;        // scaled maximum below 2^14
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

__global__ void __launch_bounds__(kThreadsH, 1)
    conv1_f16_kernel(const C1Sys *__restrict__ sys, const long *__restrict__ prefix, int n_sys,
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
    tc::mbar_init(&full[0], 17);  // one arrival per producer warp + the TMA thread's
    tc::mbar_init(&full[1], 17);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    tc::mbar_init(&accf[0], 1);
    tc::mbar_init(&accf[1], 1);
    tc::mbar_init(&acce[0], 4);  // one arrival per flush warp
    tc::mbar_init(&acce[1], 4);
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool issued = false;
  int cur = 0;

  if (warp >= 4 && warp < 20) {
    // ---- A producers: rows r0 and r0 + 64 of the tile, 16-byte unit c (8 FP16
    // values) of each 64-wide slice ----
    const int pt = tid - 128, c = pt & 7, r0 = pt >> 3;
    const uint32_t off[2] = {tc::sw128_offset(r0, c), tc::sw128_offset(r0 + 64, c)};
    uint32_t cc = 0;
    for (long w = blockIdx.x; w < items && !tc::warp_flag(abort_flag); w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      const int n = S.g.n, ld = S.g.ld, M = S.g.M, KC = (n + 63) / 64;
      const float *const S32 = S.S32;
      const int4 *const coef32 = S.coef32;
      const float fA = ldexpf(1.f, a_scale_exp(S.scale));
      const long R = (long)M * n;
      const C1Item it = c1_item(S, w - prefix[cur]);
      int ia[2], aa[2];
      bool live[2];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const long r = (long)it.t * 128 + r0 + 64 * k;
        live[k] = r < R;
        ia[k] = live[k] ? (int)(r / n) : 0;
        aa[k] = live[k] ? (int)(r % n) : 0;
      }
      const int JB = S.JB, TU = S.TU, KCf = TU ? KC - 1 : KC;
      // chunks in the order (accumulation block, 64-wide column slice, mesh point),
      // the two bracket rows of each row held in registers while the bracket stays;
      // with a packed tail the last slice follows as chunks of 8 / TU mesh points
      for (int j0 = it.j_lo; j0 < it.j_hi && !tc::warp_flag(abort_flag); j0 += JB) {
        const int j1 = min(it.j_hi, j0 + JB);
        for (int kc = 0; kc < KCf && !tc::warp_flag(abort_flag); ++kc) {
          const int l0 = kc * 64 + 8 * c;
          const bool in = l0 < n;  // units starting past n are zero padding: not fetched
          int k1[2], k2[2];        // S32 rows held in a1, a2 (-1: none)
          float4 a1[2][2], a2[2][2];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            k1[k] = k2[k] = -1;
            a1[k][0] = a1[k][1] = a2[k][0] = a2[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
          }
          for (int j = j0; j < j1; ++j, ++cc) {
            float c1[2], c2[2];  // weights times the operand scale 2^sA
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              const int4 cf = coef32[(long)ia[k] * M + j];
              c1[k] = __int_as_float(cf.z) * fA;
              c2[k] = __int_as_float(cf.w) * fA;
              if (live[k] && in) {
                // updated in place (the upper row first: it may take the old lower
                // one, when the bracket moved down by one); a bracket that moved up
                // (only where the lag wraps around) is fetched again
                if (cf.y == k1[k]) {
                  a2[k][0] = a1[k][0];
                  a2[k][1] = a1[k][1];
                } else if (cf.y != k2[k]) {
                  const float *p2 = S32 + (uint32_t)((cf.y * n + aa[k]) * ld + l0);
                  a2[k][0] = *reinterpret_cast<const float4 *>(p2);
                  a2[k][1] = *reinterpret_cast<const float4 *>(p2 + 4);
                }
                if (cf.x != k1[k]) {
                  const float *p1 = S32 + (uint32_t)((cf.x * n + aa[k]) * ld + l0);
                  a1[k][0] = *reinterpret_cast<const float4 *>(p1);
                  a1[k][1] = *reinterpret_cast<const float4 *>(p1 + 4);
                }
                k1[k] = cf.x;
                k2[k] = cf.y;
                // the bracket usually moves down by one row: ask L1 for that row now
                if (cf.x > 0) {
                  const float *pn = S32 + (uint32_t)(((cf.x - 1) * n + aa[k]) * ld + l0);
                  asm volatile("prefetch.global.L1 [%0];" ::"l"(pn));
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
            for (int k = 0; k < 2; ++k) {
              // c1 Sigma_k1 + c2 Sigma_k2 on pairs of values (packed FP32 pairs:
              // the same rounding as the scalar multiply and fused multiply-add)
              const uint64_t C1 = tc::f2_pack(c1[k], c1[k]), C2 = tc::f2_pack(c2[k], c2[k]);
              const ulonglong2 p1a = *reinterpret_cast<const ulonglong2 *>(&a1[k][0]);
              const ulonglong2 p1b = *reinterpret_cast<const ulonglong2 *>(&a1[k][1]);
              const ulonglong2 p2a = *reinterpret_cast<const ulonglong2 *>(&a2[k][0]);
              const ulonglong2 p2b = *reinterpret_cast<const ulonglong2 *>(&a2[k][1]);
              uint4 hi, lo;
              tc::f16_split2p(tc::f2_fma(C1, p1a.x, tc::f2_mul(C2, p2a.x)), hi.x, lo.x);
              tc::f16_split2p(tc::f2_fma(C1, p1a.y, tc::f2_mul(C2, p2a.y)), hi.y, lo.y);
              tc::f16_split2p(tc::f2_fma(C1, p1b.x, tc::f2_mul(C2, p2b.x)), hi.z, lo.z);
              tc::f16_split2p(tc::f2_fma(C1, p1b.y, tc::f2_mul(C2, p2b.y)), hi.w, lo.w);
              *reinterpret_cast<uint4 *>(st + off[k]) = hi;
              *reinterpret_cast<uint4 *>(st + kTileA + off[k]) = lo;
            }
            tc::fence_smem_to_async();
            tc::warp_arrive(&full[s]);
          }
        }
        if (TU) {
          // packed tail: unit c holds 8 columns of mesh point jt + c / TU
          const int jpc = 8 / TU, jo = c / TU;
          const int l0 = (KC - 1) * 64 + 8 * (c % TU);
          for (int jt = j0; jt < j1 && !tc::warp_flag(abort_flag); jt += jpc, ++cc) {
            const int j = jt + jo;
            const bool jin = jo < jpc && j < j1 && l0 < n;
            float4 p1[2][2], p2[2][2];
            float c1[2], c2[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
              c1[k] = c2[k] = 0.f;
              p1[k][0] = p1[k][1] = p2[k][0] = p2[k][1] = make_float4(0.f, 0.f, 0.f, 0.f);
              if (live[k] && jin) {
                const int4 cf = coef32[(long)ia[k] * M + j];
                c1[k] = __int_as_float(cf.z) * fA;
                c2[k] = __int_as_float(cf.w) * fA;
                const float *q1 = S32 + (uint32_t)((cf.x * n + aa[k]) * ld + l0);
                p1[k][0] = *reinterpret_cast<const float4 *>(q1);
                p1[k][1] = *reinterpret_cast<const float4 *>(q1 + 4);
                if (cf.y != cf.x) {
                  const float *q2 = S32 + (uint32_t)((cf.y * n + aa[k]) * ld + l0);
                  p2[k][0] = *reinterpret_cast<const float4 *>(q2);
                  p2[k][1] = *reinterpret_cast<const float4 *>(q2 + 4);
                } else {
                  p2[k][0] = p1[k][0];
                  p2[k][1] = p1[k][1];
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
            for (int k = 0; k < 2; ++k) {
              const uint64_t C1 = tc::f2_pack(c1[k], c1[k]), C2 = tc::f2_pack(c2[k], c2[k]);
              const ulonglong2 p1a = *reinterpret_cast<const ulonglong2 *>(&p1[k][0]);
              const ulonglong2 p1b = *reinterpret_cast<const ulonglong2 *>(&p1[k][1]);
              const ulonglong2 p2a = *reinterpret_cast<const ulonglong2 *>(&p2[k][0]);
              const ulonglong2 p2b = *reinterpret_cast<const ulonglong2 *>(&p2[k][1]);
              uint4 hi, lo;
              tc::f16_split2p(tc::f2_fma(C1, p1a.x, tc::f2_mul(C2, p2a.x)), hi.x, lo.x);
              tc::f16_split2p(tc::f2_fma(C1, p1a.y, tc::f2_mul(C2, p2a.y)), hi.y, lo.y);
              tc::f16_split2p(tc::f2_fma(C1, p1b.x, tc::f2_mul(C2, p2b.x)), hi.z, lo.z);
              tc::f16_split2p(tc::f2_fma(C1, p1b.y, tc::f2_mul(C2, p2b.y)), hi.w, lo.w);
              *reinterpret_cast<uint4 *>(st + off[k]) = hi;
              *reinterpret_cast<uint4 *>(st + kTileA + off[k]) = lo;
            }
            tc::fence_smem_to_async();
            tc::warp_arrive(&full[s]);
          }
        }
      }
    }
  } else if (warp == 20) {
    // ---- TMA: g_j FP16 split rows 0..Np-1, 64 columns per chunk, hi and lo ----
    if (lane == 0) {
      uint32_t cc = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const C1Sys &S = sys[cur];
        const C1Item it = c1_item(S, w - prefix[cur]);
        const uint32_t bytes = 2u * (uint32_t)S.g.Np * 128u;
        const int NT = S.g.NT, KC = (S.g.n + 63) / 64, n00 = S.g.n0[0], n01 = S.g.n0[1];
        const CUtensorMap *th0 = &S.hh[0], *th1 = &S.hh[1], *tl0 = &S.hl[0], *tl1 = &S.hl[1];
        const int JB = S.JB, TU = S.TU, KCf = TU ? KC - 1 : KC;
        for (int j0 = it.j_lo; j0 < it.j_hi && !*abort_flag; j0 += JB) {
          const int j1 = min(it.j_hi, j0 + JB);
          for (int kc = 0; kc < KCf && !*abort_flag; ++kc) {
            for (int j = j0; j < j1; ++j, ++cc) {
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
                tc::tma_load_3d(st + r * 128, nt ? th1 : th0, kc * 64, r, j, &full[s]);
                tc::tma_load_3d(st + tileB + r * 128, nt ? tl1 : tl0, kc * 64, r, j, &full[s]);
              }
            }
          }
          // packed tail: columns jt 8 TU .. + 63 (16-byte aligned; past the end zero-filled)
          for (int jt = j0; TU && jt < j1 && !*abort_flag; jt += 8 / TU, ++cc) {
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
              tc::tma_load_2d(st + r * 128, &S.th16[nt], jt * 8 * TU, r, &full[s]);
              tc::tma_load_2d(st + tileB + r * 128, &S.tl16[nt], jt * 8 * TU, r, &full[s]);
            }
          }
        }
      }
    }
  } else if (warp == 21) {
    // ---- MMA issue (kind::f16, K = 16 per instruction) ----
    if (lane == 0) {
      uint32_t cc = 0, tcount = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const C1Sys &S = sys[cur];
        const C1Item it = c1_item(S, w - prefix[cur]);
        const int n = S.g.n, KC = (n + 63) / 64, NT = S.g.NT, JB = S.JB, TU = S.TU;
        const int KCf = TU ? KC - 1 : KC;
        const uint32_t n00 = (uint32_t)S.g.n0[0], n01 = (uint32_t)S.g.n0[1];
        const uint32_t id0 = tc::idesc_f16(128, S.g.nsz[0]), id1 = tc::idesc_f16(128, S.g.nsz[1]);
        for (int j0 = it.j_lo; j0 < it.j_hi && !*abort_flag; j0 += JB, ++tcount) {
          const int j1 = min(it.j_hi, j0 + JB);
          const int buf = tcount & 1;
          const uint32_t tu = tcount >> 1;
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
          bool fresh = true;  // the block's first chunk overwrites the accumulator
          // full slices, mesh point by mesh point, then the packed tail's chunks
          const int nch = KCf * (j1 - j0) + (TU ? (j1 - j0 + 8 / TU - 1) / (8 / TU) : 0);
          for (int q = 0; q < nch && !*abort_flag; ++q, ++cc) {
            int ksteps;
            if (q < KCf * (j1 - j0)) {
              ksteps = min(4, (n - (q / (j1 - j0)) * 64 + 15) / 16);
            } else {
              const int jt = j0 + (q - KCf * (j1 - j0)) * (8 / TU);
              ksteps = min(4, (min(8 / TU, j1 - jt) * 8 * TU + 15) / 16);
            }
            const int s = cc & 1;
            const uint32_t use = cc >> 1;
            if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
              *abort_flag = 1;
              break;
            }
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_u32(smem + s * stage_bytes);
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
                tc::mma_f16(d, ah, bh, idesc, (fresh && kk == 0) ? 0u : 1u);
                tc::mma_f16(d, ah, bl, idesc, 1u);
                tc::mma_f16(d, al, bh, idesc, 1u);
              }
            }
            fresh = false;
            tc::mma_commit(&empty[s]);
            issued = true;
          }
          tc::mma_commit(&accf[buf]);
        }
      }
    }
  } else if (warp < 4) {
    // ---- flush: scale each FP32 block back and add it into the FP64 output rows.
    // TMEM gives each thread one row; a warp-private 32 x 16 staging tile turns
    // that into row-contiguous read-modify-writes (16 columns of two rows per
    // instruction) ----
    float *stg = reinterpret_cast<float *>(smem + 2 * stage_bytes + 256) + warp * (32 * 17);
    const int cl = lane & 15, rh = lane >> 4;
    uint32_t tcount = 0;
    for (long w = blockIdx.x; w < items && !tc::warp_flag(abort_flag); w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      const int n = S.g.n, JB = S.JB;
      const double inv = ldexp(1.0, -(a_scale_exp(S.scale) + kScaleG));
      const long R = (long)S.g.M * n;
      const C1Item it = c1_item(S, w - prefix[cur]);
      const long row0 = (long)it.t * 128 + warp * 32;
      double *const out = it.out;
      for (int j0 = it.j_lo; j0 < it.j_hi; j0 += JB, ++tcount) {
        const int buf = tcount & 1;
        const uint32_t tu = tcount >> 1;
        if (!tc::warp_wait(&accf[buf], tu & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t tbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
        const bool first = j0 == it.j_lo;
        for (int c0 = 0; c0 < n; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
          for (int t = 0; t < 16; ++t) stg[lane * 17 + t] = v[t];
          __syncwarp();
          const int b = c0 + cl;
#pragma unroll 4
          for (int i = 0; i < 16; ++i) {
            const int rr = 2 * i + rh;
            const long grow = row0 + rr;
            if (grow < R && b < n) {
              double *p = out + grow * n + b;
              const double val = (double)stg[rr * 17 + cl] * inv;
              *p = first ? val : *p + val;
            }
          }
          __syncwarp();
        }
        tc::fence_before_sync();
        tc::warp_arrive(&acce[buf]);
      }
    }
  }

  __syncthreads();
  if (*abort_flag) {
    if (warp == 21 && lane == 0) {
      if (issued) tc::mma_commit(drain);
      atomicExch(err, 1);
      if (issued) tc::mbar_wait(drain, 0, kWaitNs);
    }
    __syncthreads();
  }
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// FP16 split of g scaled by 2^kScaleG; one warp per row, two columns per lane.
// A scaled entry at or above FP16's largest finite value (|g| >= 65504 / 2^12,
// just below 16) or not finite cannot be represented: the warp raises bit 1
// (value 2) of *flag and the caller reports the input as out of range. With
// g32 the same pass also writes the FP32 copy of g (pitch ld32, zero padded):
// one read of g and one FP64-to-FP32 conversion per entry serve both, the
// scaling then being an exact FP32 multiplication by 2^kScaleG. With tw > 0
// the first tw columns of the last 64-wide slice of row (j, a) are written a
// second time at column j tw of row a of the packed tail (thi, tlo; pitch
// tpitch halves, columns from M tw on zero).
__global__ void split_f16_kernel(int n, long rows, int ld16, const double *__restrict__ G,
                                 uint32_t *__restrict__ hi, uint32_t *__restrict__ lo,
                                 int *flag, float *__restrict__ g32, int ld32,
                                 uint32_t *__restrict__ thi, uint32_t *__restrict__ tlo,
                                 int tpitch, int tw) {
  const int lane = threadIdx.x & 31;
  const long wpb = blockDim.x >> 5, nw = (long)gridDim.x * wpb;
  const float sc = (float)(1 << kScaleG);
  bool bad = false;
  for (long row = blockIdx.x * wpb + (threadIdx.x >> 5); row < rows; row += nw) {
    const double *src = G + row * n;
    const long o = row * (ld16 / 2);
    for (int c0 = 0; c0 < ld16; c0 += 64) {
      const int c = c0 + 2 * lane;
      const float x0 = (c < n) ? (float)src[c] : 0.f;
      const float x1 = (c + 1 < n) ? (float)src[c + 1] : 0.f;
      if (g32 && c < ld32) {  // ld32 is even: the pair lies inside the row
        *reinterpret_cast<float2 *>(g32 + row * ld32 + c) = make_float2(x0, x1);
      }
      const float y0 = x0 * sc, y1 = x1 * sc;
      bad |= !(fabsf(y0) < 65504.f) || !(fabsf(y1) < 65504.f);
      uint32_t h, l;
      tc::f16_split2(y0, y1, h, l);
      hi[o + c / 2] = h;
      lo[o + c / 2] = l;
      if (c0 == ld16 - 64 && 2 * lane < tw) {
        const long to = ((row % n) * tpitch + (row / n) * tw) / 2 + lane;
        thi[to] = h;
        tlo[to] = l;
      }
    }
    if (tw && row / n == rows / n - 1) {  // zero the tail row's padding past column M tw
      const long mt = (rows / n) * tw;
      for (long p = lane; p < (tpitch - mt) / 2; p += 32) {
        thi[((row % n) * tpitch + mt) / 2 + p] = 0u;
        tlo[((row % n) * tpitch + mt) / 2 + p] = 0u;
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0 && flag) atomicOr(flag, 2);
}

// scale->maxC = max over (i, j) of |c1| + |c2|; scale->maxS = 0 (one block).
__global__ void scale_init_kernel(long mm, const int4 *__restrict__ coef32, long nn,
                                  const double *__restrict__ V, TcScale *scale) {
  __shared__ float sh[2][256];
  float m = 0.f, v = 0.f;
  for (long x = threadIdx.x; x < mm; x += blockDim.x) {
    const int4 c = coef32[x];
    m = fmaxf(m, fabsf(__int_as_float(c.z)) + fabsf(__int_as_float(c.w)));
  }
  for (long x = threadIdx.x; x < nn; x += blockDim.x) v = fmaxf(v, (float)fabs(V[x]));
  sh[0][threadIdx.x] = m;
  sh[1][threadIdx.x] = v;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      sh[0][threadIdx.x] = fmaxf(sh[0][threadIdx.x], sh[0][threadIdx.x + st]);
      sh[1][threadIdx.x] = fmaxf(sh[1][threadIdx.x], sh[1][threadIdx.x + st]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scale->maxC = sh[0][0];
    scale->maxV = sh[1][0];  // the largest |V32| entry exactly: V32 = (float)V
    scale->maxS = 0u;
    scale->pad = 0u;
  }
}

}  // namespace

cudaError_t launch_sigma_to_f32(int n, int M, const double *S, float *S32, cudaStream_t s,
                                unsigned *smax) {
  const int ld = (n + 31) / 32 * 32;
  sigma_to_f32_kernel<<<1024, 256, 0, s>>>(n, (long)M * n, ld, S, S32, smax);
  return cudaGetLastError();
}

cudaError_t c1sys_fill(C1Sys *d, int n, int M, int splits, const float *ws, const float *S32,
                       const double *dHF, const int4 *coef32, double *I1, double *part,
                       const void *h16, const TcScale *scale) {
  d->g = tc_geom(n, M);
  const long stack = (long)M * n * d->g.ld;
  d->JB = conv1_block_points(n, M, h16 != nullptr);
  if (splits < 1 || splits > conv1_blocks(n, M, h16 != nullptr)) return cudaErrorInvalidValue;
  d->S = splits;
  d->RT = (int)(((long)M * n + 127) / 128);
  d->S32 = S32;
  d->dHF = dHF;
  d->coef32 = coef32;
  d->I1 = I1;
  d->part = part;
  for (int t = 0; t < 2; ++t) {
    cudaError_t e = make_tmap_rows(&d->th[t], ws + stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e == cudaSuccess) e = make_tmap_rows(&d->tl[t], ws + 2 * stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e != cudaSuccess) return e;
  }
  d->scale = scale;
  if (h16) {
    const int ld16 = ld16_of(n);
    const uint16_t *hh = reinterpret_cast<const uint16_t *>(h16);
    const uint16_t *hl = hh + (size_t)M * n * ld16;
    for (int t = 0; t < 2; ++t) {
      cudaError_t e = make_tmap_rows16(&d->hh[t], hh, n, M, ld16, d->g.nsz[t]);
      if (e == cudaSuccess) e = make_tmap_rows16(&d->hl[t], hl, n, M, ld16, d->g.nsz[t]);
      if (e != cudaSuccess) return e;
    }
    d->TU = c1_tail_units(n);
    if (d->TU) {
      const int tp = c1_tail_pitch(n, M);
      const uint16_t *th = hl + (size_t)M * n * ld16, *tl = th + (size_t)n * tp;
      for (int t = 0; t < 2; ++t) {
        // the whole pitch is mapped (at least one 64-wide box; the padding is zero)
        cudaError_t e = make_tmap_tail16(&d->th16[t], th, n, tp, tp, d->g.nsz[t]);
        if (e == cudaSuccess) e = make_tmap_tail16(&d->tl16[t], tl, n, tp, tp, d->g.nsz[t]);
        if (e != cudaSuccess) return e;
      }
    }
  }
  return cudaSuccess;
}

cudaError_t launch_split_f16(int n, int M, const double *G, void *h16, cudaStream_t s,
                             int *flag, float *g32) {
  const int ld16 = ld16_of(n), tp = c1_tail_pitch(n, M);
  uint32_t *hi = reinterpret_cast<uint32_t *>(h16);
  uint32_t *lo = hi + (size_t)M * n * ld16 / 2;
  uint32_t *thi = lo + (size_t)M * n * ld16 / 2, *tlo = thi + (size_t)n * tp / 2;
  split_f16_kernel<<<1024, 256, 0, s>>>(n, (long)M * n, ld16, G, hi, lo, flag, g32,
                                        (n + 31) / 32 * 32, thi, tlo, tp,
                                        8 * c1_tail_units(n));
  return cudaGetLastError();
}

cudaError_t launch_scale_init(int M, const int4 *coef32, int n, const double *V, TcScale *scale,
                              cudaStream_t s) {
  scale_init_kernel<<<1, 256, 0, s>>>((long)M * M, coef32, (long)n * n, V, scale);
  return cudaGetLastError();
}

cudaError_t launch_diag_f32(int n, int M, const double *dHF, const double *Sigma,
                            const double *wm, const double *wp, float *S32, cudaStream_t s,
                            unsigned *smax) {
  (void)Sigma;  // read through its FP32 copy in S32
  const int ld = (n + 31) / 32 * 32;
  const long nld = (long)n * ld;
  const int blocks = (int)((nld + 255) / 256);
  const size_t shm = 2 * (size_t)M * sizeof(float);
  if (shm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(diag_f32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
  }
  diag_f32_kernel<<<blocks, 256, shm, s>>>(n, M, ld, dHF, wm, wp, S32, smax);
  return cudaGetLastError();
}

cudaError_t launch_coef32(int M, const ConvCoef *coef, int4 *out, cudaStream_t s) {
  coef32_kernel<<<512, 256, 0, s>>>((long)M * M, M, coef, out);
  return cudaGetLastError();
}

cudaError_t conv1_sum_splits(long count, int nparts, const double *part, double *I1,
                             cudaStream_t s) {
  if (nparts < 1) return cudaSuccess;
  conv1_sum_splits_kernel<<<1024, 256, 0, s>>>(count, nparts, part, I1);
  return cudaGetLastError();
}

cudaError_t conv1_tc_launch(const C1Sys *sys, const long *prefix, int n_sys, long items,
                            int Np_max, int *err, int num_sms, cudaStream_t s, bool f16) {
  // stages + barriers (256 B) + four 32 x 17 float flush staging tiles
  const size_t smem = 1024 + 2 * (2 * (size_t)kTileA + 2 * (size_t)Np_max * 128) + 256 +
                      4 * 32 * 17 * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(conv1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(items < num_sms ? items : num_sms);
  const int nbuf = (Np_max <= 256) ? 2 : 1;
  if (f16) {
    e = cudaFuncSetAttribute(conv1_f16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    conv1_f16_kernel<<<grid, kThreadsH, smem, s>>>(sys, prefix, n_sys, items, Np_max, nbuf, err);
    return cudaGetLastError();
  }
  conv1_tc_kernel<<<grid, kThreads, smem, s>>>(sys, prefix, n_sys, items, Np_max, nbuf, err);
  return cudaGetLastError();
}

}  // namespace fedvr
