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
// then added into the FP64 result, so rounding does not grow with M.
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
constexpr uint32_t kTileA = 128 * 64;  // 128 rows x 16 floats (64-byte swizzled)
constexpr int kMaxStages = 6;
constexpr int kWarps = 14;  // 0-3 flush, 4-7 and 8-11 A producers (even / odd chunks), 12 TMA, 13 MMA
constexpr int kThreads = kWarps * 32;

// Item q of a system: split s = q / RT (split-major, so the CTAs running at
// the same time walk the same mesh points and share g_j in L2), tile t.
struct C1Item {
  int t, j_lo, j_hi;
  double *out;  // I1 or the split's partial stack
};

__device__ __forceinline__ C1Item c1_item(const C1Sys &S, long q) {
  C1Item it;
  const int s = (int)(q / S.RT);
  it.t = (int)(q % S.RT);
  it.j_lo = (int)(((long)s * S.g.M) / S.S);
  it.j_hi = (int)(((long)(s + 1) * S.g.M) / S.S);
  it.out = (s == 0) ? S.I1 : S.part + (long)(s - 1) * S.g.M * S.g.n * S.g.n;
  return it;
}

// Walk over the (item, j, chunk) sequence of one CTA for the four rows
// r0 + 32 k of each tile that a producer thread owns.
struct ProdCur {
  long w;
  int cur, n, M, ld, KC, j, j_hi, kc;
  int i[4], a[4];
  unsigned live;  // bit k: row k exists
  bool done;
};

__device__ __forceinline__ void pc_item(ProdCur &p, const C1Sys *sys, const long *prefix,
                                        int n_sys, long items, int r0) {
  while (p.w < items) {
    while (p.cur + 1 < n_sys && p.w >= prefix[p.cur + 1]) ++p.cur;
    const C1Sys &S = sys[p.cur];
    const C1Item it = c1_item(S, p.w - prefix[p.cur]);
    if (it.j_lo < it.j_hi) {
      p.n = S.g.n;
      p.M = S.g.M;
      p.ld = S.g.ld;
      p.KC = (S.g.n + 15) / 16;
      p.j = it.j_lo;
      p.j_hi = it.j_hi;
      p.kc = 0;
      const long R = (long)p.M * p.n;
      p.live = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long r = (long)it.t * 128 + r0 + 32 * k;
        const bool lv = r < R;
        p.live |= (lv ? 1u : 0u) << k;
        p.i[k] = lv ? (int)(r / p.n) : 0;
        p.a[k] = lv ? (int)(r % p.n) : 0;
      }
      return;
    }
    p.w += gridDim.x;
  }
  p.done = true;
}

// Advance by one chunk. Returns 0 (same mesh point), 1 (next mesh point of the
// same item) or 2 (another item, or the end).
__device__ __forceinline__ int pc_next(ProdCur &p, const C1Sys *sys, const long *prefix,
                                       int n_sys, long items, int r0) {
  if (++p.kc < p.KC) return 0;
  p.kc = 0;
  if (++p.j < p.j_hi) return 1;
  p.w += gridDim.x;
  pc_item(p, sys, prefix, n_sys, items, r0);
  return 2;
}

// Coefficients of the cursor's mesh point after it moved (how: 0 same mesh
// point, 1 next mesh point, 2 new item). The loads are only issued here; they
// are first used a whole group step later, when the next chunk's rows load.
__device__ __forceinline__ void pc_coefs(const ProdCur &p, const C1Sys *sys, int4 (&cf)[4],
                                         int how) {
  if (p.done || how == 0) return;
  const int4 *tab = sys[p.cur].coef32;
#pragma unroll
  for (int k = 0; k < 4; ++k) cf[k] = tab[(long)p.i[k] * p.M + p.j];
}

// Start the loads of the cursor's chunk: both source rows of the thread's
// four rows (16-byte chunk c) and their weights.
__device__ __forceinline__ void pc_load(const ProdCur &p, const C1Sys *sys, int c,
                                        const int4 (&cf)[4], float4 (&s1)[4], float4 (&s2)[4],
                                        float (&d1)[4], float (&d2)[4]) {
  const float *S32 = sys[p.cur].S32;
  const long nld = (long)p.n * p.ld;
  const int l0 = p.kc * 16 + 4 * c;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    d1[k] = __int_as_float(cf[k].z);
    d2[k] = __int_as_float(cf[k].w);
    if ((p.live >> k) & 1u) {
      const long base = (long)p.a[k] * p.ld + l0;
      s1[k] = *reinterpret_cast<const float4 *>(S32 + (long)cf[k].x * nld + base);
      s2[k] = *reinterpret_cast<const float4 *>(S32 + (long)cf[k].y * nld + base);
    } else {
      s1[k] = s2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    conv1_tc_kernel(const C1Sys *__restrict__ sys, const long *__restrict__ prefix, int n_sys,
                    long items, int Np_max, int nstage, int nbuf, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const uint32_t tileB = (uint32_t)Np_max * 64;
  const uint32_t stage_bytes = 2 * kTileA + 2 * tileB;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + nstage * stage_bytes);
  uint64_t *full = bars, *empty = bars + kMaxStages, *accf = bars + 2 * kMaxStages,
           *acce = accf + 2, *drain = acce + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < nstage; ++s) {
      tc::mbar_init(&full[s], 129);  // one producer group + the TMA thread
      tc::mbar_init(&empty[s], 1);
    }
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
  int cur = 0;

  if (warp >= 4 && warp < 12) {
    // ---- A producers. Group grp (warps 4-7 or 8-11) forms every other chunk
    // (global chunk index q = grp, grp + 2, ...); a thread owns rows r0 + 32 k
    // and 16-byte chunk c of the 16-wide slice. The two source rows of the
    // group's next chunk are loaded into registers while the stage of the
    // current one drains; a mesh point's coefficients are requested as soon as
    // the cursor reaches it, one group step before their first use. Diagonal entries j = i read the precomputed B_ii
    // (source row M + i), so every entry is c1 S_k1 + c2 S_k2. ----
    const int grp = (warp - 4) >> 2;
    const int gt = (tid - 128) & 127;
    const int c = gt & 3, r0 = gt >> 2;
    uint32_t offA[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) offA[k] = tc::sw64_offset(r0 + 32 * k, c);
    ProdCur ip{};
    ip.w = blockIdx.x;
    pc_item(ip, sys, prefix, n_sys, items, r0);
    if (grp == 1 && !ip.done) pc_next(ip, sys, prefix, n_sys, items, r0);
    int4 cf[4];  // {k1, k2, c1, c2} of ip's mesh point
    if (!ip.done) pc_coefs(ip, sys, cf, 2);
    float4 s1[4], s2[4];
    float d1[4], d2[4];
    bool have = !ip.done;
    if (have) {
      pc_load(ip, sys, c, cf, s1, s2, d1, d2);
      for (int h = 0; h < 2 && !ip.done; ++h)
        pc_coefs(ip, sys, cf, pc_next(ip, sys, prefix, n_sys, items, r0));
    }
    int st = grp % nstage;
    uint32_t u = (uint32_t)(grp / nstage);
    while (have && !*abort_flag) {
      if (u > 0 && !tc::mbar_wait(&empty[st], (u - 1) & 1, kWaitNs)) {
        *abort_flag = 1;
        break;
      }
      uint8_t *sa = smem + st * stage_bytes;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float x0 = fmaf(d1[k], s1[k].x, d2[k] * s2[k].x);
        const float x1 = fmaf(d1[k], s1[k].y, d2[k] * s2[k].y);
        const float x2 = fmaf(d1[k], s1[k].z, d2[k] * s2[k].z);
        const float x3 = fmaf(d1[k], s1[k].w, d2[k] * s2[k].w);
        const float4 hi = make_float4(tc::tf32_rna(x0), tc::tf32_rna(x1), tc::tf32_rna(x2),
                                      tc::tf32_rna(x3));
        const float4 lo = make_float4(tc::tf32_rna(x0 - hi.x), tc::tf32_rna(x1 - hi.y),
                                      tc::tf32_rna(x2 - hi.z), tc::tf32_rna(x3 - hi.w));
        *reinterpret_cast<float4 *>(sa + offA[k]) = hi;
        *reinterpret_cast<float4 *>(sa + kTileA + offA[k]) = lo;
      }
      tc::fence_smem_to_async();
      tc::mbar_arrive(&full[st]);
      st += 2;
      while (st >= nstage) {
        st -= nstage;
        ++u;
      }
      have = !ip.done;
      if (have) {  // the group's next chunk: in flight while that stage drains
        pc_load(ip, sys, c, cf, s1, s2, d1, d2);
        for (int h = 0; h < 2 && !ip.done; ++h)
          pc_coefs(ip, sys, cf, pc_next(ip, sys, prefix, n_sys, items, r0));
      }
    }
  } else if (warp == 12) {
    // ---- TMA: g_j rows 0..Np-1, 16 columns per chunk, hi and lo ----
    if (lane == 0) {
      int st = 0;
      uint32_t u = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const C1Sys &S = sys[cur];
        const C1Item it = c1_item(S, w - prefix[cur]);
        const uint32_t bytes = 2u * (uint32_t)S.g.Np * 64u;
        const int KC = (S.g.n + 15) / 16;
        for (int j = it.j_lo; j < it.j_hi && !*abort_flag; ++j) {
          for (int kc = 0; kc < KC; ++kc) {
            if (u > 0 && !tc::mbar_wait(&empty[st], (u - 1) & 1, kWaitNs)) {
              *abort_flag = 1;
              break;
            }
            uint8_t *sb = smem + st * stage_bytes + 2 * kTileA;
            tc::mbar_arrive_expect_tx(&full[st], bytes);
            for (int nt = 0; nt < S.g.NT; ++nt) {
              tc::tma_load_3d(sb + S.g.n0[nt] * 64, &S.th[nt], kc * 16, S.g.n0[nt], j, &full[st]);
              tc::tma_load_3d(sb + tileB + S.g.n0[nt] * 64, &S.tl[nt], kc * 16, S.g.n0[nt], j,
                              &full[st]);
            }
            if (++st == nstage) {
              st = 0;
              ++u;
            }
          }
        }
      }
    }
  } else if (warp == 13) {
    // ---- MMA issue: one accumulator block per JB mesh points ----
    if (lane == 0) {
      int st = 0;
      uint32_t u = 0, tcount = 0;
      for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
        while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
        const C1Sys &S = sys[cur];
        const C1Item it = c1_item(S, w - prefix[cur]);
        const int n = S.g.n, KC = (n + 15) / 16;
        for (int j0 = it.j_lo; j0 < it.j_hi && !*abort_flag; j0 += S.JB, ++tcount) {
          const int j1 = min(it.j_hi, j0 + S.JB);
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
          for (int j = j0; j < j1 && !*abort_flag; ++j) {
            for (int kc = 0; kc < KC; ++kc) {
              if (!tc::mbar_wait(&full[st], u & 1, kWaitNs)) {
                *abort_flag = 1;
                break;
              }
              tc::fence_after_sync();
              const uint32_t sa = tc::smem_u32(smem + st * stage_bytes);
              const int ksteps = min(2, (n - kc * 16 + 7) / 8);
              const bool fresh = (j == j0 && kc == 0);
              for (int kk = 0; kk < ksteps; ++kk) {
                const uint64_t ah = tc::sdesc_k64(sa + kk * 32);
                const uint64_t al = tc::sdesc_k64(sa + kTileA + kk * 32);
                for (int nt = 0; nt < S.g.NT; ++nt) {
                  const uint32_t boff = 2 * kTileA + (uint32_t)S.g.n0[nt] * 64 + kk * 32;
                  const uint64_t bh = tc::sdesc_k64(sa + boff);
                  const uint64_t bl = tc::sdesc_k64(sa + boff + tileB);
                  const uint32_t d = dbase + (uint32_t)S.g.n0[nt];
                  const uint32_t idesc = tc::idesc_tf32(128, S.g.nsz[nt]);
                  tc::mma_tf32(d, ah, bh, idesc, (fresh && kk == 0) ? 0u : 1u);
                  tc::mma_tf32(d, ah, bl, idesc, 1u);
                  tc::mma_tf32(d, al, bh, idesc, 1u);
                }
              }
              tc::mma_commit(&empty[st]);
              issued = true;
              if (++st == nstage) {
                st = 0;
                ++u;
              }
            }
          }
          tc::mma_commit(&accf[buf]);
        }
      }
    }
  } else {
    // ---- flush: add each FP32 block into the FP64 output rows ----
    uint32_t tcount = 0;
    for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      const int n = S.g.n;
      const C1Item it = c1_item(S, w - prefix[cur]);
      const long r = (long)it.t * 128 + warp * 32 + lane;
      const bool live = r < (long)S.g.M * n;
      double *row = it.out + (live ? r : 0) * n;
      for (int j0 = it.j_lo; j0 < it.j_hi; j0 += S.JB, ++tcount) {
        const int buf = tcount & 1;
        const uint32_t tu = tcount >> 1;
        if (!tc::mbar_wait(&accf[buf], tu & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t tbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
        const bool first = j0 == it.j_lo;
        for (int c0 = 0; c0 < n; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
          if (live) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const int b = c0 + t;
              if (b < n) row[b] = first ? (double)v[t] : row[b] + (double)v[t];
            }
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&acce[buf]);
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
      out[x] = make_int4(c.k, c.k + 1, __float_as_int((float)c.c1), __float_as_int((float)c.c2));
    }
  }
}

// D_i = dHF - wm_i Sigma_0 + wp_i Sigma_{M-1} at rows M + i of S32 (zero padded to ld).
__global__ void diag_f32_kernel(int n, int M, int ld, const double *__restrict__ dHF,
                                const double *__restrict__ S, const double *__restrict__ wm,
                                const double *__restrict__ wp, float *__restrict__ D) {
  const long nn = (long)n * n, total = (long)M * n * ld;
  const double *S0 = S, *S1 = S + (long)(M - 1) * nn;
  for (long x = (long)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (long)gridDim.x * blockDim.x) {
    const long row = x / ld;
    const int c = (int)(x % ld);
    const int i = (int)(row / n), a = (int)(row % n);
    float v = 0.f;
    if (c < n) {
      const long e = (long)a * n + c;
      v = (float)(dHF[e] - wm[i] * S0[e] + wp[i] * S1[e]);
    }
    D[x] = v;
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
                                    float *__restrict__ S32) {
  const long total = rows * ld;
  for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long)gridDim.x * blockDim.x) {
    const long row = idx / ld;
    const int c = (int)(idx % ld);
    S32[idx] = (c < n) ? (float)S[row * n + c] : 0.f;
  }
}

}  // namespace

cudaError_t launch_sigma_to_f32(int n, int M, const double *S, float *S32, cudaStream_t s) {
  const int ld = (n + 31) / 32 * 32;
  sigma_to_f32_kernel<<<1024, 256, 0, s>>>(n, (long)M * n, ld, S, S32);
  return cudaGetLastError();
}

cudaError_t c1sys_fill(C1Sys *d, int n, int M, int splits, const float *ws, const float *S32,
                       const double *dHF, const int4 *coef32, double *I1, double *part) {
  d->g = tc_geom(n, M);
  const long stack = (long)M * n * d->g.ld;
  d->JB = 4096 / n > 1 ? 4096 / n : 1;
  d->S = splits;
  d->RT = (int)(((long)M * n + 127) / 128);
  d->S32 = S32;
  d->dHF = dHF;
  d->coef32 = coef32;
  d->I1 = I1;
  d->part = part;
  for (int t = 0; t < 2; ++t) {
    cudaError_t e = make_tmap_rows(&d->th[t], ws + stack, n, M, d->g.ld, d->g.nsz[t], 16);
    if (e == cudaSuccess)
      e = make_tmap_rows(&d->tl[t], ws + 2 * stack, n, M, d->g.ld, d->g.nsz[t], 16);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_diag_f32(int n, int M, const double *dHF, const double *Sigma,
                            const double *wm, const double *wp, float *S32, cudaStream_t s) {
  const int ld = (n + 31) / 32 * 32;
  diag_f32_kernel<<<1024, 256, 0, s>>>(n, M, ld, dHF, Sigma, wm, wp,
                                       S32 + (long)M * n * ld);
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

// Shared memory of the convolution kernel: operand stages (as many as fit,
// at most kMaxStages) and the barriers.
static int conv1_stages(int Np_max) {
  const size_t stage = 2 * (size_t)kTileA + 2 * (size_t)Np_max * 64;
  const size_t fixed = 1024 + 256;
  int ns = (int)((232448 - fixed) / stage);
  return ns > kMaxStages ? kMaxStages : ns;
}

static size_t conv1_smem_bytes(int Np_max, int nstage) {
  return 1024 + (size_t)nstage * (2 * (size_t)kTileA + 2 * (size_t)Np_max * 64) + 256;
}

cudaError_t conv1_tc_launch(const C1Sys *sys, const long *prefix, int n_sys, long items,
                            int Np_max, int *err, int num_sms, cudaStream_t s) {
  const int nstage = conv1_stages(Np_max);
  if (nstage < 2) return cudaErrorInvalidValue;
  const size_t smem = conv1_smem_bytes(Np_max, nstage);
  cudaError_t e = cudaFuncSetAttribute(conv1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(items < num_sms ? items : num_sms);
  const int nbuf = (Np_max <= 256) ? 2 : 1;
  conv1_tc_kernel<<<grid, kThreads, smem, s>>>(sys, prefix, n_sys, items, Np_max, nstage, nbuf,
                                               err);
  return cudaGetLastError();
}

}  // namespace fedvr
