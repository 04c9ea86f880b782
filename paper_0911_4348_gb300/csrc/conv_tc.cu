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
constexpr uint32_t kTileA = 128 * 64;       // 128 rows x 16 floats (64-byte swizzled)
constexpr int kRaw = 3;                      // raw source chunks in flight per producer
constexpr uint32_t kRawSlot = 2 * 128 * 64;  // both bracket rows of 128 rows x 16 floats
constexpr int kMaxStages = 6;
constexpr int kWarps = 14;  // 0-3 flush, 4-11 A producers, 12 TMA, 13 MMA
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

// Walk over the (item, j, chunk) sequence of one CTA for the two rows r0 and
// r0 + 64 of each tile that a producer thread owns.
struct ProdCur {
  long w;
  int cur, n, M, ld, KC, j, j_hi, kc;
  int i[2], a[2];
  bool live[2], done;
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
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const long r = (long)it.t * 128 + r0 + 64 * k;
        p.live[k] = r < R;
        p.i[k] = p.live[k] ? (int)(r / p.n) : 0;
        p.a[k] = p.live[k] ? (int)(r % p.n) : 0;
      }
      return;
    }
    p.w += gridDim.x;
  }
  p.done = true;
}

// Advance by one chunk; returns true when the mesh point (or item) changed.
__device__ __forceinline__ bool pc_next(ProdCur &p, const C1Sys *sys, const long *prefix,
                                        int n_sys, long items, int r0) {
  if (++p.kc < p.KC) return false;
  p.kc = 0;
  if (++p.j < p.j_hi) return true;
  p.w += gridDim.x;
  pc_item(p, sys, prefix, n_sys, items, r0);
  return true;
}

__global__ void __launch_bounds__(kThreads, 1)
    conv1_tc_kernel(const C1Sys *__restrict__ sys, const long *__restrict__ prefix, int n_sys,
                    long items, int Np_max, int nstage, int nbuf, int *err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const uint32_t tileB = (uint32_t)Np_max * 64;
  const uint32_t stage_bytes = 2 * kTileA + 2 * tileB;
  uint8_t *raw = smem + nstage * stage_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(raw + kRaw * kRawSlot);
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
      tc::mbar_init(&full[s], 257);
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
    // ---- A producers: rows r0 and r0 + 64 of the tile, 16-byte chunk c of each
    // 16-wide slice. The bracket rows Sigma_k1, Sigma_k2 of the next kRaw
    // chunks stream into a per-thread ring by cp.async; each thread reads back
    // only what it copied, so no barrier guards the ring. ----
    const int pt = tid - 128, c = pt & 3, r0 = pt >> 2;
    const uint32_t offA[2] = {tc::sw64_offset(r0, c), tc::sw64_offset(r0 + 64, c)};
    uint32_t rofs[2][2];  // ring byte offsets: [bracket row][row k]
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      rofs[0][k] = (uint32_t)((r0 + 64 * k) * 64 + c * 16);
      rofs[1][k] = (uint32_t)((128 + r0 + 64 * k) * 64 + c * 16);
    }
    ProdCur ip{}, cp{};
    ip.w = cp.w = blockIdx.x;
    ip.done = cp.done = false;
    pc_item(ip, sys, prefix, n_sys, items, r0);
    pc_item(cp, sys, prefix, n_sys, items, r0);
    uint32_t o1[2] = {0, 0}, o2[2] = {0, 0};  // issue side: element offsets into S32
    float c1[2] = {0.f, 0.f}, c2[2] = {0.f, 0.f};
    bool dg[2] = {false, false};
    const float *iS32 = nullptr;
    const double *dHF = nullptr;
    auto issue_coefs = [&]() {
      const C1Sys &S = sys[ip.cur];
      iS32 = S.S32;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const ConvCoef cf = S.coef[(long)ip.i[k] * ip.M + ip.j];
        const int k1 = cf.k, k2 = cf.diag ? (ip.M - 1) : (cf.k + 1);
        o1[k] = (uint32_t)((k1 * ip.n + ip.a[k]) * ip.ld + 4 * c);
        o2[k] = (uint32_t)((k2 * ip.n + ip.a[k]) * ip.ld + 4 * c);
      }
    };
    auto consume_coefs = [&]() {
      const C1Sys &S = sys[cp.cur];
      dHF = S.dHF;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const ConvCoef cf = S.coef[(long)cp.i[k] * cp.M + cp.j];
        c1[k] = (float)cf.c1;
        c2[k] = (float)cf.c2;
        dg[k] = cp.live[k] && cf.diag;
      }
    };
    auto issue = [&](int slot) {
      uint8_t *rs = raw + slot * kRawSlot;
      const int l0 = ip.kc * 16;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t b = ip.live[k] ? 16u : 0u;
        tc::cp_async16(rs + rofs[0][k], iS32 + o1[k] + l0, b);
        tc::cp_async16(rs + rofs[1][k], iS32 + o2[k] + l0, b);
      }
    };
    if (!ip.done) issue_coefs();
    if (!cp.done) consume_coefs();
    for (int q = 0; q < kRaw; ++q) {
      if (!ip.done) {
        issue(q);
        if (pc_next(ip, sys, prefix, n_sys, items, r0) && !ip.done) issue_coefs();
      }
      tc::cp_async_commit();
    }
    int slot = 0, st = 0;
    uint32_t u = 0;
    while (!cp.done && !*abort_flag) {
      tc::cp_async_wait<kRaw - 1>();
      const uint8_t *rs = raw + slot * kRawSlot;
      float x[2][4];
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float4 s1 = *reinterpret_cast<const float4 *>(rs + rofs[0][k]);
        const float4 s2 = *reinterpret_cast<const float4 *>(rs + rofs[1][k]);
        x[k][0] = fmaf(c1[k], s1.x, c2[k] * s2.x);
        x[k][1] = fmaf(c1[k], s1.y, c2[k] * s2.y);
        x[k][2] = fmaf(c1[k], s1.z, c2[k] * s2.z);
        x[k][3] = fmaf(c1[k], s1.w, c2[k] * s2.w);
        if (dg[k]) {  // B_ii carries the HF self-energy change
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const int l = cp.kc * 16 + 4 * c + qq;
            if (l < cp.n) x[k][qq] += (float)dHF[(long)cp.a[k] * cp.n + l];
          }
        }
      }
      if (u > 0 && !tc::mbar_wait(&empty[st], (u - 1) & 1, kWaitNs)) {
        *abort_flag = 1;
        break;
      }
      uint8_t *sa = smem + st * stage_bytes;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float4 hi = make_float4(tc::tf32_rna(x[k][0]), tc::tf32_rna(x[k][1]),
                                      tc::tf32_rna(x[k][2]), tc::tf32_rna(x[k][3]));
        const float4 lo =
            make_float4(tc::tf32_rna(x[k][0] - hi.x), tc::tf32_rna(x[k][1] - hi.y),
                        tc::tf32_rna(x[k][2] - hi.z), tc::tf32_rna(x[k][3] - hi.w));
        *reinterpret_cast<float4 *>(sa + offA[k]) = hi;
        *reinterpret_cast<float4 *>(sa + kTileA + offA[k]) = lo;
      }
      tc::fence_smem_to_async();
      tc::mbar_arrive(&full[st]);
      // refill the ring slot just read with the chunk kRaw ahead
      if (!ip.done) {
        issue(slot);
        if (pc_next(ip, sys, prefix, n_sys, items, r0) && !ip.done) issue_coefs();
      }
      tc::cp_async_commit();
      slot = (slot + 1 == kRaw) ? 0 : slot + 1;
      if (++st == nstage) {
        st = 0;
        ++u;
      }
      if (pc_next(cp, sys, prefix, n_sys, items, r0) && !cp.done) consume_coefs();
    }
    tc::cp_async_wait<0>();
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
                       const double *dHF, const ConvCoef *coef, double *I1, double *part) {
  d->g = tc_geom(n, M);
  const long stack = (long)M * n * d->g.ld;
  d->JB = 4096 / n > 1 ? 4096 / n : 1;
  d->S = splits;
  d->RT = (int)(((long)M * n + 127) / 128);
  d->S32 = S32;
  d->dHF = dHF;
  d->coef = coef;
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

cudaError_t conv1_sum_splits(long count, int nparts, const double *part, double *I1,
                             cudaStream_t s) {
  if (nparts < 1) return cudaSuccess;
  conv1_sum_splits_kernel<<<1024, 256, 0, s>>>(count, nparts, part, I1);
  return cudaGetLastError();
}

// Shared memory of the convolution kernel: operand stages (as many as fit,
// at most kMaxStages), the raw-source ring and the barriers.
static int conv1_stages(int Np_max) {
  const size_t stage = 2 * (size_t)kTileA + 2 * (size_t)Np_max * 64;
  const size_t fixed = 1024 + (size_t)kRaw * kRawSlot + 256;
  int ns = (int)((232448 - fixed) / stage);
  return ns > kMaxStages ? kMaxStages : ns;
}

static size_t conv1_smem_bytes(int Np_max, int nstage) {
  return 1024 + (size_t)nstage * (2 * (size_t)kTileA + 2 * (size_t)Np_max * 64) +
         (size_t)kRaw * kRawSlot + 256;
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
