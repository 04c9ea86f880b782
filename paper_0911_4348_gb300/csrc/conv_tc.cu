// First Dyson convolution on the tensor cores (Sec. 2.3, Eq. deq), split TF32:
//
//   I1_i = sum_j B_ij g_j,  B_ij = c1 Sigma_k + c2 Sigma_{k+1}   (j != i)
//                           B_ii = dHF - wm_i Sigma_0 + wp_i Sigma_{M-1}
//
// with the lag bracket k and the trapezoid/interpolation weights c1, c2 of the
// FP64 path (FP64 tables, applied here in FP32). One tile = one output mesh
// point i and 128 rows a; all columns b sit in one or two N tiles. The
// contraction runs over (j, c) in 32-wide chunks: the A operand B_ij(a, c) is
// formed by the CUDA cores and split as hi + lo (TF32); B = g_j(b, c) comes
// from the split copy of g. Products hi*hi + hi*lo + lo*hi accumulate in FP32 in
// TMEM over a block of mesh points (about 4096 contraction terms) and each block
// is then added into the FP64 result, so rounding does not grow with M.
#include "common.cuh"
#include "tc.cuh"
#include "tc_sys.cuh"

namespace fedvr {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kTileA = 128 * 128;
constexpr int kWarps = 14;  // 0-3 flush, 4-11 A producers, 12 TMA, 13 MMA
constexpr int kThreads = kWarps * 32;

// Work queue: the (i, M-tile) items of every system in the table, each a
// sequence of accumulator blocks of JB mesh points j, each block a sequence
// of 32-wide chunks c. Roles as in the exchange kernel.
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
  int cur = 0;

  if (warp >= 4 && warp < 12) {
    // ---- A producers: B_ij(a, c) = c1 Sigma_k1(a, c) + c2 Sigma_k2(a, c) (+ dHF on j = i) ----
    const int pt = tid - 128, c = pt & 7, r0 = pt >> 3;
    uint32_t cc = 0;
    for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      const int n = S.g.n, ld = S.g.ld, M = S.g.M, MT = S.g.MT;
      const long nld = (long)n * ld;
      const long q = w - prefix[cur];
      const int i = (int)(q / MT), mt = (int)(q % MT);
      for (int j = 0; j < M && !*abort_flag; ++j) {
        const ConvCoef cf = S.coef[(long)i * M + j];
        const int k1 = cf.k, k2 = cf.diag ? (M - 1) : (cf.k + 1);
        const float c1 = (float)cf.c1, c2 = (float)cf.c2;
        const float *S1 = S.S32 + (long)k1 * nld, *S2 = S.S32 + (long)k2 * nld;
        for (int kc = 0; kc < S.g.KC; ++kc, ++cc) {
          const int l0 = kc * 32;
          float4 s1[4], s2[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int a = mt * 128 + r0 + 32 * k;
            if (a < n) {
              s1[k] = *reinterpret_cast<const float4 *>(S1 + (long)a * ld + l0 + 4 * c);
              s2[k] = *reinterpret_cast<const float4 *>(S2 + (long)a * ld + l0 + 4 * c);
            } else {
              s1[k] = s2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
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
            const int a = mt * 128 + r0 + 32 * k;
            float x[4] = {fmaf(c1, s1[k].x, c2 * s2[k].x), fmaf(c1, s1[k].y, c2 * s2[k].y),
                          fmaf(c1, s1[k].z, c2 * s2[k].z), fmaf(c1, s1[k].w, c2 * s2[k].w)};
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const int l = l0 + 4 * c + qq;
              if (l >= n || a >= n) x[qq] = 0.f;
              else if (cf.diag) x[qq] += (float)S.dHF[(long)a * n + l];
            }
            const float4 hi = make_float4(tc::tf32_rna(x[0]), tc::tf32_rna(x[1]),
                                          tc::tf32_rna(x[2]), tc::tf32_rna(x[3]));
            const float4 lo = make_float4(tc::tf32_rna(x[0] - hi.x), tc::tf32_rna(x[1] - hi.y),
                                          tc::tf32_rna(x[2] - hi.z), tc::tf32_rna(x[3] - hi.w));
            const uint32_t off = tc::sw128_offset(r0 + 32 * k, c);
            *reinterpret_cast<float4 *>(st + off) = hi;
            *reinterpret_cast<float4 *>(st + kTileA + off) = lo;
          }
          tc::fence_smem_to_async();
          tc::mbar_arrive(&full[s]);
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
        const uint32_t bytes = 2u * (uint32_t)S.g.Np * 128u;
        for (int j = 0; j < S.g.M && !*abort_flag; ++j) {
          for (int kc = 0; kc < S.g.KC; ++kc, ++cc) {
            const int s = cc & 1;
            const uint32_t use = cc >> 1;
            if (use > 0 && !tc::mbar_wait(&empty[s], (use - 1) & 1, kWaitNs)) {
              *abort_flag = 1;
              break;
            }
            uint8_t *st = smem + s * stage_bytes + 2 * kTileA;
            tc::mbar_arrive_expect_tx(&full[s], bytes);
            for (int nt = 0; nt < S.g.NT; ++nt) {
              tc::tma_load_3d(st + S.g.n0[nt] * 128, &S.th[nt], kc * 32, S.g.n0[nt], j, &full[s]);
              tc::tma_load_3d(st + tileB + S.g.n0[nt] * 128, &S.tl[nt], kc * 32, S.g.n0[nt], j,
                              &full[s]);
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
        const int n = S.g.n, M = S.g.M;
        for (int j0 = 0; j0 < M && !*abort_flag; j0 += S.JB, ++tcount) {
          const int j1 = min(M, j0 + S.JB);
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
            for (int kc = 0; kc < S.g.KC; ++kc, ++cc) {
              const int s = cc & 1;
              const uint32_t use = cc >> 1;
              if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
                *abort_flag = 1;
                break;
              }
              tc::fence_after_sync();
              const uint32_t sa = tc::smem_u32(smem + s * stage_bytes);
              const int ksteps = min(4, (n - kc * 32 + 7) / 8);
              const bool fresh = (j == j0 && kc == 0);
              for (int kk = 0; kk < ksteps; ++kk) {
                const uint64_t ah = tc::sdesc_k128(sa + kk * 32);
                const uint64_t al = tc::sdesc_k128(sa + kTileA + kk * 32);
                for (int nt = 0; nt < S.g.NT; ++nt) {
                  const uint32_t boff = 2 * kTileA + (uint32_t)S.g.n0[nt] * 128 + kk * 32;
                  const uint64_t bh = tc::sdesc_k128(sa + boff);
                  const uint64_t bl = tc::sdesc_k128(sa + boff + tileB);
                  const uint32_t d = dbase + (uint32_t)S.g.n0[nt];
                  const uint32_t idesc = tc::idesc_tf32(128, S.g.nsz[nt]);
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
    // ---- flush: add each FP32 block into the FP64 result ----
    uint32_t tcount = 0;
    for (long w = blockIdx.x; w < items && !*abort_flag; w += gridDim.x) {
      while (cur + 1 < n_sys && w >= prefix[cur + 1]) ++cur;
      const C1Sys &S = sys[cur];
      const int n = S.g.n, M = S.g.M, MT = S.g.MT;
      const long q = w - prefix[cur];
      const int i = (int)(q / MT), mt = (int)(q % MT);
      const int a = mt * 128 + warp * 32 + lane;
      const bool live = a < n;
      double *row = S.I1 + ((long)i * n + (live ? a : 0)) * n;
      for (int j0 = 0; j0 < M; j0 += S.JB, ++tcount) {
        const int buf = tcount & 1;
        const uint32_t tu = tcount >> 1;
        if (!tc::mbar_wait(&accf[buf], tu & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t tbase = tmem + (nbuf == 2 ? (uint32_t)(buf * 256) : 0u);
        for (int c0 = 0; c0 < n; c0 += 16) {
          float v[16];
          tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
          if (live) {
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const int b = c0 + t;
              if (b < n) row[b] = (j0 == 0) ? (double)v[t] : row[b] + (double)v[t];
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

cudaError_t c1sys_fill(C1Sys *d, int n, int M, const float *ws, const float *S32,
                       const double *dHF, const ConvCoef *coef, double *I1) {
  d->g = tc_geom(n, M);
  const long stack = (long)M * n * d->g.ld;
  d->JB = 4096 / n > 1 ? 4096 / n : 1;
  d->S32 = S32;
  d->dHF = dHF;
  d->coef = coef;
  d->I1 = I1;
  for (int t = 0; t < 2; ++t) {
    cudaError_t e = make_tmap_rows(&d->th[t], ws + stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e == cudaSuccess) e = make_tmap_rows(&d->tl[t], ws + 2 * stack, n, M, d->g.ld, d->g.nsz[t]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t conv1_tc_launch(const C1Sys *sys, const long *prefix, int n_sys, long items,
                            int Np_max, int *err, int num_sms, cudaStream_t s) {
  const size_t smem = tc_smem_bytes(Np_max, 0, false);
  cudaError_t e = cudaFuncSetAttribute(conv1_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)(items < num_sms ? items : num_sms);
  const int nbuf = (Np_max <= 256) ? 2 : 1;
  conv1_tc_kernel<<<grid, kThreads, smem, s>>>(sys, prefix, n_sys, items, Np_max, nbuf, err);
  return cudaGetLastError();
}

}  // namespace fedvr
