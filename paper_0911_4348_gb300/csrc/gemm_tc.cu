// Plain dense products of the split-precision iteration on the tensor cores:
// the direct term's V Q V (Sec. 2.3, Eq. sigma2ndb) and the three products of
// the second convolution (Sec. 2.3, Eq. deq, with the left index in the HF
// eigenbasis). Split TF32 as in the other tensor-core kernels:
//
//   O[row][col] = sum_k A(row, k) B(col, k),   x = hi + lo,
//   hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM
//
// (per-product relative error about 2^-21, the level of the FP32 CUDA-core
// products these launches replace).
//
// Rows are stacked: row r = (g, w) with g = r / G and w = r % G. The A operand
// is read either along the rows ("MC": A[g a_sg + w + k a_sk], consecutive
// rows contiguous) or along k ("KC": A[g a_sg + w a_sw + k]); with MUL2 (MC
// only) each element is multiplied by the one of the mirrored group nG-1-g.
// B is read along columns ("MC": B[k b_s + col]) or along k ("KC":
// B[col b_s + k]). The output is O[g o_sg + w + col o_sc]: the 32 lanes of an
// epilogue warp hold 32 consecutive rows, so its stores run along w. A batch
// index (blockIdx.z) adds a_sz, b_sz and o_sz. Element offsets fit in 32 bits
// (checked on the host).
//
// Optional contraction slices: with nkz > 1 the K range is cut into slices of
// kz values (a multiple of 32), blockIdx.z = batch * nkz + slice, and slice k
// writes its partial product at O + k o_kz (the caller adds the slices). With
// k_tri > 0 a tile stops its contraction at (g_max + 1) k_tri, g_max the
// largest group among its rows (a block-triangular B: the rows of group g need
// k < (g + 1) k_tri); a tile whose slice lies beyond that writes zeros.
//
// Producers take one row of A and 16 consecutive k per thread; in MC mode the 32
// lanes of a warp hold 32 consecutive rows, so every load instruction is
// coalesced along the rows.
//
// One CTA per 128 x Nt output tile (Nt <= 256, a multiple of 16): warps 0-3
// drain TMEM, warps 4-11 load, convert, split and store both operands of a
// 32-wide k chunk into the K-major 128-byte-swizzled stage layout, warp 12
// issues the MMAs. Two stages handed over with mbarriers (full: one arrival per
// producer warp; empty: MMA commit); every wait is bounded and a timeout sets
// the error flag.
#include <type_traits>

#include "common.cuh"
#include "tc.cuh"
#include "tc_sys.cuh"

namespace fedvr {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;
constexpr int kWarps = 13;  // 0-3 epilogue, 4-11 producers, 12 MMA
constexpr int kThreads = kWarps * 32;
constexpr uint32_t kTileA = 128 * 128;  // one 128-row x 32-value FP32 operand copy

struct GemmArgs {
  int R, N, K, G, nG, Nt, tcols;  // tcols: TMEM columns (power of 2 >= Nt)
  const void *A, *A2;
  int a_sg, a_sw, a_sk, a_sz;
  const void *B;
  int b_s, b_sz;
  void *O;
  int o_sg, o_sc, o_sz;
  int *err;
  int kz, nkz, k_tri;  // contraction slices and block-triangular limit (see above)
  long o_kz;
  int vec;  // FP32 operands read along k with 16-byte loads (alignment checked on the host)
};

// Split x and store the pair at element (r, k) of a 128B-swizzled K-major tile
// (lo at byte offset lo_off from hi).
__device__ __forceinline__ void put1(uint8_t *t, uint32_t lo_off, int r, int k, float x) {
  float hi, lo;
  tc::tf32_split(x, hi, lo);
  const uint32_t off = tc::sw128_offset(r, k >> 2) + (uint32_t)(k & 3) * 4u;
  *reinterpret_cast<float *>(t + off) = hi;
  *reinterpret_cast<float *>(t + lo_off + off) = lo;
}

// Four consecutive k values from row offset off of an FP32 operand (zeros
// beyond kend or for a dead row); 16-byte load when all four lie before kend.
__device__ __forceinline__ float4 ld4(const float *X, long off, int k, int kend, bool live) {
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (!live) return v;
  if (k + 4 <= kend) return *reinterpret_cast<const float4 *>(X + off + k);
  if (k < kend) v.x = X[off + k];
  if (k + 1 < kend) v.y = X[off + k + 1];
  if (k + 2 < kend) v.z = X[off + k + 2];
  if (k + 3 < kend) v.w = X[off + k + 3];
  return v;
}

// Split four consecutive k values (k0 a multiple of 4) of row r and store them
// as one 16-byte unit.
__device__ __forceinline__ void put4(uint8_t *t, uint32_t lo_off, int r, int k0, const float *x) {
  float4 hi, lo;
  tc::tf32_split(x[0], hi.x, lo.x);
  tc::tf32_split(x[1], hi.y, lo.y);
  tc::tf32_split(x[2], hi.z, lo.z);
  tc::tf32_split(x[3], hi.w, lo.w);
  const uint32_t off = tc::sw128_offset(r, k0 >> 2);
  *reinterpret_cast<float4 *>(t + off) = hi;
  *reinterpret_cast<float4 *>(t + lo_off + off) = lo;
}

template <typename TA, typename TB, typename TO, bool A_MC, bool B_MC, bool MUL2>
__global__ void __launch_bounds__(kThreads, 1) gemm_tf32x3_kernel(GemmArgs p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
  const int Nt = p.Nt;
  const uint32_t tileB = (uint32_t)Nt * 128;
  const uint32_t stage_bytes = 2 * kTileA + 2 * tileB;
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * stage_bytes);
  uint64_t *full = bars, *empty = bars + 2, *accf = bars + 4, *drain = bars + 5;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 6);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * 128, col0 = blockIdx.y * Nt;
  const int z = blockIdx.z / p.nkz, zk = blockIdx.z % p.nkz;
  const int kbeg = zk * p.kz;
  int kend = min(p.K, kbeg + p.kz);
  if (p.k_tri > 0) kend = min(kend, (min(p.R - 1, row0 + 127) / p.G + 1) * p.k_tri);
  const int KC = kend > kbeg ? (kend - kbeg + 31) / 32 : 0;

  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, (uint32_t)p.tcols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&full[0], 8);  // one arrival per producer warp
    tc::mbar_init(&full[1], 8);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    tc::mbar_init(accf, 1);
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  bool issued = false;

  if (warp >= 4 && warp < 12) {
    bool vec_done = false;
    if constexpr (!A_MC && !B_MC && std::is_same<TA, float>::value &&
                  std::is_same<TB, float>::value) {
      if (p.vec) {
        // ---- producers, FP32 operands along k: a 32-value chunk row is 8 float4, eight
        // lanes cover one 128-byte row segment (A: 4 float4 per thread, B: up to 8) ----
        vec_done = true;
        const int pt = tid - 128;
        const float *A = reinterpret_cast<const float *>(p.A) + (long)z * p.a_sz;
        const float *B = reinterpret_cast<const float *>(p.B) + (long)z * p.b_sz;
        long aoff4[4], boff4[8];
        bool alive4[4], blive4[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = row0 + ((pt + 256 * q) >> 3);
          alive4[q] = r < p.R;
          aoff4[q] = alive4[q] ? (long)(r / p.G) * p.a_sg + (long)(r % p.G) * p.a_sw : 0;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int c = (pt + 256 * q) >> 3;
          blive4[q] = c < Nt && col0 + c < p.N;
          boff4[q] = blive4[q] ? (long)(col0 + c) * p.b_s : 0;
        }
        const int c4 = (pt & 7) * 4;
        for (int kc = 0; kc < KC; ++kc) {
          const int k = kbeg + kc * 32 + c4;
          float4 av[4], bv[8];
#pragma unroll
          for (int q = 0; q < 4; ++q) av[q] = ld4(A, aoff4[q], k, kend, alive4[q]);
#pragma unroll
          for (int q = 0; q < 8; ++q) bv[q] = ld4(B, boff4[q], k, kend, blive4[q]);
          const int s = kc & 1;
          const uint32_t use = kc >> 1;
          if (use > 0 && !tc::warp_wait(&empty[s], (use - 1) & 1, kWaitNs)) {
            *abort_flag = 1;
            break;
          }
          uint8_t *st = smem + s * stage_bytes;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            put4(st, kTileA, (pt + 256 * q) >> 3, c4, reinterpret_cast<const float *>(&av[q]));
          uint8_t *sb = st + 2 * kTileA;
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int c = (pt + 256 * q) >> 3;
            if (c < Nt) put4(sb, tileB, c, c4, reinterpret_cast<const float *>(&bv[q]));
          }
          tc::fence_smem_to_async();
          tc::warp_arrive(&full[s]);
        }
      }
    }
    if (!vec_done) {
      // ---- producers ----
      const int pt = tid - 128;
      const TA *A = reinterpret_cast<const TA *>(p.A) + (long)z * p.a_sz;
      const TA *A2 = reinterpret_cast<const TA *>(p.A2);
      const TB *B = reinterpret_cast<const TB *>(p.B) + (long)z * p.b_sz;
      // A: one row and 16 consecutive k per thread. MC: warp w takes rows
      // (w & 3) * 32 + lane and k half w >> 2, so each load instruction reads 32
      // consecutive rows at one k (rows are contiguous in MC); KC: row pt / 2, k half
      // pt & 1 (k is contiguous in KC)
      const int wp = pt >> 5;
      const int ra = A_MC ? (wp & 3) * 32 + lane : (pt >> 1);
      const int kh = A_MC ? (wp >> 2) * 16 : (pt & 1) * 16;
      int aoff0 = 0, aoff20 = 0;
      bool alive0;
      {
        const int r = row0 + ra;
        const int g = r / p.G, w = r % p.G;
        alive0 = r < p.R;
        if (alive0) {
          aoff0 = g * p.a_sg + w * (A_MC ? 1 : p.a_sw);
          if (MUL2) aoff20 = (p.nG - 1 - g) * p.a_sg + w;
        }
      }
      // B columns of this thread: MC 32 consecutive local columns (one k per lane),
      // KC one local column
      const int cb = B_MC ? (pt >> 5) * 32 : pt;
      for (int kc = 0; kc < KC; ++kc) {
        const int k0 = kbeg + kc * 32;
        float av[16], bv[32];
        if (A_MC) {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int k = k0 + kh + i;
            float x = 0.f;
            if (alive0 && k < kend) {
              x = (float)A[aoff0 + k * p.a_sk];
              if (MUL2) x *= (float)A2[aoff20 + k * p.a_sk];
            }
            av[i] = x;
          }
        } else {
          const int kb = k0 + kh;
#pragma unroll
          for (int i = 0; i < 16; ++i)
            av[i] = (alive0 && kb + i < kend) ? (float)A[aoff0 + kb + i] : 0.f;
        }
        if (B_MC) {
          const int k = k0 + lane;
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int c = col0 + cb + i;
            bv[i] = (cb + i < Nt && c < p.N && k < kend) ? (float)B[k * p.b_s + c] : 0.f;
          }
        } else {
          const int c = col0 + cb;
          const bool ok = cb < Nt && c < p.N;
#pragma unroll
          for (int i = 0; i < 32; ++i)
            bv[i] = (ok && k0 + i < kend) ? (float)B[c * p.b_s + k0 + i] : 0.f;
        }
        const int s = kc & 1;
        const uint32_t use = kc >> 1;
        if (use > 0 && !tc::warp_wait(&empty[s], (use - 1) & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        uint8_t *st = smem + s * stage_bytes;
#pragma unroll
        for (int q = 0; q < 4; ++q) put4(st, kTileA, ra, kh + 4 * q, av + 4 * q);
        uint8_t *sb = st + 2 * kTileA;
        if (B_MC) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (cb + i < Nt) put1(sb, tileB, cb + i, lane, bv[i]);
        } else if (cb < Nt) {
#pragma unroll
          for (int q = 0; q < 8; ++q) put4(sb, tileB, cb, 4 * q, bv + 4 * q);
        }
        tc::fence_smem_to_async();
        tc::warp_arrive(&full[s]);
      }
    }
  } else if (warp == 12) {
    // ---- MMA issue (kind::tf32, K = 8 per instruction) ----
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, Nt);
      for (int kc = 0; kc < KC; ++kc) {
        const int s = kc & 1;
        const uint32_t use = kc >> 1;
        if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
          *abort_flag = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t sa = tc::smem_u32(smem + s * stage_bytes);
        const int ksteps = min(4, (kend - kbeg - kc * 32 + 7) / 8);
        for (int kk = 0; kk < ksteps; ++kk) {
          const uint64_t ah = tc::sdesc_k128(sa + kk * 32);
          const uint64_t al = tc::sdesc_k128(sa + kTileA + kk * 32);
          const uint64_t bh = tc::sdesc_k128(sa + 2 * kTileA + kk * 32);
          const uint64_t bl = tc::sdesc_k128(sa + 2 * kTileA + tileB + kk * 32);
          tc::mma_tf32(tmem, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
          tc::mma_tf32(tmem, ah, bl, idesc, 1u);
          tc::mma_tf32(tmem, al, bh, idesc, 1u);
        }
        tc::mma_commit(&empty[s]);
        issued = true;
      }
      if (issued) tc::mma_commit(accf);
    }
  } else {
    // ---- epilogue: TMEM lane = tile row, 16 columns per load ----
    if (KC == 0) {
      // empty contraction slice: zeros, no MMA to wait for
      const int r = row0 + warp * 32 + lane;
      if (r < p.R) {
        const long ooff = (long)zk * p.o_kz + (long)z * p.o_sz + (long)(r / p.G) * p.o_sg + (r % p.G);
        TO *O = reinterpret_cast<TO *>(p.O);
        for (int c = 0; c < Nt && col0 + c < p.N; ++c) O[ooff + (long)(col0 + c) * p.o_sc] = (TO)0;
      }
    } else if (tc::warp_wait(accf, 0, kWaitNs)) {
      tc::fence_after_sync();
      const int r = row0 + warp * 32 + lane;
      const bool live = r < p.R;
      const long ooff =
          live ? (long)zk * p.o_kz + (long)z * p.o_sz + (long)(r / p.G) * p.o_sg + (r % p.G) : 0;
      TO *O = reinterpret_cast<TO *>(p.O);
      for (int c0 = 0; c0 < Nt; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        if (live) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const int c = col0 + c0 + t;
            if (c0 + t < Nt && c < p.N) O[ooff + (long)c * p.o_sc] = (TO)v[t];
          }
        }
      }
    } else {
      *abort_flag = 1;
    }
  }

  tc::fence_before_sync();
  __syncthreads();
  if (*abort_flag) {
    // let MMAs still in flight finish (bounded) before the TMEM goes away
    if (warp == 12 && lane == 0) {
      if (issued) tc::mma_commit(drain);
      atomicExch(p.err, 1);
      if (issued) tc::mbar_wait(drain, 0, kWaitNs);
    }
    __syncthreads();
  }
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, (uint32_t)p.tcols);
}

template <typename TA, typename TB, typename TO, bool A_MC, bool B_MC, bool MUL2>
cudaError_t gemm_tf32x3(GemmArgs p, int batch, cudaStream_t s) {
  if (p.R <= 0 || p.N <= 0 || p.K <= 0) return cudaSuccess;
  if (p.N > 4096 || p.G <= 0) return cudaErrorInvalidValue;
  if (p.nkz <= 1) {
    p.nkz = 1;
    p.kz = p.K;
  } else if (p.kz <= 0 || p.kz % 32 != 0) {
    return cudaErrorInvalidValue;
  }
  const int ntile = (p.N + 255) / 256;
  p.Nt = ((p.N + ntile - 1) / ntile + 15) / 16 * 16;
  p.vec = 0;
  if (!A_MC && !B_MC && std::is_same<TA, float>::value && std::is_same<TB, float>::value) {
    const bool al = reinterpret_cast<uintptr_t>(p.A) % 16 == 0 &&
                    reinterpret_cast<uintptr_t>(p.B) % 16 == 0;
    const bool st = p.a_sg % 4 == 0 && p.a_sw % 4 == 0 && p.a_sz % 4 == 0 && p.b_s % 4 == 0 &&
                    p.b_sz % 4 == 0 && (p.nkz == 1 || p.kz % 4 == 0);
    p.vec = (al && st) ? 1 : 0;
  }
  p.tcols = 32;
  while (p.tcols < p.Nt) p.tcols *= 2;
  const size_t smem = 2 * (2 * (size_t)kTileA + 2 * (size_t)p.Nt * 128) + 1024 + 128;
  // set on every call: the attribute belongs to the current device
  cudaError_t e = cudaFuncSetAttribute(gemm_tf32x3_kernel<TA, TB, TO, A_MC, B_MC, MUL2>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((p.R + 127) / 128), (unsigned)ntile, (unsigned)(batch * p.nkz));
  gemm_tf32x3_kernel<TA, TB, TO, A_MC, B_MC, MUL2><<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

GemmArgs args0(int R, int N, int K, int *err) {
  GemmArgs p{};
  p.R = R;
  p.N = N;
  p.K = K;
  p.G = R;
  p.nG = 1;
  p.err = err;
  p.nkz = 1;
  return p;
}

// Every element offset the kernels form stays below 2^31 when the largest stack
// they touch does.
bool fits32(long elems) { return elems < (1L << 31); }

}  // namespace

cudaError_t vqv_tc(int n, int M, int ld, const float *V32, const float *g32, float *VQ, float *W,
                   int *err, cudaStream_t s) {
  const long stack = (long)M * n * ld;
  if (!fits32(stack)) return cudaErrorInvalidValue;
  // VQ_j[a][c] = sum_k V[a][k] (g_j o g_{M-1-j})[k][c]: rows (j, c), columns a
  GemmArgs p = args0(M * n, n, n, err);
  p.G = n;
  p.nG = M;
  p.A = g32;
  p.A2 = g32;
  p.a_sg = n * ld;
  p.a_sk = ld;
  p.B = V32;
  p.b_s = ld;
  p.O = VQ;
  p.o_sg = n * ld;
  p.o_sc = ld;
  cudaError_t e = gemm_tf32x3<float, float, float, true, false, true>(p, 1, s);
  if (e != cudaSuccess) return e;
  // W_j = VQ_j V is symmetric: W_j[a][c] = sum_k VQ_j[c][k] V[a][k], rows (j, c), columns a
  GemmArgs q = args0(M * n, n, n, err);
  q.G = n;
  q.nG = M;
  q.A = VQ;
  q.a_sg = n * ld;
  q.a_sw = ld;
  q.B = V32;
  q.b_s = ld;
  q.O = W;
  q.o_sg = n * ld;
  q.o_sc = ld;
  return gemm_tf32x3<float, float, float, false, false, false>(q, 1, s);
}

cudaError_t kbe_rows_tc(int n, int ncols, int K, int Tn, int sh_ld, const float *Sh, long sh_z,
                        const float *Aop, int lda, long a_z, int nkz, bool tri, double *O,
                        long o_z, long o_kz, int *err, cudaStream_t s) {
  if (!fits32((long)Tn * sh_ld + sh_ld) || !fits32(sh_z) || !fits32(a_z) || !fits32(o_z) ||
      !fits32((long)2 * n * lda))
    return cudaErrorInvalidValue;
  // O[slice][z][j][p][a][c] = sum_k Sh_z[j n + c][k] Aop_z[p n + a][k]: rows (j, c) grouped by
  // j, columns (p, a); both operands read along k; batch z = 0, 1
  GemmArgs g = args0(ncols * n, 2 * n, K, err);
  g.G = n;
  g.nG = ncols;
  g.A = Sh;
  g.a_sg = n * sh_ld;
  g.a_sw = sh_ld;
  g.a_sz = (int)sh_z;
  g.B = Aop;
  g.b_s = lda;
  g.b_sz = (int)a_z;
  g.O = O;
  g.o_sg = 2 * n * n;
  g.o_sc = n;
  g.o_sz = (int)o_z;
  g.o_kz = o_kz;
  if (nkz > 1) {
    g.nkz = nkz;
    g.kz = ((K + nkz - 1) / nkz + 31) / 32 * 32;
    g.nkz = (K + g.kz - 1) / g.kz;
  }
  g.k_tri = tri ? 2 * n : 0;
  return gemm_tf32x3<float, float, double, false, false, false>(g, 2, s);
}

cudaError_t kbe_exchange_tc(int n, int ne, int xld, const float *Ap, const float *Bp, float *P,
                            int *err, cudaStream_t s) {
  const long n2 = (long)n * n;
  if (2 * n > 128 || n2 > 4096 || xld < 2 * n || !fits32(2 * n2 * n) || !fits32(n2 * xld))
    return cudaErrorInvalidValue;
  // P_e[(b, k)][(p, a)] = sum_{(q, l)} Ap_e[(p, a)][(q, l)] Bp_e[(b, k)][(q, l)]; operand rows
  // of pitch xld
  GemmArgs g = args0(2 * n, (int)n2, 2 * n, err);
  g.A = Ap;
  g.a_sw = xld;
  g.a_sz = (int)(2 * n * xld);
  g.B = Bp;
  g.b_s = xld;
  g.b_sz = (int)(n2 * xld);
  g.O = P;
  g.o_sc = 2 * n;
  g.o_sz = (int)(2 * n2 * n);
  return gemm_tf32x3<float, float, float, false, false, false>(g, ne, s);
}

cudaError_t conv2_tc(int n, int M, const float *K32, const double *C, const double *I1,
                     double *I2, float *t1, float *t2, int *err, cudaStream_t s) {
  const long nn = (long)n * n;
  if (!fits32((long)M * nn) || !fits32((long)n * M * M)) return cudaErrorInvalidValue;
  // X_j[a][b] = sum_k C[k][a] I1_j[k][b]: rows (j, b), columns a, into t2
  GemmArgs p = args0(M * n, n, n, err);
  p.G = n;
  p.nG = M;
  p.A = I1;
  p.a_sg = (int)nn;
  p.a_sk = n;
  p.B = C;
  p.b_s = n;
  p.O = t2;
  p.o_sg = (int)nn;
  p.o_sc = n;
  cudaError_t e = gemm_tf32x3<double, double, float, true, true, false>(p, 1, s);
  if (e != cudaSuccess) return e;
  // Y[i][a][b] = sum_j K_a[i][j] X[j][a][b]: per a, rows b, columns i, into t1
  GemmArgs q = args0(n, M, M, err);
  q.A = t2;
  q.a_sk = (int)nn;
  q.a_sz = n;
  q.B = K32;
  q.b_s = M;
  q.b_sz = M * M;
  q.O = t1;
  q.o_sc = (int)nn;
  q.o_sz = n;
  e = gemm_tf32x3<float, float, float, true, false, false>(q, n, s);
  if (e != cudaSuccess) return e;
  // I2_i[x][b] = sum_a C[x][a] Y[i][a][b]: rows (i, b), columns x
  GemmArgs r = args0(M * n, n, n, err);
  r.G = n;
  r.nG = M;
  r.A = t1;
  r.a_sg = (int)nn;
  r.a_sk = n;
  r.B = C;
  r.b_s = n;
  r.O = I2;
  r.o_sg = (int)nn;
  r.o_sc = n;
  return gemm_tf32x3<float, double, double, true, false, false>(r, 1, s);
}

}  // namespace fedvr
