// Second-Born self-energy in FE-DVR two-index form, FP64 path (Sec. 2.3,
// Eq. sigma2ndb): Sigma_j = sigma g o (V Q V) - X,  Q = g o gb,
// X_ab = sum_{k,l} V_ak V_bl g_al gb_lk g_kb, with g = G[j], gb = G[M-1-j].
//
// The exchange is evaluated column by column: for fixed b,
// P^(b) = g diag(V_b,:) gb (an n x n x n product with the contraction index l
// scaled by V_bl) and X_ab = sum_k V_ak g_kb P^(b)_ak, i.e. O(n^2) work per
// element (the paper's count). X is symmetric for symmetric g, gb, so only
// rows a >= b are formed and the result is mirrored.
#include "common.cuh"

#include <mutex>

namespace fedvr {
namespace {

__global__ void polarisation_kernel(int n, int M, const double *__restrict__ G,
                                    double *__restrict__ Q) {
  long nn = (long)n * n;
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * nn) return;
  long j = idx / nn, e = idx % nn;
  Q[idx] = G[idx] * G[(M - 1 - j) * nn + e];
}

constexpr int TA = 64, TK = 64, TL = 16;

// One block: mesh point j, column b, 64 rows a. Loops over 64-wide k blocks;
// P tile (a x k) accumulates over l with A = g(a, l) * V(b, l) and B = gb(l, k);
// the epilogue folds sum_k V_ak g_kb P_ak into per-row partial sums.
__global__ void __launch_bounds__(256) exchange_fp64_kernel(int n, int M, double spin,
                                                            const double *__restrict__ V,
                                                            const double *__restrict__ G,
                                                            const double *__restrict__ W,
                                                            double *__restrict__ Sigma) {
  const int j = blockIdx.z, b = blockIdx.y;
  const int a0 = blockIdx.x * TA;
  if (a0 + TA <= b) return;  // whole block above the diagonal
  const long nn = (long)n * n;
  const double *g = G + (long)j * nn;
  const double *gb = G + (long)(M - 1 - j) * nn;
  __shared__ double As[TL][TA + 1];
  __shared__ double Bs[TL][TK + 1];
  __shared__ double Vb[TL];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double xacc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k0 = 0; k0 < n; k0 += TK) {
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] = 0.0;
    for (int l0 = 0; l0 < n; l0 += TL) {
      if (threadIdx.x < TL) {
        int l = l0 + threadIdx.x;
        Vb[threadIdx.x] = (l < n) ? V[(long)b * n + l] : 0.0;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < TA * TL; e += 256) {
        int ll = e % TL, aa = e / TL;
        int a = a0 + aa, l = l0 + ll;
        As[ll][aa] = (a < n && l < n) ? g[(long)a * n + l] * Vb[ll] : 0.0;
      }
      for (int e = threadIdx.x; e < TK * TL; e += 256) {
        int kk = e % TK, ll = e / TK;
        int k = k0 + kk, l = l0 + ll;
        Bs[ll][kk] = (k < n && l < n) ? gb[(long)l * n + k] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int ll = 0; ll < TL; ++ll) {
        double av[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) av[i] = As[ll][ty + 16 * i];
#pragma unroll
        for (int q = 0; q < 4; ++q) bv[q] = Bs[ll][tx + 16 * q];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = fma(av[i], bv[q], acc[i][q]);
      }
      __syncthreads();
    }
    // epilogue for this k block: s_i = sum_q V[a_i][k_q] g[k_q][b] P[a_i][k_q]
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int a = a0 + ty + 16 * i;
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int k = k0 + tx + 16 * q;
        if (a < n && k < n) s = fma(V[(long)a * n + k] * g[(long)k * n + b], acc[i][q], s);
      }
      // reduce over the 16 lanes (tx) that share row a
      for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      xacc[i] += s;
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int a = a0 + ty + 16 * i;
      if (a < n && a >= b) {
        long ab = (long)a * n + b;
        double v = spin * g[ab] * W[(long)j * nn + ab] - xacc[i];
        Sigma[(long)j * nn + ab] = v;
        Sigma[(long)j * nn + (long)b * n + a] = v;
      }
    }
  }
}

}  // namespace

cudaError_t sigma2_fp64(int n, int M, double spin, const double *V, const double *G,
                        double *Sigma, double *Q, double *T1, double *W, cudaStream_t s) {
  long nn = (long)n * n;
  long tot = (long)M * nn;
  polarisation_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, M, G, Q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // T1_j = Q_j V ; W_j = V T1_j
  e = dgemm(false, false, n, n, n, 1.0, Q, n, nn, V, n, 0, nullptr, 0, 0.0, T1, n, nn, M, s);
  if (e != cudaSuccess) return e;
  e = dgemm(false, false, n, n, n, 1.0, V, n, 0, T1, n, nn, nullptr, 0, 0.0, W, n, nn, M, s);
  if (e != cudaSuccess) return e;
  dim3 grid((n + TA - 1) / TA, n, M);
  exchange_fp64_kernel<<<grid, 256, 0, s>>>(n, M, spin, V, G, W, Sigma);
  return cudaGetLastError();
}

}  // namespace fedvr

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP64 Sigma^(2) build.
//
// Some callers cannot let a library call cudaMalloc: processes whose device
// memory is owned entirely by another allocator (a framework's caching
// allocator that reserves the pool up front), or loops where the implicit
// device synchronisation of cudaMalloc/cudaFree is not acceptable. For them
// this entry point runs the same kernels as fedvr_sigma2 with its workspace
// (the polarisation Q, the product Q V and V Q V) in a fixed device array
// declared below, so it allocates nothing. The array is a static device
// symbol: every GPU that loads this library holds it until the process
// exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocStack = size_t(1) << 19;  // max M * n * n per workspace matrix stack
static __device__ __align__(256) double g_sigma2_scratch[3 * kNoAllocStack];  // 12 MiB

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
double *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once per
// device (the host-side name of a __device__ array is not a device address).
cudaError_t scratch_on_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_sigma2_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double *>(ptr);
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int fedvr_sigma2_noalloc(int n, int M, double spin, const double *V, const double *G,
                                    double *Sigma, void *cuda_stream) {
  if (n < 1 || n > 1024 || M < 1 || M > 4097 || !V || !G || !Sigma || !isfinite(spin) ||
      spin < 0.0)
    return FEDVR_ERR_ARG;
  if ((size_t)M * (size_t)n * (size_t)n > kNoAllocStack) return FEDVR_ERR_ARG;
  double *scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return FEDVR_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = fedvr::sigma2_fp64(n, M, spin, V, G, Sigma, scratch, scratch + kNoAllocStack,
                                     scratch + 2 * kNoAllocStack, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FEDVR_ERR_CUDA;
  }
  return FEDVR_OK;
}
