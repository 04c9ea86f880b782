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

// One CTA per (mesh point j, column b, tile of rows a >= b): the tile's
// (a, k) pairs (rows x n) are spread over the 256 threads at up to kXQ per
// thread (pair o = tid + 256 q: row a0 + o / n, column o % n), so neither rows
// nor columns are padded. P_ak = sum_l (g_al V_bl) gb_lk accumulates over
// 16-wide slices of l staged in shared memory ([rows][16] and [16][n]); then
// v_ak = V_ak g_kb P_ak is written to shared memory and summed over k in k
// order (segments of k, then the segments in order).
constexpr int kXQ = 8, kXL = 16;
inline int xrows(int n) { return n < 256 * kXQ / n ? n : 256 * kXQ / n; }

__global__ void __launch_bounds__(256) exchange_fp64_kernel(int n, int M, int rows, double spin,
                                                            const double *__restrict__ V,
                                                            const double *__restrict__ G,
                                                            const double *__restrict__ W,
                                                            double *__restrict__ Sigma) {
  extern __shared__ double xsm[];
  double *Xs = xsm, *Ys = Xs + rows * kXL, *Vs = Ys + kXL * n, *Ps = Vs + rows * n;
  const int j = blockIdx.z, b = blockIdx.y, a0 = b + blockIdx.x * rows;
  if (a0 >= n) return;  // past the last row of this column
  const int nr = min(rows, n - a0), nout = nr * n, tid = threadIdx.x;
  const long nn = (long)n * n;
  const double *g = G + (long)j * nn;
  const double *gb = G + (long)(M - 1 - j) * nn;
  double acc[kXQ];
  int xo[kXQ], yo[kXQ];
  int nq = 0;
#pragma unroll
  for (int q = 0; q < kXQ; ++q) {
    const int o = tid + 256 * q;
    acc[q] = 0.0;
    xo[q] = o < nout ? (o / n) * kXL : 0;
    yo[q] = o < nout ? o % n : 0;
    nq += o < nout ? 1 : 0;
  }
  for (int l0 = 0; l0 < n; l0 += kXL) {
    const int nl = min(kXL, n - l0);
    for (int e = tid; e < nr * kXL; e += 256) {
      const int r = e / kXL, ll = e % kXL;
      Xs[e] = ll < nl ? g[(long)(a0 + r) * n + l0 + ll] * V[(long)b * n + l0 + ll] : 0.0;
    }
    for (int e = tid; e < nl * n; e += 256) Ys[e] = gb[(long)l0 * n + e];
    __syncthreads();
#pragma unroll 2
    for (int ll = 0; ll < nl; ++ll) {
#pragma unroll
      for (int q = 0; q < kXQ; ++q)
        if (q < nq) acc[q] = fma(Xs[xo[q] + ll], Ys[ll * n + yo[q]], acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kXQ; ++q) {
    if (q >= nq) break;
    const int o = tid + 256 * q, a = a0 + o / n, k = o % n;
    Vs[o] = V[(long)a * n + k] * g[(long)k * n + b] * acc[q];
  }
  __syncthreads();
  // row sums over k: segments of seg values by nseg threads per row, then the segments
  const int nseg = min(n, 256 / nr), seg = (n + nseg - 1) / nseg;
  if (tid < nr * nseg) {
    const int r = tid / nseg, sgi = tid % nseg, k1 = min(n, (sgi + 1) * seg);
    double p = 0.0;
    for (int k = sgi * seg; k < k1; ++k) p += Vs[r * n + k];
    Ps[tid] = p;
  }
  __syncthreads();
  if (tid < nr) {
    double x = 0.0;
    for (int sgi = 0; sgi < nseg; ++sgi) x += Ps[tid * nseg + sgi];
    const int a = a0 + tid;
    const long ab = (long)a * n + b;
    const double v = spin * g[ab] * W[(long)j * nn + ab] - x;
    Sigma[(long)j * nn + ab] = v;
    Sigma[(long)j * nn + (long)b * n + a] = v;
  }
}

// Sigma^GW = spin g o w (elementwise over the stack).
__global__ void gw_sigma_kernel(long count, double spin, const double *__restrict__ G,
                                const double *__restrict__ w, double *__restrict__ Sigma) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  Sigma[idx] = spin * G[idx] * w[idx];
}

}  // namespace

cudaError_t gw_bubble(int n, int M, const double *V, const double *G, double *Q, double *T1,
                      double *VQV, cudaStream_t s) {
  long nn = (long)n * n;
  long tot = (long)M * nn;
  polarisation_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, M, G, Q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // T1_j = Q_j V ; VQV_j = V T1_j
  e = dgemm(false, false, n, n, n, 1.0, Q, n, nn, V, n, 0, nullptr, 0, 0.0, T1, n, nn, M, s);
  if (e != cudaSuccess) return e;
  return dgemm(false, false, n, n, n, 1.0, V, n, 0, T1, n, nn, nullptr, 0, 0.0, VQV, n, nn, M, s);
}

cudaError_t launch_gw_sigma(long count, double spin, const double *G, const double *w,
                            double *Sigma, cudaStream_t s) {
  gw_sigma_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, spin, G, w, Sigma);
  return cudaGetLastError();
}

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
  const int rows = xrows(n);
  if (rows < 1) return cudaErrorInvalidValue;
  const size_t sm = (size_t)(rows * kXL + kXL * n + rows * n + 256) * sizeof(double);
  e = cudaFuncSetAttribute(exchange_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((n + rows - 1) / rows), (unsigned)n, (unsigned)M);
  exchange_fp64_kernel<<<grid, 256, sm, s>>>(n, M, rows, spin, V, G, W, Sigma);
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
