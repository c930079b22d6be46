// sipg_dot_noalloc: the column-wise FP64 dot product of sipg_dot, with its
// reduction scratch in a fixed file-scope device array instead of the
// caller-bound workspace.
//
// Who needs it: callers that cannot call cudaMalloc -- an application whose
// allocator has already reserved all device memory, or code on a latency
// path where a cudaMalloc would implicitly synchronise the device -- and that
// have not bound a workspace to the handle.  This call allocates nothing.
//
// Limits and sharing: the scratch holds kBlocks partial sums for each of at
// most kMaxCols columns (64 x 256 doubles = 128 KiB, kept by every GPU that
// loads the library until the process exits).  All calls share it: two calls
// whose kernels overlap on the GPU (different streams, no ordering between
// them) race on it.  Each call writes every partial it later reads, so
// nothing has to be cleared between calls.
//
// Set-up: the first call on a device (with that device current) looks up the
// device address of the array once with cudaGetSymbolAddress; make that
// first call before any stream capture.
#include <mutex>

#include "sipg_internal.cuh"

namespace {

constexpr int kMaxCols = 64;
constexpr int kBlocks = 256;
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;
static_assert(kThreads == kBlocks, "dot_finish reads one partial per thread");

__device__ __align__(256) double g_dot_scratch[kMaxCols * kBlocks];

double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__device__ __forceinline__ double warp_reduce(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_reduce(double v) {
  __shared__ double part[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_reduce(v);
  if (lane == 0) part[w] = v;
  __syncthreads();
  v = (threadIdx.x < kThreads / 32) ? part[threadIdx.x] : 0.0;
  if (w == 0) v = warp_reduce(v);
  return v;
}

// stage 1: one partial per (block, column), written to scratch[col * kBlocks + block]
__global__ void __launch_bounds__(kThreads) dot_partials(const double* a, const double* b, long long n,
                                                         double* scratch) {
  const long long col = (long long)blockIdx.y * n;
  double v = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)kBlocks * kThreads)
    v = fma(a[col + i], b[col + i], v);
  v = block_reduce(v);
  if (threadIdx.x == 0) scratch[blockIdx.y * kBlocks + blockIdx.x] = v;
}

// stage 2: fixed-order sum of the kBlocks partials of each column
__global__ void __launch_bounds__(kThreads) dot_finish(const double* scratch, double* out) {
  double v = scratch[blockIdx.x * kBlocks + threadIdx.x];
  v = block_reduce(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

double* scratch_address(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kMaxDevices) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    double* p = nullptr;
    *err = cudaGetSymbolAddress((void**)&p, g_dot_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" sipg_status sipg_dot_noalloc(sipg_handle* h, const double* a, const double* b, double* out,
                                        void* stream) {
  if (!h) return SIPG_EINVAL;
  if (!a || !b || !out) {
    h->err = "sipg_dot_noalloc: null vector";
    return SIPG_EINVAL;
  }
  if (h->prm.nrhs > kMaxCols) {
    h->err = "sipg_dot_noalloc: nrhs exceeds the 64 columns of its static scratch";
    return SIPG_EINVAL;
  }
  cudaError_t e;
  double* scratch = scratch_address(&e);
  if (!scratch) {
    h->err = std::string("sipg_dot_noalloc: device scratch lookup failed: ") + cudaGetErrorString(e);
    return SIPG_ECUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const long long n = (long long)h->lv[h->L].ndofs;
  dot_partials<<<dim3(kBlocks, h->prm.nrhs), kThreads, 0, s>>>(a, b, n, scratch);
  dot_finish<<<h->prm.nrhs, kThreads, 0, s>>>(scratch, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("sipg_dot_noalloc: ") + cudaGetErrorString(e);
    return SIPG_ECUDA;
  }
  h->launches += 2;
  return SIPG_OK;
}
