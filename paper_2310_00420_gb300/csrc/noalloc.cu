// cmcs_apply_noalloc: the operator Z = beta Phi^T (Phi V) + alpha * V for m vectors of one
// task, for callers that must not allocate device memory.  The intermediate W = Phi V lives in
// a fixed file-scope device array instead of memory obtained from cudaMalloc.
//
// Who needs this: code that cannot call cudaMalloc/cudaFree once it is running -- for example a
// host application whose device memory is all owned by its own pool allocator, or a
// latency-critical loop that cannot afford the implicit device synchronisation of cudaMalloc.
// Such a caller still allocates its inputs and outputs up front; this call adds nothing.
#include <mutex>
#include <stdio.h>

#include "cmcs_internal.cuh"

namespace cmcs {
void set_global_error(const char* msg);
}

// 4,194,304 floats (16 MiB): the largest m * N this entry point accepts.  Every GPU that loads
// libcmcs.so holds this array until the process exits.
constexpr size_t kNoAllocScratchFloats = size_t(1) << 22;
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once per device (with
// that device current).  Host code must not pass the symbol itself to a kernel: on the host it
// names a stand-in, not device memory.  The cached address belongs to the device's primary
// context: after cudaDeviceReset the module is loaded again and the cache is stale, so a process
// that resets a device must not call this entry point on it afterwards.
cudaError_t noalloc_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

// W[j][n] = sum_d Phi[n][d] V[j][d]; 32 x 32 output tile per block, d in chunks of 32
__global__ void __launch_bounds__(256)
k_noalloc_phiv(const float* __restrict__ phi, const float* __restrict__ V, float* __restrict__ W,
               int N, int D, int m) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int n0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int d0 = 0; d0 < D; d0 += 32) {
    for (int i = threadIdx.x; i < 1024; i += 256) {
      const int r = i >> 5, cc = i & 31;
      As[r][cc] = (n0 + r < N && d0 + cc < D) ? phi[(int64_t)(n0 + r) * D + d0 + cc] : 0.f;
      Bs[r][cc] = (j0 + r < m && d0 + cc < D) ? V[(int64_t)(j0 + r) * D + d0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int cc = 0; cc < 32; ++cc)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = fmaf(As[tx * 2 + a][cc], Bs[ty * 2 + b][cc], acc[a][b]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int n = n0 + tx * 2 + a, j = j0 + ty * 2 + b;
      if (n < N && j < m) W[(int64_t)j * N + n] = acc[a][b];
    }
}

// Z[j][d] = beta sum_n Phi[n][d] W[j][n] + alpha[d] V[j][d]
__global__ void __launch_bounds__(256)
k_noalloc_phitw(const float* __restrict__ phi, const float* __restrict__ W,
                const float* __restrict__ V, const float* __restrict__ alpha,
                float* __restrict__ Z, int N, int D, int m, float beta) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int d0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  float acc[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  for (int n0 = 0; n0 < N; n0 += 32) {
    for (int i = threadIdx.x; i < 1024; i += 256) {
      const int r = i >> 5, cc = i & 31;
      As[r][cc] = (n0 + r < N && d0 + cc < D) ? phi[(int64_t)(n0 + r) * D + d0 + cc] : 0.f;
      Bs[r][cc] = (j0 + r < m && n0 + cc < N) ? W[(int64_t)(j0 + r) * N + n0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int cc = 0; cc < 32; ++cc)
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = fmaf(As[cc][tx * 2 + a], Bs[ty * 2 + b][cc], acc[a][b]);
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int d = d0 + tx * 2 + a, j = j0 + ty * 2 + b;
      if (d < D && j < m)
        Z[(int64_t)j * D + d] = fmaf(beta, acc[a][b], alpha[d] * V[(int64_t)j * D + d]);
    }
}

// true when p is device memory (or managed memory) that kernels on device dev can address; a
// host pointer, or memory of another device, is rejected before any launch.  The query
// allocates nothing.
bool device_pointer(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" cmcs_status cmcs_apply_noalloc(const float* Phi, int N, int D, const float* alpha,
                                          double beta, const float* V, int m, float* Z,
                                          void* stream) {
  char msg[256];
  if (!Phi || !alpha || !V || !Z || N < 1 || D < 1 || m < 1 || !(beta > 0.0)) {
    cmcs::set_global_error("cmcs_apply_noalloc: null pointer or non-positive size/beta");
    return CMCS_ERR_INVALID_ARG;
  }
  if ((m + 31) / 32 > 65535) {
    cmcs::set_global_error("cmcs_apply_noalloc: m exceeds 2,097,120 vectors");
    return CMCS_ERR_INVALID_ARG;
  }
  if ((size_t)m * (size_t)N > kNoAllocScratchFloats) {
    snprintf(msg, sizeof(msg),
             "cmcs_apply_noalloc: m * N = %zu exceeds the fixed scratch of %zu floats",
             (size_t)m * (size_t)N, kNoAllocScratchFloats);
    cmcs::set_global_error(msg);
    return CMCS_ERR_INVALID_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    cmcs::set_global_error("cmcs_apply_noalloc: no current CUDA device");
    return CMCS_ERR_CUDA;
  }
  const void* ptrs[4] = {Phi, alpha, V, Z};
  const char* names[4] = {"Phi", "alpha", "V", "Z"};
  for (int i = 0; i < 4; ++i) {
    if (!device_pointer(ptrs[i], dev)) {
      snprintf(msg, sizeof(msg),
               "cmcs_apply_noalloc: %s is not device memory of the current device %d", names[i], dev);
      cmcs::set_global_error(msg);
      return CMCS_ERR_INVALID_ARG;
    }
  }
  float* W = nullptr;
  cudaError_t e = noalloc_scratch(&W);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "cmcs_apply_noalloc: scratch lookup failed: %s", cudaGetErrorString(e));
    cmcs::set_global_error(msg);
    return CMCS_ERR_CUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_noalloc_phiv<<<dim3((N + 31) / 32, (m + 31) / 32), 256, 0, st>>>(Phi, V, W, N, D, m);
  k_noalloc_phitw<<<dim3((D + 31) / 32, (m + 31) / 32), 256, 0, st>>>(Phi, W, V, alpha, Z, N, D, m,
                                                                       (float)beta);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof(msg), "cmcs_apply_noalloc: CUDA error: %s", cudaGetErrorString(e));
    cmcs::set_global_error(msg);
    return CMCS_ERR_CUDA;
  }
  return CMCS_OK;
}
