// gpa_exclusive_scan_noalloc: the library's exclusive prefix sum (the scan
// behind its edge, event and predecessor offsets) for callers that must not
// allocate device memory. Its scratch (the per-tile sums) is a fixed static
// device array instead of a cudaMalloc'd buffer; see include/gpa.h.
#include <cuda_runtime.h>

#include <mutex>

#include "gpa_internal.cuh"

namespace {

constexpr int kThreads = 1024;
constexpr int kItems = 4;
constexpr int kTile = kThreads * kItems;        // 4096 values per tile
constexpr int kMaxTiles = 4096;                 // so n <= 16,777,216
constexpr int kMaxDevices = 64;

// Tile sums of the last call, then their total at [kMaxTiles]. Every call
// writes each entry it reads before reading it, so nothing is cleared.
static __device__ __align__(256) int32_t g_scan_scratch[kMaxTiles + 64];

std::mutex g_mu;
int32_t* g_scratch_addr[kMaxDevices] = {nullptr};

// Block-wide exclusive scan of `count` values (kItems per thread); returns the
// block total through *total_out (thread 0 writes it).
__device__ void block_scan(int32_t* buf, int count, int32_t* total_out) {
  __shared__ int32_t warp_tot[32];
  const int base = threadIdx.x * kItems;
  int32_t v[kItems];
  int32_t local = 0;
#pragma unroll
  for (int t = 0; t < kItems; ++t) {
    v[t] = (base + t < count) ? buf[base + t] : 0;
    local += v[t];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int32_t wv = warp_tot[lane];
    int32_t wi = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_tot[lane] = wi - wv;
    if (lane == 31 && total_out) *total_out = wi;
  }
  __syncthreads();
  int32_t run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int t = 0; t < kItems; ++t) {
    if (base + t < count) buf[base + t] = run;
    run += v[t];
  }
}

__global__ void __launch_bounds__(kThreads) k_na_scan_tiles(int32_t* buf, int n, int32_t* scratch) {
  const int64_t off = (int64_t)blockIdx.x * kTile;
  const int64_t left = (int64_t)n - off;
  const int count = left < kTile ? (int)left : kTile;
  block_scan(buf + off, count, scratch + blockIdx.x);
}

__global__ void __launch_bounds__(kThreads) k_na_scan_sums(int32_t* scratch, int tiles, int32_t* total) {
  block_scan(scratch, tiles, scratch + kMaxTiles);
  __syncthreads();
  if (threadIdx.x == 0) *total = scratch[kMaxTiles];
}

__global__ void __launch_bounds__(kThreads) k_na_scan_add(int32_t* buf, int n, const int32_t* scratch) {
  const int64_t off = (int64_t)blockIdx.x * kTile;
  const int32_t add = scratch[blockIdx.x];
  for (int t = threadIdx.x; t < kTile && off + t < n; t += kThreads) buf[off + t] += add;
}

// Device address of the scratch array on the current device, resolved once per
// device (host code cannot use the symbol itself as a device pointer).
gpa_status scratch_address(int32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GPA_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GPA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    int32_t* p = nullptr;
    if (cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_scan_scratch) != cudaSuccess || !p)
      return GPA_ERR_CUDA;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GPA_OK;
}

}  // namespace

extern "C" gpa_status gpa_exclusive_scan_noalloc(int32_t* dev_buf, int64_t n, int32_t* dev_total, gpa_stream stream) {
  if (n < 0 || (n > 0 && !dev_buf) || !dev_total) return GPA_ERR_INVALID_ARG;
  if (n > (int64_t)kMaxTiles * kTile) return GPA_ERR_CAPACITY;
  int32_t* scratch = nullptr;
  const gpa_status s = scratch_address(&scratch);
  if (s) return s;
  // An error left pending by an earlier, unrelated call is not ours to clear:
  // report it (it stays pending for its owner) and launch nothing.
  if (cudaPeekAtLastError() != cudaSuccess) return GPA_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) return cudaMemsetAsync(dev_total, 0, sizeof(int32_t), st) == cudaSuccess ? GPA_OK : GPA_ERR_CUDA;
  const int tiles = (int)((n + kTile - 1) / kTile);
  k_na_scan_tiles<<<tiles, kThreads, 0, st>>>(dev_buf, (int)n, scratch);
  if (cudaGetLastError() != cudaSuccess) return GPA_ERR_CUDA;
  k_na_scan_sums<<<1, kThreads, 0, st>>>(scratch, tiles, dev_total);
  if (cudaGetLastError() != cudaSuccess) return GPA_ERR_CUDA;
  k_na_scan_add<<<tiles, kThreads, 0, st>>>(dev_buf, (int)n, scratch);
  return cudaGetLastError() == cudaSuccess ? GPA_OK : GPA_ERR_CUDA;
}
