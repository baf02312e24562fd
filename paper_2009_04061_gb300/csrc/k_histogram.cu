// Step (a), Sec. 2.1: aggregate packed PC samples into per-(instruction,
// stall class, latency flag) counters.
//
// HBM-bound stream: 8 bytes read per sample. Each warp reads 32 x 16-byte
// vectors per load round (two samples per lane, four rounds in flight), with
// non-allocating loads so the sample stream does not evict the counters from
// L2. Lanes holding the same counter are merged with match.any and the leader
// issues one 64-bit atomic add for the group, so hot instructions (Zipf-skewed
// hotness) cost one L2 atomic per warp rather than one per sample.
#include "gpa_internal.cuh"

namespace gpa {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;
constexpr int kSmemFuncs = 8192;
constexpr uint32_t kNoKey = 0xFFFFFFFFu;

__device__ __forceinline__ ulonglong2 load_stream(const ulonglong2* p) {
  ulonglong2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
               : "=l"(v.x), "=l"(v.y)
               : "l"(p));
  return v;
}

// Counter index of a sample, or kNoKey if the sample is malformed.
__device__ __forceinline__ uint32_t sample_key(uint64_t s, const int32_t* foff, int nf) {
  const uint32_t kernel = (uint32_t)(s >> 48);
  const uint32_t pc = (uint32_t)(s >> 24) & 0xFFFFFFu;
  const uint32_t cls = (uint32_t)(s >> 20) & 0xFu;
  const uint32_t lat = (uint32_t)(s >> 19) & 1u;
  bool ok = kernel < (uint32_t)nf && cls < 12u && !(cls == 0u && lat) && (s & 0x7FFull) == 0ull;
  if (!ok) return kNoKey;
  const int32_t lo = foff[kernel];
  if (pc >= (uint32_t)(foff[kernel + 1] - lo)) return kNoKey;
  return ((uint32_t)lo + pc) * 24u + cls * 2u + lat;
}

__device__ __forceinline__ void count(uint32_t key, bool in_range, unsigned long long* cnt, uint32_t& bad) {
  const uint32_t k = in_range ? key : kNoKey;
  if (in_range && key == kNoKey) ++bad;
  const unsigned peers = __match_any_sync(0xffffffffu, k);
  const int lane = threadIdx.x & 31;
  if (k != kNoKey && lane == __ffs(peers) - 1) atomicAdd(cnt + k, (unsigned long long)__popc(peers));
}

__global__ void __launch_bounds__(kThreads) k_histogram(Prog P, const uint64_t* __restrict__ s, int64_t n,
                                                       int head) {
  extern __shared__ int32_t s_off[];
  const bool smem = P.nf <= kSmemFuncs;
  if (smem) {
    for (int i = threadIdx.x; i <= P.nf; i += blockDim.x) s_off[i] = P.func_instr_off[i];
    __syncthreads();
  }
  const int32_t* foff = smem ? s_off : P.func_instr_off;
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0;

  // Scalar head (an 8-byte-aligned start) and tail (odd count).
  const int64_t n2 = (n - head) / 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int64_t t = 0; t < head; ++t) {
      uint32_t k = sample_key(s[t], foff, P.nf);
      if (k == kNoKey) ++bad; else atomicAdd(P.cnt + k, 1ull);
    }
    for (int64_t t = head + 2 * n2; t < n; ++t) {
      uint32_t k = sample_key(s[t], foff, P.nf);
      if (k == kNoKey) ++bad; else atomicAdd(P.cnt + k, 1ull);
    }
  }

  const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(s + head);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t step = n_warps * 32 * kUnroll;
  for (int64_t c = warp * 32 * kUnroll; c < n2; c += step) {
    ulonglong2 v[kUnroll];
    bool in[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t idx = c + u * 32 + lane;
      in[u] = idx < n2;
      v[u] = in[u] ? load_stream(v2 + idx) : make_ulonglong2(0ull, 0ull);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      count(sample_key(v[u].x, foff, P.nf), in[u], P.cnt, bad);
      count(sample_key(v[u].y, foff, P.nf), in[u], P.cnt, bad);
    }
  }
  // One invalid-count atomic per warp.
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if (lane == 0 && bad) atomicAdd(&P.stats[SS_INVALID], (unsigned long long)bad);
}

}  // namespace

void launch_histogram(const Prog& P, const uint64_t* samples, size_t n, cudaStream_t st, int sms, int64_t* launches) {
  if (n == 0) return;
  const int head = (reinterpret_cast<uintptr_t>(samples) & 15u) ? 1 : 0;
  const int64_t vecs = ((int64_t)n - head) / 2;
  int64_t blocks = (vecs + (int64_t)kThreads * kUnroll - 1) / ((int64_t)kThreads * kUnroll);
  const int64_t cap = (int64_t)sms * 8;  // 8 x 256 threads per SM resident
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const size_t smem = P.nf <= kSmemFuncs ? sizeof(int32_t) * (size_t)(P.nf + 1) : 0;
  k_histogram<<<(int)blocks, kThreads, smem, st>>>(P, samples, (int64_t)n, head);
  ++*launches;
}

}  // namespace gpa
