// Step (a), Sec. 2.1: aggregate packed PC samples into per-(instruction,
// stall class, latency flag) counters.
//
// HBM-bound stream: 8 bytes read per sample. The grid-strided variants:
// persistent CTAs stream 16-byte vectors with non-allocating loads,
// double-buffered in
// registers so the next round's loads are in flight while the current round
// is counted. Counting goes through a per-CTA shared-memory hash of hot
// counters (8,192 or 16,384 u32 key/value pairs): lanes holding the same counter are
// first merged with match.any, the group leader adds into the hash, and a key
// that finds no slot within a few probes goes straight to its 64-bit global
// counter. The hash is flushed to the global counters when three quarters
// full and at the end. With Zipf-skewed hotness most samples stay on chip.
#include "gpa_internal.cuh"

namespace gpa {

namespace {

constexpr int kUnroll = 4;           // 16-byte vectors per thread per round
constexpr int kSmemFuncs = 4096;     // function offsets cached in shared memory
constexpr uint32_t kNoKey = 0xFFFFFFFFu;

__device__ __forceinline__ ulonglong2 load_stream(const ulonglong2* p) {
  ulonglong2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
  return v;
}

// Counter index of a sample, or kNoKey if the sample is malformed.
__device__ __forceinline__ uint32_t sample_key(uint64_t s, const int32_t* foff, int nf) {
  const uint32_t kernel = (uint32_t)(s >> 48);
  const uint32_t pc = (uint32_t)(s >> 24) & 0xFFFFFFu;
  const uint32_t cls = (uint32_t)(s >> 20) & 0xFu;
  const uint32_t lat = (uint32_t)(s >> 19) & 1u;
  const bool ok = kernel < (uint32_t)nf && cls < 12u && !(cls == 0u && lat) && (s & 0x7FFull) == 0ull;
  if (!ok) return kNoKey;
  const int32_t lo = foff[kernel];
  if (pc >= (uint32_t)(foff[kernel + 1] - lo)) return kNoKey;
  return ((uint32_t)lo + pc) * 24u + cls * 2u + lat;
}

struct Hash {
  uint32_t* key;
  uint32_t* val;
  int* fill;
};

template <int HASH_LOG2, int PROBES>
__device__ __forceinline__ void hash_add(const Hash& H, uint32_t k, uint32_t c, unsigned long long* cnt) {
  constexpr int kHash = 1 << HASH_LOG2;
  uint32_t h = (k * 2654435761u) >> (32 - HASH_LOG2);
#pragma unroll 1
  for (int p = 0; p < PROBES; ++p) {
    const uint32_t cur = H.key[h];
    if (cur == k) { atomicAdd(&H.val[h], c); return; }
    if (cur == kNoKey) {
      const uint32_t prev = atomicCAS(&H.key[h], kNoKey, k);
      if (prev == kNoKey) { atomicAdd(H.fill, 1); atomicAdd(&H.val[h], c); return; }
      if (prev == k) { atomicAdd(&H.val[h], c); return; }
    }
    h = (h + 1) & (kHash - 1);
  }
  atomicAdd(cnt + k, (unsigned long long)c);  // no room nearby: count in global memory
}

template <int HASH_LOG2, int PROBES>
__device__ __forceinline__ void count(uint32_t key, bool in_range, const Hash& H, unsigned long long* cnt,
                                      uint32_t& bad) {
  const uint32_t k = in_range ? key : kNoKey;
  if (in_range && key == kNoKey) ++bad;
  const unsigned peers = __match_any_sync(0xffffffffu, k);
  const int lane = threadIdx.x & 31;
  if (k != kNoKey && lane == __ffs(peers) - 1) hash_add<HASH_LOG2, PROBES>(H, k, (uint32_t)__popc(peers), cnt);
}

template <int HASH_LOG2>
__device__ void flush(const Hash& H, unsigned long long* cnt) {
  constexpr int kHash = 1 << HASH_LOG2;
  for (int t = threadIdx.x; t < kHash; t += blockDim.x) {
    const uint32_t k = H.key[t];
    if (k != kNoKey) {
      atomicAdd(cnt + k, (unsigned long long)H.val[t]);
      H.key[t] = kNoKey;
      H.val[t] = 0u;
    }
  }
}

template <int THREADS, int HASH_LOG2, int PROBES>
__global__ void __launch_bounds__(THREADS) k_histogram(Prog P, const uint64_t* __restrict__ s, int64_t n,
                                                      int head) {
  constexpr int kHash = 1 << HASH_LOG2;
  extern __shared__ __align__(16) uint32_t sm[];
  Hash H{sm, sm + kHash, reinterpret_cast<int*>(sm + 2 * kHash)};
  int32_t* s_off = reinterpret_cast<int32_t*>(sm + 2 * kHash + 4);
  const bool smem_off = P.nf <= kSmemFuncs;
  for (int t = threadIdx.x; t < kHash; t += blockDim.x) { H.key[t] = kNoKey; H.val[t] = 0u; }
  if (threadIdx.x == 0) *H.fill = 0;
  if (smem_off)
    for (int i = threadIdx.x; i <= P.nf; i += blockDim.x) s_off[i] = P.func_instr_off[i];
  __syncthreads();
  const int32_t* foff = smem_off ? s_off : P.func_instr_off;
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0;

  // Scalar head (an 8-byte-aligned start) and tail (odd count): global atomics.
  const int64_t n2 = (n - head) / 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int64_t t = 0; t < head; ++t) {
      const uint32_t k = sample_key(s[t], foff, P.nf);
      if (k == kNoKey) ++bad; else atomicAdd(P.cnt + k, 1ull);
    }
    for (int64_t t = head + 2 * n2; t < n; ++t) {
      const uint32_t k = sample_key(s[t], foff, P.nf);
      if (k == kNoKey) ++bad; else atomicAdd(P.cnt + k, 1ull);
    }
  }

  const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(s + head);
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t step = n_warps * 32 * kUnroll;
  ulonglong2 cur[kUnroll], nxt[kUnroll];
  bool in_cur[kUnroll], in_nxt[kUnroll];
  int64_t c = warp * 32 * kUnroll;
  auto load_round = [&](int64_t base, ulonglong2* v, bool* in) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int64_t idx = base + u * 32 + lane;
      in[u] = idx < n2;
      v[u] = in[u] ? load_stream(v2 + idx) : make_ulonglong2(0ull, 0ull);
    }
  };
  load_round(c, cur, in_cur);
  int round = 0, since_flush = 0;
  // The loop bound is uniform per CTA (rounds are counted from the CTA's first
  // warp) so that every thread reaches the block-wide flush barriers.
  const int64_t cta_first = (int64_t)blockIdx.x * (blockDim.x >> 5) * 32 * kUnroll;
  const int64_t rounds = cta_first < n2 ? (n2 - cta_first + step - 1) / step : 0;
  for (int64_t r = 0; r < rounds; ++r) {
    load_round(c + step, nxt, in_nxt);
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      count<HASH_LOG2, PROBES>(sample_key(cur[u].x, foff, P.nf), in_cur[u], H, P.cnt, bad);
      count<HASH_LOG2, PROBES>(sample_key(cur[u].y, foff, P.nf), in_cur[u], H, P.cnt, bad);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) { cur[u] = nxt[u]; in_cur[u] = in_nxt[u]; }
    c += step;
    if (++round == 16) {  // every 16 rounds: flush when the hash is three quarters full
      round = 0;
      __syncthreads();
      // (also every 4,096 rounds, which keeps each 32-bit count below 2^24)
      const bool full = *H.fill > kHash * 3 / 4 || ++since_flush >= 256;
      __syncthreads();
      if (full) {
        since_flush = 0;
        flush<HASH_LOG2>(H, P.cnt);
        __syncthreads();
        if (threadIdx.x == 0) *H.fill = 0;
        __syncthreads();
      }
    }
  }
  __syncthreads();
  flush<HASH_LOG2>(H, P.cnt);
  // One invalid-count atomic per warp.
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if (lane == 0 && bad) atomicAdd(&P.stats[SS_INVALID], (unsigned long long)bad);
}

// Variant 0 (default), for streams that arrive as kernel-launch runs (a
// profiler that serializes kernels delivers them so). Each CTA (one per SM,
// 1,024 threads) claims chunks of 16 consecutive tiles of 8,192 samples. Its
// main shared-memory region serves the run it is in: as a direct-indexed
// window over the current kernel's counters when they fit (no hashing, no
// misses; 16-bit counters, two per word: the increment that brings one to
// 32,768 moves 32,768 to the global counter), else as a 16,384-entry hash.
// The first sample of each tile picks the mode; switching flushes the region
// to the 64-bit global counters.
// Samples of another kernel inside a window tile (a run boundary) go through
// a small side hash. Both hashes send keys they cannot place to the global
// counters, and are flushed when half full and at the end.
constexpr int kRunThreads = 1024;
#ifndef GPA_RUN_VEC
#define GPA_RUN_VEC 4
#endif
#ifndef GPA_RUN_CHUNK
#define GPA_RUN_CHUNK 16
#endif
constexpr int kRunVec = GPA_RUN_VEC;                  // 16-byte vectors per thread per tile
constexpr int kRunTile = kRunThreads * kRunVec;       // vectors per tile (8,192 samples)
constexpr int kMainWords = 40960;                     // 160 KB: window counters or hash pairs
constexpr uint32_t kWinCounters = 2u * kMainWords;      // 16-bit window counters, two per word
constexpr int kMainHashLog2 = 14;                     // 16,384 key/value pairs in hash mode
constexpr int kSideLog2 = 11;                         // 2,048-entry side hash
constexpr int kRunFlushTiles = 1 << 16;               // keeps 32-bit counts far from overflow
constexpr int kRunChunk = GPA_RUN_CHUNK;              // tiles per claimed chunk

template <int LOG2, int PROBES>
__device__ __forceinline__ bool table_add(uint32_t* key, uint32_t* val, uint32_t k, uint32_t c, uint32_t& inserts) {
  uint32_t h = (k * 2654435761u) >> (32 - LOG2);
#pragma unroll 1
  for (int p = 0; p < PROBES; ++p) {
    const uint32_t cur = key[h];
    if (cur == k) { atomicAdd(&val[h], c); return true; }
    if (cur == kNoKey) {
      const uint32_t prev = atomicCAS(&key[h], kNoKey, k);
      if (prev == kNoKey) { ++inserts; atomicAdd(&val[h], c); return true; }
      if (prev == k) { atomicAdd(&val[h], c); return true; }
    }
    h = (h + 1) & ((1u << LOG2) - 1u);
  }
  return false;
}

template <int LOG2>
__device__ void table_flush(uint32_t* key, uint32_t* val, unsigned long long* cnt) {
  for (int t = threadIdx.x; t < (1 << LOG2); t += kRunThreads) {
    const uint32_t k = key[t];
    if (k != kNoKey) {
      atomicAdd(cnt + k, (unsigned long long)val[t]);
      key[t] = kNoKey;
      val[t] = 0u;
    }
  }
}

__global__ void __launch_bounds__(kRunThreads, 1) k_histogram_runs(Prog P, const uint64_t* __restrict__ s,
                                                                   int64_t n, int head) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* mainr = sm;                                   // kMainWords
  uint32_t* skey = sm + kMainWords;                       // side hash
  uint32_t* sval = skey + (1 << kSideLog2);
  int* ctl = reinterpret_cast<int*>(sval + (1 << kSideLog2));  // 0 main fill, 1 side fill, 2 next mode
  int32_t* s_off = ctl + 8;
  const bool smem_off = P.nf <= kSmemFuncs;
  for (int t = threadIdx.x; t < (1 << kSideLog2); t += kRunThreads) { skey[t] = kNoKey; sval[t] = 0u; }
  for (int t = threadIdx.x; t < (1 << kMainHashLog2); t += kRunThreads) {
    mainr[t] = kNoKey;
    mainr[(1 << kMainHashLog2) + t] = 0u;
  }
  if (threadIdx.x < 8) ctl[threadIdx.x] = 0;
  if (smem_off)
    for (int i = threadIdx.x; i <= P.nf; i += kRunThreads) s_off[i] = P.func_instr_off[i];
  __syncthreads();
  const int32_t* foff = smem_off ? s_off : P.func_instr_off;
  uint32_t* hkey = mainr;
  uint32_t* hval = mainr + (1 << kMainHashLog2);
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0, main_ins = 0, side_ins = 0;

  // Scalar head (an 8-byte-aligned start) and tail (odd count): global atomics.
  const int64_t n2 = (n - head) / 2;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int64_t t = 0; t < head; ++t) {
      const uint32_t k = sample_key(s[t], foff, P.nf);
      if (k == kNoKey) ++bad; else atomicAdd(P.cnt + k, 1ull);
    }
    for (int64_t t = head + 2 * n2; t < n; ++t) {
      const uint32_t k = sample_key(s[t], foff, P.nf);
      if (k == kNoKey) ++bad; else atomicAdd(P.cnt + k, 1ull);
    }
  }

  // Mode of the main region: the kernel whose window it holds, or -1 (hash).
  int mode = -1;
  uint32_t base = 0, range = 0;
  auto flush_main = [&]() {
    if (mode >= 0) {
      for (uint32_t w = threadIdx.x; 2u * w < range; w += kRunThreads) {
        const uint32_t c = mainr[w], lo = c & 0xFFFFu, hi = c >> 16;
        if (lo) atomicAdd(P.cnt + base + 2u * w, (unsigned long long)lo);
        if (hi) atomicAdd(P.cnt + base + 2u * w + 1u, (unsigned long long)hi);
      }
    } else {
      table_flush<kMainHashLog2>(hkey, hval, P.cnt);
    }
  };

  // Tiles are handed out in chunks of kRunChunk consecutive tiles from a
  // counter (one chunk ahead, so the last tile of a chunk can prefetch the
  // first of the next): an SM that meets cheap runs takes more of them.
  const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(s + head);
  const int64_t n_tiles = (n2 + kRunTile - 1) / kRunTile;
  const int64_t n_chunks = (n_tiles + kRunChunk - 1) / kRunChunk;
  __shared__ long long s_claim;
  auto claim = [&]() -> int64_t {
    if (threadIdx.x == 0) s_claim = (long long)atomicAdd(&P.stats[SS_HIST_HEAD], 1ull);
    __syncthreads();
    const int64_t c = s_claim;
    __syncthreads();
    return c < n_chunks ? c : n_chunks;
  };
  ulonglong2 cur[kRunVec], nxt[kRunVec];
  bool in_cur[kRunVec], in_nxt[kRunVec];
  auto load_tile = [&](int64_t g, ulonglong2* v, bool* in) {
#pragma unroll
    for (int u = 0; u < kRunVec; ++u) {
      const int64_t idx = g * kRunTile + u * kRunThreads + threadIdx.x;
      in[u] = idx < n2;
      v[u] = in[u] ? load_stream(v2 + idx) : make_ulonglong2(0ull, 0ull);
    }
  };
  int64_t chunk = claim();
  int64_t upcoming = chunk < n_chunks ? claim() : n_chunks;
  int64_t g = chunk * kRunChunk, g_end = min(g + kRunChunk, n_tiles);
  if (chunk < n_chunks) load_tile(g, cur, in_cur);
  int since = 0;
  for (int64_t t = 0; chunk < n_chunks; ++t) {
    const int64_t g_next = g + 1 < g_end ? g + 1 : (upcoming < n_chunks ? upcoming * kRunChunk : -1);
    if (g_next >= 0) load_tile(g_next, nxt, in_nxt);
    // The tile's first sample picks the mode; every thread reads it (one
    // broadcast load), so all reach the same decision without a barrier.
    const uint32_t k0 = (uint32_t)(__ldg(reinterpret_cast<const unsigned long long*>(v2 + g * kRunTile)) >> 48);
    const int want = (k0 < (uint32_t)P.nf && (uint32_t)(foff[k0 + 1] - foff[k0]) * 24u <= kWinCounters)
                         ? (int)k0 : -1;
    if (want != mode || ++since >= kRunFlushTiles) {
      since = 0;
      __syncthreads();
      flush_main();
      __syncthreads();
      mode = want;
      if (mode >= 0) {
        base = (uint32_t)foff[mode] * 24u;
        range = (uint32_t)(foff[mode + 1] - foff[mode]) * 24u;
        for (uint32_t q = threadIdx.x; 2u * q < range; q += kRunThreads) mainr[q] = 0u;
      } else {
        for (int q = threadIdx.x; q < (1 << kMainHashLog2); q += kRunThreads) { hkey[q] = kNoKey; hval[q] = 0u; }
      }
      if (threadIdx.x == 0) ctl[0] = 0;
      main_ins = 0;
      __syncthreads();
    }
    if (mode >= 0) {
      // Window tile: a sample of the window's kernel indexes it directly.
      const uint32_t n_instr = range / 24u;
#pragma unroll
      for (int u = 0; u < kRunVec; ++u) {
        if (!in_cur[u]) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint64_t x = h ? cur[u].y : cur[u].x;
          if ((int)(x >> 48) == mode) {
            const uint32_t pc = (uint32_t)(x >> 24) & 0xFFFFFFu;
            const uint32_t cls = (uint32_t)(x >> 20) & 0xFu;
            const uint32_t lat = (uint32_t)(x >> 19) & 1u;
            if (pc < n_instr && cls < 12u && !(cls == 0u && lat) && (x & 0x7FFull) == 0ull) {
              const uint32_t idx = pc * 24u + cls * 2u + lat, sh = (idx & 1u) << 4;
              const uint32_t old = atomicAdd(&mainr[idx >> 1], 1u << sh);
              if (((old >> sh) & 0xFFFFu) == 32767u) {  // this increment made it 32,768
                atomicAdd(P.cnt + base + idx, 32768ull);
                atomicSub(&mainr[idx >> 1], 32768u << sh);
              }
            } else {
              ++bad;
            }
          } else {
            const uint32_t key = sample_key(x, foff, P.nf);
            if (key == kNoKey) ++bad;
            else if (!table_add<kSideLog2, 4>(skey, sval, key, 1u, side_ins)) atomicAdd(P.cnt + key, 1ull);
          }
        }
      }
    } else {
      // Hash tile: lanes holding the same counter merge first.
#pragma unroll
      for (int u = 0; u < kRunVec; ++u) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint64_t x = h ? cur[u].y : cur[u].x;
          const bool in = in_cur[u];
          const uint32_t key = in ? sample_key(x, foff, P.nf) : kNoKey;
          if (in && key == kNoKey) ++bad;
          const unsigned peers = __match_any_sync(0xffffffffu, key);
          if (key == kNoKey || lane != __ffs(peers) - 1) continue;
          const uint32_t c = (uint32_t)__popc(peers);
          if (!table_add<kMainHashLog2, 4>(hkey, hval, key, c, main_ins)) atomicAdd(P.cnt + key, (unsigned long long)c);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kRunVec; ++u) { cur[u] = nxt[u]; in_cur[u] = in_nxt[u]; }
    if (g + 1 < g_end) {
      ++g;
    } else {
      chunk = upcoming;
      if (chunk < n_chunks) {
        g = chunk * kRunChunk;
        g_end = min(g + kRunChunk, n_tiles);
        upcoming = claim();
      }
    }
    // every 32 tiles: flush a hash that is half full
    if ((t & 31) == 31) {
      if (main_ins) atomicAdd(&ctl[0], (int)main_ins);
      if (side_ins) atomicAdd(&ctl[1], (int)side_ins);
      main_ins = side_ins = 0;
      __syncthreads();
      const bool main_full = mode < 0 && ctl[0] > (1 << kMainHashLog2) / 2;
      const bool side_full = ctl[1] > (1 << kSideLog2) / 2;
      __syncthreads();
      if (main_full) table_flush<kMainHashLog2>(hkey, hval, P.cnt);
      if (side_full) table_flush<kSideLog2>(skey, sval, P.cnt);
      if (main_full || side_full) {
        __syncthreads();
        if (threadIdx.x == 0) {
          if (main_full) ctl[0] = 0;
          if (side_full) ctl[1] = 0;
        }
      }
    }
  }
  __syncthreads();
  flush_main();
  table_flush<kSideLog2>(skey, sval, P.cnt);
  for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
  if (lane == 0 && bad) atomicAdd(&P.stats[SS_INVALID], (unsigned long long)bad);
}

template <int THREADS, int HASH_LOG2, int PROBES>
static void launch_variant(const Prog& P, const uint64_t* samples, size_t n, cudaStream_t st, int sms,
                           int ctas_per_sm) {
  const int head = (reinterpret_cast<uintptr_t>(samples) & 15u) ? 1 : 0;
  const int64_t vecs = ((int64_t)n - head) / 2;
  int64_t blocks = (vecs + (int64_t)THREADS * kUnroll - 1) / ((int64_t)THREADS * kUnroll);
  const int64_t cap = (int64_t)sms * ctas_per_sm;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  const size_t smem = sizeof(uint32_t) * (2 * ((size_t)1 << HASH_LOG2) + 4) +
                      (P.nf <= kSmemFuncs ? sizeof(int32_t) * (size_t)(P.nf + 1) : 0);
  auto* k = k_histogram<THREADS, HASH_LOG2, PROBES>;
  allow_max_smem(k);
  k<<<(int)blocks, THREADS, smem, st>>>(P, samples, (int64_t)n, head);
}

}  // namespace

// variant 0 (default): contiguous segments with a per-run window or hash
// (k_histogram_runs); 1: grid-strided, 8,192-entry hash, 512 threads, 2 CTAs
// per SM, 4 probes; 2: 16,384 entries, 1,024 threads, 1 CTA per SM, 4 probes;
// 3: 8,192 entries, 256 threads, 3 CTAs per SM, 8 probes.
void launch_histogram(const Prog& P, const uint64_t* samples, size_t n, cudaStream_t st, int sms, int64_t* launches,
                      int variant) {
  if (n == 0) return;
  if (variant == 0) {
    const int head = (reinterpret_cast<uintptr_t>(samples) & 15u) ? 1 : 0;
    const int64_t vecs = ((int64_t)n - head) / 2;
    int64_t grid = (vecs + (int64_t)kRunTile * kRunChunk - 1) / ((int64_t)kRunTile * kRunChunk);
    if (grid > sms) grid = sms;
    if (grid < 1) grid = 1;
    cudaMemsetAsync(&P.stats[SS_HIST_HEAD], 0, sizeof(unsigned long long), st);
    const size_t smem = sizeof(uint32_t) * ((size_t)kMainWords + 2 * ((size_t)1 << kSideLog2) + 8) +
                        (P.nf <= kSmemFuncs ? sizeof(int32_t) * (size_t)(P.nf + 1) : 0);
    allow_max_smem(k_histogram_runs);
    k_histogram_runs<<<(int)grid, kRunThreads, smem, st>>>(P, samples, (int64_t)n, head);
    ++*launches;
    return;
  }
  if (variant == 1) launch_variant<512, 13, 4>(P, samples, n, st, sms, 2);
  else if (variant == 2) launch_variant<1024, 14, 4>(P, samples, n, st, sms, 1);
  else launch_variant<256, 13, 8>(P, samples, n, st, sms, 3);  // 3
  ++*launches;
}

}  // namespace gpa
