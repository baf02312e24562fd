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
#include <type_traits>

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
// 1,024 threads) claims chunks of consecutive tiles of 8,192 samples from a
// counter; a tile is four segments of 2,048 samples, one 16-byte vector per
// thread each. Shared memory holds a window of 32-bit counters over up to
// 1,558 consecutive instructions of one kernel, 32 words per instruction
// indexed by the sample's 5-bit (class, latency) field, and a 4,096-entry
// hash. The middle sample of each segment names the kernel that segment is
// counted for: when it differs from the window's, the window is flushed to the
// 64-bit global counters and placed for the new kernel (whole when it fits,
// else on the densest span of the 32 samples around that middle sample). A
// run boundary inside a segment thus costs at most its minority side.
// A sample inside the window is one shared-memory reduction on its word (no
// return value, predicated: no branch). The 9 field values that name no
// counter (SELECTED with the latency flag, class 12 and up) land in words the
// flush counts as invalid samples. A vector whose two samples do not both carry
// the window kernel's upper id bits and zero reserved bits, and any other
// sample (another kernel, a pc outside a partial window), takes the checked
// path: the hash, and a key that finds no slot within two probes goes to its
// global counter (measured: 1.13 ms for 5e8 samples against 1.18 with four
// probes). The hash is flushed when half full, and window and hash at least
// every 2^16 tiles (fewer than 2^30 increments: no 32-bit count wraps) and at
// the end.
constexpr int kRunThreads = 1024;
constexpr int kRunVec = 4;                            // segments per tile: vectors per thread per tile
constexpr int kRunTile = kRunThreads * kRunVec;       // vectors per tile (8,192 samples)
constexpr int kWinStride = 32;                        // window words per instruction
constexpr uint32_t kWinInstr = 1558;                  // instructions in the window
constexpr int kMainWords = (int)kWinInstr * kWinStride;  // 199,424 bytes of 32-bit counters
constexpr int kSideLog2 = 12;                         // 4,096-entry hash
constexpr int kSideProbes = 2;                        // hash probes before the global counter
constexpr int kRunFlushTiles = 1 << 16;               // forced flush: keeps 32-bit counts below 2^30
static_assert((long long)kRunFlushTiles * 2 * kRunTile < (1ll << 30), "32-bit counts could wrap between flushes");
static_assert(kMainWords % 4 == 0, "the window is read and cleared as 16-byte vectors");
static_assert(kRunVec == 4, "the per-tile kernel test reads four segment kernels");
// Bit f of kValid5 is set when the 5-bit (class, latency) field f names a
// counter: class < 12, and not SELECTED with the latency flag.
constexpr uint32_t kValid5 = 0x00FFFFFDu;

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

// Start of the window over a kernel of n instructions: 0 when it fits, else
// the start, among windows centred on lanes 12-19 of the 32 samples `x` (one
// per lane) that are of that kernel, that holds most of those 32. Every warp
// reads the same 32 samples and reaches the same answer.
__device__ __forceinline__ uint32_t window_start(uint64_t x, uint32_t kernel, uint32_t n) {
  if (n <= kWinInstr) return 0u;
  const uint32_t pc = (uint32_t)(x >> 24) & 0xFFFFFFu;
  const bool mine = (uint32_t)(x >> 48) == kernel && pc < n;
  uint32_t lo = pc > kWinInstr / 2u ? pc - kWinInstr / 2u : 0u;
  if (lo > n - kWinInstr) lo = n - kWinInstr;
  uint32_t best = 0u, best_lo = 0u;
#pragma unroll
  for (int c = 12; c < 20; ++c) {
    const uint32_t lo_c = __shfl_sync(0xffffffffu, lo, c);
    const bool cand = __shfl_sync(0xffffffffu, mine, c);
    const uint32_t hits = (uint32_t)__popc(__ballot_sync(0xffffffffu, mine && pc - lo_c < kWinInstr));
    if (cand && hits > best) { best = hits; best_lo = lo_c; }
  }
  return best_lo;
}

// One window sample: when chk == 0 and r < span, one shared-memory reduction
// (no return value) on the word at addr; otherwise BIT is set in slow.
template <uint32_t BIT>
__device__ __forceinline__ void count_window(uint32_t addr, uint32_t r, uint32_t chk, uint32_t span, uint32_t& slow) {
  asm volatile("{\n\t.reg .pred ok, p;\n\t"
               "setp.eq.u32 ok, %3, 0;\n\t"
               "setp.lt.and.u32 p, %2, %4, ok;\n\t"
               "@p red.shared.add.u32 [%1], 1;\n\t"
               "@!p or.b32 %0, %0, %5;\n\t}"
               : "+r"(slow) : "r"(addr), "r"(r), "r"(chk), "r"(span), "n"(BIT) : "memory");
}

__global__ void __launch_bounds__(kRunThreads, 1) k_histogram_runs(Prog P, const uint64_t* __restrict__ s,
                                                                   int64_t n, int head, int chunk_tiles) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* win = sm;                                     // kMainWords window counters
  const uint32_t win_base = (uint32_t)__cvta_generic_to_shared(win);
  uint32_t* skey = sm + kMainWords;                       // hash
  uint32_t* sval = skey + (1 << kSideLog2);
  int* ctl = reinterpret_cast<int*>(sval + (1 << kSideLog2));  // 1: hash fill
  // Every window word is zero whenever no kernel is being counted into it (the
  // flush zeroes what it reads), so placing the window needs no clearing.
  for (int t = threadIdx.x; t < kMainWords / 4; t += kRunThreads)
    reinterpret_cast<uint4*>(win)[t] = make_uint4(0u, 0u, 0u, 0u);
  for (int t = threadIdx.x; t < (1 << kSideLog2); t += kRunThreads) { skey[t] = kNoKey; sval[t] = 0u; }
  if (threadIdx.x < 8) ctl[threadIdx.x] = 0;
  __syncthreads();
  const int32_t* foff = P.func_instr_off;  // read through the cache: the window takes the shared memory
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0, side_ins = 0;
  // The window: mode_hi = its kernel << 16 (kNoMode: none), instructions
  // [lo, lo + wn) of it; word (pc - lo) * 32 + f5 counts (pc, f5), f5 the
  // 5-bit (class, latency) field. With r = bits 19..50 of a sample (f5 | pc << 5
  // | low 3 kernel bits << 29), a sample whose kernel bits 51..63 match is in the
  // window when r - first5 < span5, first5 = (kernel << 29) | (lo << 5), span5 =
  // wn << 5 (so lo and wn need no registers of their own). The kernel's first
  // instruction and size stay in registers: a miss of that kernel needs no
  // offset lookup.
  constexpr uint32_t kNoMode = 0xFFFF0000u;
  uint32_t mode_hi = kNoMode, first5 = 0, span5 = 0, mode_first = 0, mode_n = 0;
  // A sample that is not counted in the window: the hash, else its global counter.
  auto count_other = [&](uint64_t x) {
    uint32_t key;
    if (((uint32_t)(x >> 32) & 0xFFFF0000u) == mode_hi) {
      const uint32_t pc = (uint32_t)(x >> 24) & 0xFFFFFFu, f5 = (uint32_t)(x >> 19) & 31u;
      key = (pc < mode_n && ((kValid5 >> f5) & 1u) && (x & 0x7FFull) == 0ull) ? (mode_first + pc) * 24u + f5
                                                                                : kNoKey;
    } else {
      key = sample_key(x, foff, P.nf);
    }
    if (key == kNoKey) ++bad;
    else if (!table_add<kSideLog2, kSideProbes>(skey, sval, key, 1u, side_ins)) atomicAdd(P.cnt + key, 1ull);
  };

  // Whole tiles go through the window; what is left (an 8-byte-aligned first
  // sample, the vectors after the last whole tile, an odd last sample) is
  // counted by the first CTA through the hash.
  const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(s + head);
  const uint64_t* s2 = s + head;
  const int64_t n2 = (n - head) / 2;
  const int n_tiles = (int)(n2 / kRunTile);
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      for (int64_t t = 0; t < head; ++t) count_other(s[t]);
      for (int64_t t = head + 2 * n2; t < n; ++t) count_other(s[t]);
    }
    for (int64_t v = (int64_t)n_tiles * kRunTile + threadIdx.x; v < n2; v += kRunThreads) {
      const ulonglong2 x = load_stream(v2 + v);
      count_other(x.x);
      count_other(x.y);
    }
  }

  auto flush_win = [&]() {
    const uint32_t quads = span5 >> 2;                     // wn * 32 words, 4 per quad
    const uint32_t gfirst = mode_first + ((first5 >> 5) & 0xFFFFFFu);
    for (uint32_t q = threadIdx.x; q < quads; q += kRunThreads) {
      uint4* w = reinterpret_cast<uint4*>(win) + q;
      const uint4 v = *w;
      if ((v.x | v.y | v.z | v.w) == 0u) continue;
      *w = make_uint4(0u, 0u, 0u, 0u);
      const uint32_t c[4] = {v.x, v.y, v.z, v.w};
      const uint32_t f0 = (q % (kWinStride / 4)) * 4u;
      const uint32_t g = (gfirst + q / (kWinStride / 4)) * 24u;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (!c[e]) continue;
        const uint32_t f5 = f0 + e;
        if ((kValid5 >> f5) & 1u) atomicAdd(P.cnt + g + f5, (unsigned long long)c[e]);
        else bad += c[e];
      }
    }
  };
  // Flush the window and place it for kernel id `want` (>= nf: none), from the
  // 32 samples starting at stream index m. CTA-uniform: every thread takes part.
  auto place = [&](uint32_t want, int64_t m) {
    __syncthreads();
    flush_win();
    __syncthreads();
    mode_hi = kNoMode;
    first5 = span5 = mode_first = mode_n = 0;
    if (want < (uint32_t)P.nf) {
      const uint32_t n_instr = (uint32_t)(foff[want + 1] - foff[want]);
      mode_first = (uint32_t)foff[want];
      mode_n = n_instr;
      const uint32_t lo = window_start(__ldg(reinterpret_cast<const unsigned long long*>(s2 + m + lane)), want, n_instr);
      mode_hi = want << 16;
      first5 = (want << 29) | (lo << 5);
      span5 = min(n_instr, kWinInstr) << 5;
    }
  };

  // Tiles are handed out in chunks of chunk_tiles consecutive tiles from a
  // counter (one chunk ahead, so the last tile of a chunk can prefetch the
  // first of the next): an SM that meets cheap runs takes more of them.
  const int n_chunks = (n_tiles + chunk_tiles - 1) / chunk_tiles;
  __shared__ int s_claim;
  // A chunk claim also reports this thread's hash inserts and flushes the hash
  // when half full (the claim's barriers order both).
  auto claim = [&]() -> int {
    if (side_ins) atomicAdd(&ctl[1], (int)side_ins);
    side_ins = 0;
    if (threadIdx.x == 0) s_claim = (int)atomicAdd(&P.stats[SS_HIST_HEAD], 1ull);
    __syncthreads();
    const int c = s_claim;
    const bool side_full = ctl[1] > (1 << kSideLog2) / 2;
    __syncthreads();
    if (side_full) {
      table_flush<kSideLog2>(skey, sval, P.cnt);
      if (threadIdx.x == 0) ctl[1] = 0;
      __syncthreads();
    }
    return c < n_chunks ? c : n_chunks;
  };
  int chunk = claim();
  int upcoming = chunk < n_chunks ? claim() : n_chunks;
  int g = chunk * chunk_tiles, g_end = min(g + chunk_tiles, n_tiles);
  auto next_tile = [&]() -> int {
    return g + 1 < g_end ? g + 1 : (upcoming < n_chunks ? upcoming * chunk_tiles : -1);
  };
  auto advance = [&]() {
    if (g + 1 < g_end) {
      ++g;
    } else {
      chunk = upcoming;
      if (chunk < n_chunks) {
        g = chunk * chunk_tiles;
        g_end = min(g + chunk_tiles, n_tiles);
        upcoming = claim();
      }
    }
  };
  // The tile after next, when it is in this chunk, is fetched into L2 by one
  // bulk prefetch from one thread, so the register loads of the next tile
  // find it there.
  auto prefetch_after = [&]() {
    if (threadIdx.x == 0 && g + 2 < g_end) {
      const ulonglong2* p = v2 + (int64_t)(g + 2) * kRunTile;
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p), "r"((uint32_t)(kRunTile * 16)) : "memory");
    }
  };
  // A tile's vectors, and the kernel of each segment's middle sample: lane u
  // of every warp loads segment u's (issued with the tile's own loads).
  auto load_tile = [&](int t, ulonglong2* v, uint32_t& k) {
    const int64_t t0 = (int64_t)t * kRunTile;
#pragma unroll
    for (int u = 0; u < kRunVec; ++u) v[u] = load_stream(v2 + t0 + u * kRunThreads + threadIdx.x);
    k = lane < kRunVec ? __ldg(reinterpret_cast<const unsigned int*>(s2 + 2 * (t0 + lane * kRunThreads) +
                                                                     kRunThreads) + 1) >> 16
                       : 0u;
  };

  int since = 0;      // tiles since window and hash were last both flushed
  auto process = [&](const ulonglong2* v, uint32_t k) {
    if (++since >= kRunFlushTiles) {  // keeps the 32-bit counts small
      since = 0;
      __syncthreads();
      flush_win();
      table_flush<kSideLog2>(skey, sval, P.cnt);
      if (threadIdx.x == 0) ctl[1] = 0;
      __syncthreads();
    }
    uint32_t slow = 0;
    auto segment = [&](auto U, bool check) {
      constexpr int u = decltype(U)::value;
      if (check) {
        const uint32_t ku = __shfl_sync(0xffffffffu, k, u);
        if ((ku < (uint32_t)P.nf ? ku << 16 : kNoMode) != mode_hi)
          place(ku, 2 * ((int64_t)g * kRunTile + u * kRunThreads) + kRunThreads - 16);
      }
      // Both samples of the vector carry the window kernel's upper id bits and
      // zero reserved bits; then each is in the window when its offset is.
      const uint32_t x0l = (uint32_t)v[u].x, x0h = (uint32_t)(v[u].x >> 32);
      const uint32_t x1l = (uint32_t)v[u].y, x1h = (uint32_t)(v[u].y >> 32);
      const uint32_t chk = (((x0h ^ mode_hi) | (x1h ^ mode_hi)) & 0xFFF80000u) | ((x0l | x1l) & 0x7FFu);
      const uint32_t r0 = __funnelshift_r(x0l, x0h, 19) - first5;
      const uint32_t r1 = __funnelshift_r(x1l, x1h, 19) - first5;
      count_window<1u << (2 * u)>(win_base + 4u * r0, r0, chk, span5, slow);
      count_window<2u << (2 * u)>(win_base + 4u * r1, r1, chk, span5, slow);
    };
    // The four segments, with (check) or without a test of each segment's
    // kernel against the window's: most tiles lie inside one run. (The kernel
    // ids are the same in every warp, so the choice is uniform over the CTA.)
    auto segments = [&](bool check) {
      segment(std::integral_constant<int, 0>{}, check);
      segment(std::integral_constant<int, 1>{}, check);
      segment(std::integral_constant<int, 2>{}, check);
      segment(std::integral_constant<int, 3>{}, check);
    };
    if (__all_sync(0xffffffffu, lane >= kRunVec || k == (mode_hi >> 16))) segments(false);
    else segments(true);
    // Each lane walks its own missed samples: a warp takes as many rounds as
    // its busiest lane has misses (scattered misses cost one round).
    while (slow) {
      const int i = __ffs(slow) - 1;
      slow &= slow - 1u;
      uint64_t x = v[0].x;
#pragma unroll
      for (int q = 1; q < 2 * kRunVec; ++q)
        if (i == q) x = (q & 1) ? v[q >> 1].y : v[q >> 1].x;
      count_other(x);
    }
  };

  // Two register sets in turn: one tile is counted while the next is loaded.
  ulonglong2 va[kRunVec], vb[kRunVec];
  uint32_t ka = 0, kb = 0;
  if (chunk < n_chunks) load_tile(g, va, ka);
  while (chunk < n_chunks) {
    int nx = next_tile();
    if (nx >= 0) load_tile(nx, vb, kb);
    prefetch_after();
    process(va, ka);
    advance();
    if (chunk >= n_chunks) break;
    nx = next_tile();
    if (nx >= 0) load_tile(nx, va, ka);
    prefetch_after();
    process(vb, kb);
    advance();
  }
  __syncthreads();
  flush_win();
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

// variant 0 (default): tiles claimed in chunks of hist_chunk (0: 24), a
// per-segment window plus a hash (k_histogram_runs); 1: grid-strided, 8,192-entry hash, 512 threads, 2 CTAs
// per SM, 4 probes; 2: 16,384 entries, 1,024 threads, 1 CTA per SM, 4 probes;
// 3: 8,192 entries, 256 threads, 3 CTAs per SM, 8 probes.
void launch_histogram(const Prog& P, const uint64_t* samples, size_t n, cudaStream_t st, int sms, int64_t* launches,
                      int variant, int hist_chunk) {
  if (n == 0) return;
  if (variant == 0) {
    const int head = (reinterpret_cast<uintptr_t>(samples) & 15u) ? 1 : 0;
    const int64_t vecs = ((int64_t)n - head) / 2;
    const int chunk_tiles = hist_chunk > 0 ? hist_chunk : 24;
    int64_t grid = (vecs + (int64_t)kRunTile * chunk_tiles - 1) / ((int64_t)kRunTile * chunk_tiles);
    if (grid > sms) grid = sms;
    if (grid < 1) grid = 1;
    cudaMemsetAsync(&P.stats[SS_HIST_HEAD], 0, sizeof(unsigned long long), st);
    const size_t smem = sizeof(uint32_t) * ((size_t)kMainWords + 2 * ((size_t)1 << kSideLog2) + 8);
    allow_max_smem(k_histogram_runs);
    k_histogram_runs<<<(int)grid, kRunThreads, smem, st>>>(P, samples, (int64_t)n, head, chunk_tiles);
    ++*launches;
    return;
  }
  if (variant == 1) launch_variant<512, 13, 4>(P, samples, n, st, sms, 2);
  else if (variant == 2) launch_variant<1024, 14, 4>(P, samples, n, st, sms, 1);
  else launch_variant<256, 13, 8>(P, samples, n, st, sms, 3);  // 3
  ++*launches;
}

}  // namespace gpa
