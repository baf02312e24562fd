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
// shared memory holds a window of 32-bit counters over up to 2,078
// consecutive instructions of the run's kernel, and a 4,096-entry hash.
// A kernel that fits is windowed whole; for a larger one the window is placed
// where most of the tile's first 32 samples fall. The first sample of each
// tile names the kernel; a new kernel flushes the window to the 64-bit global
// counters and places it again.
// A sample inside the window is one shared-memory reduction (no return value,
// predicated on the window test: no branch) on its counter; any other valid
// sample (another kernel at a run boundary, or a pc outside a partial window)
// goes to the hash, and a key that finds no slot within four probes to its
// global counter. The hash is flushed when half full, and window and hash at
// least every 2^16 tiles (fewer than 2^30 increments: no 32-bit count wraps)
// and at the end.
constexpr int kRunThreads = 1024;
#ifndef GPA_RUN_VEC
#define GPA_RUN_VEC 4
#endif
#ifndef GPA_RUN_CHUNK
#define GPA_RUN_CHUNK 16
#endif
constexpr int kRunVec = GPA_RUN_VEC;                  // 16-byte vectors per thread per tile
constexpr int kRunTile = kRunThreads * kRunVec;       // vectors per tile (8,192 samples)
constexpr int kMainWords = 49872;                     // 195 KB of 32-bit window counters, 24 per instruction
constexpr uint32_t kWinInstr = kMainWords / 24u;      // 2,078 instructions
constexpr int kSideLog2 = 12;                         // 4,096-entry hash
constexpr int kRunFlushTiles = 1 << 16;               // forced flush: keeps 32-bit counts below 2^30
constexpr int kRunChunk = GPA_RUN_CHUNK;              // tiles per claimed chunk
static_assert((long long)kRunFlushTiles * 2 * kRunTile < (1ll << 30), "32-bit counts could wrap between flushes");
static_assert(kMainWords % 24 == 0, "the window holds whole instructions (24 words each)");
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

// Start of the window over a kernel of n instructions: 0 when it fits,
// else the start, among windows centred on the first 8 of the tile's first 32
// samples of that kernel, that holds most of those 32 (`x`, this lane's;
// lanes past the stream pass have ok == false). Every warp reads the same 32
// samples and reaches the same answer.
__device__ __forceinline__ uint32_t window_start(uint64_t x, bool ok, uint32_t kernel, uint32_t n) {
  if (n <= kWinInstr) return 0u;
  const uint32_t pc = (uint32_t)(x >> 24) & 0xFFFFFFu;
  const bool mine = ok && (uint32_t)(x >> 48) == kernel && pc < n;
  uint32_t lo = pc > kWinInstr / 2u ? pc - kWinInstr / 2u : 0u;
  if (lo > n - kWinInstr) lo = n - kWinInstr;
  uint32_t best = 0u, best_lo = 0u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const uint32_t lo_c = __shfl_sync(0xffffffffu, lo, c);
    const bool cand = __shfl_sync(0xffffffffu, mine, c);
    const uint32_t hits = (uint32_t)__popc(__ballot_sync(0xffffffffu, mine && pc - lo_c < kWinInstr));
    if (cand && hits > best) { best = hits; best_lo = lo_c; }
  }
  return best_lo;
}

__global__ void __launch_bounds__(kRunThreads, 1) k_histogram_runs(Prog P, const uint64_t* __restrict__ s,
                                                                   int64_t n, int head) {
  extern __shared__ __align__(16) uint32_t sm[];
  uint32_t* win = sm;                                     // kMainWords window counters
  const uint32_t win_base = (uint32_t)__cvta_generic_to_shared(win);
  uint32_t* skey = sm + kMainWords;                       // hash
  uint32_t* sval = skey + (1 << kSideLog2);
  int* ctl = reinterpret_cast<int*>(sval + (1 << kSideLog2));  // 1: hash fill
  for (int t = threadIdx.x; t < (1 << kSideLog2); t += kRunThreads) { skey[t] = kNoKey; sval[t] = 0u; }
  if (threadIdx.x < 8) ctl[threadIdx.x] = 0;
  __syncthreads();
  const int32_t* foff = P.func_instr_off;  // read through the cache: the window takes the shared memory
  const int lane = threadIdx.x & 31;
  uint32_t bad = 0, side_ins = 0;
  // The windowed kernel's first instruction and size (kept in registers: a
  // miss of that kernel needs no offset lookup).
  uint32_t mode_first = 0, mode_n = 0;
  int mode = -1;
  // A sample that is not in the window: the hash, else its global counter.
  auto count_other = [&](uint64_t x) {
    uint32_t key;
    if ((int)(x >> 48) == mode) {
      const uint32_t pc = (uint32_t)(x >> 24) & 0xFFFFFFu, f5 = (uint32_t)(x >> 19) & 31u;
      key = (pc < mode_n && ((kValid5 >> f5) & 1u) && (x & 0x7FFull) == 0ull) ? (mode_first + pc) * 24u + f5
                                                                                : kNoKey;
    } else {
      key = sample_key(x, foff, P.nf);
    }
    if (key == kNoKey) ++bad;
    else if (!table_add<kSideLog2, 4>(skey, sval, key, 1u, side_ins)) atomicAdd(P.cnt + key, 1ull);
  };

  // Whole tiles go through the window; what is left (an 8-byte-aligned first
  // sample, the vectors after the last whole tile, an odd last sample) is
  // counted by the first CTA through the hash.
  const ulonglong2* v2 = reinterpret_cast<const ulonglong2*>(s + head);
  const uint64_t* s2 = s + head;
  const int64_t n2 = (n - head) / 2;
  const int64_t n_tiles = n2 / kRunTile;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) {
      for (int64_t t = 0; t < head; ++t) count_other(s[t]);
      for (int64_t t = head + 2 * n2; t < n; ++t) count_other(s[t]);
    }
    for (int64_t v = n_tiles * kRunTile + threadIdx.x; v < n2; v += kRunThreads) {
      const ulonglong2 x = load_stream(v2 + v);
      count_other(x.x);
      count_other(x.y);
    }
  }

  // The window: kernel `mode` (-1: none), instructions [lo, lo + wn), whose
  // counters start at global index base; the counter of (pc, f5), f5 the
  // 5-bit (class, latency) field, is word (pc - lo) * 24 + f5.
  // With r = bits 19..50 of a sample (f5 | pc << 5 | low 3 kernel bits << 29),
  // a sample of kernel `mode` is in the window when r - first5 < span5,
  // first5 = (mode << 29) | (lo << 5), span5 = wn << 5.
  uint32_t lo = 0, wn = 0, base = 0, mode_hi = 0, first5 = 0, span5 = 0;
  // The window holds wn * 24 words (a multiple of 4: read and cleared as 16-byte vectors).
  auto flush_win = [&]() {
    const uint32_t quads = wn * 6u;
    for (uint32_t q = threadIdx.x; q < quads; q += kRunThreads) {
      const uint4 v = reinterpret_cast<const uint4*>(win)[q];
      const uint32_t c[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (c[e]) atomicAdd(P.cnt + base + 4u * q + e, (unsigned long long)c[e]);
    }
  };

  // Tiles are handed out in chunks of kRunChunk consecutive tiles from a
  // counter (one chunk ahead, so the last tile of a chunk can prefetch the
  // first of the next): an SM that meets cheap runs takes more of them.
  const int64_t n_chunks = (n_tiles + kRunChunk - 1) / kRunChunk;
  __shared__ long long s_claim;
  auto claim = [&]() -> int64_t {
    if (threadIdx.x == 0) s_claim = (long long)atomicAdd(&P.stats[SS_HIST_HEAD], 1ull);
    __syncthreads();
    const int64_t c = s_claim;
    __syncthreads();
    return c < n_chunks ? c : n_chunks;
  };
  int64_t chunk = claim();
  int64_t upcoming = chunk < n_chunks ? claim() : n_chunks;
  int64_t g = chunk * kRunChunk, g_end = min(g + kRunChunk, n_tiles);
  auto next_tile = [&]() -> int64_t {
    return g + 1 < g_end ? g + 1 : (upcoming < n_chunks ? upcoming * kRunChunk : -1);
  };
  auto advance = [&]() {
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
  };
  // A tile's vectors, and its first sample's kernel (every thread loads that
  // word: one broadcast load per warp, issued with the tile's own loads).
  auto load_tile = [&](int64_t t, ulonglong2* v, uint32_t& k0) {
#pragma unroll
    for (int u = 0; u < kRunVec; ++u) v[u] = load_stream(v2 + t * kRunTile + u * kRunThreads + threadIdx.x);
    k0 = __ldg(reinterpret_cast<const unsigned int*>(s2 + 2 * t * kRunTile) + 1) >> 16;
  };

  // Tiles since the hash was last flushed (the window is flushed at every
  // kernel change as well, so this bounds both).
  int since = 0;
  int64_t t_count = 0;
  auto process = [&](const ulonglong2* v, uint32_t k0) {
    const int want = k0 < (uint32_t)P.nf ? (int)k0 : -1;
    const bool periodic = ++since >= kRunFlushTiles;  // keeps the 32-bit counts small
    if (want != mode || periodic) {
      if (periodic) since = 0;
      __syncthreads();
      flush_win();
      if (periodic) table_flush<kSideLog2>(skey, sval, P.cnt);
      __syncthreads();
      if (periodic && threadIdx.x == 0) ctl[1] = 0;
      mode = want;
      lo = wn = 0;
      mode_first = mode_n = 0;
      if (mode >= 0) {
        const uint32_t n_instr = (uint32_t)(foff[mode + 1] - foff[mode]);
        mode_first = (uint32_t)foff[mode];
        mode_n = n_instr;
        lo = window_start(__ldg(reinterpret_cast<const unsigned long long*>(s2 + 2 * g * kRunTile + lane)), true,
                          (uint32_t)mode, n_instr);
        wn = min(n_instr, kWinInstr);
        base = ((uint32_t)foff[mode] + lo) * 24u;
        for (uint32_t q = threadIdx.x; q < wn * 6u; q += kRunThreads)
          reinterpret_cast<uint4*>(win)[q] = make_uint4(0u, 0u, 0u, 0u);
      }
      mode_hi = (uint32_t)max(mode, 0) << 16;
      first5 = ((uint32_t)max(mode, 0) << 29) | (lo << 5);
      span5 = wn << 5;
      __syncthreads();
    }
    // One predicated shared-memory reduction per window sample (no return
    // value to wait for, no branch).
    uint32_t slow = 0;
#pragma unroll
    for (int u = 0; u < kRunVec; ++u) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint64_t x = h ? v[u].y : v[u].x;
        const uint32_t xl = (uint32_t)x, xh = (uint32_t)(x >> 32);
        const uint32_t rel = __funnelshift_r(xl, xh, 19) - first5;
        const bool hit = rel < span5 && ((xh ^ mode_hi) >> 16) == 0u && ((kValid5 >> (rel & 31u)) & 1u) &&
                         (xl & 0x7FFu) == 0u;
        const uint32_t idx = rel - ((rel >> 5) << 3);  // (pc - lo) * 24 + f5
        const uint32_t addr = win_base + 4u * idx;
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t@p red.shared.add.u32 [%0], 1;\n\t}"
                     :: "r"(addr), "r"((uint32_t)hit) : "memory");
        if (!hit) slow |= 1u << (2 * u + h);
      }
    }
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
    // every 32 tiles: flush the hash if half full
    if ((++t_count & 31) == 0) {
      if (side_ins) atomicAdd(&ctl[1], (int)side_ins);
      side_ins = 0;
      __syncthreads();
      const bool side_full = ctl[1] > (1 << kSideLog2) / 2;
      __syncthreads();
      if (side_full) {
        table_flush<kSideLog2>(skey, sval, P.cnt);
        since = 0;
        __syncthreads();
        if (threadIdx.x == 0) ctl[1] = 0;
      }
    }
  };

  // Two register sets in turn: one tile is counted while the next is loaded.
  ulonglong2 va[kRunVec], vb[kRunVec];
  uint32_t ka = 0, kb = 0;
  if (chunk < n_chunks) load_tile(g, va, ka);
  while (chunk < n_chunks) {
    int64_t nx = next_tile();
    if (nx >= 0) load_tile(nx, vb, kb);
    process(va, ka);
    advance();
    if (chunk >= n_chunks) break;
    nx = next_tile();
    if (nx >= 0) load_tile(nx, va, ka);
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
    const size_t smem = sizeof(uint32_t) * ((size_t)kMainWords + 2 * ((size_t)1 << kSideLog2) + 8);
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
