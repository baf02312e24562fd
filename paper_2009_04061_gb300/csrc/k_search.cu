// Step (b)/(c), general backward searches (Sec. 4): immediate sources of a
// stalled use j through resource r whose value may come from outside j's
// block, with the three pruning rules evaluated over the set of source paths.
//
// One search group per (use, resource) task: a warp in the first three tiers,
// a whole CTA in the fourth (searches of tens of thousands to millions of
// nodes). The graph of (block, literal set) nodes lives in the group's arena:
// shared memory for the common small searches, global memory for the few that
// outgrow it (same code). The group's threads scan node blocks in parallel
// through per-block event lists (defs and unguarded reads, bottom-up), insert
// nodes and sources into open-addressing hashes together, relax distances and
// propagate reachability bits over frontiers with atomics, and run the
// layered longest paths as level-synchronous frontiers; rank 0 only resets
// counters between steps. The first tier's searches (at most 64 nodes, two or
// three nodes a wave) run pass A, rule 2's reachability and the longest paths
// on one thread instead (worklist queues reaching the same fixpoints): there
// the warp-wide protocol of a wave cost more than the work it spread.
//
// Node 0 is the part of j's block above j, already scanned by the local pass
// (its sources are settled there). A node's d is the shortest distance from
// the last instruction of its block to j. Pass A grows the graph in distance
// order up to `bound`, the largest latency of any def of r in the function: a
// source farther than that fails rule 3 whatever the rest of the graph holds.
// Only if some source is within its latency does pass B complete the graph,
// which rule 2 and the longest paths need; when pass B adds no node, pass A's
// distances are already those of the whole graph.
#include <algorithm>

#include "gpa_internal.cuh"

namespace gpa {

namespace {

constexpr int kInf = 0x3FFFFFFF;
constexpr uint32_t kBackBit = 0x80000000u;
constexpr int kExpanded = 1;
constexpr int kWarpsPerCta = 4;

struct Arena {
  int N, E, O, SRC, L;
  int *blk, *S, *wall, *k, *e0, *e1, *fl, *seen, *ord, *tmp, *grp, *q;  // per node
  unsigned long long* dpk;  // (shortest distance << 32) | parent node
  unsigned long long* sdb;  // per source: (shortest distance << 32) | nearest occurrence
  int *dl, *ht, *hused, *eto, *on, *ox, *onext;
  int *wblk, *wpos, *wneed;
  int *si, *sk, *sp, *shead;
  int* ctr;  // 0 nodes, 1 edges, 2 occurrences, 3 hash slots used, 4 overflow, 5 scratch
};

__host__ __device__ inline int64_t arena_bytes(int N, int SRC, int L) {
  const int64_t E = 2 * (int64_t)N, O = N;
  int64_t ints = 12 * (int64_t)N + (int64_t)L * N + 2 * (int64_t)N + N + E + 3 * O + 3 * (int64_t)N + 4 * (int64_t)SRC + 8;
  return 8 * (int64_t)N + 8 * (int64_t)SRC + ((ints * 4 + 15) & ~(int64_t)15);
}

__device__ Arena carve(char* base, int N, int SRC, int L, int* ctr) {
  Arena a;
  a.N = N; a.E = 2 * N; a.O = N; a.SRC = SRC; a.L = L;
  a.dpk = reinterpret_cast<unsigned long long*>(base);
  a.sdb = a.dpk + N;
  int* p = reinterpret_cast<int*>(base + 8 * (int64_t)N + 8 * (int64_t)SRC);
  int** node_arrays[12] = {&a.blk, &a.S, &a.wall, &a.k, &a.e0, &a.e1, &a.fl, &a.seen, &a.ord, &a.tmp, &a.grp, &a.q};
  for (int t = 0; t < 12; ++t) { *node_arrays[t] = p; p += N; }
  a.dl = p; p += (int64_t)L * N;
  a.ht = p; p += 2 * N;
  a.hused = p; p += N;
  a.eto = p; p += a.E;
  a.on = p; p += a.O; a.ox = p; p += a.O; a.onext = p; p += a.O;
  a.wblk = p; p += N; a.wpos = p; p += N; a.wneed = p; p += N;
  a.si = p; p += SRC; a.sk = p; p += SRC; a.sp = p; p += SRC; a.shead = p; p += SRC;
  a.ctr = ctr;
  return a;
}

__device__ __forceinline__ uint32_t node_hash(int blk, int S) {
  uint32_t h = (uint32_t)blk * 0x9E3779B1u ^ ((uint32_t)S * 0x85EBCA77u);
  h ^= h >> 15;
  return h;
}

// A hint that brings the line holding p into this SM's L1 (no register is
// written, so nothing waits for it).
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(__cvta_generic_to_global(p)));
}

__device__ __forceinline__ int dist_of(const Arena& a, int u) { return (int)(a.dpk[u] >> 32); }
__device__ __forceinline__ int par_of(const Arena& a, int u) { return (int)(a.dpk[u] & 0xFFFFFFFFull); }

// The threads that run one search together: a warp (tiers 1-3) or a whole
// CTA (the fourth tier's very large searches). Both give the search the same
// steps: a barrier, an any-vote, exclusive prefix counts, inclusive sums and
// reductions over the group, a read of a shared flag that every thread takes
// before any of them may change it, and a broadcast from rank 0.
struct WarpGroup {
  static constexpr int kSize = 32;
  __device__ __forceinline__ int rank() const { return threadIdx.x & 31; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
  __device__ __forceinline__ bool any(bool p) const { return __any_sync(0xffffffffu, p); }
  // exclusive prefix count of `pred`: this thread's slot; *total over the group
  __device__ __forceinline__ int slot(bool pred, int* total) const {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    *total = __popc(m);
    return __popc(m & ((1u << (threadIdx.x & 31)) - 1u));
  }
  __device__ __forceinline__ int inclusive_sum(int x, int* total) const {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    *total = __shfl_sync(0xffffffffu, x, 31);
    return x;
  }
  __device__ __forceinline__ int sum(int x) const {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  }
  __device__ __forceinline__ int max(int x) const {
    for (int o = 16; o > 0; o >>= 1) x = ::max(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
  }
  __device__ __forceinline__ int min(int x) const {
    for (int o = 16; o > 0; o >>= 1) x = ::min(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
  }
  __device__ __forceinline__ int read(const volatile int* p) const { return *p; }
  __device__ __forceinline__ unsigned long long broadcast(unsigned long long v) const {
    return __shfl_sync(0xffffffffu, v, 0);
  }
};

constexpr int kCtaThreads = 512;  // threads of a fourth-tier search CTA

// A CTA as one search group. `red` is shared scratch of kCtaThreads / 32
// ints, `cast` a shared 64-bit slot for broadcasts. Every collective ends with
// a barrier, so the scratch is free again when it returns.
struct CtaGroup {
  static constexpr int kSize = kCtaThreads;
  static constexpr int kWarps = kCtaThreads / 32;
  int* red;
  unsigned long long* cast;
  __device__ __forceinline__ int rank() const { return threadIdx.x; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
  __device__ __forceinline__ bool any(bool p) const { return __syncthreads_or(p) != 0; }
  // a value per warp (its last lane's) -> the sum over the warps before this
  // thread's; *total: the sum over all warps
  __device__ __forceinline__ int warp_offsets(int v, int* total) const {
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 31) red[w] = v;
    __syncthreads();
    int before = 0, all = 0;
#pragma unroll
    for (int i = 0; i < kWarps; ++i) {
      const int c = red[i];
      before += i < w ? c : 0;
      all += c;
    }
    __syncthreads();
    *total = all;
    return before;
  }
  __device__ __forceinline__ int slot(bool pred, int* total) const {
    const unsigned m = __ballot_sync(0xffffffffu, pred);
    const int lane = threadIdx.x & 31;
    return warp_offsets(__popc(m), total) + __popc(m & ((1u << lane) - 1u));
  }
  __device__ __forceinline__ int inclusive_sum(int x, int* total) const {
    const int lane = threadIdx.x & 31;
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    return warp_offsets(x, total) + x;
  }
  template <class Op>
  __device__ __forceinline__ int reduce(int x, Op op) const {
    for (int o = 16; o > 0; o >>= 1) x = op(x, __shfl_xor_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    int v = red[0];
#pragma unroll
    for (int i = 1; i < kWarps; ++i) v = op(v, red[i]);
    __syncthreads();
    return v;
  }
  __device__ __forceinline__ int sum(int x) const { return reduce(x, [](int p, int q) { return p + q; }); }
  __device__ __forceinline__ int max(int x) const { return reduce(x, [](int p, int q) { return ::max(p, q); }); }
  __device__ __forceinline__ int min(int x) const { return reduce(x, [](int p, int q) { return ::min(p, q); }); }
  __device__ __forceinline__ int read(const volatile int* p) const {
    const int v = *p;
    __syncthreads();
    return v;
  }
  __device__ __forceinline__ unsigned long long broadcast(unsigned long long v) const {
    if (threadIdx.x == 0) *cast = v;
    __syncthreads();
    v = *cast;
    __syncthreads();
    return v;
  }
};

// Returns false when the search outgrew the arena (nothing emitted).
// With P.diag, the search counts the sources of (j, r) before and after
// pruning into use entry e (`blocked`: an unguarded reader above j in its
// block prunes them all by rule 2) and emits nothing.
template <class G>
__device__ bool group_search(const G& g, const Prog& P, const Arch& A, const Arena& a, int j, int r, uint16_t S0,
                             int bound, uint16_t live, int tier, int e = 0, bool blocked = false) {
  const int me = g.rank();
#ifdef GPA_PHASE_TIMING
  long long t_prev = clock64();
  const long long t_begin = t_prev;
  long long t_prev_total = t_prev;
  unsigned long long ph[5] = {0, 0, 0, 0, 0};
  unsigned long long r2runs = 0;
  auto phase = [&](int i) {
    if (me == 0) {
      const long long t = clock64();
      atomicAdd(&P.stats[SS_PHASE + (min(tier, 3) - 1) * 6 + i], (unsigned long long)(t - t_prev));
      ph[i] = (unsigned long long)(t - t_prev);
      t_prev = t;
      if (i == 4 || i == 0) {
        const int nn = max(((volatile int*)a.ctr)[0], 1);
        if (i == 4 || i == 0)
          atomicAdd(&P.stats[SS_SIZE_CYC + min(15, 31 - __clz(nn))], (unsigned long long)(t - t_prev_total));
        t_prev_total = t;
        const unsigned long long key = ((unsigned long long)(t - t_begin) << 20) | (unsigned long long)min(((volatile int*)a.ctr)[0], 0xFFFFF);
        if (atomicMax(&P.stats[SS_SLOW], key) < key) {
          P.stats[SS_SLOW + 1] = r2runs;
          for (int q = 0; q < 5; ++q) P.stats[SS_SLOW + 2 + q] = ph[q];
        }
      }
    }
  };
#else
  auto phase = [](int) {};
#endif
  const int gj = P.guard[j];
  const int b0 = P.instr_block[j];
  const int first0 = P.block_meta[2 * (size_t)b0].x;
  const int w = r >> 5;
  const uint32_t bit = 1u << (r & 31);
  const uint32_t hmask = (uint32_t)(2 * a.N - 1);
  volatile int* ctr = a.ctr;

  // Unexpanded nodes are kept in a list (alternating between seen and tmp,
  // both free until rule 2): ubuf holds ctr[6] of them.
  int* ubuf = a.seen;
  int* ukeep = a.tmp;
  if (me == 0) {
    ctr[0] = 1; ctr[1] = 0; ctr[2] = 0; ctr[3] = 0; ctr[4] = 0; ctr[5] = 0; ctr[6] = 1;
    ubuf[0] = 0;
    S0 = keep_literals(S0, live);
    a.blk[0] = b0; a.S[0] = (int)S0 | ((int)S0 << 16); a.wall[0] = -1; a.fl[0] = 0;
    a.dpk[0] = 0ull; a.k[0] = 0; a.e0[0] = 0; a.e1[0] = 0;
  }
  g.sync();

  // Self-checks of the arena invariants before indexed accesses: an edge
  // range inside [0, edges) here, each target inside [0, nodes) where it is
  // read (target_ok). A violation is recorded as ST_OVERFLOW and the access
  // skipped.
  auto edges_ok = [&](int u, int) {
    const int e0 = a.e0[u], e1 = a.e1[u];
    if (e0 < 0 || e1 < e0 || e1 > a.E || e1 > ctr[1]) { set_status(P, ST_OVERFLOW); return false; }
    return true;
  };
  auto target_ok = [&](int v, int n_now) {
    if ((unsigned)v < (unsigned)n_now) return true;
    set_status(P, ST_OVERFLOW);
    return false;
  };
  auto wout = [&](int u) {
    if (u == 0) return j - first0 + 1;
    const int4 m = P.block_meta[2 * (size_t)a.blk[u]];
    return m.y - m.x;
  };
  auto last_of = [&](int u) { return P.block_meta[2 * (size_t)a.blk[u]].y - 1; };

  // Scan node u's block bottom-up through its events of r's bucket (one
  // thread). Records occurrences, the literal set leaving the top and the first
  // unguarded reader of r met (the wall). Sets a.fl[u] bit 2 if the scan
  // stopped (covered). `first` is the block's first instruction and
  // [ev_beg, ev_end) its segment of r's bucket, empty when no instruction of
  // the block defines r or reads it unguarded (loaded by the caller together
  // with the block's other records).
  auto scan = [&](int u, int first, int ev_beg, int ev_end) {
    uint16_t S = (uint16_t)(a.S[u] & 0xFFFF);
    bool stop = false;
    if (u != 0) {
      const int B = a.blk[u];
      int wall = -1;
      {
        int last_def_pos = -1;
        // Events four at a time: independent read-only loads in flight together
        // (a sentinel resource 511 pads the last group).
        for (int e0 = ev_beg; e0 < ev_end && !stop; e0 += 4) {
          uint32_t evs[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) evs[q] = e0 + q < ev_end ? __ldg(&P.events[e0 + q]) : 0x1FFu;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t ev = evs[q];
            if (stop || (int)(ev & 0x1FFu) != r) continue;
            const int pos = (int)(ev >> 16), x = first + pos;
            if (ev & 0x200u) {  // def of r
              last_def_pos = pos;
              if (!contains(S, gj) && !(B == b0 && x < j)) {  // sources above j in its block are settled
                const int o = atomicAdd((int*)&a.ctr[2], 1);
                if (o < a.O) { a.on[o] = u; a.ox[o] = x; } else { a.ctr[4] = 3; }
              }
              S = add_literal(S, (int)((ev >> 12) & 0xFu));
              if (contains(S, gj)) stop = true;
            } else if (wall < 0 && pos != last_def_pos && x != j) {  // unguarded reader of r
              wall = x;
            }
          }
        }
      }
      a.wall[u] = wall;
    }
    a.S[u] = (a.S[u] & 0xFFFF) | ((int)keep_literals(S, live) << 16);
    a.fl[u] |= kExpanded | (stop ? 4 : 0);
  };

  // Link the predecessors of the listed nodes, lanes over nodes. Edge ranges
  // come from a warp prefix count; the (block, literal set) nodes are found or
  // added with a warp-synchronous insert: a lane claims an empty slot with
  // atomicCAS, allocates and publishes the node in the same round, and lanes
  // that met a claim in progress retry the slot in the next round.
  // pm: the node's predecessor record (range, first two predecessors);
  // ro0 / ro1: the reach words of those two (loaded before the scan).
  auto link_chunk = [&](const int* lst, int cnt, int4 pm, uint32_t ro0, uint32_t ro1, bool relax) {
    const bool mine = me < cnt;
    const int u = mine ? lst[me] : 0;
    const int B = mine ? a.blk[u] : 0;
    const int Sout = mine ? ((a.S[u] >> 16) & 0xFFFF) : 0;
    const bool open = mine && !(a.fl[u] & 4);
    if (!open) pm = make_int4(0, 0, -1, -1);
    // whether a def of r reaches out of the predecessor at q, and that predecessor
    auto reaches = [&](int q) -> bool {
      const int k = q - pm.x;
      if (k == 0) return ro0 & bit;
      if (k == 1) return ro1 & bit;
      return P.rout[(size_t)__ldg(&P.pred[q]) * kWords + w] & bit;
    };
    auto pred_at = [&](int q) -> int {
      const int k = q - pm.x;
      return k == 0 ? pm.z : k == 1 ? pm.w : __ldg(&P.pred[q]);
    };
    int deg = 0;
    for (int q = pm.x; q < pm.y; ++q) deg += reaches(q) ? 1 : 0;
    int total;
    const int incl = g.inclusive_sum(deg, &total);
    const int ne = ctr[1];
    if (ne + total > a.E) { if (me == 0) ctr[4] = 2; g.sync(); return; }
    if (mine) { a.e0[u] = ne + incl - deg; a.e1[u] = ne + incl; }
    const int maxdeg = g.max(deg);
    // Pass A relaxes each new edge as it is linked, from u's distance now
    // (packed with u as the parent); an expanded target that improves is
    // queued in ord for relax_from, which carries the change on. A node whose
    // own distance improves meanwhile is such a target, so its edges are
    // relaxed again from the better distance.
    unsigned long long nd_u = ~0ull;
    if (relax && mine) {
      const int du = dist_of(a, u);
      if (du < kInf) nd_u = ((unsigned long long)(du + wout(u)) << 32) | (unsigned)u;
    }
    int qp = pm.x;
    for (int kk = 0; kk < maxdeg; ++kk) {
      bool pending = kk < deg;
      int p = -1;
      if (pending) {
        while (!reaches(qp)) ++qp;
        p = pred_at(qp++);
      }
      uint32_t h = pending ? (node_hash(p, Sout) & hmask) : 0;
      int v = -1;
      for (int round = 0; round < 4 * (int)hmask + 64; ++round) {
        if (!g.any(pending)) break;
        if (pending) {
          const int c = a.ht[h];
          if (c >= 0) {
            if (a.blk[c] == p && (a.S[c] & 0xFFFF) == Sout) { v = c; pending = false; }
            else h = (h + 1) & hmask;
          } else if (c == -1) {
            if (atomicCAS(&a.ht[h], -1, -2 - me) == -1) {
              const int nv = atomicAdd((int*)&a.ctr[0], 1);
              if (nv >= a.N) {
                a.ctr[4] = 1; a.ht[h] = -1; pending = false;
              } else {
                a.blk[nv] = p; a.S[nv] = Sout; a.wall[nv] = -1; a.fl[nv] = 0; a.k[nv] = kInf;
                a.e0[nv] = 0; a.e1[nv] = 0;  // no out-edges until the node is expanded
                a.dpk[nv] = ((unsigned long long)kInf << 32) | 0xFFFFFFFFull;
                a.hused[atomicAdd((int*)&a.ctr[3], 1)] = (int)h;
                ubuf[atomicAdd((int*)&a.ctr[6], 1)] = nv;
                __threadfence_block();
                a.ht[h] = nv;
                v = nv; pending = false;
              }
            }
          }  // c <= -2: another lane is publishing this slot; look again next round
        }
        g.sync();
      }
      if (pending) a.ctr[4] = 6;  // the round limit is a bound, not expected to be reached
      if (kk < deg && v >= 0) a.eto[a.e0[u] + kk] = v | (p >= B ? (int)kBackBit : 0);
      if (relax && kk < deg && v >= 0 && nd_u < a.dpk[v] && atomicMin(&a.dpk[v], nd_u) > nd_u &&
          (a.fl[v] & kExpanded) && !(atomicOr(&a.fl[v], 8) & 8))
        a.ord[atomicAdd((int*)&a.ctr[5], 1)] = v;
    }
    g.sync();
    if (me == 0) ctr[1] = ne + total;
    g.sync();
  };

  // Expand every listed node: parallel scans, then parallel linking.
  auto expand_list = [&](const int* list, int cnt, bool relax) {
    for (int c0 = 0; c0 < cnt; c0 += G::kSize) {
      int4 pm = make_int4(0, 0, -1, -1);
      uint32_t ro0 = 0u, ro1 = 0u;
      if (c0 + me < cnt) {
        const int u = list[c0 + me];
        const int B = a.blk[u];
        // First round of loads, all independent: the block's two records, the
        // touch word of r and the bounds of r's event segment.
        pm = __ldg(&P.block_meta[2 * (size_t)B + 1]);
        const int first = __ldg(&P.block_meta[2 * (size_t)B].x);
        const uint32_t tw = __ldg(&P.touch_mask[(size_t)B * kWords + w]);
        const size_t seg = (size_t)B * kEvBuckets + ev_bucket(r);
        const int ev_beg = __ldg(&P.ev_off[seg]);
        int ev_end = __ldg(&P.ev_off[seg + 1]);
        ev_end = (tw & bit) ? ev_end : ev_beg;  // an untouched block has nothing to scan
        // Second round: the reach words of the first two predecessors (read
        // when linking), and the first two predecessors' records, fetched into
        // L1 for the wave that expands them; the scan's event loads follow.
        if (pm.z >= 0) {
          ro0 = P.rout[(size_t)pm.z * kWords + w];
          prefetch_l1(&P.block_meta[2 * (size_t)pm.z]);
          prefetch_l1(&P.touch_mask[(size_t)pm.z * kWords + w]);
          prefetch_l1(&P.ev_off[(size_t)pm.z * kEvBuckets + ev_bucket(r)]);
        }
        if (pm.w >= 0) {
          ro1 = P.rout[(size_t)pm.w * kWords + w];
          prefetch_l1(&P.block_meta[2 * (size_t)pm.w]);
          prefetch_l1(&P.touch_mask[(size_t)pm.w * kWords + w]);
          prefetch_l1(&P.ev_off[(size_t)pm.w * kEvBuckets + ev_bucket(r)]);
        }
        scan(u, first, ev_beg, ev_end);
      }
      g.sync();
      if (ctr[4]) return;
      link_chunk(list + c0, min(G::kSize, cnt - c0), pm, ro0, ro1, relax);
      if (g.read(&ctr[4])) return;  // the next chunk's scans may set it
    }
  };

  // Worklist relaxation from the listed nodes: improved targets join the next
  // frontier once (flag bit 8 of fl). mode 0: shortest distance with parent
  // (64-bit atomicMin on (d << 32) | parent); mode 1: fewest back edges.
  // Frontiers live in ord / grp, which are free until rule 2.
  auto relax_from = [&](const int* start, int cnt, int mode) {
    int* cur = a.ord;
    int* nxt = a.grp;
    for (int t = me; t < cnt; t += G::kSize) cur[t] = start[t];
    if (me == 0) ctr[5] = 0;
    g.sync();
    int fsize = cnt;
    while (fsize > 0) {
      for (int f0 = 0; f0 < fsize; f0 += G::kSize) {
        if (f0 + me >= fsize) continue;
        const int u = cur[f0 + me];
        atomicAnd(&a.fl[u], ~8);
        const int n_now = ctr[0];
        if (!edges_ok(u, n_now)) continue;
        if (mode == 0) {
          const int du = dist_of(a, u);
          if (du >= kInf) continue;
          const unsigned long long nd = (unsigned long long)(du + wout(u)) << 32 | (unsigned)u;
          for (int e = a.e0[u]; e < a.e1[u]; ++e) {
            const int v = a.eto[e] & 0x7FFFFFFF;
            if (!target_ok(v, n_now)) break;
            if (nd < a.dpk[v] && atomicMin(&a.dpk[v], nd) > nd && !(atomicOr(&a.fl[v], 8) & 8))
              nxt[atomicAdd((int*)&a.ctr[5], 1)] = v;
          }
        } else {
          const int ku = a.k[u];
          if (ku >= kInf) continue;
          for (int e = a.e0[u]; e < a.e1[u]; ++e) {
            const int v = a.eto[e] & 0x7FFFFFFF;
            if (!target_ok(v, n_now)) break;
            const int kb = ku + (int)((uint32_t)a.eto[e] >> 31);
            if (kb < a.k[v] && atomicMin(&a.k[v], kb) > kb && !(atomicOr(&a.fl[v], 8) & 8))
              nxt[atomicAdd((int*)&a.ctr[5], 1)] = v;
          }
        }
      }
      g.sync();
      fsize = ctr[5];
      g.sync();
      if (me == 0) ctr[5] = 0;
      int* sw = cur; cur = nxt; nxt = sw;
      g.sync();
    }
  };

  // Pass B only needs the nodes that can lie on a path from a candidate
  // source up to j: the node's block must be reachable in the CFG from the
  // candidate's block, so it is not below that block's smallest reachable
  // block. cand_low is the least of these over the candidates.
  int cand_low = 0;
  auto relevant = [&](int u) { return a.blk[u] >= cand_low; };

  // Split the unexpanded list: nodes to expand now (into list) and the rest,
  // which stay unexpanded (all of them when bound < 0; in pass B, nodes off
  // every candidate's paths are dropped from the list for good).
  int* list = a.q;
  auto take_wave = [&](int lim) {
    const int m = ctr[6];
    int cnt = 0, kept = 0;
    for (int i0 = 0; i0 < m; i0 += G::kSize) {
      const int i = i0 + me;
      const int u = i < m ? ubuf[i] : 0;
      const bool now = i < m && (lim < 0 ? relevant(u) : dist_of(a, u) <= lim);
      const bool keep = i < m && !now && lim >= 0;
      int tot_now, tot_keep;
      const int at_now = g.slot(now, &tot_now);
      const int at_keep = g.slot(keep, &tot_keep);
      if (now) list[cnt + at_now] = u;
      if (keep) ukeep[kept + at_keep] = u;
      cnt += tot_now;
      kept += tot_keep;
    }
    g.sync();
    int* sw = ubuf; ubuf = ukeep; ukeep = sw;
    if (me == 0) ctr[6] = kept;
    g.sync();
    return cnt;
  };

  // Pass A by one thread, for the first tier's small searches: a
  // label-correcting queue (a node is queued when its distance improves and it
  // is expanded or within the bound; a node is expanded once, when first taken
  // within the bound; an expanded node taken again relaxes its edges from its
  // better distance). It reaches the fixpoint of the waves below (every node
  // whose shortest distance over the expanded nodes' edges is within the bound
  // is expanded), without a vote, a prefix count or a claim round per node: a
  // small search's waves are two or three nodes wide, so the warp-wide
  // protocol cost more than the work it spread. The queue is a ring over q
  // (a node is in it at most once at a time).
  auto serial_pass_a = [&]() {
    int* ring = a.q;
    int head = 0, tail = 0, inq = 0;
    int nn = ctr[0], ne = ctr[1], nh = ctr[3];
    auto push = [&](int v) {
      if (a.fl[v] & 8) return;
      a.fl[v] |= 8;
      ring[tail] = v;
      tail = tail + 1 == a.N ? 0 : tail + 1;
      ++inq;
    };
    push(0);
    while (inq > 0) {
      const int u = ring[head];
      head = head + 1 == a.N ? 0 : head + 1;
      --inq;
      a.fl[u] &= ~8;
      const int du = dist_of(a, u);
      if (!(a.fl[u] & kExpanded)) {
        if (du > bound) continue;
        const int B = a.blk[u];
        const int4 pm = __ldg(&P.block_meta[2 * (size_t)B + 1]);
        const int first = __ldg(&P.block_meta[2 * (size_t)B].x);
        const uint32_t tw = __ldg(&P.touch_mask[(size_t)B * kWords + w]);
        const size_t seg = (size_t)B * kEvBuckets + ev_bucket(r);
        const int ev_beg = __ldg(&P.ev_off[seg]);
        int ev_end = __ldg(&P.ev_off[seg + 1]);
        ev_end = (tw & bit) ? ev_end : ev_beg;
        scan(u, first, ev_beg, ev_end);
        if (ctr[4]) break;
        const int Sout = (a.S[u] >> 16) & 0xFFFF;
        a.e0[u] = ne;
        for (int q = (a.fl[u] & 4) ? pm.y : pm.x; q < pm.y; ++q) {
          const int p = q == pm.x ? pm.z : q == pm.x + 1 ? pm.w : __ldg(&P.pred[q]);
          if (!(P.rout[(size_t)p * kWords + w] & bit)) continue;
          if (ne >= a.E) { ctr[4] = 2; break; }
          uint32_t h = node_hash(p, Sout) & hmask;
          int v = -1;
          for (int probe = 0; probe <= (int)hmask; ++probe) {
            const int c = a.ht[h];
            if (c < 0) break;
            if (a.blk[c] == p && (a.S[c] & 0xFFFF) == Sout) { v = c; break; }
            h = (h + 1) & hmask;
          }
          if (v < 0) {
            if (a.ht[h] >= 0) { ctr[4] = 6; break; }  // not reached: 2N slots for at most N nodes
            if (nn >= a.N) { ctr[4] = 1; break; }
            v = nn++;
            a.blk[v] = p; a.S[v] = Sout; a.wall[v] = -1; a.fl[v] = 0; a.k[v] = kInf;
            a.e0[v] = 0; a.e1[v] = 0;
            a.dpk[v] = ((unsigned long long)kInf << 32) | 0xFFFFFFFFull;
            a.hused[nh++] = (int)h;
            a.ht[h] = v;
          }
          a.eto[ne++] = v | (p >= B ? (int)kBackBit : 0);
        }
        a.e1[u] = ne;
        if (ctr[4]) break;
      }
      if (du >= kInf) continue;
      // distance with parent, and fewest back edges, relaxed together
      const unsigned long long nd = ((unsigned long long)(du + wout(u)) << 32) | (unsigned)u;
      const int ku = a.k[u];
      for (int e = a.e0[u]; e < a.e1[u]; ++e) {
        const int v = a.eto[e] & 0x7FFFFFFF;
        const int nk = ku + (int)((uint32_t)a.eto[e] >> 31);
        bool better = false;
        if (nd < a.dpk[v]) { a.dpk[v] = nd; better = true; }
        if (nk < a.k[v]) { a.k[v] = nk; better = true; }
        if (better && ((a.fl[v] & kExpanded) || dist_of(a, v) <= bound)) push(v);
      }
    }
    ctr[0] = nn; ctr[1] = ne; ctr[3] = nh;
  };

  // Pass A expands in waves the nodes within the bound, relaxing as they
  // link (or by one thread, above); pass B, only if some source is within its
  // latency, completes the graph. Both run in this one loop, so the wave code
  // exists once in the kernel (the search kernel is bound by instruction fetch
  // when its warps spread over a larger body).
  bool cand = false, pass_b = false, grew_b = false;
  const bool serial_a = G::kSize == 32 && tier == 1;
  if (serial_a) {
    if (me == 0) serial_pass_a();
    g.sync();
    // pass B starts from the nodes pass A left unexpanded
    const int n_now = ctr[0];
    int m = 0;
    for (int i0 = 0; i0 < n_now; i0 += G::kSize) {
      const int i = i0 + me;
      const bool un = i < n_now && !(a.fl[i] & kExpanded);
      int tot;
      const int at = g.slot(un, &tot);
      if (un) ubuf[m + at] = i;
      m += tot;
    }
    g.sync();
    if (me == 0) ctr[6] = m;
    g.sync();
  }
  while (!ctr[4]) {
    const int cnt = serial_a && !pass_b ? 0 : take_wave(pass_b ? -1 : bound);
    if (cnt > 0) {
      grew_b |= pass_b;
      expand_list(list, cnt, !pass_b);
      if (ctr[4]) break;
      // pass A relaxed the wave's edges as they were linked; carry on from the
      // expanded nodes that improved (queued in ord, counted in ctr[5])
      const int n_dirty = pass_b ? 0 : ctr[5];
      if (n_dirty > 0) relax_from(a.ord, n_dirty, 0);
      continue;
    }
    if (pass_b) break;
    // End of pass A. A source within its latency? (Every candidate is found
    // by pass A: a source farther than the bound fails rule 3.)
    const int no = min(ctr[2], a.O);
    int low = 0x7FFFFFFF;
    for (int o = me; o < no; o += G::kSize) {
      const int u = a.on[o];
      if (dist_of(a, u) + (last_of(u) - a.ox[o]) <= A.lat[P.opclass[a.ox[o]]]) {
        cand = true;
        low = min(low, P.block_minreach[a.blk[u]]);
      }
    }
    cand = g.any(cand);
    cand_low = g.min(low);
    if (!cand) break;
    pass_b = true;
  }
  // Clear the hash slots this search used.
  const int nh = ctr[3];
  for (int t = me; t < nh; t += G::kSize) a.ht[a.hused[t]] = -1;
  g.sync();
  const int n = ctr[0];
  if (me == 0) {
    atomicAdd(&P.stats[SS_GENERAL], 1ull);
    atomicMax(&P.stats[SS_MAX_NODES], (unsigned long long)n);
    atomicMax(&P.stats[SS_MAX_TASK], ((unsigned long long)n << 40) | ((unsigned long long)r << 31) | (unsigned)j);
#ifdef GPA_PHASE_TIMING
    atomicAdd(&P.stats[SS_SIZES + min(15, 31 - __clz(max(n, 1)))], 1ull);
    if (cand) atomicAdd(&P.stats[SS_PASSB], 1ull);
#endif
  }
  phase(0);
  if (ctr[4]) {
    if (me == 0) ctr[7] = ctr[4];
    g.sync();
    return false;
  }
  if (!cand && !P.diag) return true;

  // Shortest distance with parents, and fewest back edges, over the whole
  // graph. When pass B expanded no node, every edge of the graph was relaxed
  // to the fixpoint in pass A, whose (distance, parent) minimum over the same
  // edges is this one; the one-thread pass A relaxes the back-edge counts
  // along with the distances, so its searches then need neither.
  const bool fresh_d = grew_b, fresh_k = grew_b || !serial_a;
  for (int u = me; u < n; u += G::kSize) {
    if (fresh_d) a.dpk[u] = u == 0 ? 0ull : (((unsigned long long)kInf << 32) | 0xFFFFFFFFull);
    if (fresh_k) a.k[u] = u == 0 ? 0 : kInf;
    a.fl[u] &= ~8;
  }
  if (me == 0) a.q[0] = 0;
  g.sync();
#pragma unroll 1
  for (int mode = fresh_d ? 0 : 1; mode < (fresh_k ? 2 : 1); ++mode) relax_from(a.q, 1, mode);
  phase(1);

  // Sources: a warp-synchronous hash keyed by instruction gives each source an
  // index; per source, 64-bit atomicMin keeps (shortest distance, its
  // occurrence), atomicMin the fewest back edges, and the occurrences are
  // chained into a list.
  const int no = ctr[2];
  if (me == 0) { ctr[3] = 0; ctr[5] = 0; }
  g.sync();
  const uint32_t smask = (uint32_t)(2 * a.SRC - 1);
  for (int o0 = 0; o0 < no; o0 += G::kSize) {
    const int o = o0 + me;
    bool pending = o < no;
    const int x = pending ? a.ox[o] : -1;
    uint32_t h = pending ? (((uint32_t)x * 0x9E3779B1u) >> 7) & smask : 0;
    int m = -1;
    for (int round = 0; round < 4 * (int)smask + 64; ++round) {
      if (!g.any(pending)) break;
      if (pending) {
        const int c = a.ht[h];
        if (c >= 0) {
          if (a.si[c] == x) { m = c; pending = false; } else h = (h + 1) & smask;
        } else if (c == -1) {
          if (atomicCAS(&a.ht[h], -1, -2 - me) == -1) {
            const int nm = atomicAdd((int*)&a.ctr[5], 1);
            if (nm >= a.SRC) {
              a.ctr[4] = 4; a.ht[h] = -1; pending = false;
            } else {
              a.si[nm] = x; a.sk[nm] = kInf; a.shead[nm] = -1; a.sp[nm] = 0;
              a.sdb[nm] = ~0ull;
              a.hused[atomicAdd((int*)&a.ctr[3], 1)] = (int)h;
              __threadfence_block();
              a.ht[h] = nm;
              m = nm; pending = false;
            }
          }
        }
      }
      g.sync();
    }
    if (pending) a.ctr[4] = 6;
    if (m >= 0) {
      const int u = a.on[o];
      const int dist = dist_of(a, u) + (last_of(u) - x);
      atomicMin(&a.sdb[m], ((unsigned long long)dist << 32) | (unsigned)o);
      atomicMin(&a.sk[m], a.k[u]);
      a.onext[o] = atomicExch(&a.shead[m], o);
    }
    g.sync();
  }
  {
    const int nh2 = ctr[3];
    for (int t = me; t < nh2; t += G::kSize) a.ht[a.hused[t]] = -1;
  }
  g.sync();
  if (ctr[4]) {
    if (me == 0) ctr[7] = ctr[4];
    g.sync();
    return false;
  }
  const int nsrc = ctr[5];
  int alive = 0;
  for (int m = me; m < nsrc; m += G::kSize) {
    a.sp[m] = (int)(a.sdb[m] >> 32) > A.lat[P.opclass[a.si[m]]] ? 1 : 0;  // rule 3
    if (P.diag == 1 && (blocked || !keeps_any(P, A, j, P.opclass[a.si[m]]))) a.sp[m] = 1;  // rule 2 above j, rule 1
    if (P.diag == 2) a.sp[m] = 0;  // export: rule 2 for every source
    alive += a.sp[m] ? 0 : 1;
  }
  alive = g.sum(alive);
  phase(2);
  if (alive == 0) {
    if (P.diag == 1 && me == 0) cov_add(P, e, nsrc, 0);
    return true;
  }

  // Rule 2. Wall groups, one per block: a hash keyed by block with atomicMax
  // of the positions (the unguarded reader met first from the bottom truncates
  // at least as much as any other reader of that block). A wall can only block
  // source i if it lies on the parent chain of i's nearest occurrence.
  if (me == 0) { ctr[3] = 0; ctr[5] = 0; }
  g.sync();
  for (int u0 = 0; u0 < n; u0 += G::kSize) {
    const int u = u0 + me;
    bool pending = u < n && u != 0 && a.wall[u] >= 0;
    const int B = pending ? a.blk[u] : -1;
    uint32_t h = pending ? (((uint32_t)B * 0x9E3779B1u) >> 5) & hmask : 0;
    int wg = -1;
    for (int round = 0; round < 4 * (int)hmask + 64; ++round) {
      if (!g.any(pending)) break;
      if (pending) {
        const int c = a.ht[h];
        if (c >= 0) {
          if (a.wblk[c] == B) { wg = c; pending = false; } else h = (h + 1) & hmask;
        } else if (c == -1) {
          if (atomicCAS(&a.ht[h], -1, -2 - me) == -1) {
            const int ng = atomicAdd((int*)&a.ctr[5], 1);
            a.wblk[ng] = B; a.wpos[ng] = -1; a.wneed[ng] = 0;
            a.hused[atomicAdd((int*)&a.ctr[3], 1)] = (int)h;
            __threadfence_block();
            a.ht[h] = ng;
            wg = ng; pending = false;
          }
        }
      }
      g.sync();
    }
    if (pending) a.ctr[4] = 6;
    if (u < n) a.grp[u] = wg;
    if (wg >= 0) atomicMax(&a.wpos[wg], a.wall[u]);
    g.sync();
  }
  {
    const int nh2 = ctr[3];
    for (int t = me; t < nh2; t += G::kSize) a.ht[a.hused[t]] = -1;
  }
  g.sync();
  if (ctr[4]) {
    if (me == 0) ctr[7] = ctr[4];
    g.sync();
    return false;
  }
  const int nw = ctr[5];
  for (int m = me; m < nsrc; m += G::kSize) {
    if (a.sp[m]) continue;
    const int o = (int)(a.sdb[m] & 0xFFFFFFFFull), u = a.on[o];
    if (u != 0 && a.wall[u] > a.ox[o]) a.wneed[a.grp[u]] = 1;
    for (int v = par_of(a, u), hops = 0; v > 0 && hops < n; v = par_of(a, v), ++hops)
      if (a.wall[v] >= 0) a.wneed[a.grp[v]] = 1;
  }
  g.sync();
  // The needed groups, compacted into ord (free until the longest paths).
  int nl = 0;
  for (int t0 = 0; t0 < nw; t0 += G::kSize) {
    const bool need = t0 + me < nw && a.wneed[t0 + me];
    int tot;
    const int at = g.slot(need, &tot);
    if (need) a.ord[nl + at] = t0 + me;
    nl += tot;
  }
  for (int t = me; t < nw; t += G::kSize) a.wneed[t] = 0;
  g.sync();
  // Bit-parallel reachability over up to 32 groups at a time: bit b of
  // reach[u] (kept in seen) says u is reachable from the root without passing
  // the wall of the batch's b-th group. A node truncated by a group (each node
  // of its block that has a wall) passes every bit on but that group's.
  // wneed[g] holds g's bit + 1 while g is in the batch.
  int* reach = a.seen;
  for (int b0 = 0; b0 < nl && alive > 0; b0 += 32) {
    const int nbits = min(32, nl - b0);
    const unsigned full = nbits == 32 ? 0xFFFFFFFFu : ((1u << nbits) - 1u);
#ifdef GPA_PHASE_TIMING
    if (me == 0) atomicAdd(&P.stats[SS_PHASE + (min(tier, 3) - 1) * 6 + 5], 1ull);
    ++r2runs;
#endif
    if (me < nbits) a.wneed[a.ord[b0 + me]] = me + 1;
    for (int u = me; u < n; u += G::kSize) reach[u] = u == 0 ? (int)full : 0;
    g.sync();
    auto pass_mask = [&](int u) {
      const int wg = u != 0 ? a.grp[u] : -1;
      const int b = wg >= 0 ? a.wneed[wg] : 0;
      return b ? ~(1u << (b - 1)) : 0xFFFFFFFFu;
    };
    // A first-tier search propagates by one thread with a worklist ring over
    // q (a node is in it at most once at a time, flag 8): the same fixpoint
    // as the frontier rounds below, without a round's barriers and counters.
    if (serial_a && me == 0) {
      int* ring = a.q;
      int head = 0, tail = 1, inq = 1;
      ring[0] = 0;
      a.fl[0] |= 8;
      while (inq > 0) {
        const int u = ring[head];
        head = head + 1 == a.N ? 0 : head + 1;
        --inq;
        a.fl[u] &= ~8;
        const unsigned m = (unsigned)reach[u] & pass_mask(u);
        if (!m || !edges_ok(u, n)) continue;
        for (int e = a.e0[u]; e < a.e1[u]; ++e) {
          const int v = a.eto[e] & 0x7FFFFFFF;
          if (!target_ok(v, n)) break;
          const unsigned add = m & ~(unsigned)reach[v];
          if (!add) continue;
          reach[v] |= (int)add;
          if (!(a.fl[v] & 8)) {
            a.fl[v] |= 8;
            ring[tail] = v;
            tail = tail + 1 == a.N ? 0 : tail + 1;
            ++inq;
          }
        }
      }
    }
    int* cur = a.q;
    int* nxt = a.tmp;
    if (me == 0) { cur[0] = 0; ctr[5] = 0; }
    int fsize = serial_a ? 0 : 1;
    g.sync();
    while (fsize > 0) {
      // Clear the queued flags of the whole frontier first: bits that arrive
      // at a frontier node during this round queue it again.
      for (int f = me; f < fsize; f += G::kSize) atomicAnd(&a.fl[cur[f]], ~8);
      g.sync();
      for (int f0 = 0; f0 < fsize; f0 += G::kSize) {
        if (f0 + me >= fsize) continue;
        const int u = cur[f0 + me];
        if (!edges_ok(u, n)) continue;
        const unsigned m = (unsigned)atomicOr(&reach[u], 0) & pass_mask(u);
        if (!m) continue;
        for (int e = a.e0[u]; e < a.e1[u]; ++e) {
          const int v = a.eto[e] & 0x7FFFFFFF;
          if (!target_ok(v, n)) break;
          const unsigned add = m & ~(unsigned)reach[v];
          if (!add) continue;
          const unsigned old = (unsigned)atomicOr(&reach[v], (int)add);
          if ((old | add) != old && !(atomicOr(&a.fl[v], 8) & 8)) nxt[atomicAdd((int*)&a.ctr[5], 1)] = v;
        }
      }
      g.sync();
      fsize = ctr[5];
      g.sync();
      if (me == 0) ctr[5] = 0;
      int* sw = cur; cur = nxt; nxt = sw;
      g.sync();
    }
    // A source survives the batch if, for every group, one of its occurrences
    // is reached without passing that group's wall (an occurrence above the
    // wall inside a truncated node is cut too).
    int dropped = 0;
    for (int m = me; m < nsrc; m += G::kSize) {
      if (a.sp[m]) continue;
      unsigned ok = 0;
      for (int o = a.shead[m]; o >= 0 && (ok & full) != full; o = a.onext[o]) {
        const int u = a.on[o];
        unsigned r = (unsigned)reach[u];
        const int wg = u != 0 ? a.grp[u] : -1;
        if (wg >= 0 && a.wneed[wg] && a.ox[o] < a.wpos[wg]) r &= ~(1u << (a.wneed[wg] - 1));
        ok |= r;
      }
      if ((ok & full) != full) { a.sp[m] = 1; ++dropped; }
    }
    alive -= g.sum(dropped);
    g.sync();
    if (me < nbits) a.wneed[a.ord[b0 + me]] = 0;
    g.sync();
  }
  phase(3);
  if (P.diag == 1) {
    if (me == 0) cov_add(P, e, nsrc, alive);
    return true;
  }
  // The export keeps every source: sp marks the rule-2 cuts (its dom flag).
  const bool every = P.diag == 2;
  if (alive == 0 && !every) return true;

  // Longest path with exactly K back edges: layer = back edges used. Each
  // layer is a DAG over the forward edges, processed in topological order by
  // level-synchronous Kahn frontiers; back edges feed the next layer.
  int maxK = 0;
  for (int m = me; m < nsrc; m += G::kSize) if (!a.sp[m] || every) maxK = max(maxK, a.sk[m]);
  maxK = g.max(maxK);
  if (maxK >= a.L) {
    if (me == 0) ctr[7] = 5;
    g.sync();
    return false;
  }
  for (int t = me; t < (maxK + 1) * n; t += G::kSize) a.dl[(t / n) * a.N + (t % n)] = -1;
  for (int u = me; u < n; u += G::kSize) a.ord[u] = 0;
  g.sync();
  for (int u = me; u < n; u += G::kSize)
    for (int e = a.e0[u]; e < a.e1[u]; ++e)
      if (!((uint32_t)a.eto[e] >> 31)) atomicAdd(&a.ord[a.eto[e] & 0x7FFFFFFF], 1);
  if (me == 0) a.dl[0] = 0;
  g.sync();
  if (serial_a) {
    // A first-tier search runs the layers by one thread: Kahn's order with a
    // queue over q (each node enters a layer's queue once, when its last
    // forward in-edge is taken), the nodes' lengths read once into tmp.
    for (int u = me; u < n; u += G::kSize) a.tmp[u] = wout(u);
    g.sync();
    if (me == 0) {
      int* ring = a.q;
      for (int l = 0; l <= maxK; ++l) {
        int* dll = a.dl + (int64_t)l * a.N;
        int head = 0, tail = 0;
        for (int u = 0; u < n; ++u) {
          a.seen[u] = a.ord[u];  // remaining forward in-edges
          if (a.ord[u] == 0) ring[tail++] = u;
        }
        while (head < tail) {
          const int u = ring[head++];
          const int cv = dll[u];
          const int nd = cv + a.tmp[u];
          for (int e = a.e0[u]; e < a.e1[u]; ++e) {
            const int v = a.eto[e] & 0x7FFFFFFF;
            if ((uint32_t)a.eto[e] >> 31) {
              int* t = &a.dl[(int64_t)(l + 1) * a.N + v];
              if (cv >= 0 && l + 1 <= maxK && nd > *t) *t = nd;
            } else {
              if (cv >= 0 && nd > dll[v]) dll[v] = nd;
              if (--a.seen[v] == 0 && tail < a.N) ring[tail++] = v;
            }
          }
        }
      }
    }
    g.sync();
  } else {
    for (int l = 0; l <= maxK; ++l) {
      int* dll = a.dl + (int64_t)l * a.N;
      if (me == 0) ctr[5] = 0;
      g.sync();
      for (int u = me; u < n; u += G::kSize) {
        a.seen[u] = a.ord[u];  // remaining forward in-edges
        if (a.ord[u] == 0) a.q[atomicAdd((int*)&a.ctr[5], 1)] = u;
      }
      g.sync();
      int fsize = ctr[5];
      int* cur = a.q;
      int* nxt = a.tmp;
      g.sync();
      if (me == 0) ctr[5] = 0;
      g.sync();
      while (fsize > 0) {
        for (int f0 = 0; f0 < fsize; f0 += G::kSize) {
          if (f0 + me < fsize) {
            const int u = cur[f0 + me];
            const int cv = dll[u];
            const int nd = cv + wout(u);
            for (int e = a.e0[u]; e < a.e1[u]; ++e) {
              const int v = a.eto[e] & 0x7FFFFFFF;
              const bool back = (uint32_t)a.eto[e] >> 31;
              if (back) {
                if (cv >= 0 && l + 1 <= maxK) atomicMax(&a.dl[(int64_t)(l + 1) * a.N + v], nd);
              } else {
                if (cv >= 0) atomicMax(&dll[v], nd);
                if (atomicSub(&a.seen[v], 1) == 1) nxt[atomicAdd((int*)&a.ctr[5], 1)] = v;
              }
            }
          }
        }
        g.sync();
        fsize = ctr[5];
        g.sync();
        if (me == 0) ctr[5] = 0;
        int* sw = cur; cur = nxt; nxt = sw;
        g.sync();
      }
    }
  }
  for (int m = me; m < nsrc; m += G::kSize) {
    if (a.sp[m] && !every) continue;
    const int K = a.sk[m];
    int best = -1;
    for (int o = a.shead[m]; o >= 0; o = a.onext[o]) {
      const int u = a.on[o];
      const int dlu = a.dl[(int64_t)K * a.N + u];
      if (dlu >= 0) best = max(best, dlu + last_of(u) - a.ox[o]);
    }
    if (best < 1) { capacity(P, 13); continue; }
    if (every) xemit(P, j, a.si[m], r, (int)(a.sdb[m] >> 32), K, best, a.sp[m] || blocked);
    else emit_raw(P, A, j, a.si[m], r, def_kind(P, a.si[m], r), (int)(a.sdb[m] >> 32), best);
  }
  g.sync();
  phase(4);
  return true;
}

// The task loop of a search group: claim (use, resource) tasks from one
// queue until it is empty. Tier 1 reads the local pass's queue; tier 2 the
// first overflow queue; tier 3 part 1 the large list and the region at the top
// of the first queue, part 2 the second overflow, which reuses the first
// queue's storage; tier 4 the third overflow (bottom of the first overflow
// queue's storage) and its top region. A search that outgrows its tier is
// queued for the next one; the last tier records why it ran out.
template <class G>
__device__ void run_tasks(const G& g, const Prog& P, const Arch& A, const Arena& a, int tier, int part) {
  const int me = g.rank();
  // The tasks of this launch, in order: nl of the large list, n0 read up
  // from the bottom of q0, n1 read down from the top of q1.
  const unsigned long long cap = (unsigned long long)P.queue_cap;
  const int4* q0 = P.queue;
  const int4* q1 = P.queue;
  unsigned long long nl = 0, n0 = 0, n1 = 0;
  int h_slot = SS_QUEUE_HEAD;
  if (tier == 1) {
    n0 = P.stats[SS_QUEUE_N];
  } else if (tier == 2) {
    q0 = P.ovf_queue, n0 = P.stats[SS_OVF_N], h_slot = SS_OVF_HEAD;
  } else if (tier == 3 && part == 1) {
    nl = min(P.stats[SS_LARGE_N], (unsigned long long)kLargeQueue);
    n1 = P.stats[SS_HINT3_N], h_slot = SS_HINT3_HEAD;
  } else if (tier == 3) {
    n0 = P.stats[SS_OVF2_N], h_slot = SS_OVF2_HEAD;
  } else {
    q0 = q1 = P.ovf_queue, n0 = P.stats[SS_OVF3_N], n1 = P.stats[SS_OVF3H_N], h_slot = SS_OVF3_HEAD;
  }
  n0 = min(n0, cap);
  n1 = min(n1, cap - n0);
  while (true) {
    unsigned long long t = 0;
    if (me == 0) t = atomicAdd(&P.stats[h_slot], 1ull);
    t = g.broadcast(t);
    if (t >= nl + n0 + n1) break;
    const int4 task = t < nl        ? P.large_queue[t]
                      : t < nl + n0 ? q0[t - nl]
                                    : q1[cap - 1 - (t - nl - n0)];
    const int f = P.block_func[P.instr_block[task.x]];
    // The coverage count needs every source: no latency bound.
    const int bound = P.diag ? kInf - 1 : P.res_maxlat[(size_t)f * kNumRes + task.y];
    const uint16_t live = live_literals(P.res_guards[(size_t)f * kNumRes + task.y], P.guard[task.x]);
    const bool ok = group_search(g, P, A, a, task.x, task.y, (uint16_t)task.z, bound, live, tier, task.w,
                                 (task.z >> 20) & 1);
    if (ok) {
      // later steps start a large third-tier search before the others
      if (me == 0 && tier == 3 && !P.diag && ((volatile int*)a.ctr)[0] >= P.large_nodes) P.large_hint[task.w] = 1;
      continue;
    }
    if (me != 0) continue;
    if (!P.diag) atomicMax(&P.tier_hint[task.w], (unsigned)(tier + 1));  // later steps queue it for a bigger tier
    if (tier < 3 || (tier == 3 && P.t4_nodes > 0)) {
      // tier 1 -> bottom of ovf_queue; tier 2 -> bottom of queue; tier 3 part 2
      // -> bottom of ovf_queue (after tier 2 read it); part 1, which may run
      // beside tier 1, -> top of ovf_queue
      const bool top = tier == 3 && part == 1;
      const int o_slot = tier == 1 ? SS_OVF_N : tier == 2 ? SS_OVF2_N : top ? SS_OVF3H_N : SS_OVF3_N;
      int4* oq = tier == 2 ? P.queue : P.ovf_queue;
      const unsigned long long o = atomicAdd(&P.stats[o_slot], 1ull);
      if (o < cap) oq[top ? cap - 1 - o : o] = task; else capacity(P, 8);
    } else {
      capacity(P, a.ctr[7] > 0 ? a.ctr[7] : 1);  // the last tier: why it ran out
    }
  }
}

// Persistent work-stealing warps, one search each. Tiers 1 and 2 keep the
// arena in shared memory (tier 1: several warps per CTA, small arenas; tier 2:
// one warp per CTA, a large arena); tier 3 uses global-memory arenas. Tier 3
// runs in two parts: part 1 takes the searches queued straight for it (the
// large list first) and may run beside tiers 1 and 2; part 2 takes the second
// tier's overflow.
// Registers: at least six 128-thread CTAs per SM, i.e. 80 registers a thread
// (96 without the bound). The first tier and the third tier's hinted part run
// side by side and together fill the SM's registers, so fewer registers a warp
// keep more warps in flight (measured: 40.7 against 41.9 ms a step).
#ifndef GPA_SEARCH_MIN_CTAS
#define GPA_SEARCH_MIN_CTAS 6
#endif
__global__ void __launch_bounds__(kWarpsPerCta * 32, GPA_SEARCH_MIN_CTAS)
    k_search_warp(Prog P, Arch A, SearchArena SA, int tier, int part) {
  extern __shared__ __align__(16) char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wid;
  char* base = tier < 3 ? smem + (int64_t)wid * SA.bytes : SA.global + (int64_t)gw * SA.bytes;
  // The search counters live in shared memory in every tier (the arena of
  // tier 3 is in global memory): frontier sizes are read after every round.
  __shared__ int s_ctr[kWarpsPerCta][8];
  const Arena a = carve(base, SA.nodes, SA.src, SA.layers, s_ctr[wid]);
  for (int t = lane; t < 2 * SA.nodes; t += 32) a.ht[t] = -1;
  __syncwarp();
  run_tasks(WarpGroup{}, P, A, a, tier, part);
}

// The fourth tier: a CTA per search, over a global-memory arena of its own
// (the searches that outgrow the third tier's arenas have tens of thousands to
// millions of (block, literal set) nodes: their waves, frontiers and source
// lists are wide enough for a CTA's threads).
__global__ void __launch_bounds__(kCtaThreads, 1) k_search_cta(Prog P, Arch A, SearchArena SA) {
  __shared__ int s_ctr[8];
  __shared__ int s_red[CtaGroup::kWarps];
  __shared__ unsigned long long s_cast;
  const CtaGroup g{s_red, &s_cast};
  const Arena a = carve(SA.global + (int64_t)blockIdx.x * SA.bytes, SA.nodes, SA.src, SA.layers, s_ctr);
  for (int t = threadIdx.x; t < 2 * SA.nodes; t += kCtaThreads) a.ht[t] = -1;
  __syncthreads();
  run_tasks(g, P, A, a, 4, 0);
}

}  // namespace

int64_t search_arena_bytes(int nodes, int src, int layers) { return arena_bytes(nodes, src, layers); }

int search_warps_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_search_warp, 32, 0) != cudaSuccess || n < 1) n = 4;
  return n;
}

void launch_search(const Prog& P, const Arch& A, const SearchArena* tiers, const SearchFork* fork, cudaStream_t st,
                   int sms, int64_t* launches) {
  // Each launch requests its own tier's arena size.
  const size_t smem1 = (size_t)tiers[0].bytes * kWarpsPerCta;
  const size_t smem2 = (size_t)tiers[1].bytes;
  allow_max_smem(k_search_warp);
  // The searches queued straight for the third tier depend on nothing the
  // first two tiers do: with a second stream they run beside them (no kernel
  // waits on another; the join only orders the third tier's second part,
  // which shares its arenas, after them).
  // Tier 1 is submitted first, so its CTAs take their share of each SM and the
  // third tier's warps fill the registers left beside them.
  cudaStream_t s3 = st;
  if (fork) {
    cudaEventRecord(fork->fork, st);
    cudaStreamWaitEvent(fork->side, fork->fork, 0);
    s3 = fork->side;
  }
  k_search_warp<<<tiers[0].warps / kWarpsPerCta, kWarpsPerCta * 32, smem1, st>>>(P, A, tiers[0], 1, 0);
  k_search_warp<<<tiers[2].warps, 32, 0, s3>>>(P, A, tiers[2], 3, 1);
  if (fork) cudaEventRecord(fork->join, fork->side);
  k_search_warp<<<tiers[1].warps, 32, smem2, st>>>(P, A, tiers[1], 2, 0);
  if (fork) cudaStreamWaitEvent(st, fork->join, 0);
  k_search_warp<<<tiers[2].warps, 32, 0, st>>>(P, A, tiers[2], 3, 2);
  *launches += 4;
  if (P.t4_nodes > 0) {
    // The fourth tier runs after the third on this stream, so the third tier's
    // arena pool is free by then: when it holds more fourth-tier arenas than the
    // program's own, the CTAs carve theirs from it (at most one CTA per SM).
    SearchArena t4{P.t4_nodes, P.t4_src, kMaxLayers, P.t4_ctas, P.t4_bytes, P.t4_arena};
    const int64_t in_pool = (int64_t)tiers[2].warps * tiers[2].bytes / P.t4_bytes;
    if (in_pool > t4.warps && tiers[2].global) {
      t4.warps = (int)std::min<int64_t>(in_pool, std::max(sms, 1));
      t4.global = tiers[2].global;
    }
    k_search_cta<<<t4.warps, kCtaThreads, 0, st>>>(P, A, t4);
    ++*launches;
  }
}

}  // namespace gpa
