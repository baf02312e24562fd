// Steps (b) and (c), Sec. 4: backward slicing with virtual barrier registers
// and predicate coverage, the three pruning rules, and Eq. 1 apportioning.
//
// For each stalled use j and each resource r it reads, the immediate sources
// are the defs of r reached backwards from j while the union P of the guard
// literals of the defs met so far does not contain j's guard (Sec. 4,
// "Predicated instructions"); "_" is contained by everything and Pi with !Pi
// makes "_". A source i survives if (rule 2) no single unguarded reader k of r
// (k not i, j) lies on every source path from i to j, and (rule 3) its
// shortest source path is at most latency(i). Sources reached through several
// resources merge into one source i; Eq. 1 then splits each dependency class
// and latency flag of j by issue_i / longest_path_i among the sources that
// (rule 1) match the class's opcode rule.
//
// Work split:
//  * k_search_local: one thread per stalled use, one linear scan per
//    resource inside j's block. It settles every source of that block
//    (their only path is the straight segment) and stops at coverage or at
//    the first unguarded reader of r (that reader lies on every path beyond,
//    so nothing further can survive rule 2). Uses whose value may come from
//    another block are queued.
//  * k_search_general: persistent threads pull queued (use, resource) pairs
//    and explore the (block, literal set) graph with per-slot scratch:
//    shortest paths and fewest back edges by label correcting, rule 2 by
//    re-running reachability with each block's highest unguarded reader as a
//    wall, longest path with exactly K back edges over layers.
//  * k_merge_count / scan / k_apportion: merge sources per use, apportion in
//    integers, scatter blame with warp-aggregated 64-bit atomics.
#include <cooperative_groups.h>
#include <cooperative_groups/reduce.h>

#include "gpa_internal.cuh"

namespace cg = cooperative_groups;

namespace gpa {

namespace {

__device__ __forceinline__ int dep_class(int ci) {
  return ci == 0 ? GPA_EXEC_DEPENDENCY : ci == 1 ? GPA_MEMORY_DEPENDENCY : ci == 2 ? GPA_SYNC : GPA_CONSTANT_MEMORY_DEPENDENCY;
}
constexpr int kInf = 0x3FFFFFFF;
constexpr uint32_t kBackBit = 0x80000000u;

__device__ __forceinline__ bool stalled(const Prog& P, int j) {
  const unsigned long long* c = P.cnt + (size_t)j * kCnt;
  return (c[4] | c[5] | c[6] | c[7] | c[10] | c[11] | c[12] | c[13]) != 0ull;
}

// Raw edge (j <- i through r) onto j's list.
__device__ void emit_raw(const Prog& P, const Arch& A, int j, int i, int r, int kind, int dmin, int dlong) {
  uint32_t fl = r >= kBarBase ? 2u : (r >= kPredBase ? 8u : 4u);
  // Write-after-read (Sec. 4, Fig. 6): the variable-latency def reads a
  // register that the use writes, and they are linked through a read barrier.
  if (r >= kBarBase && kind == 2 && (A.flags[P.opclass[i]] & GPA_F_VARLAT)) {
    for (int e = P.def_off[j]; e < P.def_off[j + 1]; ++e) {
      const int rr = P.def_res[e] & 0x1FF;
      if (rr < kPredBase && uses_res(P, i, rr)) { fl |= 1u; break; }
    }
  }
  if (dmin >= (1 << 24) || dlong >= (1 << 24)) { set_status(P, ST_CAPACITY); return; }
  const unsigned long long slot = atomicAdd(&P.stats[SS_RAW_N], 1ull);
  if (slot >= (unsigned long long)P.raw_cap) { set_status(P, ST_CAPACITY); return; }
  const int next = atomicExch(&P.head[j], (int)slot);
  P.raw[slot] = make_int4(i, next, dmin, dlong | (int)(fl << 24));
}

__global__ void k_search_local(Prog P, Arch A) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.ni; j += gridDim.x * blockDim.x) {
    if (!stalled(P, j)) continue;
    const int gj = P.guard[j];
    const int b0 = P.instr_block[j];
    const int first = P.block_instr_off[b0];
    for (int e = P.use_off[j]; e < P.use_off[j + 1]; ++e) {
      const int r = P.use_res[e] & 0x1FF;
      uint16_t S = 0;
      bool blocked = false;
      for (int x = j - 1; x >= first; --x) {
        const int kind = def_kind(P, x, r);
        if (kind >= 0) {
          if (!contains(S, gj)) {
            const int d = j - x;
            if (d <= A.lat[P.opclass[x]]) emit_raw(P, A, j, x, r, kind, d, d);
          }
          S = add_literal(S, P.guard[x]);
          if (contains(S, gj)) { blocked = true; break; }
        } else if (P.guard[x] == 0 && uses_res(P, x, r)) {
          blocked = true;  // unguarded reader on every path beyond this point
          break;
        }
      }
      if (blocked) continue;
      const int w = r >> 5;
      const uint32_t bit = 1u << (r & 31);
      for (int q = P.pred_off[b0]; q < P.pred_off[b0 + 1]; ++q) {
        if (P.rout[(size_t)P.pred[q] * kWords + w] & bit) {
          const unsigned long long t = atomicAdd(&P.stats[SS_QUEUE_N], 1ull);
          if (t < (unsigned long long)P.queue_cap) P.queue[t] = make_int4(j, r, (int)S, 0);
          else set_status(P, ST_CAPACITY);
          break;
        }
      }
    }
  }
}

// ---------------------------------------------------------------- general search
struct Slot {
  int *blk, *S, *cov, *wall, *d, *k, *e0, *e1, *seen, *ord, *tmp, *q, *hused, *par, *fl, *dl, *ht;
  int *eto, *onode, *ox, *si, *sd, *sk, *sl, *sp, *wblk, *wpos, *wneed;
};

__device__ __forceinline__ Slot slot_at(const SearchScratch& SS, int slot) {
  int* p = SS.base + (int64_t)slot * SS.slot_ints;
  const int N = SS.max_nodes;
  Slot s;
  s.blk = p; p += N; s.S = p; p += N; s.cov = p; p += N; s.wall = p; p += N;
  s.d = p; p += N; s.k = p; p += N; s.e0 = p; p += N; s.e1 = p; p += N;
  s.seen = p; p += N; s.ord = p; p += N; s.tmp = p; p += N; s.q = p; p += N; s.hused = p; p += N;
  s.par = p; p += N; s.fl = p; p += N;
  s.dl = p; p += (int64_t)kMaxLayers * N;
  s.ht = p; p += 2 * N;
  s.eto = p; p += SS.edge_cap;
  s.onode = p; p += SS.occ_cap; s.ox = p; p += SS.occ_cap;
  s.si = p; p += SS.src_cap; s.sd = p; p += SS.src_cap; s.sk = p; p += SS.src_cap;
  s.sl = p; p += SS.src_cap; s.sp = p; p += SS.src_cap;
  s.wblk = p; p += SS.wall_cap; s.wpos = p; p += SS.wall_cap; s.wneed = p;
  return s;
}

__device__ __forceinline__ uint32_t node_hash(int blk, int S) {
  uint32_t h = (uint32_t)blk * 0x9E3779B1u ^ ((uint32_t)S * 0x85EBCA77u);
  h ^= h >> 15;
  return h;
}

// Stable merge sort of node ids by (block descending, id ascending).
__device__ void sort_nodes(int* a, int* tmp, int n, const int* blk) {
  for (int w = 1; w < n; w <<= 1) {
    for (int lo = 0; lo < n; lo += 2 * w) {
      int mid = min(lo + w, n), hi = min(lo + 2 * w, n);
      int i = lo, j = mid, k = lo;
      while (i < mid && j < hi) {
        const int x = a[i], y = a[j];
        const bool take_y = blk[y] > blk[x] || (blk[y] == blk[x] && y < x);
        tmp[k++] = take_y ? a[j++] : a[i++];
      }
      while (i < mid) tmp[k++] = a[i++];
      while (j < hi) tmp[k++] = a[j++];
    }
    for (int t = 0; t < n; ++t) a[t] = tmp[t];
  }
}

constexpr int kExpanded = 1, kQueued = 2;

// Explores the graph of (block, literal set) nodes backwards from j for
// resource r. Node 0 is the part of j's block above j, already scanned by
// the local pass (its sources are settled there). A node's d is the shortest
// distance from the last instruction of its block to j.
//
// Pass A grows the graph in shortest-distance order up to `bound`, the largest
// latency of any def of r in the function: a source farther than that fails
// rule 3 whatever the rest of the graph holds. Only if some source is within
// its latency does pass B complete the graph, which rule 2 and the longest
// paths need. Returns false when the search outgrew this scratch slot
// (nothing was emitted); the caller retries it in a larger slot.
__device__ bool general_search(const Prog& P, const Arch& A, const SearchScratch& SS, int slot_id, int j, int r,
                               uint16_t S0, int bound) {
  Slot s = slot_at(SS, slot_id);
  const int N = SS.max_nodes;
  const uint32_t hmask = (uint32_t)(2 * N - 1);
  const int gj = P.guard[j];
  const int b0 = P.instr_block[j];
  const int first0 = P.block_instr_off[b0];
  const int w = r >> 5;
  const uint32_t bit = 1u << (r & 31);
  int n = 0, ne = 0, no = 0, nh = 0;
  bool overflow = false;

  s.blk[0] = b0; s.S[0] = (int)S0 | ((int)S0 << 16); s.cov[0] = first0; s.wall[0] = -1;
  s.d[0] = 0; s.fl[0] = 0;
  n = 1;

  auto wout = [&](int u) {
    return u == 0 ? (j - first0 + 1) : (P.block_instr_off[s.blk[u] + 1] - P.block_instr_off[s.blk[u]]);
  };
  auto last_of = [&](int u) { return P.block_instr_off[s.blk[u] + 1] - 1; };
  auto find_or_add = [&](int blk, int Sv) -> int {
    uint32_t h = node_hash(blk, Sv) & hmask;
    for (int probe = 0; probe <= (int)hmask; ++probe) {
      const int v = s.ht[h];
      if (v < 0) {
        if (n >= N) return -1;
        const int u = n++;
        s.blk[u] = blk; s.S[u] = Sv; s.wall[u] = -1; s.cov[u] = 0; s.d[u] = kInf; s.fl[u] = 0;
        s.ht[h] = u;
        s.hused[nh++] = (int)h;
        return u;
      }
      if (s.blk[v] == blk && (s.S[v] & 0xFFFF) == Sv) return v;
      h = (h + 1) & hmask;
    }
    return -1;
  };
  // Scan node u's block bottom-up (not for the root), then link its predecessors.
  auto scan_expand = [&](int u) {
    s.fl[u] |= kExpanded;
    uint16_t S = (uint16_t)(s.S[u] & 0xFFFF);
    bool stop = false;
    if (u != 0) {
      const int B = s.blk[u];
      const int first = P.block_instr_off[B], last = P.block_instr_off[B + 1] - 1;
      int cov = first, wall = -1;
      if ((P.def_mask[(size_t)B * kWords + w] | P.uuse_mask[(size_t)B * kWords + w]) & bit) {
        for (int x = last; x >= first; --x) {
          const int kind = def_kind(P, x, r);
          if (kind >= 0) {
            if (!contains(S, gj) && !(B == b0 && x < j)) {  // sources above j in its block are settled
              if (no >= SS.occ_cap) { overflow = true; return; }
              s.onode[no] = u; s.ox[no] = x; ++no;
            }
            S = add_literal(S, P.guard[x]);
            if (contains(S, gj)) { stop = true; cov = x; break; }
          } else if (wall < 0 && x != j && P.guard[x] == 0 && uses_res(P, x, r)) {
            wall = x;
          }
        }
      }
      s.S[u] = (s.S[u] & 0xFFFF) | ((int)S << 16);
      s.cov[u] = cov;
      s.wall[u] = wall;
    }
    s.e0[u] = ne;
    if (!stop) {
      const int B = s.blk[u];
      for (int q = P.pred_off[B]; q < P.pred_off[B + 1]; ++q) {
        const int p = P.pred[q];
        if (!(P.rout[(size_t)p * kWords + w] & bit)) continue;  // no def of r leaves p
        const int v = find_or_add(p, S);
        if (v < 0 || ne >= SS.edge_cap) { overflow = true; break; }
        s.eto[ne++] = v | (p >= B ? (int)kBackBit : 0);
      }
    }
    s.e1[u] = ne;
  };

  // Pass A: label-correcting growth limited to d <= bound (circular queue, a node at most once in it).
  int qh = 0, qc = 0;
  s.q[0] = 0; qc = 1; s.fl[0] |= kQueued;
  while (qc > 0 && !overflow) {
    const int u = s.q[qh];
    qh = (qh + 1 == N) ? 0 : qh + 1;
    --qc;
    s.fl[u] &= ~kQueued;
    if (s.d[u] > bound) continue;
    if (!(s.fl[u] & kExpanded)) scan_expand(u);
    if (overflow) break;
    const int du = s.d[u] + wout(u);
    for (int e = s.e0[u]; e < s.e1[u]; ++e) {
      const int v = s.eto[e] & 0x7FFFFFFF;
      if (du < s.d[v]) {
        s.d[v] = du;
        if (!(s.fl[v] & kQueued)) {
          int at = qh + qc;
          if (at >= N) at -= N;
          s.q[at] = v; ++qc; s.fl[v] |= kQueued;
        }
      }
    }
  }
  bool candidate = false;
  for (int o = 0; o < no && !overflow && !candidate; ++o) {
    const int u = s.onode[o];
    candidate = s.d[u] + (last_of(u) - s.ox[o]) <= A.lat[P.opclass[s.ox[o]]];
  }
  // Pass B: complete the graph when a source may survive.
  if (candidate)
    for (int u = 0; u < n && !overflow; ++u)
      if (!(s.fl[u] & kExpanded)) scan_expand(u);
  for (int t = 0; t < nh; ++t) s.ht[s.hused[t]] = -1;
  atomicAdd(&P.stats[SS_GENERAL], 1ull);
  atomicMax(&P.stats[SS_MAX_NODES], (unsigned long long)n);
  if (overflow) return false;
  if (!candidate) return true;

  // Shortest distance, fewest back edges and a shortest-path parent per node.
  for (int u = 0; u < n; ++u) { s.d[u] = kInf; s.k[u] = kInf; s.par[u] = -1; }
  s.d[0] = 0; s.k[0] = 0;
  bool changed = true;
  for (int pass = 0; changed; ++pass) {
    if (pass > n + 1) { set_status(P, ST_CAPACITY); return true; }
    changed = false;
    for (int u = 0; u < n; ++u) {
      if (s.d[u] >= kInf) continue;
      const int du = s.d[u] + wout(u), ku = s.k[u];
      for (int e = s.e0[u]; e < s.e1[u]; ++e) {
        const int v = s.eto[e] & 0x7FFFFFFF;
        const int kb = ku + (int)((uint32_t)s.eto[e] >> 31);
        if (du < s.d[v]) { s.d[v] = du; s.par[v] = u; changed = true; }
        if (kb < s.k[v]) { s.k[v] = kb; changed = true; }
      }
    }
  }
  // Sources: shortest path and fewest back edges over their occurrences; the
  // occurrence with the shortest path is kept for the rule-2 wall filter.
  int nsrc = 0;
  for (int o = 0; o < no; ++o) {
    const int u = s.onode[o], x = s.ox[o];
    const int dist = s.d[u] + (last_of(u) - x), kk = s.k[u];
    int t = 0;
    while (t < nsrc && s.si[t] != x) ++t;
    if (t == nsrc) {
      if (nsrc >= SS.src_cap) return false;
      s.si[t] = x; s.sd[t] = dist; s.sk[t] = kk; s.sl[t] = o; s.sp[t] = 0; ++nsrc;
    } else {
      if (dist < s.sd[t]) { s.sd[t] = dist; s.sl[t] = o; }
      s.sk[t] = min(s.sk[t], kk);
    }
  }
  int alive = 0;
  for (int t = 0; t < nsrc; ++t) {
    if (s.sd[t] > A.lat[P.opclass[s.si[t]]]) s.sp[t] = 1;  // rule 3
    else ++alive;
  }
  if (alive == 0) return true;

  // Rule 2. Nodes sorted by block; per block, the unguarded reader of r met
  // first from the bottom truncates at least as much as any other reader of
  // that block, so one wall per block is enough. A wall can only block source
  // i if it lies on the shortest path to i (it must lie on every path), so
  // only walls met along the parent chain of that path are re-tested.
  for (int u = 0; u < n; ++u) s.ord[u] = u;
  sort_nodes(s.ord, s.tmp, n, s.blk);
  int* grp = s.tmp;  // node -> wall group, after the sort
  int nw = 0;
  for (int t = 0; t < n;) {
    const int B = s.blk[s.ord[t]];
    int e = t, mx = -1;
    while (e < n && s.blk[s.ord[e]] == B) { if (s.ord[e] != 0) mx = max(mx, s.wall[s.ord[e]]); ++e; }
    int g = -1;
    if (mx >= 0) {
      if (nw >= SS.wall_cap) return false;
      g = nw++;
      s.wblk[g] = B; s.wpos[g] = mx; s.wneed[g] = 0;
    }
    for (int q = t; q < e; ++q) grp[s.ord[q]] = g;
    t = e;
  }
  for (int m = 0; m < nsrc; ++m) {
    if (s.sp[m]) continue;
    const int o = s.sl[m];
    const int u = s.onode[o];
    if (u != 0 && s.wall[u] > s.ox[o]) s.wneed[grp[u]] = 1;
    for (int v = s.par[u], hops = 0; v > 0 && hops < n; v = s.par[v], ++hops)
      if (s.wall[v] >= 0) s.wneed[grp[v]] = 1;
  }
  for (int u = 0; u < n; ++u) s.seen[u] = 0;
  for (int t = 0; t < nw && alive > 0; ++t) {
    if (!s.wneed[t]) continue;
    const int WB = s.wblk[t], WP = s.wpos[t], epoch = t + 1;
    auto trunc = [&](int u) { return u != 0 && s.blk[u] == WB && s.cov[u] <= WP; };
    int h = 0, tl = 0;
    s.q[tl++] = 0; s.seen[0] = epoch;
    while (h < tl) {
      const int u = s.q[h++];
      if (trunc(u)) continue;
      for (int e = s.e0[u]; e < s.e1[u]; ++e) {
        const int v = s.eto[e] & 0x7FFFFFFF;
        if (s.seen[v] != epoch) { s.seen[v] = epoch; s.q[tl++] = v; }
      }
    }
    for (int m = 0; m < nsrc; ++m) {
      if (s.sp[m]) continue;
      bool reach = false;
      for (int o = 0; o < no && !reach; ++o) {
        if (s.ox[o] != s.si[m]) continue;
        const int u = s.onode[o];
        if (s.seen[u] == epoch && !(trunc(u) && s.ox[o] < WP)) reach = true;
      }
      if (!reach) { s.sp[m] = 1; --alive; }
    }
  }
  if (alive == 0) return true;

  // Longest path with exactly K back edges: layer = back edges used; within a
  // layer edges go from higher to lower block ids, so the block-descending
  // order is a topological order.
  int maxK = 0;
  for (int m = 0; m < nsrc; ++m) if (!s.sp[m]) maxK = max(maxK, s.sk[m]);
  if (maxK >= kMaxLayers) { set_status(P, ST_CAPACITY); return true; }
  for (int l = 0; l <= maxK; ++l)
    for (int u = 0; u < n; ++u) s.dl[l * N + u] = -1;
  s.dl[0] = 0;
  for (int l = 0; l <= maxK; ++l) {
    for (int t = 0; t < n; ++t) {
      const int u = s.ord[t];
      const int cur = s.dl[l * N + u];
      if (cur < 0) continue;
      const int nd = cur + wout(u);
      for (int e = s.e0[u]; e < s.e1[u]; ++e) {
        const int v = s.eto[e] & 0x7FFFFFFF;
        const int nl = l + (int)((uint32_t)s.eto[e] >> 31);
        if (nl <= maxK && nd > s.dl[nl * N + v]) s.dl[nl * N + v] = nd;
      }
    }
  }
  for (int m = 0; m < nsrc; ++m) {
    if (s.sp[m]) continue;
    const int K = s.sk[m];
    int best = -1;
    for (int o = 0; o < no; ++o) {
      if (s.ox[o] != s.si[m]) continue;
      const int u = s.onode[o];
      const int dlu = s.dl[K * N + u];
      if (dlu >= 0) best = max(best, dlu + last_of(u) - s.ox[o]);
    }
    if (best < 1) { set_status(P, ST_CAPACITY); continue; }
    emit_raw(P, A, j, s.si[m], r, def_kind(P, s.si[m], r), s.sd[m], best);
  }
  return true;
}

// Persistent work-stealing: each thread owns one scratch slot and pulls
// queued searches until the queue is drained. Tier 1 (small slots) hands
// searches it cannot hold to tier 2 (large slots).
__global__ void k_search_general(Prog P, Arch A, SearchScratch SS, int tier) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= SS.n_slots) return;
  const int4* q = tier == 1 ? P.queue : P.ovf_queue;
  unsigned long long nq = P.stats[tier == 1 ? SS_QUEUE_N : SS_OVF_N];
  if (nq > (unsigned long long)P.queue_cap) nq = (unsigned long long)P.queue_cap;
  unsigned long long* head = &P.stats[tier == 1 ? SS_QUEUE_HEAD : SS_OVF_HEAD];
  while (true) {
    const unsigned long long t = atomicAdd(head, 1ull);
    if (t >= nq) break;
    const int4 task = q[t];
    const int f = P.block_func[P.instr_block[task.x]];
    const int bound = P.res_maxlat[(size_t)f * kNumRes + task.y];
    if (general_search(P, A, SS, slot, task.x, task.y, (uint16_t)task.z, bound)) continue;
    if (tier == 1) {
      const unsigned long long o = atomicAdd(&P.stats[SS_OVF_N], 1ull);
      if (o < (unsigned long long)P.queue_cap) P.ovf_queue[o] = task; else set_status(P, ST_CAPACITY);
    } else {
      set_status(P, ST_CAPACITY);
    }
  }
}

// ---------------------------------------------------------------- merge and apportion
__global__ void k_blame_init(Prog P) {
  const int64_t n = (int64_t)P.ni * kCnt;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(t % kCnt) >> 1;
    const bool dep = c == GPA_EXEC_DEPENDENCY || c == GPA_MEMORY_DEPENDENCY || c == GPA_SYNC ||
                     c == GPA_CONSTANT_MEMORY_DEPENDENCY;
    P.blame[t] = dep ? 0ull : P.cnt[t];
  }
}

__global__ void k_merge_count(Prog P, int max_src) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.ni; j += gridDim.x * blockDim.x) {
    int c = 0;
    int ids[kMaxSrc];
    for (int t = P.head[j]; t >= 0; t = P.raw[t].y) {
      const int i = P.raw[t].x;
      bool seen = false;
      for (int q = 0; q < c; ++q) seen |= ids[q] == i;
      if (seen) continue;
      if (c >= max_src) { set_status(P, ST_CAPACITY); break; }
      ids[c++] = i;
    }
    P.edge_off[j] = c;
  }
}

__device__ __forceinline__ void blame_add(unsigned long long* addr, unsigned long long v) {
  cg::coalesced_group g = cg::coalesced_threads();
  cg::coalesced_group grp = cg::labeled_partition(g, (unsigned long long)(uintptr_t)addr);
  const unsigned long long sum = cg::reduce(grp, v, cg::plus<unsigned long long>());
  if (grp.thread_rank() == 0) atomicAdd(addr, sum);
}

__device__ __forceinline__ bool opcode_keeps(const Arch& A, int cls, int op) {
  if (cls == GPA_MEMORY_DEPENDENCY || cls == GPA_CONSTANT_MEMORY_DEPENDENCY) return (A.flags[op] & GPA_F_MEM) != 0;
  if (cls == GPA_SYNC) return (A.flags[op] & GPA_F_SYNC) != 0;
  return true;
}

__global__ void k_apportion(Prog P, Arch A, int max_src) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.ni; j += gridDim.x * blockDim.x) {
    const unsigned long long* cj = P.cnt + (size_t)j * kCnt;
    const int off = P.edge_off[j];
    int c = P.edge_off[j + 1] - off;
    if (c == 0 && !stalled(P, j)) continue;
    if (off + c > P.edge_cap) { set_status(P, ST_CAPACITY); c = 0; }
    int mi[kMaxSrc], md[kMaxSrc], ml[kMaxSrc];
    uint32_t mf[kMaxSrc];
    int m = 0;
    if (c > 0) {
      for (int t = P.head[j]; t >= 0; t = P.raw[t].y) {
        const int4 R = P.raw[t];
        const int dl = R.w & 0xFFFFFF;
        const uint32_t fl = (uint32_t)R.w >> 24;
        int q = 0;
        while (q < m && mi[q] != R.x) ++q;
        if (q == m) {
          if (m >= c) continue;  // capacity already reported by the count pass
          mi[m] = R.x; md[m] = R.z; ml[m] = dl; mf[m] = fl; ++m;
        } else {
          md[q] = min(md[q], R.z); ml[q] = max(ml[q], dl); mf[q] |= fl;
        }
      }
      // ascending def index
      for (int a = 1; a < m; ++a) {
        const int xi = mi[a], xd = md[a], xl = ml[a];
        const uint32_t xf = mf[a];
        int b = a - 1;
        while (b >= 0 && mi[b] > xi) { mi[b + 1] = mi[b]; md[b + 1] = md[b]; ml[b + 1] = ml[b]; mf[b + 1] = mf[b]; --b; }
        mi[b + 1] = xi; md[b + 1] = xd; ml[b + 1] = xl; mf[b + 1] = xf;
      }
      for (int t = 0; t < m; ++t) {
        const int64_t e = off + t;
        P.e_use[e] = j; P.e_def[e] = mi[t]; P.e_dmin[e] = md[t]; P.e_dlong[e] = ml[t]; P.e_flags[e] = mf[t];
#pragma unroll
        for (int q = 0; q < 8; ++q) P.e_share[e * 8 + q] = 0ull;
      }
    }
    for (int ci = 0; ci < 4; ++ci) {
      const int cls = dep_class(ci);
      for (int lat = 0; lat < 2; ++lat) {
        const unsigned long long S = cj[cls * 2 + lat];
        if (!S) continue;
        int sel[kMaxSrc];
        int ns = 0;
        for (int t = 0; t < m; ++t)
          if (opcode_keeps(A, cls, P.opclass[mi[t]])) sel[ns++] = t;
        if (ns == 0) {  // no surviving source: the samples stay on j
          blame_add(P.blame + (size_t)j * kCnt + cls * 2 + lat, S);
          continue;
        }
        // Eq. 1: weight = issued samples / longest path, in units of 2^-20.
        unsigned long long wt[kMaxSrc];
        unsigned __int128 W = 0;
        for (int q = 0; q < ns; ++q) {
          const unsigned long long issue = P.cnt[(size_t)mi[sel[q]] * kCnt];
          const unsigned long long len = (unsigned long long)max(ml[sel[q]], 1);
          if (issue >> 43) set_status(P, ST_OVERFLOW);
          wt[q] = (unsigned long long)(((unsigned __int128)issue << 20) / len);
          W += wt[q];
        }
        if (W == 0) {
          for (int q = 0; q < ns; ++q) {
            wt[q] = (1ull << 20) / (unsigned long long)max(ml[sel[q]], 1);
            W += wt[q];
          }
        }
        if (W == 0) {
          for (int q = 0; q < ns; ++q) wt[q] = 1ull;
          W = (unsigned __int128)ns;
        }
        unsigned __int128 rem[kMaxSrc];
        unsigned long long sh[kMaxSrc];
        unsigned long long given = 0;
        for (int q = 0; q < ns; ++q) {
          const unsigned __int128 num = (unsigned __int128)S * wt[q];
          sh[q] = (unsigned long long)(num / W);
          rem[q] = num % W;
          given += sh[q];
        }
        // Largest remainders get the leftover units; ties go to the lower def index.
        unsigned long long left = S - given;
        while (left > 0) {
          int best = -1;
          for (int q = 0; q < ns; ++q) {
            if (rem[q] == (unsigned __int128)-1) continue;
            if (best < 0 || rem[q] > rem[best]) best = q;  // sel is in ascending def order
          }
          if (best < 0) break;  // cannot happen: fewer leftover units than sources
          sh[best] += 1;
          rem[best] = (unsigned __int128)-1;
          --left;
        }
        for (int q = 0; q < ns; ++q) {
          const int t = sel[q];
          P.e_share[(int64_t)(off + t) * 8 + ci * 2 + lat] = sh[q];
          if (sh[q]) blame_add(P.blame + (size_t)mi[t] * kCnt + cls * 2 + lat, sh[q]);
        }
      }
    }
  }
}

}  // namespace

void launch_blame(const Prog& P, const Arch& A, const SearchScratch& tier1, const SearchScratch& tier2, int max_src,
                  int32_t* scan_tmp, cudaStream_t st, int sms, int64_t* launches) {
  const int threads = 128;
  const int g_instr = grid_for(P.ni, threads, sms);
  cudaMemsetAsync(P.head, 0xFF, sizeof(int32_t) * (size_t)P.ni, st);
  k_blame_init<<<grid_for((int64_t)P.ni * kCnt, 256, sms), 256, 0, st>>>(P);
  k_search_local<<<g_instr, threads, 0, st>>>(P, A);
  k_search_general<<<(tier1.n_slots + 63) / 64, 64, 0, st>>>(P, A, tier1, 1);
  k_search_general<<<(tier2.n_slots + 31) / 32, 32, 0, st>>>(P, A, tier2, 2);
  k_merge_count<<<g_instr, threads, 0, st>>>(P, max_src);
  *launches += 5;
  scan_exclusive_inplace(P.edge_off, P.ni, scan_tmp, st, launches);
  k_apportion<<<g_instr, threads, 0, st>>>(P, A, max_src);
  ++*launches;
}

}  // namespace gpa
