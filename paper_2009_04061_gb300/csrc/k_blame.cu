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
//    so nothing further can survive rule 2). If every predecessor block
//    through which a def of r arrives covers j's guard, those predecessors
//    are settled here too (one path per source); otherwise the (use,
//    resource) pair is queued.
//  * k_search_warp (k_search.cu): persistent warps pull queued (use,
//    resource) pairs and explore the (block, literal set) graph.
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

// Scans predecessor block p of j's block b0 bottom-up for resource r, from
// the literal set S left at the top of b0. Returns true if p covers j's
// guard. With emit, emits p's sources that survive rules 2 and 3: when every
// predecessor covers, a source has exactly one def-clear path (from j up to
// the top of b0, into p at its bottom and up to the source), so its shortest
// and longest distances are that path's length d0 + (last(p) - x), and
// rule 2 reduces to an unguarded reader of r below it in p (met first in the
// bottom-up scan). Defs above j in b0 are settled by the in-block scan.
__device__ bool scan_pred(const Prog& P, const Arch& A, int j, int r, int gj, int b0, int p, uint16_t S, int d0,
                          bool emit, int* n_all = nullptr, int* n_kept = nullptr, bool blocked = false) {
  const int first = P.block_instr_off[p], last = P.block_instr_off[p + 1] - 1;
  bool wall = false;
  int last_def_pos = -1;
  const size_t seg = (size_t)p * kEvBuckets + ev_bucket(r);  // p's events of r's bucket
  const int ev1 = P.ev_off[seg + 1];
  for (int t = P.ev_off[seg]; t < ev1; ++t) {
    const uint32_t ev = P.events[t];
    if ((int)(ev & 0x1FFu) != r) continue;
    const int pos = (int)(ev >> 16), x = first + pos;
    if (ev & 0x200u) {
      last_def_pos = pos;
      if (!contains(S, gj) && !(p == b0 && x < j)) {
        const int d = d0 + (last - x);
        const bool keep = !wall && d <= A.lat[P.opclass[x]];
        if (emit && keep) emit_raw(P, A, j, x, r, (int)((ev >> 10) & 3u), d, d);
        if (n_all) {  // coverage count
          ++*n_all;
          if (keep && !blocked && keeps_any(P, A, j, P.opclass[x])) ++*n_kept;
        }
        if (P.diag == 2 && n_all) xemit(P, j, x, r, d, p >= b0 ? 1 : 0, d, wall || blocked);
      }
      S = add_literal(S, (int)((ev >> 12) & 0xFu));
      if (contains(S, gj)) return true;
    } else if (!wall && pos != last_def_pos && x != j) {
      wall = true;
    }
  }
  return false;
}

// The stalled uses (instructions with dependency-class samples), appended a
// warp at a time: a tenth of the instructions on the batched workload, so the
// kernels that work per stalled use take them from this list with every lane
// busy instead of striding over all instructions. One instruction a thread
// over a grid that covers them all (the loads of many CTAs in flight); the
// dependency-class counters are words 4-7 and 10-13 of a row, read as four
// 16-byte pairs.
__global__ void k_stalled_list(Prog P) {
  static_assert(2 * GPA_EXEC_DEPENDENCY == 4 && 2 * GPA_MEMORY_DEPENDENCY == 6 && 2 * GPA_SYNC == 10 &&
                    2 * GPA_CONSTANT_MEMORY_DEPENDENCY == 12,
                "dependency-class words 4-7 and 10-13");
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  bool s = false;
  if (j < P.ni) {
    const ulonglong2* c = reinterpret_cast<const ulonglong2*>(P.cnt + (size_t)j * kCnt);
    const ulonglong2 a = c[2], b = c[3], d = c[5], e = c[6];
    s = (a.x | a.y | b.x | b.y | d.x | d.y | e.x | e.y) != 0ull;
  }
  const unsigned m = __ballot_sync(0xffffffffu, s);
  if (!m) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&P.stats[SS_SUSE_N], (unsigned long long)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (s) P.suse[base + __popc(m & ((1u << lane) - 1u))] = j;
}

// Thread per stalled use (from the stalled-use list).
__global__ void k_search_local(Prog P, Arch A) {
  const int n_suse = (int)P.stats[SS_SUSE_N];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_suse; k += gridDim.x * blockDim.x) {
    const int j = P.suse[k];
    const int gj = P.guard[j];
    const int b0 = P.instr_block[j];
    const int first = P.block_instr_off[b0];
    const int pj = j - first;
    for (int e = P.use_off[j]; e < P.use_off[j + 1]; ++e) {
      const int r = P.use_res[e] & 0x1FF;
      const size_t seg = (size_t)b0 * kEvBuckets + ev_bucket(r);  // b0's events of r's bucket
      const int ev0 = P.ev_off[seg], ev1 = P.ev_off[seg + 1];
      uint16_t S = 0;
      bool blocked = false, covered = false;
      int last_def_pos = -1;
      int n_all = 0, n_kept = 0;  // coverage count (P.diag)
      for (int t = ev0; t < ev1; ++t) {  // bottom-up
        const uint32_t ev = P.events[t];
        const int pos = (int)(ev >> 16);
        if (pos >= pj || (int)(ev & 0x1FFu) != r) continue;
        const int x = first + pos;
        if (ev & 0x200u) {
          last_def_pos = pos;
          if (!contains(S, gj)) {
            const int d = pj - pos;
            if (!P.diag) {
              if (d <= A.lat[P.opclass[x]]) emit_raw(P, A, j, x, r, (int)((ev >> 10) & 3u), d, d);
            } else {
              ++n_all;
              if (!blocked && d <= A.lat[P.opclass[x]] && keeps_any(P, A, j, P.opclass[x])) ++n_kept;
              if (P.diag == 2) xemit(P, j, x, r, d, 0, d, blocked);
            }
          }
          S = add_literal(S, (int)((ev >> 12) & 0xFu));
          if (contains(S, gj)) { covered = true; break; }
        } else if (pos != last_def_pos && !blocked) {
          // An unguarded reader on every path beyond this point: nothing
          // further survives rule 2 (the coverage count still counts it).
          blocked = true;
          if (!P.diag) break;
        }
      }
      if (P.diag && covered) { cov_add(P, e, n_all, n_kept); continue; }
      if (covered || (blocked && !P.diag)) continue;
      // Predecessors through which a def of r reaches b0 (distinct blocks).
      // If each covers j's guard inside itself, resolve here; otherwise queue
      // the general search.
      const int w = r >> 5;
      const uint32_t bit = 1u << (r & 31);
      const int q0 = P.pred_off[b0], q1 = P.pred_off[b0 + 1];
      auto counts = [&](int q) {
        const int p = P.pred[q];
        if (!(P.rout[(size_t)p * kWords + w] & bit)) return false;
        for (int q2 = q0; q2 < q; ++q2) if (P.pred[q2] == p) return false;
        return true;
      };
      bool any = false, all_cover = true;
      for (int q = q0; q < q1 && all_cover; ++q) {
        if (!counts(q)) continue;
        any = true;
        all_cover = scan_pred(P, A, j, r, gj, b0, P.pred[q], S, pj + 1, false);
      }
      if (!any) {
        if (P.diag) cov_add(P, e, n_all, n_kept);
        continue;
      }
      if (all_cover) {
        for (int q = q0; q < q1; ++q)
          if (counts(q))
            scan_pred(P, A, j, r, gj, b0, P.pred[q], S, pj + 1, !P.diag, P.diag ? &n_all : nullptr, &n_kept, blocked);
        if (P.diag) cov_add(P, e, n_all, n_kept);
        continue;
      }
      if (P.diag) cov_add(P, e, n_all, n_kept);  // the in-block part; the search adds the rest
      // A search known to outgrow the first tier goes straight to the tier
      // that held it before: the second tier's queue; the third tier's large
      // list (searches that had large_nodes nodes or more, started first) or
      // its region at the top of the first queue; or the fourth tier's region
      // at the top of the overflow queue.
      const uint32_t hint = P.tier_hint[e];
      const int4 task = make_int4(j, r, (int)S | (blocked ? 1 << 20 : 0), e);
      if (hint >= 4 && P.t4_nodes > 0) {
        const unsigned long long t = atomicAdd(&P.stats[SS_OVF3H_N], 1ull);
        if (t < (unsigned long long)P.queue_cap) P.ovf_queue[P.queue_cap - 1 - (int64_t)t] = task;
        else capacity(P, 8);
      } else if (hint >= 3) {
        bool placed = false;
        if (P.large_hint[e]) {
          const unsigned long long t = atomicAdd(&P.stats[SS_LARGE_N], 1ull);
          if (t < (unsigned long long)kLargeQueue) {
            P.large_queue[t] = task;
            placed = true;
          }
        }
        if (!placed) {
          const unsigned long long t = atomicAdd(&P.stats[SS_HINT3_N], 1ull);
          if (t < (unsigned long long)P.queue_cap) P.queue[P.queue_cap - 1 - (int64_t)t] = task;
          else capacity(P, 8);
        }
      } else {
        const int slot = hint == 2 ? SS_OVF_N : SS_QUEUE_N;
        int4* q = hint == 2 ? P.ovf_queue : P.queue;
        const unsigned long long t = atomicAdd(&P.stats[slot], 1ull);
        if (t < (unsigned long long)P.queue_cap) q[t] = task;
        else capacity(P, 8);
      }
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

__device__ __forceinline__ void blame_add(unsigned long long* addr, unsigned long long v) {
  cg::coalesced_group g = cg::coalesced_threads();
  cg::coalesced_group grp = cg::labeled_partition(g, (unsigned long long)(uintptr_t)addr);
  const unsigned long long sum = cg::reduce(grp, v, cg::plus<unsigned long long>());
  if (grp.thread_rank() == 0) atomicAdd(addr, sum);
}

// Distinct sources of use j over its raw edge list, using ids[cap] as scratch:
// the count, or -1 if there are more than cap.
__device__ int distinct_sources(const Prog& P, int j, int* ids, int cap) {
  int c = 0;
  for (int t = P.head[j]; t >= 0; t = P.raw[t].y) {
    const int i = P.raw[t].x;
    bool seen = false;
    for (int q = 0; q < c; ++q) seen |= ids[q] == i;
    if (seen) continue;
    if (c >= cap) return -1;
    ids[c++] = i;
  }
  return c;
}

// Uses with more distinct sources than a thread's arrays hold are listed for
// k_merge_big / k_apportion_big (shared-memory arrays, one CTA per use).
__global__ void k_merge_count(Prog P, int max_src) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.ni; j += gridDim.x * blockDim.x) {
    int ids[kMaxSrc];
    int c = distinct_sources(P, j, ids, min(max_src, kMaxSrc));
    if (c < 0 && max_src > kMaxSrc) {
      const unsigned long long k = atomicAdd(&P.stats[SS_BIG_N], 1ull);
      P.big_use[k] = j;  // k < ni: each use is listed at most once
      c = 0;             // k_merge_big writes the count
    } else if (c < 0) {
      capacity(P, 9);
      c = 0;
    }
    P.edge_off[j] = c;
  }
}

__global__ void k_merge_big(Prog P, int max_src) {
  __shared__ int ids[kBigSrc];
  const unsigned long long nbig = P.stats[SS_BIG_N];
  for (unsigned long long k = blockIdx.x; k < nbig; k += gridDim.x) {
    if (threadIdx.x == 0) {
      const int j = P.big_use[k];
      int c = distinct_sources(P, j, ids, min(max_src, kBigSrc));
      if (c < 0) { capacity(P, 9); c = 0; }
      P.edge_off[j] = c;
    }
    __syncthreads();
  }
}

// Merged edges of use j (ascending def index) and Eq. 1 shares of each of its
// dependency classes and latency flags, with arrays of capacity cap.
__device__ void apportion_use(const Prog& P, const Arch& A, int j, int off, int c, int* mi, int* md, int* ml,
                              uint32_t* mf, int* sel, unsigned long long* wt, unsigned __int128* rem,
                              unsigned long long* sh) {
  const unsigned long long* cj = P.cnt + (size_t)j * kCnt;
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
      int ns = 0;
      for (int t = 0; t < m; ++t)
        if (opcode_keeps(A, cls, P.opclass[mi[t]])) sel[ns++] = t;
      if (ns == 0) {  // no surviving source: the samples stay on j
        blame_add(P.blame + (size_t)j * kCnt + cls * 2 + lat, S);
        continue;
      }
      // Eq. 1: weight = issued samples / longest path, in units of 2^-20.
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

// Thread per stalled use (a use with edges is stalled: searches run for
// stalled uses only).
__global__ void k_apportion(Prog P, Arch A, int max_src) {
  const int n_suse = (int)P.stats[SS_SUSE_N];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_suse; k += gridDim.x * blockDim.x) {
    const int j = P.suse[k];
    const int off = P.edge_off[j];
    int c = P.edge_off[j + 1] - off;
    if (c > kMaxSrc) continue;  // k_apportion_big
    if (off + c > P.edge_cap) { capacity(P, 10); c = 0; }
    int mi[kMaxSrc], md[kMaxSrc], ml[kMaxSrc], sel[kMaxSrc];
    uint32_t mf[kMaxSrc];
    unsigned long long wt[kMaxSrc], sh[kMaxSrc];
    unsigned __int128 rem[kMaxSrc];
    apportion_use(P, A, j, off, c, mi, md, ml, mf, sel, wt, rem, sh);
  }
}

__global__ void k_apportion_big(Prog P, Arch A) {
  extern __shared__ __align__(16) unsigned char big_sm[];
  unsigned __int128* rem = reinterpret_cast<unsigned __int128*>(big_sm);
  unsigned long long* wt = reinterpret_cast<unsigned long long*>(rem + kBigSrc);
  unsigned long long* sh = wt + kBigSrc;
  int* mi = reinterpret_cast<int*>(sh + kBigSrc);
  int* md = mi + kBigSrc;
  int* ml = md + kBigSrc;
  int* sel = ml + kBigSrc;
  uint32_t* mf = reinterpret_cast<uint32_t*>(sel + kBigSrc);
  const unsigned long long nbig = P.stats[SS_BIG_N];
  for (unsigned long long k = blockIdx.x; k < nbig; k += gridDim.x) {
    if (threadIdx.x == 0) {
      const int j = P.big_use[k];
      const int off = P.edge_off[j];
      int c = P.edge_off[j + 1] - off;
      if (off + c > P.edge_cap) { capacity(P, 10); c = 0; }
      if (c > kMaxSrc) apportion_use(P, A, j, off, c, mi, md, ml, mf, sel, wt, rem, sh);
    }
    __syncthreads();
  }
}

// Single dependency coverage: a stalled use is a single dependency node when
// no resource it reads has more than one source (before pruning) or more than
// one kept source (after).
__global__ void k_coverage(Prog P) {
  unsigned long long nodes = 0, before = 0, after = 0, total = 0;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < P.ni; j += gridDim.x * blockDim.x) {
    if (!stalled(P, j)) continue;
    uint32_t most_all = 0, most_kept = 0;
    for (int e = P.use_off[j]; e < P.use_off[j + 1]; ++e) {
      const uint32_t c = P.cov_cnt[e];
      most_all = max(most_all, c & 0xFFFFu);
      most_kept = max(most_kept, c >> 16);
      total += c & 0xFFFFu;
    }
    ++nodes;
    before += most_all <= 1u;
    after += most_kept <= 1u;
  }
  for (int o = 16; o > 0; o >>= 1) {
    nodes += __shfl_xor_sync(0xffffffffu, nodes, o);
    before += __shfl_xor_sync(0xffffffffu, before, o);
    after += __shfl_xor_sync(0xffffffffu, after, o);
    total += __shfl_xor_sync(0xffffffffu, total, o);
  }
  if ((threadIdx.x & 31) == 0 && nodes) {
    atomicAdd(&P.stats[SS_COV], nodes);
    atomicAdd(&P.stats[SS_COV + 1], before);
    atomicAdd(&P.stats[SS_COV + 2], after);
    atomicAdd(&P.stats[SS_COV_ALL], total);
  }
}

}  // namespace

void launch_coverage(const Prog& P, const Arch& A, const SearchArena* tiers, const SearchFork* fork, cudaStream_t st,
                     int sms, int64_t* launches) {
  const int threads = 128;
  const int g_instr = grid_for(P.ni, threads, sms);
  // The per-use kernels take the stalled-use list (its length is known on the
  // device only): enough CTAs for every SM to hold as many warps as their
  // registers allow, each thread taking about one use on the batched workload.
  const int g_use = std::max(1, std::min(grid_for(P.ni, threads, sms) * 4, (P.ni + threads - 1) / threads));
  k_stalled_list<<<std::max(1, (P.ni + 255) / 256), 256, 0, st>>>(P);
  k_search_local<<<g_use, threads, 0, st>>>(P, A);
  *launches += 2;
  launch_search(P, A, tiers, fork, st, sms, launches);
  k_coverage<<<g_instr, threads, 0, st>>>(P);
  ++*launches;
}

void launch_blame(const Prog& P, const Arch& A, const SearchArena* tiers, const SearchFork* fork, int max_src,
                  int32_t* scan_tmp, cudaStream_t st, int sms, int64_t* launches) {
  const int threads = 128;
  const int g_instr = grid_for(P.ni, threads, sms);
  // The per-use kernels take the stalled-use list (its length is known on the
  // device only): enough CTAs for every SM to hold as many warps as their
  // registers allow, each thread taking about one use on the batched workload.
  const int g_use = std::max(1, std::min(grid_for(P.ni, threads, sms) * 4, (P.ni + threads - 1) / threads));
  cudaMemsetAsync(P.head, 0xFF, sizeof(int32_t) * (size_t)P.ni, st);
  k_blame_init<<<grid_for((int64_t)P.ni * kCnt, 256, sms), 256, 0, st>>>(P);
  k_stalled_list<<<std::max(1, (P.ni + 255) / 256), 256, 0, st>>>(P);
  k_search_local<<<g_use, threads, 0, st>>>(P, A);
  *launches += 3;
  launch_search(P, A, tiers, fork, st, sms, launches);
  k_merge_count<<<g_instr, threads, 0, st>>>(P, max_src);
  k_merge_big<<<sms, 32, 0, st>>>(P, max_src);
  *launches += 2;
  scan_exclusive_inplace(P.edge_off, P.ni, scan_tmp, st, launches);
  k_apportion<<<g_use, threads, 0, st>>>(P, A, max_src);
  const size_t big_smem = (size_t)kBigSrc * (16 + 8 + 8 + 4 * 5);
  allow_max_smem(k_apportion_big);
  k_apportion_big<<<sms, 32, big_smem, st>>>(P, A);
  *launches += 2;
}

}  // namespace gpa
