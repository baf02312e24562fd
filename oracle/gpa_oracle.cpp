// CPU ORACLE for the GPA stall-blame path — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, literal restatement of what the dynamic analyzer computes
// (Zhou et al., "GPA: A GPU Performance Advisor Based on Instruction
// Sampling"): sample aggregation (Sec. 2.1), backward slicing with virtual
// barrier registers and predicate coverage (Sec. 4), the three pruning rules
// and the apportioning of Eq. 1 (Sec. 4), the detailed dependency classes
// (Sec. 4, Fig. 6), the optimizers of Table 2 and the estimators of Eq. 2, 4
// and 5 (Sec. 5). Only the tests, the package smoke check and the bench's CPU
// baseline may load this library; the product path never does. It shares no
// code, header or table with the CUDA implementation: both are fed the same
// arrays by the synthetic-input module and nothing else.
//
// Everything is done at instruction granularity with std::map/std::set and
// explicit graph searches; nothing is blocked, fused or reordered.

#include <algorithm>
#include <array>
#include <cstdint>
#include <cstring>
#include <deque>
#include <limits>
#include <map>
#include <set>
#include <vector>

namespace {

constexpr int kNumRes = 268;
constexpr int kPredBase = 255;
constexpr int kBarBase = 262;
constexpr int kNumClass = 12;
constexpr uint16_t kAll = 0xFFFF;  // the literal set that contains "_"

// Opcode-class property bits (values of the architecture table).
constexpr uint32_t F_MEM = 1, F_SYNC = 2, F_GLOBAL = 4, F_LOCAL = 8, F_CONST = 16, F_SHARED = 32,
                   F_LONG_ARITH = 64, F_VARLAT = 128;

enum { C_SELECTED = 0, C_INST_FETCH = 1, C_EXEC = 2, C_MEM = 3, C_SYNC = 5, C_CONST_MEM = 6,
       C_MEM_THROTTLE = 8 };
// Optimizers of Table 2 built here, in this fixed enumeration order.
enum { O_REG_REUSE, O_STRENGTH_RED, O_FUNC_SPLIT, O_FAST_MATH, O_WARP_BALANCE, O_MEM_TXN_RED,
       O_LOOP_UNROLL, O_CODE_REORDER, O_FUNC_INLINE, N_OPT };
constexpr int kDepClass[4] = {C_EXEC, C_MEM, C_SYNC, C_CONST_MEM};

}  // namespace

extern "C" {

struct OProg {
  int32_t nf, ni, nb, nl, n_lines;
  const int32_t *func_instr_off, *func_block_off, *func_loop_off;
  const int32_t *block_instr_off, *succ_off, *succ;
  const uint8_t *opclass, *guard, *iflags;
  const int32_t* line;
  const int32_t* def_off;
  const uint16_t* def_res;
  const int32_t* use_off;
  const uint16_t* use_res;
  const int32_t *block_loop, *loop_parent, *loop_header;
  int32_t n_calls;                          // call table: call instruction -> called function
  const int32_t *call_site, *call_callee;
};

struct OArch {
  int32_t n_op;
  const int32_t* latency;
  const uint32_t* flags;
};

}  // extern "C"

namespace {

// ------------------------------------------------------------------ Sec. 2.1
// Sample layout (most significant first): kernel 16 | pc 24 | class 4 |
// latency flag 1 | sm 8 | 11 reserved bits.
struct Decoded { uint64_t kernel, pc, cls, lat, sm, reserved; };
Decoded decode(uint64_t s) {
  return {s >> 48, (s >> 24) & 0xFFFFFF, (s >> 20) & 0xF, (s >> 19) & 1, (s >> 11) & 0xFF, s & 0x7FF};
}

// ------------------------------------------------------------------ helpers
bool defines(const OProg& P, int x, int r) {
  for (int e = P.def_off[x]; e < P.def_off[x + 1]; ++e)
    if ((P.def_res[e] & 0x1FF) == r) return true;
  return false;
}
int def_kind(const OProg& P, int x, int r) {
  for (int e = P.def_off[x]; e < P.def_off[x + 1]; ++e)
    if ((P.def_res[e] & 0x1FF) == r) return (P.def_res[e] >> 12) & 3;
  return -1;
}
bool uses(const OProg& P, int x, int r) {
  for (int e = P.use_off[x]; e < P.use_off[x + 1]; ++e)
    if ((P.use_res[e] & 0x1FF) == r) return true;
  return false;
}

// ------------------------------------------------------------------ Sec. 4, predicates
// A literal set P is a 14-bit mask: bit i = Pi, bit 7+i = !Pi; kAll stands for
// a set containing "_" (no guard, or both Pi and !Pi).
int lit_bit(int g) { return g <= 7 ? g - 1 : 7 + (g - 8); }
uint16_t add_literal(uint16_t S, int g) {
  if (S == kAll || g == 0) return kAll;
  S = (uint16_t)(S | (1u << lit_bit(g)));
  for (int i = 0; i < 7; ++i)
    if ((S >> i & 1) && (S >> (7 + i) & 1)) return kAll;
  return S;
}
// "P contains p'" iff p' in P or "_" in P.
bool contains(uint16_t S, int pguard) {
  if (S == kAll) return true;
  if (pguard == 0) return false;
  return (S >> lit_bit(pguard)) & 1;
}

// ------------------------------------------------------------------ per-function CFG facts
struct Fn {
  const OProg* P;
  int f, i0, i1, b0, b1;
  int nbf;
  std::vector<std::vector<int>> bsucc, bpred;      // local block ids
  std::vector<std::vector<uint64_t>> dom;          // bit d of dom[b]: d dominates b
  std::vector<int> iblock;                         // local instruction -> local block
  std::vector<int> topo;                           // local instruction -> forward topological position
  std::vector<char> reach;                         // block reachable from the entry

  int first(int b) const { return P->block_instr_off[b0 + b] - i0; }
  int last(int b) const { return P->block_instr_off[b0 + b + 1] - 1 - i0; }
  // Edge u -> v is a back edge iff v dominates u.
  bool back(int u, int v) const { return (dom[u][v >> 6] >> (v & 63)) & 1; }

  explicit Fn(const OProg& prog, int fid) : P(&prog), f(fid) {
    i0 = prog.func_instr_off[f]; i1 = prog.func_instr_off[f + 1];
    b0 = prog.func_block_off[f]; b1 = prog.func_block_off[f + 1];
    nbf = b1 - b0;
    bsucc.assign(nbf, {}); bpred.assign(nbf, {});
    for (int b = 0; b < nbf; ++b)
      for (int e = prog.succ_off[b0 + b]; e < prog.succ_off[b0 + b + 1]; ++e) {
        int s = prog.succ[e] - b0;
        bsucc[b].push_back(s);
        bpred[s].push_back(b);
      }
    iblock.assign(i1 - i0, 0);
    for (int b = 0; b < nbf; ++b)
      for (int x = first(b); x <= last(b); ++x) iblock[x] = b;
    // Reachability from the entry block.
    reach.assign(nbf, 0);
    std::vector<int> st = {0};
    reach[0] = 1;
    while (!st.empty()) {
      int b = st.back(); st.pop_back();
      for (int s : bsucc[b]) if (!reach[s]) { reach[s] = 1; st.push_back(s); }
    }
    // Dominators by the textbook iterative data-flow definition:
    // Dom(entry) = {entry}; Dom(b) = {b} U intersection of Dom(p) over reachable preds p.
    const int nw = (nbf + 63) / 64;
    dom.assign(nbf, std::vector<uint64_t>(nw, ~0ULL));
    std::fill(dom[0].begin(), dom[0].end(), 0ULL);
    dom[0][0] = 1;
    for (bool changed = true; changed;) {
      changed = false;
      for (int b = 1; b < nbf; ++b) {
        if (!reach[b]) continue;
        std::vector<uint64_t> nd(nw, ~0ULL);
        bool any = false;
        for (int p : bpred[b]) {
          if (!reach[p]) continue;
          any = true;
          for (int w = 0; w < nw; ++w) nd[w] &= dom[p][w];
        }
        if (!any) std::fill(nd.begin(), nd.end(), 0ULL);
        nd[b >> 6] |= 1ULL << (b & 63);
        if (nd != dom[b]) { dom[b] = nd; changed = true; }
      }
    }
    // Forward topological order of the instruction graph without back edges (Kahn).
    std::vector<int> indeg(nbf, 0);
    for (int b = 0; b < nbf; ++b)
      for (int s : bsucc[b]) if (!back(b, s)) ++indeg[s];
    std::deque<int> q;
    for (int b = 0; b < nbf; ++b) if (indeg[b] == 0) q.push_back(b);
    std::vector<int> border;
    while (!q.empty()) {
      int b = q.front(); q.pop_front();
      border.push_back(b);
      for (int s : bsucc[b]) if (!back(b, s) && --indeg[s] == 0) q.push_back(s);
    }
    topo.assign(i1 - i0, 0);
    int pos = 0;
    for (int b : border)
      for (int x = first(b); x <= last(b); ++x) topo[x] = pos++;
  }

  // Instruction-level predecessors of local instruction x, with back-edge flags.
  void ipreds(int x, std::vector<std::pair<int, int>>& out) const {
    out.clear();
    int b = iblock[x];
    if (x > first(b)) { out.push_back({x - 1, 0}); return; }
    for (int p : bpred[b]) out.push_back({last(p), back(p, b) ? 1 : 0});
  }
};

// ------------------------------------------------------------------ Sec. 4, backward slicing
struct SrcRes {
  int i;        // local instruction index of the source (def)
  int dmin;     // shortest source path, in instructions (adjacent = 1)
  int K;        // fewest loop back edges on any source path
  int dlong;    // longest source path that uses exactly K back edges
  bool dom;     // dominator-based pruning removes i -> j for this resource
};

// For use j (local) and resource r, search backward over states (x, S), S the
// union of guard literals of the defs of r met so far (Sec. 4, predicated
// instructions). A def x of r met while S does not contain j's guard is an
// immediate source; the path stops once S contains it. Then distances, back
// edge counts, longest paths and the single-k dominator rule are computed over
// the set of source paths.
//
// With `latency` given, the dominator rule is only evaluated for sources whose
// shortest path passes the latency rule (the others are dropped by rule 3
// whatever rule 2 says); without it, for every source.
std::vector<SrcRes> search(const Fn& F, int j, int r, const int32_t* latency = nullptr) {
  const OProg& P = *F.P;
  const int gj = P.guard[F.i0 + j];
  std::map<std::pair<int, uint16_t>, int> id;
  std::vector<int> sx;
  std::vector<uint16_t> sS;
  std::vector<std::vector<std::pair<int, int>>> adj;
  std::deque<int> work;
  auto get = [&](int x, uint16_t S) {
    auto key = std::make_pair(x, S);
    auto it = id.find(key);
    if (it != id.end()) return it->second;
    int s = (int)sx.size();
    id[key] = s;
    sx.push_back(x); sS.push_back(S); adj.emplace_back();
    work.push_back(s);
    return s;
  };
  std::vector<std::pair<int, int>> pr;
  std::vector<std::pair<int, int>> roots;  // (state, back flag of the edge into j)
  F.ipreds(j, pr);
  for (auto [y, bk] : pr) roots.push_back({get(y, 0), bk});
  while (!work.empty()) {
    int s = work.front(); work.pop_front();
    int x = sx[s];
    uint16_t S = sS[s];
    if (defines(P, F.i0 + x, r)) {
      S = add_literal(S, P.guard[F.i0 + x]);
      if (contains(S, gj)) continue;  // covered: this path stops here
    }
    std::vector<std::pair<int, int>> pp;
    F.ipreds(x, pp);
    for (auto [y, bk] : pp) {
      int t = get(y, S);
      adj[s].push_back({t, bk});
    }
  }
  const int ns = (int)sx.size();
  auto is_occ = [&](int s) { return defines(P, F.i0 + sx[s], r) && !contains(sS[s], gj); };

  // Shortest distance (unit edges; a root is one instruction away from j).
  std::vector<int> dist(ns, -1);
  {
    std::deque<int> q;
    for (auto [s, bk] : roots) if (dist[s] < 0) { dist[s] = 1; q.push_back(s); }
    while (!q.empty()) {
      int s = q.front(); q.pop_front();
      for (auto [t, bk] : adj[s]) if (dist[t] < 0) { dist[t] = dist[s] + 1; q.push_back(t); }
    }
  }
  // Fewest back edges (0-1 BFS).
  std::vector<int> kmin(ns, std::numeric_limits<int>::max());
  {
    std::deque<int> q;
    for (auto [s, bk] : roots) if (bk < kmin[s]) { kmin[s] = bk; if (bk) q.push_back(s); else q.push_front(s); }
    while (!q.empty()) {
      int s = q.front(); q.pop_front();
      for (auto [t, bk] : adj[s]) {
        int nk = kmin[s] + bk;
        if (nk < kmin[t]) { kmin[t] = nk; if (bk) q.push_back(t); else q.push_front(t); }
      }
    }
  }
  std::map<int, SrcRes> src;
  for (int s = 0; s < ns; ++s) {
    if (!is_occ(s)) continue;
    int i = sx[s];
    auto it = src.find(i);
    if (it == src.end()) src[i] = SrcRes{i, dist[s], kmin[s], -1, false};
    else { it->second.dmin = std::min(it->second.dmin, dist[s]); it->second.K = std::min(it->second.K, kmin[s]); }
  }
  if (src.empty()) return {};
  // Longest path with exactly K back edges: layered graph, layer = back edges
  // used so far. Within a layer, edges follow forward CFG edges backwards, so
  // decreasing forward-topological position is a valid processing order.
  int maxK = 0;
  for (auto& kv : src) maxK = std::max(maxK, kv.second.K);
  std::vector<int> order(ns);
  for (int s = 0; s < ns; ++s) order[s] = s;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (F.topo[sx[a]] != F.topo[sx[b]]) return F.topo[sx[a]] > F.topo[sx[b]];
    return a < b;
  });
  std::vector<std::vector<int>> dl(maxK + 1, std::vector<int>(ns, -1));
  for (auto [s, bk] : roots) if (bk <= maxK) dl[bk][s] = std::max(dl[bk][s], 1);
  for (int layer = 0; layer <= maxK; ++layer)
    for (int s : order) {
      if (dl[layer][s] < 0) continue;
      for (auto [t, bk] : adj[s]) {
        int nl = layer + bk;
        if (nl <= maxK) dl[nl][t] = std::max(dl[nl][t], dl[layer][s] + 1);
      }
    }
  for (int s = 0; s < ns; ++s) {
    if (!is_occ(s)) continue;
    SrcRes& R = src[sx[s]];
    R.dlong = std::max(R.dlong, dl[R.K][s]);
  }
  // Dominator-based pruning: remove i -> j if an unguarded instruction k
  // (k not i, not j) that uses r lies on every source path from i to j, i.e.
  // removing k's states disconnects j from every source state of i.
  auto needs_dom = [&](const SrcRes& R) {
    return !R.dom && (!latency || R.dmin <= latency[P.opclass[F.i0 + R.i]]);
  };
  std::set<int> cand;
  for (int s = 0; s < ns; ++s) {
    int k = sx[s];
    if (k != j && P.guard[F.i0 + k] == 0 && uses(P, F.i0 + k, r)) cand.insert(k);
  }
  for (int k : cand) {
    bool any = false;
    for (auto& kv : src) any = any || needs_dom(kv.second);
    if (!any) break;
    std::vector<char> seen(ns, 0);
    std::deque<int> q;
    for (auto [s, bk] : roots) if (sx[s] != k && !seen[s]) { seen[s] = 1; q.push_back(s); }
    while (!q.empty()) {
      int s = q.front(); q.pop_front();
      for (auto [t, bk] : adj[s]) if (sx[t] != k && !seen[t]) { seen[t] = 1; q.push_back(t); }
    }
    std::set<int> still;
    for (int s = 0; s < ns; ++s) if (seen[s] && is_occ(s)) still.insert(sx[s]);
    for (auto& kv : src)
      if (needs_dom(kv.second) && kv.first != k && !still.count(kv.first)) kv.second.dom = true;
  }
  std::vector<SrcRes> out;
  for (auto& kv : src) out.push_back(kv.second);
  return out;
}

// ------------------------------------------------------------------ Sec. 4, blame
struct Edge {
  int j, i;           // global instruction indices
  int dmin, dlong;
  uint32_t flags;     // 1 WAR, 2 via barrier, 4 via register, 8 via predicate
  uint64_t share[4][2];
};

struct Advice {
  uint64_t T = 0, A = 0, L = 0, issued = 0;
  uint64_t M[N_OPT] = {0};
  double speedup[N_OPT] = {0};
  int32_t rank[N_OPT] = {0};
  // hotspots[o][h] = def pc, use pc, def line, use line, distance, samples
  int64_t hot[N_OPT][5][6];
  int32_t n_hot[N_OPT] = {0};
};

struct Result {
  int f_lo, f_hi, i_lo, i_hi, l_lo, l_hi;
  std::vector<Edge> edges;
  std::vector<uint64_t> blame;           // (i_hi - i_lo) * 24
  std::vector<Advice> adv;               // per function
  std::vector<uint64_t> loop_A, loop_ML; // per loop of the range
  std::vector<double> loop_S;
  std::vector<uint64_t> line_stall, line_lat;  // per line of the whole program (only this range filled)
};

bool opcode_keeps(const OArch& arch, int c, int op) {
  uint32_t fl = arch.flags[op];
  if (c == C_MEM || c == C_CONST_MEM) return (fl & F_MEM) != 0;   // memory instructions only
  if (c == C_SYNC) return (fl & F_SYNC) != 0;                      // synchronization instructions only
  return true;                                                      // execution dependency: no opcode rule
}

// Eq. 1 in integers: weight_i = floor(issue_i * 2^20 / longest path_i); shares
// floor(S * w_i / W), remainder one unit at a time to the largest
// (S * w_i mod W), ties to the lower def index.
void apportion(uint64_t S, const std::vector<uint64_t>& issue, const std::vector<int>& dlong,
               const std::vector<int>& def_idx, std::vector<uint64_t>& share) {
  const size_t n = issue.size();
  std::vector<uint64_t> w(n);
  unsigned __int128 W = 0;
  for (size_t t = 0; t < n; ++t) { w[t] = (uint64_t)(((unsigned __int128)issue[t] << 20) / (uint64_t)dlong[t]); W += w[t]; }
  if (W == 0) {
    for (size_t t = 0; t < n; ++t) { w[t] = ((uint64_t)1 << 20) / (uint64_t)dlong[t]; W += w[t]; }
  }
  if (W == 0) { for (size_t t = 0; t < n; ++t) w[t] = 1; W = n; }
  share.assign(n, 0);
  std::vector<unsigned __int128> rem(n);
  uint64_t given = 0;
  for (size_t t = 0; t < n; ++t) {
    unsigned __int128 num = (unsigned __int128)S * w[t];
    share[t] = (uint64_t)(num / W);
    rem[t] = num % W;
    given += share[t];
  }
  uint64_t R = S - given;
  std::vector<size_t> ord(n);
  for (size_t t = 0; t < n; ++t) ord[t] = t;
  std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) {
    if (rem[a] != rem[b]) return rem[a] > rem[b];
    return def_idx[a] < def_idx[b];
  });
  for (uint64_t t = 0; t < R; ++t) share[ord[t]] += 1;
}

int innermost_loop(const OProg& P, const Fn& F, int x_local) {
  return P.block_loop[F.b0 + F.iblock[x_local]];
}
bool loop_within(const OProg& P, int l, int anc) {  // l nested in anc (or equal)
  for (int q = l; q >= 0; q = P.loop_parent[q]) if (q == anc) return true;
  return false;
}
int lca_loop(const OProg& P, int a, int b) {
  for (int q = a; q >= 0; q = P.loop_parent[q]) if (loop_within(P, b, q)) return q;
  return -1;
}

double est(uint64_t T, uint64_t M) {
  if (T == 0) return 1.0;
  if (T == M) return std::numeric_limits<double>::infinity();
  return (double)T / (double)(T - M);
}

// Sec. 4 for one use j (local index) of function F: immediate sources over
// every resource j reads, the three pruning rules, and Eq. 1 for each
// dependency class and latency flag. Appends the surviving merged edges (with
// their shares) to `edges` and hands every share to add(def, class, latency
// flag, samples), or the samples to j itself when no source survives.
template <class AddBlame>
void blame_use(const OProg& P, const OArch& arch, const uint64_t* cnt, const Fn& F, int j, std::vector<Edge>& edges,
               AddBlame add) {
  const int i0 = F.i0;
  auto C = [&](int x, int c, int lat) { return cnt[(size_t)(i0 + x) * 24 + c * 2 + lat]; };
  bool stalled = false;
  for (int c : kDepClass) stalled = stalled || C(j, c, 0) || C(j, c, 1);
  if (!stalled) return;
  // Immediate sources over every resource j uses; parallel edges (i, j)
  // through several resources merge into one source i.
  std::map<int, Edge> m;
  for (int e = P.use_off[i0 + j]; e < P.use_off[i0 + j + 1]; ++e) {
    int r = P.use_res[e] & 0x1FF;
    for (const SrcRes& s : search(F, j, r, arch.latency)) {
      int op = P.opclass[i0 + s.i];
      bool survive = !s.dom && s.dmin <= arch.latency[op];  // dominator and latency pruning
      if (!survive) continue;
      auto it = m.find(s.i);
      if (it == m.end()) {
        Edge E{};
        E.j = i0 + j; E.i = i0 + s.i; E.dmin = s.dmin; E.dlong = s.dlong; E.flags = 0;
        it = m.emplace(s.i, E).first;
      } else {
        it->second.dmin = std::min(it->second.dmin, s.dmin);
        it->second.dlong = std::max(it->second.dlong, s.dlong);
      }
      Edge& E = it->second;
      if (r >= kBarBase) E.flags |= 2;
      else if (r >= kPredBase) E.flags |= 8;
      else E.flags |= 4;
      // Write-after-read: a variable-latency def reads a register that the use writes,
      // linked through a read barrier (Sec. 4, Fig. 6).
      if (r >= kBarBase && def_kind(P, i0 + s.i, r) == 2 && (arch.flags[op] & F_VARLAT)) {
        for (int d = P.def_off[i0 + j]; d < P.def_off[i0 + j + 1]; ++d) {
          int rr = P.def_res[d] & 0x1FF;
          if (rr < kPredBase && uses(P, i0 + s.i, rr)) E.flags |= 1;
        }
      }
    }
  }
  std::vector<Edge> ej;
  for (auto& kv : m) ej.push_back(kv.second);
  // Apportion each dependency class and latency flag separately (Eq. 1).
  for (int ci = 0; ci < 4; ++ci) {
    int c = kDepClass[ci];
    for (int lat = 0; lat < 2; ++lat) {
      uint64_t S = C(j, c, lat);
      if (!S) continue;
      std::vector<int> idx, dl, di;
      std::vector<uint64_t> iss;
      for (size_t t = 0; t < ej.size(); ++t) {
        if (!opcode_keeps(arch, c, P.opclass[ej[t].i])) continue;  // opcode pruning
        idx.push_back((int)t);
        iss.push_back(cnt[(size_t)ej[t].i * 24 + 0]);
        dl.push_back(ej[t].dlong);
        di.push_back(ej[t].i);
      }
      if (idx.empty()) { add(j, c, lat, S); continue; }  // no source survives: stays on j
      std::vector<uint64_t> sh;
      apportion(S, iss, dl, di, sh);
      for (size_t t = 0; t < idx.size(); ++t) {
        ej[idx[t]].share[ci][lat] = sh[t];
        add(ej[idx[t]].i - i0, c, lat, sh[t]);
      }
    }
  }
  for (auto& E : ej) edges.push_back(E);
}

void analyze_function(const OProg& P, const OArch& arch, const uint64_t* cnt, int f, Result& R) {
  Fn F(P, f);
  const int i0 = F.i0, n = F.i1 - F.i0;
  auto C = [&](int x, int c, int lat) { return cnt[(size_t)(i0 + x) * 24 + c * 2 + lat]; };
  auto Bl = [&](int x, int c, int lat) -> uint64_t& { return R.blame[(size_t)(i0 + x - R.i_lo) * 24 + c * 2 + lat]; };
  size_t e_begin = R.edges.size();

  // Non-dependency reasons stay where they were observed.
  for (int x = 0; x < n; ++x)
    for (int c = 0; c < kNumClass; ++c) {
      if (c == C_EXEC || c == C_MEM || c == C_SYNC || c == C_CONST_MEM) continue;
      for (int lat = 0; lat < 2; ++lat) Bl(x, c, lat) += C(x, c, lat);
    }

  for (int j = 0; j < n; ++j)
    blame_use(P, arch, cnt, F, j, R.edges, [&](int x, int c, int lat, uint64_t v) { Bl(x, c, lat) += v; });

  // ---------------------------------------------------------------- Sec. 5
  Advice A;
  for (int x = 0; x < n; ++x)
    for (int c = 0; c < kNumClass; ++c)
      for (int lat = 0; lat < 2; ++lat) {
        uint64_t v = C(x, c, lat);
        A.T += v;
        if (lat) A.L += v; else A.A += v;
        if (c == C_SELECTED && !lat) A.issued += v;
      }
  // Per-edge matched amounts for the edge-based optimizers.
  auto mem_detail = [&](const Edge& E, int c) {  // 0 local, 1 constant, 2 global
    uint32_t fl = arch.flags[P.opclass[E.i]];
    if (fl & F_LOCAL) return 0;
    if ((fl & F_CONST) || c == C_CONST_MEM) return 1;
    return 2;
  };
  auto edge_match = [&](const Edge& E, int o) -> uint64_t {
    uint32_t fl = arch.flags[P.opclass[E.i]];
    uint64_t v = 0;
    switch (o) {
      case O_REG_REUSE:
        for (int lat = 0; lat < 2; ++lat) {
          if (mem_detail(E, C_MEM) == 0) v += E.share[1][lat];
          if (mem_detail(E, C_CONST_MEM) == 0) v += E.share[3][lat];
        }
        return v;
      case O_STRENGTH_RED:
        if (fl & F_LONG_ARITH) v = E.share[0][0] + E.share[0][1];
        return v;
      case O_LOOP_UNROLL:
      case O_CODE_REORDER: {
        v = E.share[0][1];
        if (mem_detail(E, C_MEM) == 2) v += E.share[1][1];
        if (mem_detail(E, C_CONST_MEM) == 2) v += E.share[3][1];
        if (o == O_LOOP_UNROLL) {
          int li = innermost_loop(P, F, E.i - i0), lj = innermost_loop(P, F, E.j - i0);
          if (li < 0 || lj < 0 || lca_loop(P, li, lj) < 0) v = 0;
        }
        return v;
      }
    }
    return 0;
  };
  // Function Inlining (Table 2): is f a device function, is local x a call site
  // (a site or callee of -1 stands for one outside the program: it matches nothing).
  bool device_fn = false;
  for (int c = 0; c < P.n_calls; ++c) device_fn = device_fn || P.call_callee[c] == f;
  auto is_call_site = [&](int x) {
    for (int c = 0; c < P.n_calls; ++c)
      if (P.call_site[c] == i0 + x) return true;
    return false;
  };
  auto instr_match = [&](int x, int o) -> uint64_t {
    uint64_t v = 0;
    switch (o) {
      case O_FUNC_SPLIT: return C(x, C_INST_FETCH, 0) + C(x, C_INST_FETCH, 1);
      case O_FAST_MATH:
        if (P.iflags[i0 + x] & 1)
          for (int c = 1; c < kNumClass; ++c) v += C(x, c, 0) + C(x, c, 1);
        return v;
      case O_WARP_BALANCE: return C(x, C_SYNC, 0) + C(x, C_SYNC, 1);
      case O_MEM_TXN_RED:
        if (arch.flags[P.opclass[i0 + x]] & F_GLOBAL) v = C(x, C_MEM_THROTTLE, 0) + C(x, C_MEM_THROTTLE, 1);
        return v;
      case O_FUNC_INLINE:
        // Latency stall samples sampled in a device function (one that some
        // call site calls) or at a call instruction.
        if (device_fn || is_call_site(x))
          for (int c = 1; c < kNumClass; ++c) v += C(x, c, 1);
        return v;
    }
    return 0;
  };
  const bool edge_based[N_OPT] = {true, true, false, false, false, false, true, true, false};
  for (int o = 0; o < N_OPT; ++o) {
    std::vector<std::array<int64_t, 6>> cand;
    if (edge_based[o]) {
      for (size_t t = e_begin; t < R.edges.size(); ++t) {
        const Edge& E = R.edges[t];
        uint64_t v = edge_match(E, o);
        A.M[o] += v;
        if (v) cand.push_back({E.i - i0, E.j - i0, P.line[E.i], P.line[E.j], E.dmin, (int64_t)v});
      }
    } else {
      for (int x = 0; x < n; ++x) {
        uint64_t v = instr_match(x, o);
        A.M[o] += v;
        if (v) cand.push_back({x, x, P.line[i0 + x], P.line[i0 + x], 0, (int64_t)v});
      }
    }
    std::sort(cand.begin(), cand.end(), [](const std::array<int64_t, 6>& a, const std::array<int64_t, 6>& b) {
      if (a[5] != b[5]) return a[5] > b[5];
      if (a[0] != b[0]) return a[0] < b[0];
      return a[1] < b[1];
    });
    A.n_hot[o] = (int32_t)std::min<size_t>(5, cand.size());
    for (int h = 0; h < 5; ++h)
      for (int q = 0; q < 6; ++q) A.hot[o][h][q] = h < A.n_hot[o] ? cand[h][q] : -1;
    // Eq. 2 for stall elimination; Eq. 4 for latency hiding.
    const bool hiding = o == O_LOOP_UNROLL || o == O_CODE_REORDER || o == O_FUNC_INLINE;
    if (hiding) A.speedup[o] = est(A.T, std::min(A.A, A.M[o]));
    else A.speedup[o] = est(A.T, A.M[o]);
  }
  std::vector<int> ord(N_OPT);
  for (int o = 0; o < N_OPT; ++o) ord[o] = o;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return A.speedup[a] > A.speedup[b]; });
  for (int o = 0; o < N_OPT; ++o) A.rank[o] = ord[o];
  R.adv.push_back(A);

  // Scopes (Eq. 5): active samples of the loop body including nested loops, and
  // matched latency samples of edges whose innermost common loop is nested in l.
  const int l0 = P.func_loop_off[f], l1 = P.func_loop_off[f + 1];
  for (int l = l0; l < l1; ++l) {
    uint64_t Al = 0, MLl = 0;
    for (int x = 0; x < n; ++x) {
      int li = innermost_loop(P, F, x);
      if (li >= 0 && loop_within(P, li, l))
        for (int c = 0; c < kNumClass; ++c) Al += C(x, c, 0);
    }
    for (size_t t = e_begin; t < R.edges.size(); ++t) {
      const Edge& E = R.edges[t];
      int li = innermost_loop(P, F, E.i - i0), lj = innermost_loop(P, F, E.j - i0);
      if (li < 0 || lj < 0) continue;
      int q = lca_loop(P, li, lj);
      if (q >= 0 && loop_within(P, q, l)) MLl += edge_match(E, O_LOOP_UNROLL);
    }
    R.loop_A[l - R.l_lo] = Al;
    R.loop_ML[l - R.l_lo] = MLl;
    R.loop_S[l - R.l_lo] = est(A.T, std::min(Al, MLl));
  }
  // Lines: blamed stall samples (every reason but SELECTED) and their latency part.
  for (int x = 0; x < n; ++x)
    for (int c = 1; c < kNumClass; ++c) {
      R.line_stall[P.line[i0 + x]] += Bl(x, c, 0) + Bl(x, c, 1);
      R.line_lat[P.line[i0 + x]] += Bl(x, c, 1);
    }
}

}  // namespace

extern "C" {

// Counts per (instruction, class, latency flag), dense: cnt[global pc * 24 + class * 2 + lat].
// Invalid samples (unknown kernel, pc past the function, class >= 12, SELECTED
// with the latency flag, nonzero reserved bits) are counted apart.
int oracle_histogram(const OProg* P, const uint64_t* s, int64_t n, uint64_t* cnt, uint64_t* invalid) {
  std::map<uint64_t, uint64_t> h;
  uint64_t bad = 0;
  for (int64_t t = 0; t < n; ++t) {
    Decoded d = decode(s[t]);
    bool ok = d.kernel < (uint64_t)P->nf && d.cls < (uint64_t)kNumClass && !(d.cls == 0 && d.lat == 1) &&
              d.reserved == 0;
    if (ok) ok = d.pc < (uint64_t)(P->func_instr_off[d.kernel + 1] - P->func_instr_off[d.kernel]);
    if (!ok) { ++bad; continue; }
    ++h[s[t] >> 19];
  }
  std::memset(cnt, 0, sizeof(uint64_t) * (size_t)P->ni * 24);
  for (auto& kv : h) {
    uint64_t k = kv.first;
    uint64_t kernel = k >> 29, pc = (k >> 5) & 0xFFFFFF, cls = (k >> 1) & 0xF, lat = k & 1;
    cnt[((size_t)P->func_instr_off[kernel] + pc) * 24 + cls * 2 + lat] = kv.second;
  }
  *invalid = bad;
  return 0;
}

// Classic reaching definitions over def sites (predicated defs do not kill),
// worklist to the fixpoint, then the resource projection: bit r of RIN[b]
// (ROUT[b]) is set iff some def of r reaches the entry (exit) of b. 9 words per block.
int oracle_reaching(const OProg* P, int32_t f_lo, int32_t f_hi, uint32_t* rin, uint32_t* rout) {
  const int bb0 = P->func_block_off[f_lo];
  for (int f = f_lo; f < f_hi; ++f) {
    const int b0 = P->func_block_off[f], b1 = P->func_block_off[f + 1];
    const int i0 = P->func_instr_off[f], i1 = P->func_instr_off[f + 1];
    const int nbf = b1 - b0;
    // Def sites of the function: (instruction, resource), numbered in order.
    std::vector<int> site_res;
    std::vector<int> site_first(i1 - i0 + 1, 0);
    for (int x = i0; x < i1; ++x) {
      site_first[x - i0] = (int)site_res.size();
      for (int e = P->def_off[x]; e < P->def_off[x + 1]; ++e) site_res.push_back(P->def_res[e] & 0x1FF);
    }
    site_first[i1 - i0] = (int)site_res.size();
    const int ns = (int)site_res.size();
    const int nw = (ns + 63) / 64;
    std::vector<std::vector<uint64_t>> of_res(kNumRes, std::vector<uint64_t>(nw, 0));  // all sites of r
    for (int t = 0; t < ns; ++t) of_res[site_res[t]][t >> 6] |= 1ULL << (t & 63);
    using Bits = std::vector<uint64_t>;
    std::vector<Bits> IN(nbf, Bits(nw, 0)), OUT(nbf, Bits(nw, 0));
    std::vector<std::vector<int>> pred(nbf), succ(nbf);
    for (int b = 0; b < nbf; ++b)
      for (int e = P->succ_off[b0 + b]; e < P->succ_off[b0 + b + 1]; ++e) {
        succ[b].push_back(P->succ[e] - b0);
        pred[P->succ[e] - b0].push_back(b);
      }
    // Transfer through a block, instruction by instruction: an unguarded def
    // kills every other def site of its resource; every def generates its site.
    auto transfer = [&](int b, const Bits& in) {
      Bits cur = in;
      for (int x = P->block_instr_off[b0 + b]; x < P->block_instr_off[b0 + b + 1]; ++x)
        for (int t = site_first[x - i0]; t < site_first[x - i0 + 1]; ++t) {
          if (P->guard[x] == 0)
            for (int w = 0; w < nw; ++w) cur[w] &= ~of_res[site_res[t]][w];
          cur[t >> 6] |= 1ULL << (t & 63);
        }
      return cur;
    };
    std::deque<int> wl;
    std::vector<char> inwl(nbf, 1);
    for (int b = 0; b < nbf; ++b) wl.push_back(b);
    while (!wl.empty()) {
      int b = wl.front(); wl.pop_front(); inwl[b] = 0;
      Bits in(nw, 0);
      for (int p : pred[b])
        for (int w = 0; w < nw; ++w) in[w] |= OUT[p][w];
      IN[b] = in;
      Bits out = transfer(b, in);
      if (out != OUT[b]) {
        OUT[b] = out;
        for (int s2 : succ[b]) if (!inwl[s2]) { inwl[s2] = 1; wl.push_back(s2); }
      }
    }
    // Resource projection: r is set iff some def site of r is in the set.
    for (int b = 0; b < nbf; ++b) {
      uint32_t* wi = rin + (size_t)(b0 + b - bb0) * 9;
      uint32_t* wo = rout + (size_t)(b0 + b - bb0) * 9;
      std::memset(wi, 0, 36); std::memset(wo, 0, 36);
      for (int t = 0; t < ns; ++t) {
        const int r = site_res[t];
        if (IN[b][t >> 6] >> (t & 63) & 1) wi[r >> 5] |= 1u << (r & 31);
        if (OUT[b][t >> 6] >> (t & 63) & 1) wo[r >> 5] |= 1u << (r & 31);
      }
    }
  }
  return 0;
}

// Sources of global use j through resource r; returns the number written.
int oracle_search(const OProg* P, int32_t j, int32_t r, int32_t max_out, int32_t* i_out, int32_t* dmin,
                  int32_t* K, int32_t* dlong, uint8_t* dom) {
  int f = 0;
  while (P->func_instr_off[f + 1] <= j) ++f;
  Fn F(*P, f);
  std::vector<SrcRes> v = search(F, j - F.i0, r);
  int n = 0;
  for (const SrcRes& s : v) {
    if (n >= max_out) break;
    i_out[n] = F.i0 + s.i; dmin[n] = s.dmin; K[n] = s.K; dlong[n] = s.dlong; dom[n] = s.dom ? 1 : 0;
    ++n;
  }
  return (int)v.size();
}

// Single dependency coverage (Sec. 6, "Single Dependency Coverage"). The nodes
// of the dependency graph are the stalled uses (instructions with samples of a
// dependency class); a node is a single dependency node if no resource it
// reads has more than one incoming edge. Counted over the immediate sources of
// the backward slice (before pruning) and over the sources that survive the
// three rules: dominator, latency, and opcode for at least one of the use's
// stalled classes (after). out: nodes, single before, single after.
int oracle_coverage(const OProg* P, const OArch* arch, const uint64_t* cnt, int32_t f_lo, int32_t f_hi,
                    int64_t* out) {
  out[0] = out[1] = out[2] = 0;
  for (int f = f_lo; f < f_hi; ++f) {
    Fn F(*P, f);
    const int i0 = F.i0, n = F.i1 - F.i0;
    auto C = [&](int x, int c, int lat) { return cnt[(size_t)(i0 + x) * 24 + c * 2 + lat]; };
    for (int j = 0; j < n; ++j) {
      bool stalled = false;
      for (int c : kDepClass) stalled = stalled || C(j, c, 0) || C(j, c, 1);
      if (!stalled) continue;
      ++out[0];
      size_t most_all = 0, most_kept = 0;
      for (int e = P->use_off[i0 + j]; e < P->use_off[i0 + j + 1]; ++e) {
        const int r = P->use_res[e] & 0x1FF;
        const std::vector<SrcRes> v = search(F, j, r, arch->latency);
        size_t kept = 0;
        for (const SrcRes& s : v) {
          const int op = P->opclass[i0 + s.i];
          if (s.dom || s.dmin > arch->latency[op]) continue;  // dominator and latency pruning
          bool any_class = false;                            // opcode pruning
          for (int c : kDepClass)
            if ((C(j, c, 0) || C(j, c, 1)) && opcode_keeps(*arch, c, op)) any_class = true;
          if (any_class) ++kept;
        }
        most_all = std::max(most_all, v.size());
        most_kept = std::max(most_kept, kept);
      }
      if (most_all <= 1) ++out[1];
      if (most_kept <= 1) ++out[2];
    }
  }
  return 0;
}

// Checks the loop-nest input of function f against natural loops derived from
// dominators and back edges. Returns 0 when they agree; otherwise a code.
int oracle_check_loops(const OProg* P, int32_t f) {
  Fn F(*P, f);
  for (int b = 0; b < F.nbf; ++b) if (!F.reach[b]) return 1;
  std::map<int, std::set<int>> nat;  // header -> body
  for (int u = 0; u < F.nbf; ++u)
    for (int v : F.bsucc[u]) {
      if (!F.back(u, v)) { if (v <= u) return 2; continue; }
      std::set<int>& body = nat[v];
      body.insert(v);
      std::vector<int> st;
      if (!body.count(u)) { body.insert(u); st.push_back(u); }
      while (!st.empty()) {
        int x = st.back(); st.pop_back();
        for (int p : F.bpred[x]) if (!body.count(p)) { body.insert(p); st.push_back(p); }
      }
    }
  const int l0 = P->func_loop_off[f], l1 = P->func_loop_off[f + 1];
  if ((int)nat.size() != l1 - l0) return 3;
  for (int l = l0; l < l1; ++l) {
    int h = P->loop_header[l] - F.b0;
    auto it = nat.find(h);
    if (it == nat.end()) return 4;
    std::set<int> body;
    for (int b = 0; b < F.nbf; ++b) {
      int q = P->block_loop[F.b0 + b];
      if (q >= 0 && loop_within(*P, q, l)) body.insert(b);
    }
    if (body != it->second) return 5;
    int par = P->loop_parent[l];
    if (par >= 0) {
      // Parent must be the smallest loop strictly containing this one.
      std::set<int> pb;
      for (int b = 0; b < F.nbf; ++b) {
        int q = P->block_loop[F.b0 + b];
        if (q >= 0 && loop_within(*P, q, par)) pb.insert(b);
      }
      if (!std::includes(pb.begin(), pb.end(), body.begin(), body.end()) || pb == body) return 6;
    }
  }
  return 0;
}

// Blame, edges and advice for functions [f_lo, f_hi).
void* oracle_analyze(const OProg* P, const OArch* arch, const uint64_t* cnt, int32_t f_lo, int32_t f_hi) {
  auto* R = new Result();
  R->f_lo = f_lo; R->f_hi = f_hi;
  R->i_lo = P->func_instr_off[f_lo]; R->i_hi = P->func_instr_off[f_hi];
  R->l_lo = P->func_loop_off[f_lo]; R->l_hi = P->func_loop_off[f_hi];
  R->blame.assign((size_t)(R->i_hi - R->i_lo) * 24, 0);
  R->loop_A.assign(R->l_hi - R->l_lo, 0);
  R->loop_ML.assign(R->l_hi - R->l_lo, 0);
  R->loop_S.assign(R->l_hi - R->l_lo, 0);
  R->line_stall.assign(P->n_lines, 0);
  R->line_lat.assign(P->n_lines, 0);
  for (int f = f_lo; f < f_hi; ++f) analyze_function(*P, *arch, cnt, f, *R);
  return R;
}

// Surviving merged edges (with their Eq. 1 shares) of the given stalled uses
// only (global instruction indices, ascending): what oracle_analyze gives for
// those uses, without analyzing the others. Read with oracle_n_edges /
// oracle_get_edges; the handle holds no blame or advice.
void* oracle_edges_of_uses(const OProg* P, const OArch* arch, const uint64_t* cnt, int32_t n_uses,
                           const int32_t* uses) {
  auto* R = new Result();
  R->f_lo = R->f_hi = R->i_lo = R->i_hi = R->l_lo = R->l_hi = 0;
  int f = -1;
  Fn* F = nullptr;
  for (int t = 0; t < n_uses; ++t) {
    const int j = uses[t];
    if (f < 0 || j < P->func_instr_off[f] || j >= P->func_instr_off[f + 1]) {
      f = 0;
      while (P->func_instr_off[f + 1] <= j) ++f;
      delete F;
      F = new Fn(*P, f);
    }
    blame_use(*P, *arch, cnt, *F, j - F->i0, R->edges, [](int, int, int, uint64_t) {});
  }
  delete F;
  return R;
}

int64_t oracle_n_edges(void* h) { return (int64_t)((Result*)h)->edges.size(); }

void oracle_get_edges(void* h, int32_t* j, int32_t* i, int32_t* dmin, int32_t* dlong, uint32_t* flags,
                      uint64_t* share) {
  auto* R = (Result*)h;
  for (size_t t = 0; t < R->edges.size(); ++t) {
    const Edge& E = R->edges[t];
    j[t] = E.j; i[t] = E.i; dmin[t] = E.dmin; dlong[t] = E.dlong; flags[t] = E.flags;
    for (int c = 0; c < 4; ++c)
      for (int l = 0; l < 2; ++l) share[t * 8 + c * 2 + l] = E.share[c][l];
  }
}

void oracle_get_blame(void* h, uint64_t* out) {
  auto* R = (Result*)h;
  std::memcpy(out, R->blame.data(), R->blame.size() * sizeof(uint64_t));
}

// Per function of the range: tot[4] (T, A, L, issued), M[8], speedup[8],
// rank[8], n_hot[8], hot[8*5*6]; per loop: A, ML, S; per line: stall, latency.
void oracle_get_advice(void* h, uint64_t* tot, uint64_t* M, double* speedup, int32_t* rank, int32_t* n_hot,
                       int64_t* hot, uint64_t* loop_A, uint64_t* loop_ML, double* loop_S, uint64_t* line_stall,
                       uint64_t* line_lat) {
  auto* R = (Result*)h;
  for (size_t f = 0; f < R->adv.size(); ++f) {
    const Advice& A = R->adv[f];
    tot[f * 4 + 0] = A.T; tot[f * 4 + 1] = A.A; tot[f * 4 + 2] = A.L; tot[f * 4 + 3] = A.issued;
    for (int o = 0; o < N_OPT; ++o) {
      M[f * N_OPT + o] = A.M[o];
      speedup[f * N_OPT + o] = A.speedup[o];
      rank[f * N_OPT + o] = A.rank[o];
      n_hot[f * N_OPT + o] = A.n_hot[o];
      for (int t = 0; t < 5; ++t)
        for (int q = 0; q < 6; ++q) hot[((f * N_OPT + o) * 5 + t) * 6 + q] = A.hot[o][t][q];
    }
  }
  for (size_t l = 0; l < R->loop_A.size(); ++l) { loop_A[l] = R->loop_A[l]; loop_ML[l] = R->loop_ML[l]; loop_S[l] = R->loop_S[l]; }
  std::memcpy(line_stall, R->line_stall.data(), R->line_stall.size() * sizeof(uint64_t));
  std::memcpy(line_lat, R->line_lat.data(), R->line_lat.size() * sizeof(uint64_t));
}

void oracle_free(void* h) { delete (Result*)h; }

}  // extern "C"
