// Seeded synthetic workload generator for the GPA stall-blame path.
//
// Produces (1) SASS-like programs: structured CFGs (sequences, if/else
// diamonds, if-then, while and do-while natural loops) whose instructions
// carry opcode class, guard predicate, def list and use list over the
// 268 resources R0-R254, P0-P6 and the virtual barrier registers B0-B5
// (Sec. 2.2, Table 1; Sec. 4 "Virtual barrier registers"), and (2) packed
// 64-bit PC samples (Sec. 2.1) drawn from per-instruction hotness.
//
// This module holds none of the analysis arithmetic. It is shared input
// plumbing: both the CPU oracle and the CUDA path consume what it writes.
// Randomness is splitmix64 (Steele, Lea, Flood 2014), counter based for the
// samples so that any slice [n0, n0+n) of a stream can be regenerated alone.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ULL;

inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

struct Rng {
  uint64_t s;
  explicit Rng(uint64_t seed) : s(mix64(seed ^ 0x5851f42d4c957f2dULL)) {}
  uint64_t next() { s += kGolden; return mix64(s); }
  double uni() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
  int below(int n) { return n <= 1 ? 0 : (int)((next() >> 33) % (uint64_t)n); }
  int range(int lo, int hi) { return hi <= lo ? lo : lo + below(hi - lo + 1); }
  bool coin(double p) { return uni() < p; }
};

// Opcode classes (values are part of the data format, see synth/__init__.py).
enum Op : int {
  IADD, IMAD, FFMA, ISETP, MOV, BRA, BAR, MEMBAR, LDG, STG, LDS, STS,
  LDL, STL, LDC, ATOM, F2F, MUFU, DFMA, EXIT_, N_OP
};

constexpr int kRegBase = 0, kPredBase = 255, kBarBase = 262;
constexpr int kKindWrite = 1, kKindRead = 2;

struct Ins {
  uint8_t op = 0, guard = 0, flags = 0, prof = 0;
  int32_t line = 0;
  std::vector<uint16_t> defs, uses;
};
struct Blk {
  std::vector<Ins> ins;
  int term = 0;     // 0 fall-through, 1 conditional branch + fall, 2 branch, 3 exit
  int target = -1;
};
struct LoopRec { int header = -1, first = -1, last = -1, parent = -1; };

struct FnParams {
  int32_t n_instr, n_loops, max_depth, n_regs, ldg_pct, tmpl, guard_pct, pad_;
  double zipf_s;
  uint64_t seed;
};

struct LNode { std::vector<int> kids; int weight = 1; };

struct Fn {
  std::vector<Blk> blocks;
  std::vector<LoopRec> loops;
  std::vector<uint64_t> wcum;  // inclusive cumulative sampling weight per instruction
  int n_lines = 0;
};

struct Gen {
  Rng rng;
  FnParams p;
  Fn fn;
  // Register allocation model: temporaries have short live ranges and their
  // registers are reused once dead; parameters (base pointers, sizes) are
  // loaded at entry and never redefined; each loop owns an induction variable.
  std::vector<int> live_reg, live_uses;   // live temporaries, oldest first
  std::vector<int> addr_reg, addr_uses;   // live 64-bit address temporaries (first register of the pair)
  uint8_t rstate[256];                    // 0 free, 1 temporary, 2 long lived
  std::vector<int> params, param_pairs, ivs;
  int8_t wbar[256], rbar[256];
  int bar_prod[6];
  bool bar_read[6];
  std::vector<int> preds;
  int bar_rr = 0;
  int64_t icount = 0;
  int64_t arith_at[256];
  int line = 0;
  int cur_loop = -1;
  int sync_bar = -1, sync_left = 0;
  double mix[N_OP];
  std::vector<LNode> lnodes;

  explicit Gen(const FnParams& fp) : rng(fp.seed), p(fp) {
    std::memset(wbar, -1, sizeof wbar);
    std::memset(rbar, -1, sizeof rbar);
    std::memset(rstate, 0, sizeof rstate);
    for (int k = 0; k < 6; ++k) { bar_prod[k] = -1; bar_read[k] = false; }
    for (int r = 0; r < 256; ++r) arith_at[r] = -1000000;
    for (int o = 0; o < N_OP; ++o) mix[o] = 0;
    // Body opcode mix (percent): 15% LDG/STG (+LDC), 10% LDS/STS, 50% FFMA/IMAD/IADD,
    // 5% BAR, the rest ISETP/MOV and a sprinkle of local/const/conversion/MUFU.
    mix[LDG] = 9; mix[STG] = 5; mix[LDC] = 1; mix[LDS] = 6; mix[STS] = 4;
    mix[FFMA] = 20; mix[IMAD] = 15; mix[IADD] = 15; mix[BAR] = 5; mix[ISETP] = 12;
    mix[MOV] = 4; mix[LDL] = 1; mix[STL] = 1; mix[F2F] = 1; mix[MUFU] = 1;
    if (p.ldg_pct > 0 && p.ldg_pct != 9) {
      double others = 0;
      for (int o = 0; o < N_OP; ++o) if (o != LDG) others += mix[o];
      double scale = (100.0 - p.ldg_pct) / others;
      for (int o = 0; o < N_OP; ++o) if (o != LDG) mix[o] *= scale;
      mix[LDG] = p.ldg_pct;
    }
  }

  Op body_op() {
    double tot = 0;
    for (int o = 0; o < N_OP; ++o) tot += mix[o];
    double u = rng.uni() * tot;
    for (int o = 0; o < N_OP; ++o) { u -= mix[o]; if (u < 0) return (Op)o; }
    return IADD;
  }

  void free_reg(int r) { if (rstate[r] == 1) rstate[r] = 0; }
  int pick_src() {
    const double u = rng.uni();
    if (u < 0.08 && !params.empty()) return params[rng.below((int)params.size())];
    if (u < 0.16 && !ivs.empty()) return ivs[rng.below((int)ivs.size())];
    if (!live_reg.empty()) {
      const int w = (int)std::min<size_t>(6, live_reg.size());
      const int k = std::min(rng.below(w), rng.below(w));
      const int idx = (int)live_reg.size() - 1 - k;
      const int r = live_reg[idx];
      if (--live_uses[idx] <= 0) {
        free_reg(r);
        live_reg.erase(live_reg.begin() + idx);
        live_uses.erase(live_uses.begin() + idx);
      }
      return r;
    }
    if (!params.empty()) return params[rng.below((int)params.size())];
    return 0;
  }
  int n_uses() { int k = 1; while (k < 6 && rng.coin(0.45)) ++k; return k; }
  void evict_oldest() {
    if (!live_reg.empty()) {
      free_reg(live_reg[0]);
      live_reg.erase(live_reg.begin()); live_uses.erase(live_uses.begin());
    } else if (!addr_reg.empty()) {
      free_reg(addr_reg[0]); free_reg(addr_reg[0] + 1);
      addr_reg.erase(addr_reg.begin()); addr_uses.erase(addr_uses.begin());
    }
  }
  // An aligned run of `width` free registers, preferring low numbers as an allocator does.
  int alloc(int width) {
    for (int tries = 0; tries < 64; ++tries) {
      int seen = 0, pick = -1;
      const int skip = rng.below(4);
      for (int r = 0; r + width <= p.n_regs; r += width) {
        bool ok = true;
        for (int t = 0; t < width; ++t) ok = ok && rstate[r + t] == 0;
        if (!ok) continue;
        pick = r;
        if (seen++ == skip) break;
      }
      if (pick >= 0) return pick;
      if (live_reg.empty() && addr_reg.empty()) break;
      evict_oldest();
    }
    return 0;
  }
  int new_temp(int width) {
    const int d = alloc(width);
    for (int t = 0; t < width; ++t) {
      rstate[d + t] = 1;
      live_reg.push_back(d + t);
      live_uses.push_back(n_uses());
    }
    return d;
  }
  int pick_pair() {
    if (!addr_reg.empty() && rng.coin(0.6)) {
      const int idx = (int)addr_reg.size() - 1;
      const int r = addr_reg[idx];
      if (--addr_uses[idx] <= 0) {
        free_reg(r); free_reg(r + 1);
        addr_reg.erase(addr_reg.begin() + idx); addr_uses.erase(addr_uses.begin() + idx);
      }
      return r;
    }
    if (!param_pairs.empty()) return param_pairs[rng.below((int)param_pairs.size())];
    return 0;
  }
  static void add_unique(std::vector<uint16_t>& v, int x) {
    for (uint16_t y : v) if ((y & 0x1FF) == (x & 0x1FF)) return;
    v.push_back((uint16_t)x);
  }
  int fresh_barrier(const std::vector<int>& avoid) {
    for (int t = 0; t < 6; ++t) {
      int k = (bar_rr + t) % 6;
      if (std::find(avoid.begin(), avoid.end(), k) == avoid.end()) { bar_rr = (k + 1) % 6; return k; }
    }
    int k = bar_rr; bar_rr = (bar_rr + 1) % 6; return k;
  }
  void release_barrier(int k) {
    for (int r = 0; r < 256; ++r) {
      if (wbar[r] == k) wbar[r] = -1;
      if (rbar[r] == k) rbar[r] = -1;
    }
    bar_prod[k] = -1;
    bar_read[k] = false;
  }

  // guard: -1 draw at random, 0 none, else the literal (1+i for Pi, 8+i for !Pi).
  Ins build(Op op, int guard, int forced_dst = -1, int forced_w = 1) {
    Ins in;
    in.op = (uint8_t)op;
    std::vector<int> srcs, dsts;
    int pdef = -1;
    auto dst_w = [&](int w) {
      const int d = forced_dst >= 0 ? forced_dst : new_temp(w);
      for (int t = 0; t < (forced_dst >= 0 ? forced_w : w); ++t) dsts.push_back(d + t);
    };
    auto pair = [&]() { int a = pick_pair(); srcs.push_back(a); srcs.push_back(a + 1); };
    switch (op) {
      case IADD: dst_w(1); srcs.push_back(pick_src()); srcs.push_back(pick_src()); break;
      case IMAD:
        if (forced_dst < 0 && rng.coin(0.3)) {  // wide multiply-add producing a 64-bit address
          const int a = alloc(2);
          rstate[a] = rstate[a + 1] = 1;
          addr_reg.push_back(a); addr_uses.push_back(n_uses());
          dsts.push_back(a); dsts.push_back(a + 1);
          srcs.push_back(pick_src()); srcs.push_back(pick_src());
          const int b = pick_pair(); srcs.push_back(b); srcs.push_back(b + 1);
        } else {
          dst_w(1); for (int t = 0; t < 3; ++t) srcs.push_back(pick_src());
        }
        break;
      case FFMA:
        dst_w(1); for (int t = 0; t < 3; ++t) srcs.push_back(pick_src()); break;
      case DFMA: dst_w(2); pair(); pair(); break;
      case MOV: dst_w(1); srcs.push_back(pick_src()); break;
      case ISETP: pdef = rng.below(7); srcs.push_back(pick_src()); srcs.push_back(pick_src()); break;
      case F2F: dst_w(1); pair(); break;
      case MUFU: dst_w(1); srcs.push_back(pick_src()); break;
      case LDG: { int u = rng.below(10); dst_w(u < 6 ? 1 : (u < 9 ? 2 : 4)); pair(); break; }
      case STG: { pair(); srcs.push_back(pick_src()); if (rng.coin(0.3)) srcs.push_back(pick_src()); break; }
      case LDS: dst_w(rng.coin(0.7) ? 1 : 2); srcs.push_back(pick_src()); break;
      case STS: srcs.push_back(pick_src()); srcs.push_back(pick_src()); break;
      case LDL: dst_w(1); srcs.push_back(pick_src()); break;
      case STL: srcs.push_back(pick_src()); srcs.push_back(pick_src()); break;
      case LDC: dst_w(rng.coin(0.7) ? 1 : 2); if (forced_dst < 0 && rng.coin(0.5)) srcs.push_back(pick_src()); break;
      case ATOM: dst_w(1); pair(); srcs.push_back(pick_src()); break;
      default: break;  // BRA, BAR, MEMBAR, EXIT
    }
    if (guard < 0) {
      guard = 0;
      if (op != BAR && op != MEMBAR && op != BRA && op != EXIT_ && !preds.empty() && rng.coin(p.guard_pct / 100.0)) {
        int pk = preds[rng.below((int)preds.size())];
        guard = rng.coin(0.5) ? 1 + pk : 8 + pk;
      }
    }
    in.guard = (uint8_t)guard;

    // Wait mask: read-after-write on pending write barriers, write-after-read on
    // pending read barriers, and the trailing waits of a BAR that set a barrier.
    std::vector<int> waits;
    auto add_wait = [&](int k) { if (k >= 0 && std::find(waits.begin(), waits.end(), k) == waits.end()) waits.push_back(k); };
    for (int s : srcs) add_wait(wbar[s]);
    for (int d : dsts) add_wait(rbar[d]);
    if (sync_bar >= 0) { add_wait(sync_bar); if (--sync_left <= 0) sync_bar = -1; }

    bool e_mem = false, e_const = false, e_sync = (op == BAR), e_exec = false;
    for (int k : waits) {
      int pr = bar_prod[k];
      if (bar_read[k]) e_exec = true;
      else if (pr == LDG || pr == LDL || pr == ATOM) e_mem = true;
      else if (pr == LDC) e_const = true;
      else if (pr == BAR || pr == MEMBAR) e_sync = true;
      else if (pr == LDS || pr == F2F || pr == MUFU) e_exec = true;
    }
    for (int s : srcs) if (icount - arith_at[s] <= 6) e_exec = true;
    bool memop = (op == LDG || op == STG || op == ATOM || op == LDL || op == STL);
    in.prof = (uint8_t)((e_mem ? 1 : 0) | (e_const ? 2 : 0) | (e_sync ? 4 : 0) | (e_exec ? 8 : 0) | (memop ? 16 : 0));

    for (int s : srcs) add_unique(in.uses, kRegBase + s);
    if (guard) add_unique(in.uses, kPredBase + (guard <= 7 ? guard - 1 : guard - 8));
    for (int k : waits) add_unique(in.uses, kBarBase + k);
    for (int k : waits) if (bar_prod[k] >= 0 || bar_read[k]) release_barrier(k);

    for (int d : dsts) add_unique(in.defs, kRegBase + d);
    if (pdef >= 0) add_unique(in.defs, kPredBase + pdef);

    bool wset = (op == LDG || op == LDS || op == LDL || op == LDC || op == ATOM || op == F2F || op == MUFU);
    bool rset = (op == STG || op == STS || op == STL);
    bool bset = (op == BAR && rng.coin(0.5));
    if (wset || rset || bset) {
      int k = fresh_barrier(waits);
      release_barrier(k);
      bar_prod[k] = op;
      bar_read[k] = rset;
      in.defs.push_back((uint16_t)((kBarBase + k) | ((rset ? kKindRead : kKindWrite) << 12)));
      if (wset) for (int d : dsts) wbar[d] = (int8_t)k;
      if (rset) for (int s : srcs) rbar[s] = (int8_t)k;
      if (bset) { sync_bar = k; sync_left = rng.range(1, 3); }
    }
    bool fixed_lat = (op == IADD || op == IMAD || op == FFMA || op == MOV || op == DFMA);
    for (int d : dsts) {
      if (!wset) wbar[d] = -1;
      rbar[d] = -1;
      arith_at[d] = fixed_lat ? icount : -1000000;
    }
    if (pdef >= 0 && std::find(preds.begin(), preds.end(), pdef) == preds.end()) preds.push_back(pdef);
    if (op == MUFU) in.flags |= 1;  // instruction stands for a math-library call
    if (rng.coin(0.35)) ++line;
    in.line = line;
    ++icount;
    return in;
  }

  int new_block() { fn.blocks.emplace_back(); return (int)fn.blocks.size() - 1; }

  void fill(int b, int n) {
    for (int t = 0; t < n; ++t) {
      if (t + 1 < n && !preds.empty() && rng.coin(0.3 * p.guard_pct / 100.0)) {
        // A complementary guarded pair defining one register (the Fig. 4a shape).
        int pk = preds[rng.below((int)preds.size())];
        int d = new_temp(1);
        fn.blocks[b].ins.push_back(build(LDG, 1 + pk, d));
        fn.blocks[b].ins.push_back(build(rng.coin(0.5) ? LDC : IMAD, 8 + pk, d));
        ++t;
        continue;
      }
      fn.blocks[b].ins.push_back(build(body_op(), -1));
    }
  }

  void end_cbr(int b, int target, bool negate, int cond_src = -1) {
    Ins s = build(ISETP, 0);
    if (cond_src >= 0) add_unique(s.uses, kRegBase + cond_src);
    int pk = -1;
    for (uint16_t d : s.defs) if ((d & 0x1FF) >= kPredBase && (d & 0x1FF) < kBarBase) pk = (d & 0x1FF) - kPredBase;
    fn.blocks[b].ins.push_back(s);
    fn.blocks[b].ins.push_back(build(BRA, negate ? 8 + pk : 1 + pk));
    fn.blocks[b].term = 1;
    fn.blocks[b].target = target;
  }
  void end_br(int b, int target) {
    fn.blocks[b].ins.push_back(build(BRA, 0));
    fn.blocks[b].term = 2;
    fn.blocks[b].target = target;
  }

  void straight(int n) {
    n = std::max(n, 1);
    while (n > 0) {
      int sz = std::min(n, rng.range(5, 14));
      if (n - sz < 3) sz = n;
      int b = new_block();
      fill(b, sz);
      n -= sz;
    }
  }

  void filler(int budget) {
    if (budget < 16) { straight(budget); return; }
    double u = rng.uni();
    if (u < 0.40) {
      int a = rng.range(budget / 4, budget * 3 / 4);
      filler(a);
      filler(budget - a);
    } else if (u < 0.75 && budget >= 24) {
      int csz = rng.range(4, 11);
      int c = new_block(); fill(c, csz - 2); end_cbr(c, -1, rng.coin(0.5));
      int jsz = rng.range(3, 10);
      int rem = std::max(4, budget - csz - jsz);
      int tb = std::max(2, rng.range(rem / 3, rem * 2 / 3));
      int eb = std::max(2, rem - tb);
      filler(tb - 1);
      int tl = (int)fn.blocks.size() - 1;
      end_br(tl, -1);
      int else_start = (int)fn.blocks.size();
      filler(eb);
      int join = new_block(); fill(join, jsz);
      fn.blocks[c].target = else_start;
      fn.blocks[tl].target = join;
    } else {
      int csz = rng.range(4, 11);
      int c = new_block(); fill(c, csz - 2); end_cbr(c, -1, rng.coin(0.5));
      int jsz = rng.range(3, 10);
      filler(std::max(2, budget - csz - jsz));
      int join = new_block(); fill(join, jsz);
      fn.blocks[c].target = join;
    }
  }

  // Induction variable: set in the block that falls into the loop, stepped in the latch.
  int iv_begin() {
    const int iv = alloc(1);
    rstate[iv] = 2;
    fn.blocks.back().ins.push_back(build(MOV, 0, iv));
    ivs.push_back(iv);
    return iv;
  }
  void iv_step(int b, int iv) {
    Ins st = build(IADD, 0, iv);
    add_unique(st.uses, kRegBase + iv);
    fn.blocks[b].ins.push_back(st);
  }
  void iv_end(int iv) { ivs.pop_back(); rstate[iv] = 0; }

  void loop(int node, int budget) {
    int parent = cur_loop;
    int id = (int)fn.loops.size();
    fn.loops.emplace_back();
    fn.loops[id].parent = parent;
    cur_loop = id;
    const int iv = iv_begin();
    if (rng.coin(0.4)) {  // while loop: test at the top, unconditional latch
      int h = new_block(); fill(h, rng.range(0, 2)); end_cbr(h, -1, true, iv);
      fn.loops[id].header = h; fn.loops[id].first = h;
      seq(std::max(6, budget - 8), lnodes[node].kids);
      int l = new_block(); fill(l, rng.range(1, 3)); iv_step(l, iv); end_br(l, h);
      fn.loops[id].last = l;
      fn.blocks[h].target = l + 1;
    } else {              // do-while loop: test in the latch
      int first = (int)fn.blocks.size();
      seq(std::max(6, budget - 6), lnodes[node].kids);
      int l = new_block(); fill(l, rng.range(1, 3)); iv_step(l, iv); end_cbr(l, first, false, iv);
      fn.loops[id].header = first; fn.loops[id].first = first; fn.loops[id].last = l;
    }
    iv_end(iv);
    cur_loop = parent;
  }

  // Kernel parameters: base-pointer pairs and scalars loaded from constant
  // memory at entry and live for the whole function.
  void prologue(int b) {
    const int npairs = std::max(1, std::min(4, p.n_regs / 24));
    const int nsingle = std::max(1, std::min(4, p.n_regs / 24));
    for (int k = 0; k < npairs; ++k) {
      const int r = alloc(2);
      rstate[r] = rstate[r + 1] = 2;
      param_pairs.push_back(r);
      fn.blocks[b].ins.push_back(build(LDC, 0, r, 2));
    }
    for (int k = 0; k < nsingle; ++k) {
      const int r = alloc(1);
      rstate[r] = 2;
      params.push_back(r);
      fn.blocks[b].ins.push_back(build(LDC, 0, r, 1));
    }
  }

  void seq(int budget, const std::vector<int>& kids) {
    int nk = (int)kids.size();
    if (nk == 0) { filler(budget); return; }
    int wsum = 0;
    for (int k : kids) wsum += lnodes[k].weight;
    int kid_total = (int)(budget * 0.75);
    int fill_total = std::max(3 * (nk + 1), budget - kid_total);
    std::vector<int> fb(nk + 1, fill_total / (nk + 1));
    fb[0] += fill_total % (nk + 1);
    filler(std::max(3, fb[0]));
    for (int t = 0; t < nk; ++t) {
      int kb = std::max(12, (int)((int64_t)kid_total * lnodes[kids[t]].weight / wsum));
      loop(kids[t], kb);
      filler(std::max(3, fb[t + 1]));
    }
  }

  int compute_weight(int n) {
    int w = 1;
    for (int k : lnodes[n].kids) w += compute_weight(k);
    lnodes[n].weight = w;
    return w;
  }

  void generate() {
    if (p.tmpl == 1) { template_c1(); return; }
    // Random loop tree with n_loops nodes and depth at most max_depth.
    std::vector<int> roots, depth;
    for (int l = 0; l < p.n_loops; ++l) {
      lnodes.emplace_back();
      depth.push_back(1);
      std::vector<int> cand;
      for (int q = 0; q < l; ++q) if (depth[q] < p.max_depth) cand.push_back(q);
      if (!cand.empty() && rng.coin(0.55)) {
        int par = cand[rng.below((int)cand.size())];
        lnodes[par].kids.push_back(l);
        depth[l] = depth[par] + 1;
      } else {
        roots.push_back(l);
      }
    }
    for (int r : roots) compute_weight(r);
    const int e0 = new_block();
    prologue(e0);
    fill(e0, rng.range(2, 6));
    seq(std::max(8, p.n_instr - 4 - (int)fn.blocks[e0].ins.size()), roots);
    int e = new_block(); fill(e, 2); fn.blocks[e].ins.push_back(build(EXIT_, 0)); fn.blocks[e].term = 3;
  }

  // One function of 200 instructions in 12 blocks: two entry blocks, an
  // if/else diamond, a do-while loop of four blocks, two tail blocks.
  void template_c1() {
    int b0 = new_block(); prologue(b0); fill(b0, 18 - (int)fn.blocks[b0].ins.size());
    int b1 = new_block(); fill(b1, 16);
    int c = new_block(); fill(c, 12); end_cbr(c, -1, rng.coin(0.5));
    int t = new_block(); fill(t, 19); end_br(t, -1);
    int e = new_block(); fill(e, 18);
    int j = new_block(); fill(j, 15);
    fn.blocks[c].target = e; fn.blocks[t].target = j;
    fn.loops.emplace_back();
    const int iv = iv_begin();
    int h = new_block(); fill(h, 20);
    int m1 = new_block(); fill(m1, 18);
    int m2 = new_block(); fill(m2, 20);
    int l = new_block(); fill(l, 13); iv_step(l, iv); end_cbr(l, h, false, iv);
    iv_end(iv);
    fn.loops[0].header = h; fn.loops[0].first = h; fn.loops[0].last = l; fn.loops[0].parent = -1;
    int x1 = new_block(); fill(x1, 14);
    int x2 = new_block(); fill(x2, 9); fn.blocks[x2].ins.push_back(build(EXIT_, 0)); fn.blocks[x2].term = 3;
    (void)b1; (void)m1; (void)m2; (void)x1;
  }

  // Sampling weight: Zipf(s) over a seeded permutation of ranks, times 32 per
  // enclosing loop level; quantised so that a function's total stays below 2^47.
  void weights() {
    int n = 0;
    for (auto& b : fn.blocks) n += (int)b.ins.size();
    std::vector<int> depth_of(n, 0);
    int x = 0;
    for (int b = 0; b < (int)fn.blocks.size(); ++b) {
      int d = 0;
      for (auto& L : fn.loops) if (b >= L.first && b <= L.last) ++d;
      for (size_t t = 0; t < fn.blocks[b].ins.size(); ++t) depth_of[x++] = d;
    }
    std::vector<int> rank(n);
    for (int i = 0; i < n; ++i) rank[i] = i;
    for (int i = n - 1; i > 0; --i) std::swap(rank[i], rank[rng.below(i + 1)]);
    std::vector<double> w(n);
    double tot = 0;
    for (int i = 0; i < n; ++i) {
      w[i] = std::pow(32.0, depth_of[i]) / std::pow((double)rank[i] + 1.0, p.zipf_s);
      tot += w[i];
    }
    fn.wcum.resize(n);
    uint64_t acc = 0;
    const double scale = std::ldexp(1.0, 47) / tot;
    for (int i = 0; i < n; ++i) {
      uint64_t q = (uint64_t)std::floor(w[i] * scale);
      if (q == 0) q = 1;
      acc += q;
      fn.wcum[i] = acc;
    }
    fn.n_lines = line + 1;
  }
};

struct Program {
  int32_t nf = 0, ni = 0, nb = 0, nl = 0, ne = 0, nd = 0, nu = 0, n_lines = 0;
  std::vector<int32_t> func_instr_off, func_block_off, func_loop_off, func_line_off;
  std::vector<int32_t> block_instr_off, succ_off, succ;
  std::vector<uint8_t> opclass, guard, iflags, prof;
  std::vector<int32_t> line, def_off, use_off;
  std::vector<uint16_t> def_res, use_res;
  std::vector<int32_t> block_loop, loop_parent, loop_header;
  std::vector<uint64_t> wcum;    // per-instruction inclusive cumulative weight (function local)
  std::vector<uint64_t> kcum;    // per-function inclusive cumulative weight
  uint64_t pcum[32][24];         // per stall profile inclusive cumulative over (class, lat)
};

void build_profiles(Program& P) {
  // 30% SELECTED; 40% dependency stalls split over the classes the instruction
  // is eligible for; the rest over non-dependency reasons. Latency flag: 0 for
  // SELECTED, else a fair coin.
  for (int pf = 0; pf < 32; ++pf) {
    double pr[12] = {0};
    bool mem = pf & 1, cst = pf & 2, syn = pf & 4, exe = pf & 8, memop = pf & 16;
    pr[0] = 0.30;
    std::vector<int> dep;
    if (mem) dep.push_back(3);
    if (cst) dep.push_back(6);
    if (syn) dep.push_back(5);
    if (exe) dep.push_back(2);
    double other = 0.30;
    if (dep.empty()) other += 0.40;
    else for (int c : dep) pr[c] += 0.40 / dep.size();
    double ow[12] = {0};
    ow[1] = 0.25; ow[7] = 0.20; ow[9] = 0.25; ow[10] = 0.15; ow[4] = 0.05; ow[11] = 0.05;
    if (memop) ow[8] = 0.30;
    double os = 0;
    for (int c = 0; c < 12; ++c) os += ow[c];
    for (int c = 0; c < 12; ++c) pr[c] += other * ow[c] / os;
    double e[24] = {0};
    e[0] = pr[0];
    for (int c = 1; c < 12; ++c) { e[2 * c] = pr[c] * 0.5; e[2 * c + 1] = pr[c] * 0.5; }
    const double two32 = 4294967296.0;
    uint64_t acc = 0;
    int last_nz = 0;
    for (int t = 0; t < 24; ++t) {
      acc += (uint64_t)std::floor(e[t] * two32);
      P.pcum[pf][t] = acc;
      if (e[t] > 0) last_nz = t;
    }
    uint64_t fix = (uint64_t)1 << 32;
    for (int t = last_nz; t < 24; ++t) P.pcum[pf][t] += fix - acc;
  }
}

}  // namespace

extern "C" {

// Generates nf functions; params is an array of nf FnParams. kernel_zipf_s
// weighs kernels for sampling (Zipf over a seeded permutation). Returns a handle.
void* synth_program_new(int32_t nf, const FnParams* params, double kernel_zipf_s, uint64_t kseed, int32_t n_threads) {
  std::vector<Fn> fns(nf);
  int nt = std::max(1, std::min<int>(n_threads, nf));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    th.emplace_back([&, t]() {
      for (int f = t; f < nf; f += nt) {
        Gen g(params[f]);
        g.generate();
        g.weights();
        fns[f] = std::move(g.fn);
      }
    });
  }
  for (auto& x : th) x.join();

  auto* P = new Program();
  P->nf = nf;
  P->func_instr_off.push_back(0); P->func_block_off.push_back(0);
  P->func_loop_off.push_back(0); P->func_line_off.push_back(0);
  P->block_instr_off.push_back(0); P->succ_off.push_back(0);
  P->def_off.push_back(0); P->use_off.push_back(0);
  for (int f = 0; f < nf; ++f) {
    Fn& F = fns[f];
    int bbase = P->nb, lbase = P->nl, linebase = P->n_lines;
    for (int b = 0; b < (int)F.blocks.size(); ++b) {
      Blk& B = F.blocks[b];
      for (Ins& in : B.ins) {
        P->opclass.push_back(in.op); P->guard.push_back(in.guard);
        P->iflags.push_back(in.flags); P->prof.push_back(in.prof);
        P->line.push_back(linebase + in.line);
        for (uint16_t d : in.defs) P->def_res.push_back(d);
        for (uint16_t u : in.uses) P->use_res.push_back(u);
        P->def_off.push_back((int32_t)P->def_res.size());
        P->use_off.push_back((int32_t)P->use_res.size());
      }
      P->ni += (int)B.ins.size();
      P->block_instr_off.push_back(P->ni);
      std::vector<int> s;
      if (B.term == 0) s.push_back(b + 1);
      else if (B.term == 1) { s.push_back(b + 1); if (B.target != b + 1) s.push_back(B.target); }
      else if (B.term == 2) s.push_back(B.target);
      for (int x : s) P->succ.push_back(bbase + x);
      P->succ_off.push_back((int32_t)P->succ.size());
      int inner = -1, idepth = 0;
      for (int l = 0; l < (int)F.loops.size(); ++l) {
        if (b >= F.loops[l].first && b <= F.loops[l].last) {
          int d = 0;
          for (int q = l; q >= 0; q = F.loops[q].parent) ++d;
          if (d > idepth) { idepth = d; inner = l; }
        }
      }
      P->block_loop.push_back(inner < 0 ? -1 : lbase + inner);
    }
    for (auto& L : F.loops) {
      P->loop_parent.push_back(L.parent < 0 ? -1 : lbase + L.parent);
      P->loop_header.push_back(bbase + L.header);
    }
    for (uint64_t w : F.wcum) P->wcum.push_back(w);
    P->nb += (int)F.blocks.size();
    P->nl += (int)F.loops.size();
    P->n_lines += F.n_lines;
    P->func_instr_off.push_back(P->ni);
    P->func_block_off.push_back(P->nb);
    P->func_loop_off.push_back(P->nl);
    P->func_line_off.push_back(P->n_lines);
  }
  P->ne = (int)P->succ.size();
  P->nd = (int)P->def_res.size();
  P->nu = (int)P->use_res.size();

  // Kernel weights: Zipf(kernel_zipf_s) over a seeded permutation of function ids.
  Rng kr(kseed);
  std::vector<int> rank(nf);
  for (int i = 0; i < nf; ++i) rank[i] = i;
  for (int i = nf - 1; i > 0; --i) std::swap(rank[i], rank[kr.below(i + 1)]);
  std::vector<double> w(nf);
  double tot = 0;
  for (int i = 0; i < nf; ++i) { w[i] = 1.0 / std::pow((double)rank[i] + 1.0, kernel_zipf_s); tot += w[i]; }
  uint64_t acc = 0;
  for (int i = 0; i < nf; ++i) {
    uint64_t q = (uint64_t)std::floor(w[i] / tot * std::ldexp(1.0, 47));
    if (q == 0) q = 1;
    acc += q;
    P->kcum.push_back(acc);
  }
  build_profiles(*P);
  return P;
}

void synth_program_free(void* h) { delete (Program*)h; }

// sizes: nf, ni, nb, nl, ne(succ entries), nd(def entries), nu(use entries), n_lines
void synth_program_sizes(void* h, int64_t* out) {
  auto* P = (Program*)h;
  out[0] = P->nf; out[1] = P->ni; out[2] = P->nb; out[3] = P->nl;
  out[4] = P->ne; out[5] = P->nd; out[6] = P->nu; out[7] = P->n_lines;
}

void synth_program_copy(void* h, int32_t* func_instr_off, int32_t* func_block_off, int32_t* func_loop_off,
                        int32_t* func_line_off, int32_t* block_instr_off, int32_t* succ_off, int32_t* succ,
                        uint8_t* opclass, uint8_t* guard, uint8_t* iflags, uint8_t* prof, int32_t* line,
                        int32_t* def_off, uint16_t* def_res, int32_t* use_off, uint16_t* use_res,
                        int32_t* block_loop, int32_t* loop_parent, int32_t* loop_header) {
  auto* P = (Program*)h;
  auto cp = [](auto* dst, const auto& v) { if (!v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0])); };
  cp(func_instr_off, P->func_instr_off); cp(func_block_off, P->func_block_off);
  cp(func_loop_off, P->func_loop_off); cp(func_line_off, P->func_line_off);
  cp(block_instr_off, P->block_instr_off); cp(succ_off, P->succ_off); cp(succ, P->succ);
  cp(opclass, P->opclass); cp(guard, P->guard); cp(iflags, P->iflags); cp(prof, P->prof);
  cp(line, P->line); cp(def_off, P->def_off); cp(def_res, P->def_res);
  cp(use_off, P->use_off); cp(use_res, P->use_res);
  cp(block_loop, P->block_loop); cp(loop_parent, P->loop_parent); cp(loop_header, P->loop_header);
}

// Launch layout of a stream of `total` samples (Sec. 2.1: the profiler
// serializes kernel executions, so each launch's samples arrive as one run).
// Kernel k receives its share of `total` by cumulative rounding of the Zipf
// kernel weights, split into 1-8 launches (seeded); the launches of all
// kernels run in a seeded random order. starts has n_runs + 1 entries.
static void launch_runs(const Program& P, uint64_t seed, int64_t total, std::vector<int64_t>& starts,
                        std::vector<int32_t>& kernels) {
  const uint64_t ktot = P.kcum.back();
  auto share_end = [&](int k) {  // floor(total * kcum[k] / ktot) without overflow
    const unsigned __int128 x = (unsigned __int128)(uint64_t)total * P.kcum[k];
    return (int64_t)(x / ktot);
  };
  std::vector<std::pair<int32_t, int64_t>> runs;  // (kernel, length)
  int64_t prev = 0;
  const uint64_t ls = mix64(seed ^ 0xA0761D6478BD642FULL);
  for (int k = 0; k < P.nf; ++k) {
    const int64_t end = share_end(k), nk = end - prev;
    prev = end;
    if (nk <= 0) continue;
    int64_t L = 1 + (int64_t)(mix64(ls + (uint64_t)(k + 1) * kGolden) % 8);
    if (L > nk) L = nk;
    for (int64_t t = 0; t < L; ++t) runs.emplace_back(k, nk * (t + 1) / L - nk * t / L);
  }
  Rng r(seed ^ 0xE7037ED1A0B428DBULL);
  for (size_t i = runs.size(); i > 1; --i) std::swap(runs[i - 1], runs[r.below((int)i)]);
  starts.assign(1, 0);
  kernels.clear();
  for (auto& x : runs) { kernels.push_back(x.first); starts.push_back(starts.back() + x.second); }
}

// Run layout for callers: returns the number of runs; fills starts[0..n_runs]
// and kernels[0..n_runs-1] when cap >= n_runs.
int64_t synth_launch_runs(void* h, uint64_t seed, int64_t total, int64_t* starts, int32_t* kernels, int64_t cap) {
  std::vector<int64_t> st;
  std::vector<int32_t> kr;
  launch_runs(*(Program*)h, seed, total, st, kr);
  const int64_t nr = (int64_t)kr.size();
  if (cap >= nr) {
    std::memcpy(starts, st.data(), sizeof(int64_t) * (size_t)(nr + 1));
    if (nr) std::memcpy(kernels, kr.data(), sizeof(int32_t) * (size_t)nr);
  }
  return nr;
}

// Packed samples [n0, n0+n) of stream `seed`:
//   kernel (16b) | pc (24b) | class (4b) | latency flag (1b) | sm (8b) | 11 reserved zero bits.
// order 0: the kernel of every sample is drawn independently (kernels interleaved);
// order 1: launch runs as laid out by launch_runs for a stream of `total` samples
// (total <= 0 means n0 + n).
// invalid_ppm injects malformed samples (bad kernel, pc, class, or SELECTED+latency).
void synth_samples(void* h, uint64_t seed, int64_t n0, int64_t n, uint64_t* out, uint32_t invalid_ppm,
                   int32_t n_threads, int64_t total, int32_t order) {
  auto* P = (Program*)h;
  const uint64_t base = mix64(seed ^ 0xD1B54A32D192ED03ULL);
  const uint64_t ktot = P->kcum.back();
  std::vector<int64_t> rstart;
  std::vector<int32_t> rkern;
  if (order == 1) launch_runs(*P, seed, std::max<int64_t>(total, n0 + n), rstart, rkern);
  int nt = std::max<int64_t>(1, std::min<int64_t>(n_threads, (n + 65535) / 65536));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) {
    th.emplace_back([&, t]() {
      int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
      size_t run = 0;
      for (int64_t q = lo; q < hi; ++q) {
        uint64_t idx = (uint64_t)(n0 + q);
        uint64_t d0 = mix64(base + (3 * idx + 1) * kGolden);
        uint64_t d1 = mix64(base + (3 * idx + 2) * kGolden);
        uint64_t d2 = mix64(base + (3 * idx + 3) * kGolden);
        int k;
        if (order == 1) {
          if (q == lo || (int64_t)idx >= rstart[run + 1])
            run = (size_t)(std::upper_bound(rstart.begin(), rstart.end(), (int64_t)idx) - rstart.begin()) - 1;
          k = run < rkern.size() ? rkern[run] : rkern.back();
        } else {
          uint64_t v0 = (d0 >> 16) % ktot;
          k = (int)(std::upper_bound(P->kcum.begin(), P->kcum.end(), v0) - P->kcum.begin());
        }
        int lo_i = P->func_instr_off[k], hi_i = P->func_instr_off[k + 1];
        uint64_t ftot = P->wcum[hi_i - 1];
        uint64_t v1 = (d1 >> 16) % ftot;
        int x = (int)(std::upper_bound(P->wcum.begin() + lo_i, P->wcum.begin() + hi_i, v1) - P->wcum.begin());
        int pc = x - lo_i;
        const uint64_t* pc24 = P->pcum[P->prof[x]];
        uint64_t r = d2 & 0xFFFFFFFFULL;
        int e = (int)(std::upper_bound(pc24, pc24 + 24, r) - pc24);
        uint64_t cls = (uint64_t)(e >> 1), lat = (uint64_t)(e & 1);
        uint64_t sm = (d2 >> 32) % 152;
        uint64_t kk = (uint64_t)k, pp = (uint64_t)pc;
        if (invalid_ppm && ((((d0 & 0xFFFFF) * 1000000ULL) >> 20) < invalid_ppm)) {
          switch ((d1 >> 3) & 3) {
            case 0: kk = (uint64_t)P->nf + ((d1 >> 40) & 7); if (kk > 0xFFFF) kk = 0xFFFF; break;
            case 1: pp = (uint64_t)(hi_i - lo_i) + ((d1 >> 40) & 63); break;
            case 2: cls = 12 + ((d1 >> 40) & 3); break;
            default: cls = 0; lat = 1; break;
          }
        }
        out[q] = (kk << 48) | ((pp & 0xFFFFFF) << 24) | (cls << 20) | (lat << 19) | (sm << 11);
      }
    });
  }
  for (auto& x : th) x.join();
}

}  // extern "C"
