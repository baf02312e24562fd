// Step (d), Sec. 5: roll blame up to lines, loops and functions, match the
// code optimizers of Table 2 (Function Inlining from the program's call
// table), estimate their speedups (Eq. 2 for stall elimination, Eq. 4 for
// latency hiding, Eq. 5 per loop scope), rank them and
// pick each optimizer's top five hotspots (def, use, distance); with launch
// statistics, the parallel optimizers (Eqs. 6-10).
//
// One CTA per function: threads stride over the function's instructions and
// its merged edges (contiguous, since edges are ordered by use), reduce the
// sums in shared memory, and thread 0 finishes the per-function results
// (warp 0 merges the hotspot lists). The
// CTAs take functions largest first from a counter, so the largest ones start
// at once and the rest fill in behind them.
#include "gpa_internal.cuh"

namespace gpa {

namespace {

constexpr int kThreads = 512;
constexpr int kHot = 5;
enum { O_RR = 0, O_SR, O_FS, O_FM, O_WB, O_MT, O_LU, O_CR, O_FI, N_O = 9 };
constexpr int kAcc = 13;  // per-function sums, see k_advise

struct Cand { unsigned long long v; int def, use, dist; };

__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {  // a ranks before b
  if (a.v != b.v) return a.v > b.v;
  if (a.def != b.def) return a.def < b.def;
  return a.use < b.use;
}
__device__ __forceinline__ void top_insert(Cand* top, int& n, const Cand& c) {
  if (c.v == 0) return;
  if (n == kHot && !better(c, top[kHot - 1])) return;
  int p = n < kHot ? n++ : kHot - 1;
  while (p > 0 && better(c, top[p - 1])) { top[p] = top[p - 1]; --p; }
  top[p] = c;
}

__device__ __forceinline__ double est(unsigned long long T, unsigned long long M) {
  if (T == 0) return 1.0;
  if (T == M) return __longlong_as_double(0x7FF0000000000000LL);  // +inf
  return (double)T / (double)(T - M);
}

__device__ int innermost_loop(const Prog& P, int x) { return P.block_loop[P.instr_block[x]]; }

__device__ int lca_loop(const Prog& P, int a, int b) {
  if (a < 0 || b < 0) return -1;
  int da = P.loop_depth[a], db = P.loop_depth[b];
  while (da > db) { a = P.loop_parent[a]; --da; }
  while (db > da) { b = P.loop_parent[b]; --db; }
  while (a != b && a >= 0 && b >= 0) { a = P.loop_parent[a]; b = P.loop_parent[b]; }
  return (a == b) ? a : -1;
}

// Matched samples of an edge per edge-based optimizer. Shares are indexed
// class slot (exec, memory, sync, constant memory) * 2 + latency flag. The
// def and use's innermost common loop (a walk up the loop nest) is found
// only with `loops` (lu is 0 without it); `lca` receives it.
struct EdgeMatch { unsigned long long rr, sr, lu, cr; };
__device__ __forceinline__ EdgeMatch edge_match(const Prog& P, const Arch& A, int64_t e, bool loops = true,
                                                int* lca = nullptr) {
  const unsigned long long* sh = P.e_share + e * 8;
  const uint32_t fl = A.flags[P.opclass[P.e_def[e]]];
  const bool local = fl & GPA_F_LOCAL;
  const bool global_mem = !local && !(fl & GPA_F_CONST);  // constant-memory stalls are never global
  EdgeMatch m;
  m.rr = local ? (sh[2] + sh[3] + sh[6] + sh[7]) : 0ull;                       // Register Reuse
  m.sr = (fl & GPA_F_LONG_ARITH) ? (sh[0] + sh[1]) : 0ull;                    // Strength Reduction
  m.cr = sh[1] + (global_mem ? sh[3] : 0ull);                                 // latency samples
  const int q = loops && m.cr ? lca_loop(P, innermost_loop(P, P.e_def[e]), innermost_loop(P, P.e_use[e])) : -1;
  m.lu = q >= 0 ? m.cr : 0ull;
  if (lca) *lca = q;
  return m;
}

// Parallel optimizers of function f (Table 2; Sec. 5.2, Eqs. 6-10 with f = 1),
// from its launch statistics, the SM model and its totals (T samples, issued).
// Occupancy: blocks per SM is the least of the warp, register, shared-memory
// and block-count limits (the binding one is reported, lowest id on ties).
// W = resident blocks per SM * warps per block / schedulers; R_I = issued / T;
// I(W) = 1 - (1 - R_I)^W (Eqs. 8-9).
//  Block Increase (fewer blocks than SMs): the same threads in one block per
//  SM, W_new = W * blocks / SMs; every SM runs one wave, so a scheduler's
//  warps over the run are its resident warps: C_W = W_new / W (Eq. 6).
//  Thread Increase (the block-count limit binds, and the grid reaches it): the
//  same threads in larger blocks, W_new = the warps per SM the warp, register
//  and shared-memory limits (per warp) and the grid allow, / schedulers; a
//  scheduler's warps over the run are unchanged: C_W = 1.
//  S = (1 / C_W) * C_I (Eq. 10), C_I = I(W_new) / I(W) (Eq. 7).
__device__ void parallel_advice(const Prog& P, int f, unsigned long long T, unsigned long long issued) {
  int match[2] = {0, 0}, limit = -1;
  double sp[2] = {1.0, 1.0}, w[4] = {0.0, 0.0, 0.0, 0.0};
  if (P.launch) {
    const LaunchRec L = P.launch[f];
    const SmModel& M = P.sm;
    const long long big = 1ll << 40;
    const long long wpb = (L.threads + 31) / 32;
    long long lim[4];
    lim[0] = M.max_warps / wpb;
    long long warps_by_regs = M.max_warps;  // warps per SM the registers allow
    if (L.regs > 0) {
      const long long rpw = ((long long)L.regs * 32 + M.reg_unit - 1) / M.reg_unit * M.reg_unit;
      warps_by_regs = (long long)M.schedulers * ((M.regs / M.schedulers) / rpw);
      lim[1] = warps_by_regs / wpb;
    } else {
      lim[1] = big;
    }
    long long warps_by_smem = big;          // warps per SM the shared memory allows
    if (L.smem > 0) {
      const long long per = ((long long)L.smem + M.smem_reserved + M.smem_unit - 1) / M.smem_unit * M.smem_unit;
      lim[2] = M.smem / per;
      warps_by_smem = lim[2] * wpb;
    } else {
      lim[2] = big;
    }
    lim[3] = M.max_blocks;
    long long bps = lim[0];
    limit = 0;
    for (int q = 1; q < 4; ++q)
      if (lim[q] < bps) { bps = lim[q]; limit = q; }
    const long long per_sm = (L.blocks + M.n_sms - 1) / M.n_sms;  // blocks per SM the grid gives
    const long long rb = bps < per_sm ? bps : per_sm;
    const double W = (double)(rb * wpb) / (double)M.schedulers;
    match[0] = L.blocks < M.n_sms;
    match[1] = limit == 3 && per_sm >= bps;
    double Wn[2] = {0.0, 0.0};
    Wn[0] = W * (double)L.blocks / (double)M.n_sms;
    long long wn = M.max_warps;
    if (warps_by_regs < wn) wn = warps_by_regs;
    if (warps_by_smem < wn) wn = warps_by_smem;
    const long long grid_warps = (L.blocks * wpb + M.n_sms - 1) / M.n_sms;
    if (grid_warps < wn) wn = grid_warps;
    Wn[1] = (double)wn / (double)M.schedulers;
    // an estimate needs a resident warp and an issue rate above zero
    const bool est_ok = bps > 0 && T > 0 && issued > 0;
    const double R = T ? (double)issued / (double)T : 0.0;
    const double I = 1.0 - pow(1.0 - R, W);
    for (int k = 0; k < 2; ++k) {
      if (!match[k]) continue;
      w[2 * k] = W;
      w[2 * k + 1] = Wn[k];
      if (!est_ok) continue;
      const double cw = k == 0 ? Wn[0] / W : 1.0, ci = (1.0 - pow(1.0 - R, Wn[k])) / I;
      sp[k] = (1.0 / cw) * ci;
    }
  }
  for (int k = 0; k < 2; ++k) {
    P.a_par_match[(size_t)f * 2 + k] = match[k];
    P.a_par_speedup[(size_t)f * 2 + k] = sp[k];
  }
  for (int k = 0; k < 4; ++k) P.a_par_warps[(size_t)f * 4 + k] = w[k];
  P.a_par_limit[f] = limit;
}

__global__ void __launch_bounds__(kThreads) k_advise(Prog P, Arch A) {
  __shared__ unsigned long long red[kAcc][kThreads / 32];
  __shared__ unsigned long long tot[kAcc];
  // each warp's top five (v == 0: none), two sets: warp 0 merges one optimizer's
  // while the other warps fill the other with the next optimizer's
  __shared__ Cand wtop[2][kThreads / 32][kHot];
  __shared__ int s_f;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  while (true) {
    __syncthreads();  // every thread has read s_f
    if (tid == 0) {
      const unsigned long long q = atomicAdd(&P.stats[SS_ADV_HEAD], 1ull);
      s_f = q < (unsigned long long)P.nf ? P.reach_order[q] : -1;
    }
    __syncthreads();
    const int f = s_f;
    if (f < 0) break;
    const int i0 = P.func_instr_off[f], i1 = P.func_instr_off[f + 1];
    // Edge ranges are clamped to the edge capacity (overflow is reported in the status word).
    const int64_t e0 = min((int64_t)P.edge_off[i0], P.edge_cap), e1 = min((int64_t)P.edge_off[i1], P.edge_cap);
    unsigned long long acc[kAcc];
#pragma unroll
    for (int q = 0; q < kAcc; ++q) acc[q] = 0ull;
    // acc: 0 T, 1 A, 2 L, 3 issued, 4 FS, 5 FM, 6 WB, 7 MT, 8 RR, 9 SR, 10 LU, 11 CR, 12 FI
    for (int x = i0 + tid; x < i1; x += kThreads) {
      const unsigned long long* c = P.cnt + (size_t)x * kCnt;
      unsigned long long a = 0, l = 0, stall = 0;
#pragma unroll
      for (int e = 0; e < kCnt; ++e) {
        if (e & 1) l += c[e]; else a += c[e];
        if (e >= 2) stall += c[e];
      }
      acc[0] += a + l; acc[1] += a; acc[2] += l; acc[3] += c[0];
      acc[4] += c[2] + c[3];
      if (P.iflags[x] & 1) acc[5] += stall;
      acc[6] += c[10] + c[11];
      if (A.flags[P.opclass[x]] & GPA_F_GLOBAL) acc[7] += c[16] + c[17];
      if (P.iflags[x] & 6) acc[12] += l;  // latency stalls in a device function or at a call site
      for (int lp = innermost_loop(P, x); lp >= 0; lp = P.loop_parent[lp])
        if (a) atomicAdd(&P.a_loop_active[lp], a);
      const unsigned long long* b = P.blame + (size_t)x * kCnt;
      unsigned long long bs = 0, bl = 0;
#pragma unroll
      for (int e = 2; e < kCnt; ++e) { bs += b[e]; if (e & 1) bl += b[e]; }
      if (bs) atomicAdd(&P.a_line_stall[P.line[x]], bs);
      if (bl) atomicAdd(&P.a_line_lat[P.line[x]], bl);
    }
    for (int64_t e = e0 + tid; e < e1; e += kThreads) {
      int q;
      const EdgeMatch m = edge_match(P, A, e, true, &q);
      acc[8] += m.rr; acc[9] += m.sr; acc[10] += m.lu; acc[11] += m.cr;
      if (m.lu)
        for (int lp = q; lp >= 0; lp = P.loop_parent[lp]) atomicAdd(&P.a_loop_matched[lp], m.lu);
    }
#pragma unroll
    for (int q = 0; q < kAcc; ++q) {
      unsigned long long v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[q][warp] = v;
    }
    __syncthreads();
    if (tid < kAcc) {
      unsigned long long v = 0;
      for (int w = 0; w < kThreads / 32; ++w) v += red[tid][w];
      tot[tid] = v;
    }
    __syncthreads();
    const unsigned long long T = tot[0], Aact = tot[1];
    if (tid == 0) {
      unsigned long long M[N_O];
      M[O_RR] = tot[8]; M[O_SR] = tot[9]; M[O_FS] = tot[4]; M[O_FM] = tot[5];
      M[O_WB] = tot[6]; M[O_MT] = tot[7]; M[O_LU] = tot[10]; M[O_CR] = tot[11]; M[O_FI] = tot[12];
      double sp[N_O];
      for (int o = 0; o < N_O; ++o) {
        const bool hide = (o == O_LU || o == O_CR || o == O_FI);
        sp[o] = est(T, hide ? min(Aact, M[o]) : M[o]);
        P.a_matched[(size_t)f * N_O + o] = M[o];
        P.a_speedup[(size_t)f * N_O + o] = sp[o];
      }
      int ord[N_O];
      for (int o = 0; o < N_O; ++o) ord[o] = o;
      for (int a = 1; a < N_O; ++a) {  // stable: ties keep the lower id first
        int v = ord[a], b = a - 1;
        while (b >= 0 && sp[ord[b]] < sp[v]) { ord[b + 1] = ord[b]; --b; }
        ord[b + 1] = v;
      }
      for (int o = 0; o < N_O; ++o) P.a_rank[(size_t)f * N_O + o] = ord[o];
      for (int q = 0; q < 4; ++q) P.a_totals[(size_t)f * 4 + q] = tot[q];
      parallel_advice(P, f, T, tot[3]);
    }
    // Hotspots, one optimizer at a time: thread-local top five, a warp-level
    // merge, then thread 0 merges the warps' lists.
    for (int o = 0; o < N_O; ++o) {
      Cand top[kHot];
      int nt = 0;
      const bool edge_based = (o == O_RR || o == O_SR || o == O_LU || o == O_CR);
      if (edge_based) {
        for (int64_t e = e0 + tid; e < e1; e += kThreads) {
          const EdgeMatch m = edge_match(P, A, e, o == O_LU);
          const unsigned long long v = o == O_RR ? m.rr : o == O_SR ? m.sr : o == O_LU ? m.lu : m.cr;
          top_insert(top, nt, Cand{v, P.e_def[e] - i0, P.e_use[e] - i0, P.e_dmin[e]});
        }
      } else {
        for (int x = i0 + tid; x < i1; x += kThreads) {
          const unsigned long long* c = P.cnt + (size_t)x * kCnt;
          unsigned long long v = 0;
          if (o == O_FS) v = c[2] + c[3];
          else if (o == O_FM) { if (P.iflags[x] & 1) for (int e = 2; e < kCnt; ++e) v += c[e]; }
          else if (o == O_WB) v = c[10] + c[11];
          else if (o == O_FI) { if (P.iflags[x] & 6) for (int e = 3; e < kCnt; e += 2) v += c[e]; }
          else if (A.flags[P.opclass[x]] & GPA_F_GLOBAL) v = c[16] + c[17];
          top_insert(top, nt, Cand{v, x - i0, x - i0, 0});
        }
      }
      // The warp's top five: five rounds of a butterfly maximum over the lanes'
      // next candidates (candidates are distinct, so the order is total; lanes
      // out of candidates offer v = 0, ties between those go to the lower lane).
      int ptr = 0;
      for (int h = 0; h < kHot; ++h) {
        Cand b = ptr < nt ? top[ptr] : Cand{0ull, 0, 0, 0};
        int owner = lane;
        for (int sh = 16; sh > 0; sh >>= 1) {
          Cand y;
          y.v = __shfl_xor_sync(0xffffffffu, b.v, sh);
          y.def = __shfl_xor_sync(0xffffffffu, b.def, sh);
          y.use = __shfl_xor_sync(0xffffffffu, b.use, sh);
          y.dist = __shfl_xor_sync(0xffffffffu, b.dist, sh);
          const int yo = __shfl_xor_sync(0xffffffffu, owner, sh);
          if (better(y, b) || (!better(b, y) && yo < owner)) { b = y; owner = yo; }
        }
        if (lane == owner && b.v != 0ull) ++ptr;
        if (lane == 0) wtop[o & 1][warp][h] = b;
      }
      __syncthreads();
      // The CTA's top five: warp 0 merges the warps' sorted lists the same way
      // (lane w offers the next entry of warp w's list).
      if (warp == 0) {
        static_assert(kThreads / 32 <= 32, "one lane per warp's list");
        long long* out = P.a_hot + ((size_t)f * N_O + o) * kHot * 6;
        int wp = 0, nb = 0;
        for (int h = 0; h < kHot; ++h) {
          Cand b = lane < kThreads / 32 && wp < kHot ? wtop[o & 1][lane][wp] : Cand{0ull, 0, 0, 0};
          int owner = lane;
          for (int sh = 16; sh > 0; sh >>= 1) {
            Cand y;
            y.v = __shfl_xor_sync(0xffffffffu, b.v, sh);
            y.def = __shfl_xor_sync(0xffffffffu, b.def, sh);
            y.use = __shfl_xor_sync(0xffffffffu, b.use, sh);
            y.dist = __shfl_xor_sync(0xffffffffu, b.dist, sh);
            const int yo = __shfl_xor_sync(0xffffffffu, owner, sh);
            if (better(y, b) || (!better(b, y) && yo < owner)) { b = y; owner = yo; }
          }
          if (lane == owner && b.v != 0ull) ++wp;
          if (lane == 0) {
            if (b.v != 0ull) {
              out[h * 6 + 0] = b.def; out[h * 6 + 1] = b.use;
              out[h * 6 + 2] = P.line[i0 + b.def]; out[h * 6 + 3] = P.line[i0 + b.use];
              out[h * 6 + 4] = b.dist; out[h * 6 + 5] = (long long)b.v;
              ++nb;
            } else {
              for (int q = 0; q < 6; ++q) out[h * 6 + q] = -1;
            }
          }
        }
        if (lane == 0) P.a_nhot[(size_t)f * N_O + o] = nb;
      }
      // No barrier here: the next pass fills the other set, and warp 0 reaches
      // the barrier after that pass only once this merge is done, before the
      // pass after next fills this set again.
    }
    // Eq. 5 per loop scope of this function (its loop counters were only touched by this CTA).
    __threadfence_block();
    __syncthreads();
    for (int lp = P.func_loop_off[f] + tid; lp < P.func_loop_off[f + 1]; lp += kThreads) {
      const unsigned long long al = __ldcg(&P.a_loop_active[lp]);
      const unsigned long long ml = __ldcg(&P.a_loop_matched[lp]);
      P.a_loop_speedup[lp] = est(T, min(al, ml));
    }
    __syncthreads();
  }
}

}  // namespace

void launch_advise(const Prog& P, const Arch& A, cudaStream_t st, int sms, int64_t* launches) {
  if (P.nl > 0) {
    cudaMemsetAsync(P.a_loop_active, 0, sizeof(unsigned long long) * P.nl, st);
    cudaMemsetAsync(P.a_loop_matched, 0, sizeof(unsigned long long) * P.nl, st);
  }
  cudaMemsetAsync(P.a_line_stall, 0, sizeof(unsigned long long) * P.n_lines, st);
  cudaMemsetAsync(P.a_line_lat, 0, sizeof(unsigned long long) * P.n_lines, st);
  cudaMemsetAsync(&P.stats[SS_ADV_HEAD], 0, sizeof(unsigned long long), st);
  int blocks = P.nf < sms * 2 ? P.nf : sms * 2;
  k_advise<<<blocks > 0 ? blocks : 1, kThreads, 0, st>>>(P, A);
  ++*launches;
}

}  // namespace gpa
