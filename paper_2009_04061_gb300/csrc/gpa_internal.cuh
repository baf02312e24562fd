// Internal device-side layout and helpers of libgpa (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gpa.h"

namespace gpa {

constexpr int kNumRes = 268;     // R0..R254, P0..P6, B0..B5
constexpr int kPredBase = 255;
constexpr int kBarBase = 262;
constexpr int kWords = 9;        // 268 bits in 32-bit words
constexpr int kEvBuckets = 16;   // event segments per block: resources by r mod 16
__host__ __device__ inline int ev_bucket(int r) { return r & (kEvBuckets - 1); }
constexpr int kCnt = 24;         // counters per instruction: class * 2 + latency flag
constexpr uint16_t kAllLits = 0xFFFF;
constexpr int kMaxLayers = 8;    // back-edge layers for longest paths (K <= 7)
constexpr int kMaxSrc = 64;      // merged sources per stalled use in the thread-per-use kernels
constexpr int kBigSrc = 2048;    // merged sources per stalled use (hard upper bound; beyond kMaxSrc
                                 // a CTA per use with shared-memory arrays)

// Bits of the per-program device status word.
enum : unsigned long long {
  ST_NOT_CONVERGED = 1, ST_CAPACITY = 2, ST_TIMEOUT = 4, ST_OVERFLOW = 8
};
// Slots of the per-program stats array (unsigned long long).
enum {
  SS_INVALID = 0, SS_GENERAL = 1, SS_MAX_NODES = 2, SS_SWEEPS = 3, SS_STATUS = 4,
  SS_RAW_N = 5, SS_QUEUE_N = 6, SS_QUEUE_HEAD = 7, SS_OVF_N = 8, SS_OVF_HEAD = 9, SS_OVF2_N = 10,
  SS_OVF2_HEAD = 11, SS_MAX_TASK = 12,
  // Per-tier search phase cycles (3 tiers x 6; the fourth tier adds to the
  // third's), filled only when built with -DGPA_PHASE_TIMING: graph,
  // distances, sources, rule 2, longest paths, and the count of rule-2
  // reachability runs.
  // With -DGPA_PHASE_TIMING also: searches by log2 of their node count (16
  // slots) and the searches that needed pass B (1 slot).
  // And the slowest search: (cycles << 20 | nodes), its rule-2 runs and the
  // cycles of its five phases.
  SS_PHASE = 13, SS_SIZES = 31, SS_PASSB = 47, SS_SLOW = 48,
  // 55: unused
  SS_OVF3_N = 56, SS_OVF3_HEAD = 57,  // searches handed on to the program's own fourth tier
  SS_SIZE_CYC = 58,  // with -DGPA_PHASE_TIMING: cycles of the searches by log2 of their node count (16)
  SS_HINT3_N = 74,   // searches queued straight for the third tier (from the top of `queue`)
  SS_FAILBITS = 75,  // why a step reported GPA_ERR_CAPACITY: the last search tier ran out of
                     // 1 nodes, 2 edges, 3 occurrences, 4 sources, 5 back-edge layers,
                     // 6 hash rounds; 8 queue, 9 sources per use, 10 merged edges,
                     // 11 distance range, 12 raw edges, 13 no path length
  SS_BIG_N = 76,     // uses with more than kMaxSrc distinct sources (listed in big_use)
  SS_COV = 77,       // gpa_dependency_coverage: stalled uses, single before, single after pruning
  SS_COV_ALL = 80,   // the counting pass's total of sources before pruning
  SS_XN = 81,        // unpruned edges written by the export pass
  SS_HIST_HEAD = 82, // next chunk of the run-aware aggregation kernel (reset before each launch)
  SS_HINT3_HEAD = 83,  // next of the searches queued straight for the third tier
  SS_OVF3H_N = 84,     // searches for the fourth tier stored from the top of `ovf_queue`
  SS_LARGE_N = 85,     // entries of large_queue
  SS_REACH_CLS = 86,   // next entry of reach_order for each of the staged fixpoint's 4 launches
  SS_SUSE_N = 90,      // entries of suse (the stalled uses of this step)
  SS_ADV_HEAD = 91,    // next entry of reach_order for the advice kernel's CTAs
  SS_N = 92
};

struct Arch {
  int32_t n_op;
  int32_t lat[GPA_MAX_OPCLASSES];
  uint32_t flags[GPA_MAX_OPCLASSES];
};

// Device view of one loaded program and its per-step buffers.
// One function's launch statistics (the layout of gpa_launch_stats) and the
// SM of the occupancy model (the fields of gpa_sm_model).
struct LaunchRec {
  long long blocks;
  int32_t threads, regs, smem, reserved;
};
struct SmModel {
  int32_t n_sms, schedulers, max_warps, max_blocks, regs, reg_unit, smem, smem_unit, smem_reserved;
};

struct Prog {
  int32_t nf, ni, nb, nl, n_lines;
  int32_t diag;                   // 1: the searches count sources (gpa_dependency_coverage), 2: they export
                                  // every source (gpa_export_unpruned_edges); both emit no raw edges
  int4* xedges;                   // export: 2 per edge, {use, def, resource, dmin}, {K, dlong, dom, 0}
  int64_t xcap;                   // edges the export buffer holds
  uint32_t* cov_cnt;              // n_use: that run's sources per use entry, before pruning (low 16 bits)
                                  // and kept after pruning (high 16 bits)
  int32_t reach_smem;             // shared memory of the staged fixpoint: the largest need that fits
  int32_t reach_cls[5];           // the staged fixpoint's launches: reach_order[reach_cls[c], reach_cls[c + 1])
  int32_t reach_cls_smem[4];      // and the largest need among them (0: no launch)
  const uint8_t* func_natural;    // nf: 1 when every loop body of the function is a natural loop
                                  // (functions needing more use the global-memory fixpoint)
  // Fourth search tier, sized for this program's largest function (0 nodes:
  // none): searches that outgrow the context's third tier, a CTA each.
  int32_t t4_nodes, t4_src, t4_ctas;
  int64_t t4_bytes;               // per CTA
  char* t4_arena;                 // t4_ctas * t4_bytes, global memory
  const int32_t* func_instr_off;
  const int32_t* func_block_off;
  const int32_t* func_loop_off;
  const int32_t* block_instr_off;
  const int32_t* succ_off;
  const int32_t* succ;
  const int32_t* pred_off;
  const int32_t* pred;
  const uint8_t* opclass;
  const uint8_t* guard;
  const uint8_t* iflags;          // bit 0 math-library code, 1 call site, 2 in a device function
  const int32_t* line;
  const int32_t* def_off;
  const uint16_t* def_res;
  const int32_t* use_off;
  const uint16_t* use_res;
  const int32_t* block_loop;
  const int32_t* loop_parent;
  const int32_t* loop_header;
  const int32_t* loop_depth;
  const int32_t* instr_block;
  const int32_t* block_func;
  const int32_t* reach_order;     // nf: functions by the staged fixpoint's shared memory need, largest first
  const int32_t* block_minreach;  // nb: smallest block reachable from the block (itself included)
  const int4* block_meta;         // 2 per block: {first instr, end instr, first event, end event},
                                  // {first pred, end pred, first two predecessors or -1} (one
                                  // 32-byte line for the searches)
  const int32_t* ev_off;          // nb * 16 + 1: event segments of (block, resource bucket)
  const uint32_t* events;         // per segment, the defs and unguarded reads of the bucket's
                                  // resources, bottom-up: resource | def << 9 | kind << 10 |
                                  // guard << 12 | position in block << 16
  // step state
  unsigned long long* cnt;        // ni * 24
  unsigned long long* stats;      // SS_N
  uint32_t* def_mask;             // nb * 9: resources defined in the block
  uint32_t* uuse_mask;            // nb * 9: resources read by an unguarded instruction
  uint32_t* touch_mask;           // nb * 9: DEF | UUSE (blocks a search must scan)
  int32_t* res_maxlat;            // nf * 268: largest latency of any def of the resource in the function
  uint32_t* res_guards;           // nf * 268: guard literals of the resource's defs in the function
  uint32_t* rin;                  // nb * 9
  uint32_t* rout;                 // nb * 9
  int32_t* head;                  // ni: raw-edge list head per use (-1 = none)
  int4* raw;                      // raw edges: def, next, dmin, dlong | flags << 24
  int64_t raw_cap;
  int4* queue;                    // general searches: use, resource, start literal set, use entry
  int32_t large_nodes;            // node count from which a third-tier search is started early
  uint8_t* large_hint;            // n_use: 1 when the entry's last third-tier search had large_nodes nodes or more
  int4* large_queue;              // kLargeQueue: such searches, started before the other third-tier ones
  uint32_t* tier_hint;            // n_use: smallest search tier known to hold the entry's search (0: none);
                                  // kept across steps (a search's size depends only on the program)
  int4* ovf_queue;                // general searches that outgrew a small scratch slot
  int64_t queue_cap;
  int32_t* edge_cnt;              // ni + 1 (exclusive scan in place -> offsets)
  int32_t* big_use;               // ni: uses with more than kMaxSrc sources (SS_BIG_N of them)
  int32_t* suse;                  // ni: the stalled uses of this step, SS_SUSE_N of them (any order)
  int32_t* edge_off;              // ni + 1
  int32_t* e_use;
  int32_t* e_def;
  int32_t* e_dmin;
  int32_t* e_dlong;
  uint32_t* e_flags;
  unsigned long long* e_share;    // edges * 8
  int64_t edge_cap;
  unsigned long long* blame;      // ni * 24
  // advice
  unsigned long long* a_totals;   // nf * 4
  unsigned long long* a_matched;  // nf * 8
  double* a_speedup;              // nf * 8
  int32_t* a_rank;                // nf * 8
  int32_t* a_nhot;                // nf * 8
  long long* a_hot;               // nf * 8 * 5 * 6
  unsigned long long* a_loop_active;
  unsigned long long* a_loop_matched;
  double* a_loop_speedup;
  unsigned long long* a_line_stall;
  unsigned long long* a_line_lat;
  // parallel optimizers (Table 2, Eqs. 6-10): launch statistics per function
  // (nullptr: none set) and the SM they ran on
  const LaunchRec* launch;
  SmModel sm;
  int32_t* a_par_match;           // nf * 2
  double* a_par_speedup;          // nf * 2
  double* a_par_warps;            // nf * 4
  int32_t* a_par_limit;           // nf
};

// Per-warp arenas of the general (multi-block) search.
struct SearchArena {
  int32_t nodes, src, layers, warps;  // warps: search groups (the fourth tier's are CTAs)
  int64_t bytes;   // per group
  char* global;    // global-memory tiers: warps * bytes
};

__device__ __forceinline__ void set_status(const Prog& P, unsigned long long bits) {
  atomicOr(&P.stats[SS_STATUS], bits);
}
// GPA_ERR_CAPACITY with its reason (bit `why` of SS_FAILBITS).
__device__ __forceinline__ void capacity(const Prog& P, int why) {
  atomicOr(&P.stats[SS_STATUS], (unsigned long long)ST_CAPACITY);
  atomicOr(&P.stats[SS_FAILBITS], 1ull << why);
}

// ---------------------------------------------------------------- Sec. 4 predicate literals
// Literal set: bit i = Pi, bit 7+i = !Pi; kAllLits = the set holds "_".
__device__ __forceinline__ uint16_t add_literal(uint16_t S, int g) {
  if (S == kAllLits || g == 0) return kAllLits;
  S = (uint16_t)(S | (1u << (g - 1)));  // literal 1..7 -> bit 0..6 (Pi), 8..14 -> bit 7..13 (!Pi)
  uint32_t pos = S & 0x7Fu, neg = (S >> 7) & 0x7Fu;
  return (pos & neg) ? kAllLits : S;
}
// Literals of a set that can still matter to a search for a use guarded by
// g through a resource whose defs carry the guard literals `guards`: g
// itself, and each literal whose complement some def may still add (only
// such a literal can complete a Pi / !Pi pair). Dropping the others merges
// literal sets that give every continuation the same coverage outcomes.
__device__ __forceinline__ uint16_t live_literals(uint32_t guards, int g) {
  const uint32_t comp = ((guards & 0x7Fu) << 7) | ((guards >> 7) & 0x7Fu);
  return (uint16_t)(comp | (g ? 1u << (g - 1) : 0u));
}
__device__ __forceinline__ uint16_t keep_literals(uint16_t S, uint16_t live) {
  return S == kAllLits ? S : (uint16_t)(S & live);
}
// "P contains p'": p' in P or "_" in P.
__device__ __forceinline__ bool contains(uint16_t S, int g) {
  if (S == kAllLits) return true;
  if (g == 0) return false;
  return (S >> (g - 1)) & 1u;
}

// Rule 1, opcode pruning: can instruction class op cause stalls of class cls?
__device__ __forceinline__ bool opcode_keeps(const Arch& A, int cls, int op) {
  if (cls == GPA_MEMORY_DEPENDENCY || cls == GPA_CONSTANT_MEMORY_DEPENDENCY) return (A.flags[op] & GPA_F_MEM) != 0;
  if (cls == GPA_SYNC) return (A.flags[op] & GPA_F_SYNC) != 0;
  return true;
}
// Rule 1 for the coverage count: does op survive for some dependency class stalled at j?
__device__ __forceinline__ bool keeps_any(const Prog& P, const Arch& A, int j, int op) {
  const unsigned long long* c = P.cnt + (size_t)j * kCnt;
  return ((c[2 * GPA_EXEC_DEPENDENCY] | c[2 * GPA_EXEC_DEPENDENCY + 1]) && opcode_keeps(A, GPA_EXEC_DEPENDENCY, op)) ||
         ((c[2 * GPA_MEMORY_DEPENDENCY] | c[2 * GPA_MEMORY_DEPENDENCY + 1]) && opcode_keeps(A, GPA_MEMORY_DEPENDENCY, op)) ||
         ((c[2 * GPA_SYNC] | c[2 * GPA_SYNC + 1]) && opcode_keeps(A, GPA_SYNC, op)) ||
         ((c[2 * GPA_CONSTANT_MEMORY_DEPENDENCY] | c[2 * GPA_CONSTANT_MEMORY_DEPENDENCY + 1]) &&
          opcode_keeps(A, GPA_CONSTANT_MEMORY_DEPENDENCY, op));
}
// One unpruned edge for the export (GPA_ERR_CAPACITY if the buffer is full).
__device__ __forceinline__ void xemit(const Prog& P, int j, int i, int r, int dmin, int K, int dlong, bool dom) {
  const unsigned long long k = atomicAdd(&P.stats[SS_XN], 1ull);
  if (k >= (unsigned long long)P.xcap) {
    atomicOr(&P.stats[SS_STATUS], (unsigned long long)ST_CAPACITY);
    return;
  }
  P.xedges[2 * k] = make_int4(j, i, r, dmin);
  P.xedges[2 * k + 1] = make_int4(K, dlong, dom ? 1 : 0, 0);
}
// Adds a (use entry) contribution to the coverage count.
__device__ __forceinline__ void cov_add(const Prog& P, int e, int n_all, int n_kept) {
  atomicAdd(&P.cov_cnt[e], (uint32_t)min(n_all, 0xFFFF) | ((uint32_t)min(n_kept, 0xFFFF) << 16));
}

// Def kind of resource r at instruction x: -1 not defined, else 0/1/2.
__device__ __forceinline__ int def_kind(const Prog& P, int x, int r) {
  const int e1 = P.def_off[x + 1];
  for (int e = P.def_off[x]; e < e1; ++e) {
    uint32_t v = P.def_res[e];
    if ((int)(v & 0x1FFu) == r) return (int)((v >> 12) & 3u);
  }
  return -1;
}
__device__ __forceinline__ bool uses_res(const Prog& P, int x, int r) {
  const int e1 = P.use_off[x + 1];
  for (int e = P.use_off[x]; e < e1; ++e)
    if ((int)(P.use_res[e] & 0x1FFu) == r) return true;
  return false;
}

__device__ __forceinline__ bool stalled(const Prog& P, int j) {
  const unsigned long long* c = P.cnt + (size_t)j * kCnt;
  return (c[4] | c[5] | c[6] | c[7] | c[10] | c[11] | c[12] | c[13]) != 0ull;
}

// Raw edge (j <- i through r) onto j's list.
__device__ __forceinline__ void emit_raw(const Prog& P, const Arch& A, int j, int i, int r, int kind, int dmin,
                                         int dlong) {
  uint32_t fl = r >= kBarBase ? 2u : (r >= kPredBase ? 8u : 4u);
  // Write-after-read (Sec. 4, Fig. 6): the variable-latency def reads a
  // register that the use writes, and they are linked through a read barrier.
  if (r >= kBarBase && kind == 2 && (A.flags[P.opclass[i]] & GPA_F_VARLAT)) {
    for (int e = P.def_off[j]; e < P.def_off[j + 1]; ++e) {
      const int rr = P.def_res[e] & 0x1FF;
      if (rr < kPredBase && uses_res(P, i, rr)) { fl |= 1u; break; }
    }
  }
  if (dmin >= (1 << 24) || dlong >= (1 << 24)) { capacity(P, 11); return; }
  const unsigned long long slot = atomicAdd(&P.stats[SS_RAW_N], 1ull);
  if (slot >= (unsigned long long)P.raw_cap) { capacity(P, 12); return; }
  const int next = atomicExch(&P.head[j], (int)slot);
  P.raw[slot] = make_int4(i, next, dmin, dlong | (int)(fl << 24));
}

// ---------------------------------------------------------------- launchers
int grid_for(int64_t n, int threads, int sms);
void launch_build_layout(const Prog& P, cudaStream_t st, int sms, int64_t* launches);
void launch_store_u64(unsigned long long* p, unsigned long long v, cudaStream_t st, int64_t* launches);
void launch_build_preds(const Prog& P, int n_succ, int32_t* pred_off, int32_t* cursor, int32_t* tmp, cudaStream_t st,
                        int sms, int64_t* launches);
void launch_histogram(const Prog& P, const uint64_t* samples, size_t n, cudaStream_t st, int sms, int64_t* launches,
                      int variant, int hist_chunk);
void launch_dataflow(const Prog& P, const Arch& A, int max_sweeps, int schedule, cudaStream_t st, int sms,
                     int64_t* launches);

// Lets kernel func take up to the device's opt-in shared memory per block.
// Every launch and captured graph node of a kernel then sees the same limit
// (each requests only what it uses), whatever ran before it.
// The dynamic limit is the opt-in maximum less the kernel's static shared memory.
template <class F>
inline void allow_max_smem(F func) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, func);
  cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

// Shared memory of the staged fixpoint for a function of nbf blocks, ne
// predecessor entries and nlf loops: ROUT (9 words a block), a 16-byte record
// per block (16-byte aligned: up to 12 bytes of padding), the predecessor CSR,
// each block's innermost loop, and per loop its parent and two 9-word masks (the
// definitions in its body; those of its body and enclosing loops).
__host__ __device__ inline int64_t reach_smem_need(int64_t nbf, int64_t ne, int64_t nlf) {
  return 4 * kWords * nbf + 12 + 16 * nbf + 4 * (nbf + 1) + 4 * ne + 4 * nbf + 4 * nlf + 2 * 4 * kWords * nlf;
}
// Size classes of the staged fixpoint's launches (upper bounds of the need):
// the larger a function, the fewer warps per SM its launch runs.
constexpr int64_t kReachClassCap[4] = {200 * 1024, 64 * 1024, 28 * 1024, 12 * 1024};
constexpr int64_t kReachSmemCap = 200 * 1024;
// A second stream (and two events) on which the searches queued straight for
// the third tier run beside the first two tiers.
struct SearchFork {
  cudaStream_t side;
  cudaEvent_t fork, join;
};
constexpr int kLargeQueue = 4096;  // capacity of large_queue
constexpr int kLargeNodes = 1024;  // default of large_nodes
void launch_blame(const Prog& P, const Arch& A, const SearchArena* tiers, const SearchFork* fork, int max_src,
                  int32_t* scan_tmp, cudaStream_t st, int sms, int64_t* launches);
void launch_search(const Prog& P, const Arch& A, const SearchArena* tiers, const SearchFork* fork, cudaStream_t st,
                   int sms, int64_t* launches);
void launch_coverage(const Prog& P, const Arch& A, const SearchArena* tiers, const SearchFork* fork, cudaStream_t st,
                     int sms, int64_t* launches);
int64_t search_arena_bytes(int nodes, int src, int layers);
int search_warps_per_sm();  // resident one-warp CTAs of the search kernel per SM (global-memory tiers)
void launch_build_meta(const Prog& P, int4* meta, cudaStream_t st, int sms, int64_t* launches);
void launch_build_events(const Prog& P, int32_t* ev_off, uint32_t* events, int32_t* tmp, cudaStream_t st, int sms,
                         int64_t* launches);
void launch_advise(const Prog& P, const Arch& A, cudaStream_t st, int sms, int64_t* launches);
// Exclusive scan of n int32 values in place over buf[0..n], buf[n] receives the total.
void scan_exclusive_inplace(int32_t* buf, int n, int32_t* tmp, cudaStream_t st, int64_t* launches);
size_t scan_tmp_ints(int n);

}  // namespace gpa
