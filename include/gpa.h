/*
 * gpa.h — C ABI of the GB300-native GPA stall-blame library (libgpa.so).
 *
 * The library turns packed PC samples into attributed stall blame and
 * speedup advice, following Zhou et al., "GPA: A GPU Performance Advisor
 * Based on Instruction Sampling": sample aggregation (Sec. 2.1), backward
 * slicing over registers, predicates and virtual barrier registers with
 * predicate coverage (Sec. 4), opcode/dominator/latency pruning and the
 * apportioning of Eq. 1 (Sec. 4), the detailed dependency classes (Sec. 4,
 * Fig. 6), the code optimizers of Table 2 and the estimators of Eq. 2, 4 and 5
 * (Sec. 5). Every step runs in CUDA kernels on the current device; there is
 * no CPU fallback.
 *
 * Conventions for every entry point:
 *  - Return value: GPA_OK (0) or a negative gpa_status. Argument and program
 *    validation errors are returned synchronously and leave all state
 *    unchanged. CUDA runtime failures return GPA_ERR_CUDA.
 *  - Device-side anomalies (invalid samples, iteration or capacity limits
 *    reached inside a kernel) never trap: kernels record them in a per-program
 *    status word that gpa_sync_status() reads.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    device memory of the current device. Pinned host memory makes the host
 *    copies asynchronous.
 *  - gpa_stream is a cudaStream_t (NULL = legacy default stream). Work is
 *    enqueued on it and completes asynchronously unless stated otherwise.
 *  - A context and its programs are not thread safe: serialize calls on one
 *    gpa_ctx from the host.
 */
#ifndef GPA_H_
#define GPA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gpa_ctx gpa_ctx;
typedef int32_t gpa_status;
typedef uint32_t gpa_pid;
typedef void* gpa_stream;

enum {
  GPA_OK = 0,
  GPA_ERR_INVALID_ARG = -1,      /* bad pointer, size or handle */
  GPA_ERR_INVALID_PROGRAM = -2,  /* program arrays violate the format below */
  GPA_ERR_CUDA = -3,             /* a CUDA runtime call failed */
  GPA_ERR_NOT_CONVERGED = -4,    /* reaching-definitions sweeps hit their limit */
  GPA_ERR_CAPACITY = -5,         /* a per-search or per-use capacity was exceeded */
  GPA_ERR_TIMEOUT = -6,          /* a bounded device-side wait gave up */
  GPA_ERR_NO_PROGRAM = -7,       /* pid is not loaded */
  GPA_ERR_OOM = -8               /* device allocation failed or budget exceeded */
};

#define GPA_NUM_RES 268      /* R0..R254 = 0..254, P0..P6 = 255..261, B0..B5 = 262..267 */
#define GPA_NUM_CLASSES 12   /* stall reasons, see below */
#define GPA_NUM_OPT 9        /* optimizers, see below */
#define GPA_MAX_OPCLASSES 64

/* Stall reasons (class field of a sample). Sec. 4 names memory dependency,
 * execution dependency and synchronization as the reasons caused by other
 * instructions; the list follows the public CUPTI PC-sampling reasons. */
enum {
  GPA_SELECTED = 0, GPA_INST_FETCH = 1, GPA_EXEC_DEPENDENCY = 2, GPA_MEMORY_DEPENDENCY = 3,
  GPA_TEXTURE = 4, GPA_SYNC = 5, GPA_CONSTANT_MEMORY_DEPENDENCY = 6, GPA_PIPE_BUSY = 7,
  GPA_MEMORY_THROTTLE = 8, GPA_NOT_SELECTED = 9, GPA_OTHER = 10, GPA_SLEEPING = 11
};

/* Optimizers of Table 2 (code optimizers), in result order. Function Inlining
 * (a latency-hiding optimizer, Eq. 4) matches the latency stall samples taken
 * at instructions of device functions and at call sites. */
enum {
  GPA_OPT_REGISTER_REUSE = 0, GPA_OPT_STRENGTH_REDUCTION = 1, GPA_OPT_FUNCTION_SPLIT = 2,
  GPA_OPT_FAST_MATH = 3, GPA_OPT_WARP_BALANCE = 4, GPA_OPT_MEMORY_TRANSACTION_REDUCTION = 5,
  GPA_OPT_LOOP_UNROLLING = 6, GPA_OPT_CODE_REORDERING = 7, GPA_OPT_FUNCTION_INLINING = 8
};

/* Opcode-class property bits of gpa_arch_desc.flags. */
enum {
  GPA_F_MEM = 1,         /* memory instruction: may take memory-dependency blame (Sec. 4 rule 1) */
  GPA_F_SYNC = 2,        /* synchronization instruction: may take sync blame (Sec. 4 rule 1) */
  GPA_F_GLOBAL = 4,      /* global memory (detailed class, Memory Transaction Reduction) */
  GPA_F_LOCAL = 8,       /* local memory (detailed class, Register Reuse) */
  GPA_F_CONST = 16,      /* constant memory (detailed class) */
  GPA_F_SHARED = 32,     /* shared memory (detailed execution-dependency class) */
  GPA_F_LONG_ARITH = 64, /* long-latency arithmetic (Strength Reduction) */
  GPA_F_VARLAT = 128     /* variable latency (write-after-read detection) */
};

/* Architecture table (Sec. 3 "Architectural features"; Sec. 4 latency rule).
 * latency[op]: instructions a def of opcode class op needs before its result
 * is ready; an edge whose shortest path is longer is pruned. Both arrays are
 * host memory of n_opclasses entries, copied by gpa_create. */
typedef struct {
  int32_t n_opclasses;       /* 1..GPA_MAX_OPCLASSES */
  const int32_t* latency;    /* host, >= 0 */
  const uint32_t* flags;     /* host, GPA_F_* bits */
} gpa_arch_desc;

typedef struct {
  int32_t max_fixpoint_sweeps;  /* reaching-definitions sweep limit; 0 = 64 */
  int32_t max_search_nodes;     /* (block, predicate-set) nodes of the largest general search; 0 = 32768 */
  int32_t search_slots;         /* warps with a max_search_nodes global-memory arena; 0 = as many as the
                                   search kernel keeps resident (24 per SM on GB300, about 16 GB of arenas
                                   at the default max_search_nodes) */
  int32_t max_sources_per_use;  /* distinct sources merged per stalled use; 0 = 2048 (max 2048) */
  int32_t small_search_nodes;   /* nodes of the shared-memory arena of a first-tier search warp; 0 = 64
                                   (max 1024). A search that outgrows it is redone in the next tier */
  int32_t mid_search_nodes;     /* nodes of the second tier's shared-memory arenas (three warps per SM
                                   up to 512 nodes, one up to 1024); 0 = small_search_nodes (searches that
                                   outgrow the first tier go on to the global-memory warps, which are
                                   faster than few large shared-memory arenas) */
  int32_t hist_variant;         /* aggregation kernel: 0 (default) = one CTA per SM taking chunks of
                                   tiles of 8,192 samples from a counter, shared memory used per
                                   2,048-sample segment as a direct-indexed window over up to 1,558
                                   instructions of the segment's kernel plus a hash for the rest;
                                   grid-strided with a shared-memory hash: 1 = 8,192 entries, 512
                                   threads, 2 CTAs per SM; 2 = 16,384 entries, 1,024 threads, 1 CTA
                                   per SM; 3 = 8,192 entries, 256 threads, 3 CTAs per SM */
  int32_t large_search_nodes;   /* a global-memory search that reached this many nodes is started
                                   before the others on later steps of its program; 0 = 1024 */
  int32_t hist_chunk;           /* aggregation variant 0: tiles per claimed chunk, 0 = 24 (max 4096) */
  int32_t reach_schedule;       /* reaching-definitions fixpoint: 0 (default) = a CTA per function staged
                                   in shared memory (launches by size class; functions beyond 200 KB of
                                   stage take the windowed kernel); 1 = the windowed kernel for every
                                   function (a lane per basic block, windows of 32 blocks in global
                                   memory) */
  int32_t small_search_warps;   /* first-tier search warps per SM (a multiple of 4, at most 32); 0 = 24.
                                   The first tier shares the SMs with the third tier's searches known
                                   from earlier steps, which take the registers it leaves */
} gpa_options;

/* A program: n_functions functions laid out one after another. All arrays are
 * host memory, read during gpa_load_program and copied; the caller may free
 * them on return. Indices are global (over the whole program), int32 unless
 * noted.
 *  func_instr_off[n_functions+1], func_block_off[n_functions+1],
 *  func_loop_off[n_functions+1]   ranges of each function's instructions,
 *                                 blocks and loops (pc = index - func_instr_off[f]).
 *  block_instr_off[n_blocks+1]    instructions of block b; every block has at least one.
 *  succ_off[n_blocks+1], succ[n_succ]  CFG successors (blocks of the same function).
 *                                 Block order: an edge u->v with v > u is a forward edge;
 *                                 an edge with v <= u must go to the header of a loop
 *                                 that contains u (a back edge). Every block must be
 *                                 reachable from its function's first block.
 *  opclass[n_instr] (uint8)       opcode class, < n_opclasses of the architecture table.
 *  guard[n_instr] (uint8)         guard literal: 0 none, 1+i = @Pi, 8+i = @!Pi (i < 7).
 *  iflags[n_instr] (uint8)        bit 0: instruction belongs to a math-library routine.
 *  line[n_instr]                  source line id, < n_lines.
 *  def_off[n_instr+1], def_res[n_def] (uint16)  resources written: resource | kind << 12,
 *                                 kind 1 = write barrier, 2 = read barrier (B resources only).
 *  use_off[n_instr+1], use_res[n_use] (uint16)  resources read: source registers, the guard
 *                                 predicate, barriers in the wait mask. No duplicates in a list.
 *  block_loop[n_blocks]           innermost loop containing the block, or -1.
 *  loop_parent[n_loops]           enclosing loop or -1; loop_header[n_loops] its header block.
 *  call_site[n_calls], call_callee[n_calls]  optional call table (n_calls = 0: none): the
 *                                 global index of a call instruction and the function it
 *                                 calls. A function that some call site calls is a device
 *                                 function (Table 2, Function Inlining). A call into or out of
 *                                 the program (as in one shard of a larger one) has site -1
 *                                 (called from elsewhere) or callee -1 (calls elsewhere), not
 *                                 both. Sites ascend: -1 entries first, the others distinct.
 * Limits: n_functions < 65536, instructions per function < 2^24, instructions per block
 * < 65536, n_instr * 24 < 2^32, n_blocks * 16 < 2^31 - 1, n_def + n_use < 2^31 - 1. */
typedef struct {
  int32_t n_functions, n_instr, n_blocks, n_loops, n_lines;
  int32_t n_succ, n_def, n_use;
  const int32_t* func_instr_off;
  const int32_t* func_block_off;
  const int32_t* func_loop_off;
  const int32_t* block_instr_off;
  const int32_t* succ_off;
  const int32_t* succ;
  const uint8_t* opclass;
  const uint8_t* guard;
  const uint8_t* iflags;
  const int32_t* line;
  const int32_t* def_off;
  const uint16_t* def_res;
  const int32_t* use_off;
  const uint16_t* use_res;
  const int32_t* block_loop;
  const int32_t* loop_parent;
  const int32_t* loop_header;
  int32_t n_calls;
  const int32_t* call_site;
  const int32_t* call_callee;
} gpa_program_desc;

/* Launch statistics of one function (kernel) as the profiler's kernel
 * records give them, input of the parallel optimizers (Table 2 "Parallel
 * Optimizers", Sec. 5.2 "Parallel Optimization Estimator"). */
typedef struct {
  int64_t blocks;             /* blocks in the grid, >= 1 */
  int32_t threads_per_block;  /* 1..1024 */
  int32_t regs_per_thread;    /* 0..255 */
  int32_t smem_per_block;     /* shared memory per block in bytes (static + dynamic), >= 0 */
  int32_t reserved;           /* must be 0 */
} gpa_launch_stats;

/* The SM of the occupancy model behind the parallel estimators (the public
 * occupancy-calculator rules): blocks per SM = the least of
 *   max_blocks_per_sm,
 *   floor(max_warps_per_sm / warps per block),
 *   floor(schedulers_per_sm * floor(regs_per_sm / schedulers_per_sm / regs per warp) / warps per block)
 *     with regs per warp = regs_per_thread * 32 rounded up to reg_alloc_unit (no limit if 0),
 *   floor(smem_per_sm / (smem_per_block + smem_reserved_per_block rounded up to smem_alloc_unit))
 *     (no limit if smem_per_block is 0).
 * All fields > 0 except smem_reserved_per_block (>= 0). */
typedef struct {
  int32_t n_sms, schedulers_per_sm, max_warps_per_sm, max_blocks_per_sm;
  int32_t regs_per_sm, reg_alloc_unit;
  int32_t smem_per_sm, smem_alloc_unit, smem_reserved_per_block;
} gpa_sm_model;

/* Advice destination (host memory); any NULL field is skipped.
 *  totals[n_functions*4]           T, A (active), L (latency), issued samples (Sec. 2.1, 5.2).
 *  matched[n_functions*9]          matched samples M (Eq. 2) or M^L (Eq. 4) per optimizer.
 *  speedup[n_functions*9]          Eq. 2 for optimizers 0-5, Eq. 4 for 6-8; T = 0 gives 1.0,
 *                                  T = M gives +inf.
 *  rank[n_functions*9]             optimizer ids by speedup, descending (ties: lower id).
 *  n_hot[n_functions*9]            hotspots filled (0..5).
 *  hot[n_functions*9*5*6]          per hotspot: def pc, use pc, def line, use line,
 *                                  distance (shortest path), matched samples; -1 when unused.
 *  loop_active[n_loops], loop_matched[n_loops], loop_speedup[n_loops]  Eq. 5 per loop scope.
 *  line_stall[n_lines], line_latency[n_lines]  blamed stall samples per source line and their
 *                                  latency-sample part.
 *  par_match[n_functions*2] (int32)  parallel optimizers (0 Block Increase, 1 Thread Increase):
 *                                  1 when Table 2's condition holds (fewer blocks than SMs; the
 *                                  per-SM block limit binds before the warp, register and
 *                                  shared-memory limits, with blocks enough to reach it).
 *  par_speedup[n_functions*2]      Eq. 10 with f = 1 when matched, else 1.0 (also without launch
 *                                  statistics). Not part of rank (kept apart from the code
 *                                  optimizers).
 *  par_warps[n_functions*4]        per optimizer: resident warps per scheduler before and after
 *                                  (W of Eq. 8 and W_new of Eq. 9); 0 without launch statistics.
 *  par_limit[n_functions] (int32)  the binding occupancy limit: 0 warps, 1 registers, 2 shared
 *                                  memory, 3 blocks per SM (lowest id on ties); -1 without
 *                                  launch statistics. */
typedef struct {
  uint64_t* totals;
  uint64_t* matched;
  double* speedup;
  int32_t* rank;
  int32_t* n_hot;
  int64_t* hot;
  uint64_t* loop_active;
  uint64_t* loop_matched;
  double* loop_speedup;
  uint64_t* line_stall;
  uint64_t* line_latency;
  int32_t* par_match;
  double* par_speedup;
  double* par_warps;
  int32_t* par_limit;
} gpa_advice;

const char* gpa_status_string(gpa_status s);

/* Fills *arch with the library's default table (host pointers to static
 * storage): opcode classes IADD, IMAD, FFMA, ISETP, MOV, BRA, BAR, MEMBAR, LDG,
 * STG, LDS, STS, LDL, STL, LDC, ATOM, F2F, MUFU, DFMA, EXIT, CALL in that order. */
gpa_status gpa_arch_default(gpa_arch_desc* arch);

/* Creates a context on the current CUDA device. arch (the architecture table of
 * Sec. 3 "Architectural features", with the latencies the latency rule of Sec. 4
 * uses) and opts are copied; opts may be NULL. *out owns device memory until
 * gpa_destroy. */
gpa_status gpa_create(const gpa_arch_desc* arch, const gpa_options* opts, gpa_ctx** out);

/* Synchronizes the device, frees every program and the context (resource
 * management; the paper has no counterpart). */
gpa_status gpa_destroy(gpa_ctx* ctx);

/* Validates and copies a program to the device and allocates its counters
 * and result buffers (stream-ordered allocations on the context's own build
 * stream; returns when they are done, without waiting for other streams).
 * The program is what the paper's static analyzer provides to the dynamic one
 * (Sec. 3: control flow graphs, loop nests, line maps; Sec. 2.2 and Sec. 4:
 * per-instruction operands, virtual barrier registers, predicates).
 * *out receives the program id. */
gpa_status gpa_load_program(gpa_ctx* ctx, const gpa_program_desc* prog, gpa_pid* out);

/* Device bytes gpa_load_program would request for prog under ctx (validated
 * like a load; nothing is allocated or copied), for admission control. It reads
 * only the context's architecture table and options, so unlike the other calls
 * it may run on another host thread while the context is in use. */
gpa_status gpa_program_footprint(gpa_ctx* ctx, const gpa_program_desc* prog, int64_t* bytes);

/* Device bytes requested for a loaded program (equal to its footprint). */
gpa_status gpa_program_bytes(gpa_ctx* ctx, gpa_pid pid, int64_t* bytes);

/* Frees a program (synchronizes the device first; resource management, no
 * counterpart in the paper). */
gpa_status gpa_unload_program(gpa_ctx* ctx, gpa_pid pid);

/* Frees a program in stream order: its device memory is released once the
 * work queued on stream so far has finished, without waiting on the host.
 * All of the program's work must have been queued on stream, or on streams
 * that stream waits for. The program id is invalid on return. */
gpa_status gpa_unload_program_async(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream);

/* Zeroes the program's sample counters, invalid count and status word. */
gpa_status gpa_reset_counts(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream);

/* Step (a), Sec. 2.1: adds n packed samples (device pointer, 8-byte aligned;
 * borrowed until stream passes this call) to the program's counters.
 * Layout, most significant bit first: kernel 16 | pc 24 | class 4 |
 * latency flag 1 | sm 8 | 11 reserved bits. Samples with an unknown kernel,
 * a pc past its function, class >= 12, SELECTED with the latency flag, or
 * nonzero reserved bits are counted as invalid, not fatal. Counters
 * accumulate across calls. */
gpa_status gpa_ingest_samples(gpa_ctx* ctx, gpa_pid pid, const uint64_t* dev_samples, size_t n,
                              gpa_stream stream);

/* Step (a) from host memory (8-byte aligned). Pinned host memory that the
 * current device can address is read by the aggregation kernel directly over
 * the host link, on at most 32 SMs (the link needs no more; work on other
 * streams can use the rest); other memory is copied in chunks through library staging
 * buffers, the copy of one chunk overlapping the aggregation of the last.
 * Returns when the work is enqueued; host_samples must stay valid and
 * unchanged until stream completes this call. */
gpa_status gpa_ingest_host_samples(gpa_ctx* ctx, gpa_pid pid, const uint64_t* host_samples, size_t n,
                                   gpa_stream stream);

/* The program's counters (n_instr*24 uint64, the layout of gpa_get_counts) as
 * device data, for a batch sharded over several GPUs (Sec. 2.1 aggregation is a
 * sum over samples, so counts of disjoint sample chunks add up): every rank
 * aggregates its chunk of the samples over the whole program and copies the
 * counters out with gpa_copy_counts (dev_dst: device memory of the current
 * device, 8-byte aligned, n_instr*24 entries); the owner of a function receives
 * the sum of the ranks' counts of that function in one exchange, and loads them
 * into its own program of the functions it owns with gpa_set_counts, which
 * replaces the counters, sets the invalid-sample count and clears the status
 * word (as gpa_reset_counts plus an ingest would). Both are asynchronous on
 * stream; dev_counts must stay valid until stream passes the call. */
gpa_status gpa_copy_counts(gpa_ctx* ctx, gpa_pid pid, uint64_t* dev_dst, gpa_stream stream);
gpa_status gpa_set_counts(gpa_ctx* ctx, gpa_pid pid, const uint64_t* dev_counts, uint64_t invalid,
                          gpa_stream stream);

/* Steps (b)-(c), Sec. 4: reaching definitions, backward slicing, pruning and
 * apportioning over the counters ingested so far. Replaces any previous blame. */
gpa_status gpa_blame(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream);

/* Step (d), Sec. 5: roll-up, optimizer matching, estimators and ranking. If out
 * is not NULL the results are copied to it and the call synchronizes stream;
 * with out == NULL they stay on the device (fetch later with gpa_get_advice). */
gpa_status gpa_advise(gpa_ctx* ctx, gpa_pid pid, const gpa_advice* out, gpa_stream stream);

/* Synchronizes stream and returns the program's device status word as a
 * gpa_status (GPA_OK, GPA_ERR_NOT_CONVERGED, GPA_ERR_CAPACITY, ...). If info is
 * not NULL it must have room for 8 values: info[0] = invalid samples,
 * info[1] = general (multi-block) searches run, info[2] = largest search in
 * nodes, info[3] = fixpoint sweeps, info[4] and info[5] = searches run by the
 * second and third search tiers in the last gpa_blame (handed on by a smaller
 * tier, or queued there directly because an earlier step of the program found
 * them that large), info[6] and
 * info[7] = the stalled use (global instruction index) and the resource of
 * the largest search. */
gpa_status gpa_sync_status(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream, int64_t* info);

/* Single dependency coverage (Sec. 6) of the program's current counts: out[0]
 * = stalled uses (instructions with dependency-class samples, the nodes of the
 * dependency graph), out[1] = those with at most one source through every
 * resource they read before pruning (all immediate sources of the backward
 * slice), out[2] = the same after pruning (sources that survive the dominator
 * and latency rules, and the opcode rule for one of the use's stalled
 * classes). A diagnostic: it runs unbounded searches (slower than gpa_blame),
 * leaves blame, edges and advice as they were, and overwrites the search
 * statistics of gpa_sync_status. out must hold 3 values; synchronizes stream.
 * The paper reports the ratios out[1] / out[0] and out[2] / out[0] (Sec. 6,
 * "Single Dependency Coverage"). */
gpa_status gpa_dependency_coverage(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream, int64_t* out);

/* The dependency graph before pruning (Sec. 4, "construct a dependency
 * graph"): every immediate source of every (stalled use, resource) of the
 * current counts, with its shortest distance, fewest back edges, the longest
 * distance with exactly that many back edges, and whether the dominator rule
 * cuts it (an unguarded reader of the resource on all its source paths; the
 * latency and opcode rules are left to the caller, from dmin and the def's
 * opcode class). Runs the unbounded searches twice (a counting pass sizes the
 * program-owned export buffer); *n_edges receives the edge count. Blame, edges
 * and advice stay as they were. Synchronizes stream. */
gpa_status gpa_export_unpruned_edges(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream, int64_t* n_edges);

/* Copies the last export, ordered by (use, resource, def), into arrays of
 * n_edges entries (NULL pointers are skipped): global use and def instruction
 * indices, resource id, dmin, back edges, dlong, dom (0/1). */
gpa_status gpa_get_unpruned_edges(gpa_ctx* ctx, gpa_pid pid, int32_t* use, int32_t* def, int32_t* res,
                                  int32_t* dmin, int32_t* back_edges, int32_t* dlong, uint8_t* dom,
                                  gpa_stream stream);

/* Captures one whole step of the program into a CUDA graph owned by the
 * program (replacing any earlier one): zero the counters, ingest n samples
 * from dev_samples (device pointer, 8-byte aligned, which must stay valid
 * and hold the step's input whenever the graph runs), blame, and compute the
 * advice (left on the device; gpa_get_advice copies it). Nothing runs at
 * capture, and nothing on the step path allocates, so the graph needs no
 * warm-up. Capture errors return GPA_ERR_CUDA and leave the previous graph
 * in place. */
gpa_status gpa_step_capture(gpa_ctx* ctx, gpa_pid pid, const uint64_t* dev_samples, size_t n);

/* Launches the captured step on stream, ordered after earlier users of the
 * context's search scratch. GPA_ERR_INVALID_ARG if nothing was captured. */
gpa_status gpa_step_launch(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream);

/* Diagnostic: per search tier (3) the SM cycles summed over the searches of the
 * last gpa_blame in six phases: building the graph, shortest distances and
 * fewest back edges, sources and rule 3, rule 2, longest paths and emission,
 * and (not cycles) the number of rule-2 reachability runs; out[0..17],
 * tier-major. Then out[18..33] = searches by floor(log2(nodes)) (the last
 * slot holds 2^15 nodes and more) and out[34] = searches that completed their
 * graph past the latency bound; out[35] = the slowest search's cycles << 20 |
 * its nodes, out[36] its rule-2 runs, out[37..41] its cycles in the first
 * five phases; out[42..57] the cycles of the searches by floor(log2(nodes)).
 * out[58] (kept in every build): why searches outgrew their arena in the last
 * gpa_blame, bit 1 nodes, 2 edges, 3 occurrences, 4 sources, 5 back-edge
 * layers, 6 hash round limit. out must hold 59 values. The others are zero unless the
 * library was built with -DGPA_PHASE_TIMING (the timers cost a few atomics per
 * search). Synchronizes stream. */
gpa_status gpa_get_search_profile(gpa_ctx* ctx, gpa_pid pid, uint64_t* out, gpa_stream stream);

/* Parity getters: synchronize stream and copy device results to host memory.
 * counts[n_instr*24]: the aggregated samples of Sec. 2.1 (Fig. 1), counts[pc*24 +
 * class*2 + latency]; *invalid may be NULL. */
gpa_status gpa_get_counts(gpa_ctx* ctx, gpa_pid pid, uint64_t* counts, uint64_t* invalid, gpa_stream stream);
/* rin/rout[n_blocks*9]: reaching definitions at resource granularity (Sec. 4,
 * "Backward slicing"): bit r of block b's 9 words set iff some def of resource r
 * reaches the entry/exit of b. */
gpa_status gpa_get_reaching(gpa_ctx* ctx, gpa_pid pid, uint32_t* rin, uint32_t* rout, gpa_stream stream);
/* blame[n_instr*24], same layout as counts: each instruction's own samples outside
 * the dependency classes plus what Eq. 1 apportions to it (Sec. 4). */
gpa_status gpa_get_blame(gpa_ctx* ctx, gpa_pid pid, uint64_t* blame, gpa_stream stream);
/* The dependency graph after pruning (Sec. 4, Fig. 4b-d): surviving merged edges,
 * sorted by (use, def). With all arrays NULL, only
 * *n_edges is written. Otherwise each array has room for cap entries:
 * use[], def[] global instruction indices; dmin/dlong shortest and longest
 * source path; flags bit 0 write-after-read, 1 via barrier, 2 via register,
 * 3 via predicate; share[cap*8] = blamed samples per (class 2,3,5,6) x latency flag. */
gpa_status gpa_get_edges(gpa_ctx* ctx, gpa_pid pid, int64_t* n_edges, int64_t cap, int32_t* use, int32_t* def,
                         int32_t* dmin, int32_t* dlong, uint32_t* flags, uint64_t* share, gpa_stream stream);
/* Copies the advice computed by the last gpa_advise (see gpa_advice). */
gpa_status gpa_get_advice(gpa_ctx* ctx, gpa_pid pid, const gpa_advice* out, gpa_stream stream);

/* Sets the launch statistics of the program's functions (stats[n_functions],
 * host, copied) and the SM they ran on, for the parallel optimizers of later
 * gpa_advise calls; stats == NULL clears them. Synchronous (waits for the
 * device). A step captured with gpa_step_capture is dropped (capture it
 * again; gpa_step_launch returns GPA_ERR_INVALID_ARG until then). Returns
 * GPA_ERR_INVALID_ARG, changing nothing, for a field out of its range. */
gpa_status gpa_set_launch_stats(gpa_ctx* ctx, gpa_pid pid, const gpa_launch_stats* stats, const gpa_sm_model* sm);

/* The SM model of a CUDA device: counts and sizes from the device properties;
 * register allocation in units of 256 per warp, shared memory in units of 128
 * bytes (the allocation granularities of this GPU generation). */
gpa_status gpa_sm_model_of_device(int device, gpa_sm_model* out);

/* Kernel launches issued by this context since creation (for accounting). */
int64_t gpa_launch_count(gpa_ctx* ctx);

/* In-place exclusive prefix sum of n int32 values on the device: dev_buf[k]
 * becomes the sum of the inputs before k and *dev_total (device memory) the sum
 * of all n. The sums are int32 and wrap silently on overflow: the running
 * total of the inputs must fit in int32. The paper has no counterpart: this is
 * the scan the library uses for its own offsets (edges per use, events per
 * block, predecessors).
 *
 * It allocates nothing, unlike the rest of the library, which owns
 * cudaMalloc'd buffers. It is for callers that cannot call cudaMalloc at the
 * point where they need a scan: code that runs inside another framework's
 * memory pool and must not grow the process's device footprint, or a profiler
 * callback that must not perturb the application it measures (an allocation
 * there can synchronize the device or change the memory the application sees).
 * Its scratch (the per-tile sums) is a fixed static device array of
 * (4096 + 64) int32 that every device loading the library holds until exit.
 *
 * Limits and behaviour: 0 <= n <= 16,777,216; larger n returns
 * GPA_ERR_CAPACITY, a null pointer or negative n GPA_ERR_INVALID_ARG, and
 * nothing is launched. The first call on a device looks up the scratch
 * address on that device (cudaGetSymbolAddress); make that first call before
 * any stream capture. Every call shares the one scratch array and leaves its
 * contents behind (nothing in it needs to start at zero): calls that overlap on
 * the GPU, on different streams or from different threads, race and give
 * wrong results. The call is asynchronous on stream. A CUDA error already
 * pending when it is called (from an earlier, unrelated call) makes it return
 * GPA_ERR_CUDA without launching, and leaves that error pending. */
gpa_status gpa_exclusive_scan_noalloc(int32_t* dev_buf, int64_t n, int32_t* dev_total, gpa_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* GPA_H_ */
