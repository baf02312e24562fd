// Host runtime behind the C ABI in include/gpa.h: context and program
// registry, input validation, device memory, stream-ordered launches, the
// chunked host-sample ingest, status words and parity getters.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "gpa_internal.cuh"

using namespace gpa;

namespace {

struct ProgramRec {
  Prog P{};
  bool dry = false;                     // count bytes only (gpa_program_footprint)
  int4* xbuf = nullptr;                 // export buffer of gpa_export_unpruned_edges (grown on demand)
  int64_t xbuf_cap = 0, x_n = 0;
  cudaStream_t build = nullptr;         // stream of the stream-ordered allocations and copies
  int64_t bytes = 0;                    // device bytes requested for the program
  cudaGraphExec_t step_exec = nullptr;  // captured step (gpa_step_capture)
  LaunchRec* launch = nullptr;          // launch statistics (gpa_set_launch_stats)
  int64_t step_launches = 0;            // kernels in it
  int32_t *pred_off = nullptr, *cursor = nullptr, *ev_off = nullptr;  // build scratch kept from allocation
  uint32_t* events = nullptr;
  int4* meta = nullptr;
  int n_succ = 0, n_def = 0, n_use = 0;
  int32_t* scan_tmp = nullptr;
  std::vector<void*> allocs;
};

}  // namespace

struct gpa_ctx {
  int device = 0;
  int sms = 0;
  Arch arch{};
  gpa_options opts{};
  SearchArena tier[3]{};
  cudaEvent_t scratch_ev = nullptr;
  std::map<gpa_pid, ProgramRec*> progs;
  gpa_pid next_pid = 1;
  int64_t launches = 0;
  // staging for gpa_ingest_host_samples
  uint64_t* stage[2] = {nullptr, nullptr};
  size_t stage_n = 0;
  cudaStream_t copy_stream = nullptr;
  cudaStream_t capture_stream = nullptr;  // private stream for gpa_step_capture
  cudaStream_t build_stream = nullptr;    // program allocation, copies and layout builds
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  gpa::SearchFork fork{nullptr, nullptr, nullptr};  // third-tier searches beside tiers 1-2
};

namespace {

constexpr size_t kStageSamples = (size_t)64 << 20;  // 64M samples (512 MB) per staging buffer

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return GPA_ERR_CUDA; \
  } while (0)

template <class T>
gpa_status dev_alloc(ProgramRec* R, T** p, size_t n) {
  const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
  R->bytes += (int64_t)bytes;
  if (R->dry) {  // counting only: a pointer that is never used
    *p = nullptr;
    return GPA_OK;
  }
  void* q = nullptr;
  if (cudaMallocAsync(&q, bytes, R->build) != cudaSuccess) return GPA_ERR_OOM;
  R->allocs.push_back(q);
  *p = (T*)q;
  return GPA_OK;
}
template <class T>
gpa_status dev_copy(ProgramRec* R, const T** dst, const T* src, size_t n) {
  T* p = nullptr;
  gpa_status s = dev_alloc(R, &p, n);
  if (s) return s;
  if (!R->dry && n && cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyHostToDevice, R->build) != cudaSuccess)
    return GPA_ERR_CUDA;
  *dst = p;
  return GPA_OK;
}

// Frees a program whose work has finished (the callers synchronize first).
void free_program(ProgramRec* R) {
  if (R->step_exec) cudaGraphExecDestroy(R->step_exec);
  if (R->xbuf) cudaFree(R->xbuf);
  if (R->launch) cudaFree(R->launch);
  if (R->build) cudaStreamSynchronize(R->build);
  for (void* p : R->allocs) cudaFree(p);
  delete R;
}

ProgramRec* find(gpa_ctx* ctx, gpa_pid pid) {
  if (!ctx) return nullptr;
  auto it = ctx->progs.find(pid);
  return it == ctx->progs.end() ? nullptr : it->second;
}

// ---------------------------------------------------------------- validation
gpa_status validate(const gpa_program_desc* d, const Arch& A) {
  const int nf = d->n_functions, ni = d->n_instr, nb = d->n_blocks, nl = d->n_loops;
  if (nf < 1 || nf >= 65536 || ni < 1 || nb < nf || nl < 0 || d->n_lines < 1 || d->n_succ < 0 || d->n_def < 0 ||
      d->n_use < 0)
    return GPA_ERR_INVALID_PROGRAM;
  if ((int64_t)ni * kCnt >= ((int64_t)1 << 32)) return GPA_ERR_INVALID_PROGRAM;
  // event lists: int32 offsets over (block, resource bucket) segments and events
  if ((int64_t)nb * kEvBuckets >= INT32_MAX || (int64_t)d->n_def + d->n_use >= INT32_MAX)
    return GPA_ERR_INVALID_PROGRAM;
  if (!d->func_instr_off || !d->func_block_off || !d->func_loop_off || !d->block_instr_off || !d->succ_off ||
      !d->opclass || !d->guard || !d->iflags || !d->line || !d->def_off || !d->use_off || !d->block_loop)
    return GPA_ERR_INVALID_ARG;
  if ((d->n_succ && !d->succ) || (d->n_def && !d->def_res) || (d->n_use && !d->use_res) ||
      (nl && (!d->loop_parent || !d->loop_header)) || d->n_calls < 0 ||
      (d->n_calls && (!d->call_site || !d->call_callee)))
    return GPA_ERR_INVALID_ARG;
  for (int c = 0; c < d->n_calls; ++c) {
    const int x = d->call_site[c], g = d->call_callee[c];
    if (x < -1 || x >= ni || g < -1 || g >= nf || (x < 0 && g < 0)) return GPA_ERR_INVALID_PROGRAM;
    if (c && (x < d->call_site[c - 1] || (x >= 0 && x == d->call_site[c - 1]))) return GPA_ERR_INVALID_PROGRAM;
  }
  auto mono = [](const int32_t* a, int n, int last, bool strict) {
    if (a[0] != 0 || a[n] != last) return false;
    for (int i = 0; i < n; ++i)
      if (strict ? a[i + 1] <= a[i] : a[i + 1] < a[i]) return false;
    return true;
  };
  if (!mono(d->func_instr_off, nf, ni, true) || !mono(d->func_block_off, nf, nb, true) ||
      !mono(d->func_loop_off, nf, nl, false) || !mono(d->block_instr_off, nb, ni, true) ||
      !mono(d->succ_off, nb, d->n_succ, false) || !mono(d->def_off, ni, d->n_def, false) ||
      !mono(d->use_off, ni, d->n_use, false))
    return GPA_ERR_INVALID_PROGRAM;
  std::vector<int> bfunc(nb), lfunc(nl);
  for (int b = 0; b < nb; ++b)
    if (d->block_instr_off[b + 1] - d->block_instr_off[b] > 65535) return GPA_ERR_INVALID_PROGRAM;
  for (int f = 0; f < nf; ++f) {
    if (d->func_instr_off[f + 1] - d->func_instr_off[f] >= (1 << 24)) return GPA_ERR_INVALID_PROGRAM;
    if (d->block_instr_off[d->func_block_off[f]] != d->func_instr_off[f]) return GPA_ERR_INVALID_PROGRAM;
    for (int b = d->func_block_off[f]; b < d->func_block_off[f + 1]; ++b) bfunc[b] = f;
    for (int l = d->func_loop_off[f]; l < d->func_loop_off[f + 1]; ++l) lfunc[l] = f;
  }
  for (int x = 0; x < ni; ++x) {
    if (d->opclass[x] >= A.n_op || d->guard[x] > 14 || d->line[x] < 0 || d->line[x] >= d->n_lines)
      return GPA_ERR_INVALID_PROGRAM;
    uint32_t seen[kWords];
    std::memset(seen, 0, sizeof seen);
    for (int e = d->def_off[x]; e < d->def_off[x + 1]; ++e) {
      const int r = d->def_res[e] & 0x1FF, kind = (d->def_res[e] >> 12) & 0xF;
      if (r >= kNumRes || (d->def_res[e] & 0x0E00) || kind > 2 || (kind && r < kBarBase)) return GPA_ERR_INVALID_PROGRAM;
      if (seen[r >> 5] >> (r & 31) & 1) return GPA_ERR_INVALID_PROGRAM;
      seen[r >> 5] |= 1u << (r & 31);
    }
    std::memset(seen, 0, sizeof seen);
    for (int e = d->use_off[x]; e < d->use_off[x + 1]; ++e) {
      const int r = d->use_res[e];
      if (r >= kNumRes) return GPA_ERR_INVALID_PROGRAM;
      if (seen[r >> 5] >> (r & 31) & 1) return GPA_ERR_INVALID_PROGRAM;
      seen[r >> 5] |= 1u << (r & 31);
    }
  }
  for (int l = 0; l < nl; ++l) {
    const int p = d->loop_parent[l], h = d->loop_header[l];
    if (p < -1 || p >= nl || p == l || (p >= 0 && lfunc[p] != lfunc[l])) return GPA_ERR_INVALID_PROGRAM;
    if (h < 0 || h >= nb || bfunc[h] != lfunc[l]) return GPA_ERR_INVALID_PROGRAM;
    int depth = 0;
    for (int q = l; q >= 0; q = d->loop_parent[q])
      if (++depth > nl) return GPA_ERR_INVALID_PROGRAM;  // parent cycle
  }
  auto in_loop = [&](int b, int l) {
    for (int q = d->block_loop[b]; q >= 0; q = d->loop_parent[q])
      if (q == l) return true;
    return false;
  };
  for (int b = 0; b < nb; ++b) {
    const int q = d->block_loop[b];
    if (q < -1 || q >= nl || (q >= 0 && lfunc[q] != bfunc[b])) return GPA_ERR_INVALID_PROGRAM;
  }
  for (int l = 0; l < nl; ++l)
    if (!in_loop(d->loop_header[l], l)) return GPA_ERR_INVALID_PROGRAM;
  for (int u = 0; u < nb; ++u) {
    for (int e = d->succ_off[u]; e < d->succ_off[u + 1]; ++e) {
      const int v = d->succ[e];
      if (v < 0 || v >= nb || bfunc[v] != bfunc[u]) return GPA_ERR_INVALID_PROGRAM;
      for (int e2 = d->succ_off[u]; e2 < e; ++e2)
        if (d->succ[e2] == v) return GPA_ERR_INVALID_PROGRAM;
      if (v <= u) {  // must be a back edge: v heads a loop that contains u
        bool ok = false;
        for (int q = d->block_loop[u]; q >= 0 && !ok; q = d->loop_parent[q]) ok = d->loop_header[q] == v;
        if (!ok) return GPA_ERR_INVALID_PROGRAM;
      }
    }
  }
  // every block reachable from its function's entry
  std::vector<char> reach(nb, 0);
  std::vector<int> st;
  for (int f = 0; f < nf; ++f) {
    st.push_back(d->func_block_off[f]);
    reach[d->func_block_off[f]] = 1;
  }
  while (!st.empty()) {
    int b = st.back();
    st.pop_back();
    for (int e = d->succ_off[b]; e < d->succ_off[b + 1]; ++e)
      if (!reach[d->succ[e]]) { reach[d->succ[e]] = 1; st.push_back(d->succ[e]); }
  }
  for (int b = 0; b < nb; ++b)
    if (!reach[b]) return GPA_ERR_INVALID_PROGRAM;
  return GPA_OK;
}

gpa_status status_from(unsigned long long st) {
  if (st & ST_NOT_CONVERGED) return GPA_ERR_NOT_CONVERGED;
  if (st & (ST_CAPACITY | ST_OVERFLOW)) return GPA_ERR_CAPACITY;
  if (st & ST_TIMEOUT) return GPA_ERR_TIMEOUT;
  return GPA_OK;
}

// Default opcode classes (order documented in gpa.h).
const int32_t kDefLat[21] = {4, 5, 4, 4, 2, 0, 32, 32, 1024, 1024, 32, 32, 1024, 1024, 64, 1024, 16, 16, 8, 0, 1024};
const uint32_t kDefFlags[21] = {
    0, 0, 0, 0, 0, 0, GPA_F_SYNC, GPA_F_SYNC,
    GPA_F_MEM | GPA_F_GLOBAL | GPA_F_VARLAT, GPA_F_MEM | GPA_F_GLOBAL | GPA_F_VARLAT,
    GPA_F_SHARED | GPA_F_VARLAT, GPA_F_SHARED | GPA_F_VARLAT,
    GPA_F_MEM | GPA_F_LOCAL | GPA_F_VARLAT, GPA_F_MEM | GPA_F_LOCAL | GPA_F_VARLAT,
    GPA_F_MEM | GPA_F_CONST | GPA_F_VARLAT, GPA_F_MEM | GPA_F_GLOBAL | GPA_F_VARLAT,
    GPA_F_LONG_ARITH | GPA_F_VARLAT, GPA_F_LONG_ARITH | GPA_F_VARLAT, 0, 0, 0};

}  // namespace

extern "C" {

const char* gpa_status_string(gpa_status s) {
  switch (s) {
    case GPA_OK: return "ok";
    case GPA_ERR_INVALID_ARG: return "invalid argument";
    case GPA_ERR_INVALID_PROGRAM: return "invalid program";
    case GPA_ERR_CUDA: return "CUDA runtime error";
    case GPA_ERR_NOT_CONVERGED: return "reaching-definitions fixpoint did not converge";
    case GPA_ERR_CAPACITY: return "capacity exceeded";
    case GPA_ERR_TIMEOUT: return "device wait timed out";
    case GPA_ERR_NO_PROGRAM: return "no such program";
    case GPA_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}

gpa_status gpa_arch_default(gpa_arch_desc* arch) {
  if (!arch) return GPA_ERR_INVALID_ARG;
  arch->n_opclasses = 21;
  arch->latency = kDefLat;
  arch->flags = kDefFlags;
  return GPA_OK;
}

gpa_status gpa_create(const gpa_arch_desc* arch, const gpa_options* opts, gpa_ctx** out) {
  if (!arch || !out || arch->n_opclasses < 1 || arch->n_opclasses > GPA_MAX_OPCLASSES || !arch->latency ||
      !arch->flags)
    return GPA_ERR_INVALID_ARG;
  for (int o = 0; o < arch->n_opclasses; ++o)
    if (arch->latency[o] < 0) return GPA_ERR_INVALID_ARG;
  gpa_options o{};
  if (opts) {
    o = *opts;
    if (o.max_fixpoint_sweeps < 0 || o.max_search_nodes < 0 || o.search_slots < 0 || o.max_sources_per_use < 0 ||
        o.max_sources_per_use > kBigSrc || o.small_search_nodes < 0 || o.mid_search_nodes < 0 ||
        o.hist_variant < 0 || o.hist_variant > 3 || o.large_search_nodes < 0 || o.hist_chunk < 0 ||
        o.hist_chunk > 4096 || o.reach_schedule < 0 || o.reach_schedule > 1 || o.small_search_warps < 0 ||
        o.small_search_warps > 32 || o.small_search_warps % 4 != 0)
      return GPA_ERR_INVALID_ARG;
  }
  auto* c = new (std::nothrow) gpa_ctx();
  if (!c) return GPA_ERR_OOM;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return GPA_ERR_CUDA;
  }
  c->arch.n_op = arch->n_opclasses;
  for (int k = 0; k < arch->n_opclasses; ++k) { c->arch.lat[k] = arch->latency[k]; c->arch.flags[k] = arch->flags[k]; }
  if (o.max_fixpoint_sweeps == 0) o.max_fixpoint_sweeps = 64;
  if (o.max_search_nodes == 0) o.max_search_nodes = 32768;
  // Global-memory search warps: as many as the search kernel keeps resident
  // (its registers allow 24 one-warp CTAs per SM on GB300). Many warps on
  // global-memory arenas hide latency better than few on shared memory.
  if (o.search_slots == 0) o.search_slots = search_warps_per_sm() * c->sms;
  if (o.max_sources_per_use == 0) o.max_sources_per_use = kBigSrc;
  if (o.large_search_nodes == 0) o.large_search_nodes = kLargeNodes;
  if (o.small_search_nodes == 0) o.small_search_nodes = 64;
  if (o.small_search_warps == 0) o.small_search_warps = 24;
  c->opts = o;
  // Tier 1: four warps per CTA with small shared-memory arenas, six CTAs per
  // SM by default (small_search_warps): as many warps as the search kernel's
  // registers allow. The searches are chains of dependent steps, so more warps
  // in flight finish more of them (on the batched workload, 64-node arenas at
  // 24 warps per SM take the first tier from 26.0 to 22.2 ms against 128-node
  // arenas at 12, while the third tier's hinted part runs beside it). Tier 2: three one-warp CTAs per SM with larger shared-memory arenas
  // (one per SM beyond 512 nodes). Tier 3: warps
  // with global-memory arenas for the rare searches beyond that. Node
  // capacities are powers of two (hash masks).
  int n1 = 2, n3 = 2;
  while (n1 < o.small_search_nodes && n1 < 1024) n1 <<= 1;
  while (n3 < o.max_search_nodes) n3 <<= 1;
  int n2 = 2;
  const int want2 = o.mid_search_nodes ? o.mid_search_nodes : n1;
  while (n2 < want2 && n2 < 1024) n2 <<= 1;
  n2 = std::max(n1, n2);
  SearchArena* T = c->tier;
  T[0].nodes = n1; T[0].src = std::min(n1, 64); T[0].layers = 4; T[0].warps = o.small_search_warps * c->sms;
  T[1].nodes = n2; T[1].src = std::min(n2, 256); T[1].layers = 4; T[1].warps = (n2 <= 512 ? 3 : 1) * c->sms;
  T[2].nodes = n3; T[2].src = std::min(n3, 1024); T[2].layers = kMaxLayers; T[2].warps = o.search_slots;
  for (int t = 0; t < 3; ++t) {
    T[t].bytes = search_arena_bytes(T[t].nodes, T[t].src, T[t].layers);
    T[t].global = nullptr;
  }
  gpa_status s = GPA_OK;
  if (T[0].bytes * 4 > 220 * 1024 || T[1].bytes > 220 * 1024) s = GPA_ERR_INVALID_ARG;
  if (!s && cudaMalloc(&T[2].global, (size_t)T[2].bytes * T[2].warps) != cudaSuccess) {
    T[2].global = nullptr;
    s = GPA_ERR_OOM;
  }
  if (!s && cudaMemset(T[2].global, 0, (size_t)T[2].bytes * T[2].warps) != cudaSuccess) s = GPA_ERR_CUDA;
  if (!s && cudaEventCreateWithFlags(&c->scratch_ev, cudaEventDisableTiming) != cudaSuccess) s = GPA_ERR_CUDA;
  if (!s && cudaStreamCreateWithFlags(&c->build_stream, cudaStreamNonBlocking) != cudaSuccess) s = GPA_ERR_CUDA;
  if (!s && cudaStreamCreateWithFlags(&c->fork.side, cudaStreamNonBlocking) != cudaSuccess) s = GPA_ERR_CUDA;
  if (!s && cudaEventCreateWithFlags(&c->fork.fork, cudaEventDisableTiming) != cudaSuccess) s = GPA_ERR_CUDA;
  if (!s && cudaEventCreateWithFlags(&c->fork.join, cudaEventDisableTiming) != cudaSuccess) s = GPA_ERR_CUDA;
  if (s) {
    if (c->tier[2].global) cudaFree(c->tier[2].global);
    if (c->scratch_ev) cudaEventDestroy(c->scratch_ev);
    if (c->build_stream) cudaStreamDestroy(c->build_stream);
    if (c->fork.side) cudaStreamDestroy(c->fork.side);
    if (c->fork.fork) cudaEventDestroy(c->fork.fork);
    if (c->fork.join) cudaEventDestroy(c->fork.join);
    delete c;
    return s;
  }
  *out = c;
  return GPA_OK;
}

gpa_status gpa_destroy(gpa_ctx* ctx) {
  if (!ctx) return GPA_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  for (auto& kv : ctx->progs) free_program(kv.second);
  if (ctx->tier[2].global) cudaFree(ctx->tier[2].global);
  for (int k = 0; k < 2; ++k) {
    if (ctx->stage[k]) cudaFree(ctx->stage[k]);
    if (ctx->ev_copied[k]) cudaEventDestroy(ctx->ev_copied[k]);
    if (ctx->ev_used[k]) cudaEventDestroy(ctx->ev_used[k]);
  }
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  if (ctx->build_stream) cudaStreamDestroy(ctx->build_stream);
  if (ctx->scratch_ev) cudaEventDestroy(ctx->scratch_ev);
  if (ctx->fork.side) cudaStreamDestroy(ctx->fork.side);
  if (ctx->fork.fork) cudaEventDestroy(ctx->fork.fork);
  if (ctx->fork.join) cudaEventDestroy(ctx->fork.join);
  delete ctx;
  return GPA_OK;
}

// Allocates (or, with R->dry, only counts) the program's device memory and
// copies its arrays. On failure the caller frees R.
static gpa_status alloc_program(const gpa_program_desc* d, ProgramRec* R, int tier3_nodes) {
  Prog& P = R->P;
  P.nf = d->n_functions; P.ni = d->n_instr; P.nb = d->n_blocks; P.nl = d->n_loops; P.n_lines = d->n_lines;
  // Staged fixpoint: the largest per-function need within the cap (edges stay
  // inside their function, so a function's predecessor entries are its
  // blocks' successor entries).
  auto reach_need = [&](int f) {
    const int b0 = d->func_block_off[f], b1 = d->func_block_off[f + 1];
    return reach_smem_need(b1 - b0, (int64_t)d->succ_off[b1] - d->succ_off[b0],
                           (int64_t)d->func_loop_off[f + 1] - d->func_loop_off[f]);
  };
  // Staged fixpoint: functions needing at most this much shared memory (the
  // others take the windowed global-memory kernel).
  P.reach_smem = 0;
  for (int f = 0; f < d->n_functions; ++f) {
    const int64_t need = reach_need(f);
    if (need <= kReachClassCap[0] && need > P.reach_smem) P.reach_smem = (int32_t)need;
  }
  R->n_succ = d->n_succ; R->n_def = d->n_def; R->n_use = d->n_use;
  const size_t ni = P.ni, nb = P.nb, nl = P.nl, nf = P.nf;
#define TRY(x)                        \
  do {                                \
    gpa_status t_ = (x);              \
    if (t_) return t_;                \
  } while (0)
  TRY(dev_copy(R, &P.func_instr_off, d->func_instr_off, nf + 1));
  {
    // The staged fixpoint takes the functions by shared memory need, largest
    // first, in four launches by size class (kReachClassCap): class c holds the
    // needs in (cap[c + 1], cap[c]], and its launch sizes its stage for the
    // largest of them. Functions beyond cap[0] are left to the windowed kernel.
    std::vector<int64_t> need(nf);
    for (size_t f = 0; f < nf; ++f) need[f] = reach_need((int)f);
    std::vector<int32_t> order(nf);
    for (size_t f = 0; f < nf; ++f) order[f] = (int32_t)f;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return need[a] > need[b]; });
    TRY(dev_copy(R, &P.reach_order, order.data(), nf));
    int q = 0;
    while (q < (int)nf && need[order[q]] > kReachClassCap[0]) ++q;
    for (int c = 0; c < 4; ++c) {
      P.reach_cls[c] = q;
      P.reach_cls_smem[c] = 0;
      const int64_t lo = c < 3 ? kReachClassCap[c + 1] : -1;
      while (q < (int)nf && need[order[q]] > lo) {
        P.reach_cls_smem[c] = std::max<int32_t>(P.reach_cls_smem[c], (int32_t)need[order[q]]);
        ++q;
      }
    }
    P.reach_cls[4] = q;
    // Natural loops: a loop body is the header and the blocks that reach one of
    // its latches (a body block with an edge to the header) without passing the
    // header. Then every body block reaches every other one, which lets the
    // fixpoint seed a block with the definitions of its enclosing loops.
    std::vector<uint8_t> natural(nf, 1);
    if (!R->dry) {  // (a footprint needs only the sizes)
      std::vector<int32_t> pcnt(nb + 1, 0), pl((size_t)d->n_succ);
      for (size_t u = 0; u < nb; ++u)
        for (int e = d->succ_off[u]; e < d->succ_off[u + 1]; ++e) ++pcnt[d->succ[e] + 1];
      for (size_t b = 0; b < nb; ++b) pcnt[b + 1] += pcnt[b];
      std::vector<int32_t> fill(pcnt.begin(), pcnt.end() - 1);
      for (size_t u = 0; u < nb; ++u)
        for (int e = d->succ_off[u]; e < d->succ_off[u + 1]; ++e) pl[fill[d->succ[e]]++] = (int32_t)u;
      auto in_body = [&](int b, int l) {
        for (int q = d->block_loop[b]; q >= 0; q = d->loop_parent[q])
          if (q == l) return true;
        return false;
      };
      std::vector<int32_t> body_n(nl, 0), stamp(nb, -1), st;
      for (size_t b = 0; b < nb; ++b)
        for (int q = d->block_loop[b]; q >= 0; q = d->loop_parent[q]) ++body_n[q];
      for (size_t f = 0; f < nf; ++f)
        for (int l = d->func_loop_off[f]; l < d->func_loop_off[f + 1] && natural[f]; ++l) {
          const int h = d->loop_header[l];
          int seen = 1;
          stamp[h] = l;
          st.clear();
          for (int e = pcnt[h]; e < pcnt[h + 1]; ++e)
            if (in_body(pl[e], l) && stamp[pl[e]] != l) { stamp[pl[e]] = l; ++seen; st.push_back(pl[e]); }
          while (!st.empty() && natural[f]) {
            const int x = st.back();
            st.pop_back();
            if (!in_body(x, l)) { natural[f] = 0; break; }
            for (int e = pcnt[x]; e < pcnt[x + 1]; ++e)
              if (stamp[pl[e]] != l) { stamp[pl[e]] = l; ++seen; st.push_back(pl[e]); }
          }
          if (seen != body_n[l]) natural[f] = 0;
        }
    }
    TRY(dev_copy(R, &P.func_natural, natural.data(), nf));
    // Smallest block reachable from each block: a min fixpoint over
    // successors, swept in descending block order (forward edges point up, so
    // each sweep settles every forward path; back edges need a few more).
    std::vector<int32_t> mr(nb);
    for (size_t b = 0; b < nb; ++b) mr[b] = (int32_t)b;
    for (bool changed = true; changed;) {
      changed = false;
      for (size_t b = nb; b-- > 0;)
        for (int e = d->succ_off[b]; e < d->succ_off[b + 1]; ++e)
          if (mr[d->succ[e]] < mr[b]) { mr[b] = mr[d->succ[e]]; changed = true; }
    }
    TRY(dev_copy(R, &P.block_minreach, mr.data(), nb));
  }
  TRY(dev_copy(R, &P.func_block_off, d->func_block_off, nf + 1));
  TRY(dev_copy(R, &P.func_loop_off, d->func_loop_off, nf + 1));
  TRY(dev_copy(R, &P.block_instr_off, d->block_instr_off, nb + 1));
  TRY(dev_copy(R, &P.succ_off, d->succ_off, nb + 1));
  TRY(dev_copy(R, &P.succ, d->succ, (size_t)d->n_succ));
  TRY(dev_copy(R, &P.opclass, d->opclass, ni));
  TRY(dev_copy(R, &P.guard, d->guard, ni));
  {
    // Instruction flags on the device: bit 0 math-library code (the caller's
    // bit 0), bit 1 call site, bit 2 in a device function (a function some call
    // site calls): Function Inlining matches bits 1-2.
    std::vector<uint8_t> fl(ni);
    std::vector<char> dev(nf, 0);
    for (int c = 0; c < d->n_calls; ++c)
      if (d->call_callee[c] >= 0) dev[d->call_callee[c]] = 1;
    for (size_t f = 0; f < nf; ++f)
      for (int x = d->func_instr_off[f]; x < d->func_instr_off[f + 1]; ++x)
        fl[x] = (uint8_t)((d->iflags[x] & 1) | (dev[f] ? 4 : 0));
    for (int c = 0; c < d->n_calls; ++c)
      if (d->call_site[c] >= 0) fl[d->call_site[c]] |= 2;
    TRY(dev_copy(R, &P.iflags, fl.data(), ni));
  }
  TRY(dev_copy(R, &P.line, d->line, ni));
  TRY(dev_copy(R, &P.def_off, d->def_off, ni + 1));
  TRY(dev_copy(R, &P.def_res, d->def_res, (size_t)d->n_def));
  TRY(dev_copy(R, &P.use_off, d->use_off, ni + 1));
  TRY(dev_copy(R, &P.use_res, d->use_res, (size_t)d->n_use));
  TRY(dev_copy(R, &P.block_loop, d->block_loop, nb));
  TRY(dev_copy(R, &P.loop_parent, d->loop_parent, nl));
  TRY(dev_copy(R, &P.loop_header, d->loop_header, nl));
  int32_t *pred_off = nullptr, *pred = nullptr, *cursor = nullptr, *ldepth = nullptr, *iblock = nullptr,
          *bfunc = nullptr;
  TRY(dev_alloc(R, &pred_off, nb + 1));
  TRY(dev_alloc(R, &pred, (size_t)d->n_succ));
  TRY(dev_alloc(R, &cursor, nb));
  TRY(dev_alloc(R, &ldepth, nl));
  TRY(dev_alloc(R, &iblock, ni));
  TRY(dev_alloc(R, &bfunc, nb));
  int32_t* ev_off = nullptr;
  uint32_t* events = nullptr;
  TRY(dev_alloc(R, &ev_off, nb * kEvBuckets + 1));
  TRY(dev_alloc(R, &events, (size_t)d->n_def + (size_t)d->n_use));
  P.ev_off = ev_off; P.events = events;
  TRY(dev_alloc(R, &P.res_maxlat, nf * kNumRes));
  TRY(dev_alloc(R, &P.res_guards, nf * kNumRes));
  P.pred_off = pred_off; P.pred = pred; P.loop_depth = ldepth; P.instr_block = iblock; P.block_func = bfunc;
  TRY(dev_alloc(R, &R->scan_tmp, scan_tmp_ints((int)std::max(ni, nb * kEvBuckets) + 1)));
  TRY(dev_alloc(R, &P.cnt, ni * kCnt));
  TRY(dev_alloc(R, &P.stats, (size_t)SS_N));
  TRY(dev_alloc(R, &P.def_mask, nb * kWords));
  TRY(dev_alloc(R, &P.touch_mask, nb * kWords));
  TRY(dev_alloc(R, &R->meta, 2 * nb));
  P.block_meta = R->meta;
  TRY(dev_alloc(R, &P.uuse_mask, nb * kWords));
  TRY(dev_alloc(R, &P.rin, nb * kWords));
  TRY(dev_alloc(R, &P.rout, nb * kWords));
  TRY(dev_alloc(R, &P.head, ni));
  P.raw_cap = 2 * (int64_t)d->n_use + 1024;
  TRY(dev_alloc(R, &P.raw, (size_t)P.raw_cap));
  P.queue_cap = (int64_t)d->n_use + 1;
  TRY(dev_alloc(R, &P.queue, (size_t)P.queue_cap));
  TRY(dev_alloc(R, &P.ovf_queue, (size_t)P.queue_cap));
  TRY(dev_alloc(R, &P.tier_hint, (size_t)std::max<int64_t>(d->n_use, 1)));
  TRY(dev_alloc(R, &P.large_hint, (size_t)std::max<int64_t>(d->n_use, 1)));
  TRY(dev_alloc(R, &P.large_queue, (size_t)kLargeQueue));
  TRY(dev_alloc(R, &P.cov_cnt, (size_t)std::max<int64_t>(d->n_use, 1)));
  P.diag = 0;
  TRY(dev_alloc(R, &P.edge_off, ni + 1));
  TRY(dev_alloc(R, &P.big_use, ni));
  TRY(dev_alloc(R, &P.suse, ni));
  P.edge_cnt = P.edge_off;
  P.edge_cap = P.raw_cap;
  TRY(dev_alloc(R, &P.e_use, (size_t)P.edge_cap));
  TRY(dev_alloc(R, &P.e_def, (size_t)P.edge_cap));
  TRY(dev_alloc(R, &P.e_dmin, (size_t)P.edge_cap));
  TRY(dev_alloc(R, &P.e_dlong, (size_t)P.edge_cap));
  TRY(dev_alloc(R, &P.e_flags, (size_t)P.edge_cap));
  TRY(dev_alloc(R, &P.e_share, (size_t)P.edge_cap * 8));
  TRY(dev_alloc(R, &P.blame, ni * kCnt));
  TRY(dev_alloc(R, &P.a_totals, nf * 4));
  TRY(dev_alloc(R, &P.a_matched, nf * GPA_NUM_OPT));
  TRY(dev_alloc(R, &P.a_speedup, nf * GPA_NUM_OPT));
  TRY(dev_alloc(R, &P.a_rank, nf * GPA_NUM_OPT));
  TRY(dev_alloc(R, &P.a_nhot, nf * GPA_NUM_OPT));
  TRY(dev_alloc(R, &P.a_hot, nf * GPA_NUM_OPT * 5 * 6));
  TRY(dev_alloc(R, &P.a_loop_active, nl));
  TRY(dev_alloc(R, &P.a_loop_matched, nl));
  TRY(dev_alloc(R, &P.a_loop_speedup, nl));
  TRY(dev_alloc(R, &P.a_line_stall, (size_t)P.n_lines));
  TRY(dev_alloc(R, &P.a_line_lat, (size_t)P.n_lines));
  TRY(dev_alloc(R, &P.a_par_match, nf * 2));
  TRY(dev_alloc(R, &P.a_par_speedup, nf * 2));
  TRY(dev_alloc(R, &P.a_par_warps, nf * 4));
  TRY(dev_alloc(R, &P.a_par_limit, nf));
  P.launch = nullptr;
  P.sm = SmModel{};
  // Fourth search tier: room for 64 literal sets per block of the largest
  // function (at most 2^22 nodes), when that is more than the context's
  // third tier holds; fewer CTAs for bigger arenas (about 2 GB at most).
  {
    int64_t mb = 1;
    for (int f = 0; f < d->n_functions; ++f) mb = std::max<int64_t>(mb, d->func_block_off[f + 1] - d->func_block_off[f]);
    int64_t n4 = 2;
    while (n4 < 64 * mb && n4 < ((int64_t)1 << 22)) n4 <<= 1;
    P.t4_nodes = 0; P.t4_arena = nullptr; P.t4_bytes = 0; P.t4_ctas = 0; P.t4_src = 0;
    if (n4 > tier3_nodes) {
      P.t4_nodes = (int32_t)n4;
      P.t4_src = (int32_t)std::min<int64_t>(n4, 4096);
      P.t4_ctas = n4 <= ((int64_t)1 << 18) ? 16 : n4 <= ((int64_t)1 << 20) ? 8 : 4;
      P.t4_bytes = search_arena_bytes(P.t4_nodes, P.t4_src, kMaxLayers);
      TRY(dev_alloc(R, &P.t4_arena, (size_t)P.t4_bytes * P.t4_ctas));
    }
  }
#undef TRY
  R->pred_off = pred_off; R->cursor = cursor; R->ev_off = ev_off; R->events = events;
  return GPA_OK;
}

gpa_status gpa_program_footprint(gpa_ctx* ctx, const gpa_program_desc* d, int64_t* bytes) {
  if (!ctx || !d || !bytes) return GPA_ERR_INVALID_ARG;
  gpa_status s = validate(d, ctx->arch);
  if (s) return s;
  ProgramRec R;
  R.dry = true;
  s = alloc_program(d, &R, ctx->tier[2].nodes);
  if (s) return s;
  *bytes = R.bytes;
  return GPA_OK;
}

gpa_status gpa_program_bytes(gpa_ctx* ctx, gpa_pid pid, int64_t* bytes) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!bytes) return GPA_ERR_INVALID_ARG;
  *bytes = R->bytes;
  return GPA_OK;
}

gpa_status gpa_load_program(gpa_ctx* ctx, const gpa_program_desc* d, gpa_pid* out) {
  if (!ctx || !d || !out) return GPA_ERR_INVALID_ARG;
  gpa_status s = validate(d, ctx->arch);
  if (s) return s;
  auto* R = new (std::nothrow) ProgramRec();
  if (!R) return GPA_ERR_OOM;
  R->build = ctx->build_stream;
  s = alloc_program(d, R, ctx->tier[2].nodes);
  if (s) { free_program(R); return s; }
  Prog& P = R->P;
  P.large_nodes = ctx->opts.large_search_nodes;
  const size_t ni = P.ni;
  int32_t *pred_off = R->pred_off, *cursor = R->cursor, *ev_off = R->ev_off;
  uint32_t* events = R->events;
  // Everything of the load runs on the context's build stream, which is then
  // synchronized: other streams' work is not waited for.
  cudaStream_t st = R->build;
  if (cudaMemsetAsync(P.cnt, 0, ni * kCnt * sizeof(unsigned long long), st) != cudaSuccess ||
      cudaMemsetAsync(P.stats, 0, SS_N * sizeof(unsigned long long), st) != cudaSuccess ||
      cudaMemsetAsync(P.edge_off, 0, (ni + 1) * sizeof(int32_t), st) != cudaSuccess) {
    free_program(R);
    return GPA_ERR_CUDA;
  }
  if (cudaMemsetAsync(P.tier_hint, 0, sizeof(uint32_t) * (size_t)std::max<int64_t>(R->n_use, 1), st) != cudaSuccess ||
      cudaMemsetAsync(P.large_hint, 0, (size_t)std::max<int64_t>(R->n_use, 1), st) != cudaSuccess) {
    free_program(R);
    return GPA_ERR_CUDA;
  }
  if (P.t4_arena && cudaMemsetAsync(P.t4_arena, 0, (size_t)P.t4_bytes * P.t4_ctas, st) != cudaSuccess) {
    free_program(R);
    return GPA_ERR_CUDA;
  }
  launch_build_layout(P, st, ctx->sms, &ctx->launches);
  launch_build_preds(P, R->n_succ, pred_off, cursor, R->scan_tmp, st, ctx->sms, &ctx->launches);
  launch_build_events(P, ev_off, events, R->scan_tmp, st, ctx->sms, &ctx->launches);
  launch_build_meta(P, R->meta, st, ctx->sms, &ctx->launches);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    free_program(R);
    return GPA_ERR_CUDA;
  }
  const gpa_pid pid = ctx->next_pid++;
  ctx->progs[pid] = R;
  *out = pid;
  return GPA_OK;
}

gpa_status gpa_unload_program(gpa_ctx* ctx, gpa_pid pid) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  cudaDeviceSynchronize();
  free_program(R);
  ctx->progs.erase(pid);
  return GPA_OK;
}

gpa_status gpa_unload_program_async(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  cudaStream_t st = (cudaStream_t)stream;
  // The captured graph, if any, is freed when an in-flight launch completes.
  if (R->step_exec) cudaGraphExecDestroy(R->step_exec);
  R->step_exec = nullptr;
  gpa_status s = GPA_OK;
  for (void* p : R->allocs)
    if (cudaFreeAsync(p, st) != cudaSuccess) s = GPA_ERR_CUDA;
  R->allocs.clear();
  delete R;
  ctx->progs.erase(pid);
  return s;
}

gpa_status gpa_reset_counts(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(R->P.cnt, 0, (size_t)R->P.ni * kCnt * sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(R->P.stats, 0, SS_N * sizeof(unsigned long long), st));
  return GPA_OK;
}

gpa_status gpa_copy_counts(gpa_ctx* ctx, gpa_pid pid, uint64_t* dev_dst, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!dev_dst || (reinterpret_cast<uintptr_t>(dev_dst) & 7u)) return GPA_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(dev_dst, R->P.cnt, (size_t)R->P.ni * kCnt * sizeof(unsigned long long),
                     cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return GPA_OK;
}

gpa_status gpa_set_counts(gpa_ctx* ctx, gpa_pid pid, const uint64_t* dev_counts, uint64_t invalid,
                          gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!dev_counts || (reinterpret_cast<uintptr_t>(dev_counts) & 7u)) return GPA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(R->P.stats, 0, SS_N * sizeof(unsigned long long), st));
  CK(cudaMemcpyAsync(R->P.cnt, dev_counts, (size_t)R->P.ni * kCnt * sizeof(unsigned long long),
                     cudaMemcpyDeviceToDevice, st));
  launch_store_u64(&R->P.stats[SS_INVALID], (unsigned long long)invalid, st, &ctx->launches);
  CK(cudaGetLastError());
  return GPA_OK;
}

gpa_status gpa_ingest_samples(gpa_ctx* ctx, gpa_pid pid, const uint64_t* dev_samples, size_t n, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (n == 0) return GPA_OK;
  if (!dev_samples || (reinterpret_cast<uintptr_t>(dev_samples) & 7u)) return GPA_ERR_INVALID_ARG;
  launch_histogram(R->P, dev_samples, n, (cudaStream_t)stream, ctx->sms, &ctx->launches, ctx->opts.hist_variant,
                   ctx->opts.hist_chunk);
  CK(cudaGetLastError());
  return GPA_OK;
}

constexpr int kHostIngestCtas = 32;  // SMs an ingest over the host link takes

gpa_status gpa_ingest_host_samples(gpa_ctx* ctx, gpa_pid pid, const uint64_t* host, size_t n, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (n == 0) return GPA_OK;
  if (!host) return GPA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // Pinned host memory that this device can address (page-locked allocations
  // are mapped under unified addressing) is read by the aggregation kernel
  // itself over the host link: no staging buffer, no copy engine. The link
  // (about 210 GB/s) needs far fewer SMs than HBM (about 23 GB/s an SM), so the
  // launch takes at most kHostIngestCtas of them and leaves the rest to other
  // work, such as the blame of the batch before. Other memory goes through the
  // staging buffers.
  cudaPointerAttributes at{};
  int dev = -1;
  if (cudaPointerGetAttributes(&at, host) == cudaSuccess && at.type == cudaMemoryTypeHost && at.devicePointer &&
      cudaGetDevice(&dev) == cudaSuccess && dev == ctx->device) {
    launch_histogram(R->P, static_cast<const uint64_t*>(at.devicePointer), n, st,
                     std::min(ctx->sms, kHostIngestCtas), &ctx->launches, ctx->opts.hist_variant,
                     ctx->opts.hist_chunk);
    CK(cudaGetLastError());
    return GPA_OK;
  }
  cudaGetLastError();  // a failed query is not an error here
  if (!ctx->stage[0]) {
    ctx->stage_n = kStageSamples;
    for (int k = 0; k < 2; ++k) {
      if (cudaMalloc(&ctx->stage[k], ctx->stage_n * sizeof(uint64_t)) != cudaSuccess) return GPA_ERR_OOM;
      CK(cudaEventCreateWithFlags(&ctx->ev_copied[k], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_used[k], cudaEventDisableTiming));
      CK(cudaEventRecord(ctx->ev_used[k], st));
    }
    CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  }
  // Double buffering: the copy of chunk c+1 overlaps the aggregation of chunk c.
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_used[0], 0));
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_used[1], 0));
  size_t off = 0;
  for (int c = 0; off < n; ++c) {
    const int k = c & 1;
    const size_t m = std::min(ctx->stage_n, n - off);
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_used[k], 0));
    CK(cudaMemcpyAsync(ctx->stage[k], host + off, m * sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->copy_stream));
    CK(cudaEventRecord(ctx->ev_copied[k], ctx->copy_stream));
    CK(cudaStreamWaitEvent(st, ctx->ev_copied[k], 0));
    launch_histogram(R->P, ctx->stage[k], m, st, ctx->sms, &ctx->launches, ctx->opts.hist_variant,
                     ctx->opts.hist_chunk);
    CK(cudaEventRecord(ctx->ev_used[k], st));
    off += m;
  }
  CK(cudaGetLastError());
  return GPA_OK;
}

// Steps (b)-(c) on stream st. With order_scratch, waits for and marks the
// context's shared search scratch (a captured step does this around its
// graph launch instead).
static gpa_status blame_body(gpa_ctx* ctx, ProgramRec* R, cudaStream_t st, bool order_scratch) {
  // per-step counters: general searches, largest search, sweeps, raw edges, queues
  CK(cudaMemsetAsync(R->P.stats + SS_GENERAL, 0, sizeof(unsigned long long) * 3, st));
  CK(cudaMemsetAsync(R->P.stats + SS_RAW_N, 0, sizeof(unsigned long long) * (SS_N - SS_RAW_N), st));
  launch_dataflow(R->P, ctx->arch, ctx->opts.max_fixpoint_sweeps, ctx->opts.reach_schedule, st, ctx->sms,
                  &ctx->launches);
  // The search scratch is shared by the context's programs: order its users.
  if (order_scratch) CK(cudaStreamWaitEvent(st, ctx->scratch_ev, 0));
  launch_blame(R->P, ctx->arch, ctx->tier, &ctx->fork, ctx->opts.max_sources_per_use, R->scan_tmp, st, ctx->sms,
               &ctx->launches);
  if (order_scratch) CK(cudaEventRecord(ctx->scratch_ev, st));
  CK(cudaGetLastError());
  return GPA_OK;
}

gpa_status gpa_blame(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  return blame_body(ctx, R, (cudaStream_t)stream, true);
}

// The counting run of the searches (P.diag = 1) behind gpa_dependency_coverage
// and gpa_export_unpruned_edges; h receives the stats words.
static gpa_status coverage_run(gpa_ctx* ctx, ProgramRec* R, cudaStream_t st, int diag, unsigned long long* h) {
  Prog D = R->P;
  D.diag = diag;
  D.xedges = R->xbuf;
  D.xcap = diag == 2 ? R->xbuf_cap : 0;
  CK(cudaMemsetAsync(D.cov_cnt, 0, sizeof(uint32_t) * (size_t)std::max(R->n_use, 1), st));
  CK(cudaMemsetAsync(D.stats + SS_GENERAL, 0, sizeof(unsigned long long) * 3, st));
  CK(cudaMemsetAsync(D.stats + SS_RAW_N, 0, sizeof(unsigned long long) * (SS_N - SS_RAW_N), st));
  launch_dataflow(D, ctx->arch, ctx->opts.max_fixpoint_sweeps, ctx->opts.reach_schedule, st, ctx->sms,
                  &ctx->launches);
  CK(cudaStreamWaitEvent(st, ctx->scratch_ev, 0));
  launch_coverage(D, ctx->arch, ctx->tier, &ctx->fork, st, ctx->sms, &ctx->launches);
  CK(cudaEventRecord(ctx->scratch_ev, st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(h, D.stats, sizeof(unsigned long long) * SS_N, cudaMemcpyDeviceToHost));
  return status_from(h[SS_STATUS]);
}

gpa_status gpa_dependency_coverage(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream, int64_t* out) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!out) return GPA_ERR_INVALID_ARG;
  unsigned long long h[SS_N];
  const gpa_status s = coverage_run(ctx, R, (cudaStream_t)stream, 1, h);
  out[0] = (int64_t)h[SS_COV];
  out[1] = (int64_t)h[SS_COV + 1];
  out[2] = (int64_t)h[SS_COV + 2];
  return s;
}

gpa_status gpa_export_unpruned_edges(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream, int64_t* n_edges) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!n_edges) return GPA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[SS_N];
  gpa_status s = coverage_run(ctx, R, st, 1, h);  // sizes the export
  if (s) return s;
  const int64_t need = (int64_t)h[SS_COV_ALL];
  if (need > R->xbuf_cap) {
    if (R->xbuf) cudaFree(R->xbuf);
    R->xbuf = nullptr;
    R->xbuf_cap = 0;
    if (cudaMalloc(&R->xbuf, sizeof(int4) * 2 * (size_t)std::max<int64_t>(need, 1)) != cudaSuccess) return GPA_ERR_OOM;
    R->xbuf_cap = std::max<int64_t>(need, 1);
  }
  s = coverage_run(ctx, R, st, 2, h);
  R->x_n = std::min<int64_t>((int64_t)h[SS_XN], R->xbuf_cap);
  *n_edges = R->x_n;
  return s;
}

gpa_status gpa_get_unpruned_edges(gpa_ctx* ctx, gpa_pid pid, int32_t* use, int32_t* def, int32_t* res,
                                  int32_t* dmin, int32_t* back_edges, int32_t* dlong, uint8_t* dom, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  const int64_t n = R->x_n;
  std::vector<int4> x(2 * (size_t)n);
  if (n) CK(cudaMemcpy(x.data(), R->xbuf, sizeof(int4) * 2 * (size_t)n, cudaMemcpyDeviceToHost));
  std::vector<int64_t> order(n);
  for (int64_t k = 0; k < n; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    const int4 &p = x[2 * a], &q = x[2 * b];
    if (p.x != q.x) return p.x < q.x;
    if (p.z != q.z) return p.z < q.z;
    return p.y < q.y;
  });
  for (int64_t t = 0; t < n; ++t) {
    const int4 a = x[2 * order[t]], b = x[2 * order[t] + 1];
    if (use) use[t] = a.x;
    if (def) def[t] = a.y;
    if (res) res[t] = a.z;
    if (dmin) dmin[t] = a.w;
    if (back_edges) back_edges[t] = b.x;
    if (dlong) dlong[t] = b.y;
    if (dom) dom[t] = (uint8_t)b.z;
  }
  return GPA_OK;
}

gpa_status gpa_step_capture(gpa_ctx* ctx, gpa_pid pid, const uint64_t* dev_samples, size_t n) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (n && (!dev_samples || (reinterpret_cast<uintptr_t>(dev_samples) & 7u))) return GPA_ERR_INVALID_ARG;
  if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
  cudaStream_t cs = ctx->capture_stream;
  const int64_t l0 = ctx->launches;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  gpa_status s = GPA_OK;
  if (cudaMemsetAsync(R->P.cnt, 0, (size_t)R->P.ni * kCnt * sizeof(unsigned long long), cs) != cudaSuccess ||
      cudaMemsetAsync(R->P.stats, 0, SS_N * sizeof(unsigned long long), cs) != cudaSuccess)
    s = GPA_ERR_CUDA;
  if (!s && n)
    launch_histogram(R->P, dev_samples, n, cs, ctx->sms, &ctx->launches, ctx->opts.hist_variant,
                     ctx->opts.hist_chunk);
  if (!s) s = blame_body(ctx, R, cs, false);
  if (!s) launch_advise(R->P, ctx->arch, cs, ctx->sms, &ctx->launches);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(cs, &g);
  const int64_t kernels = ctx->launches - l0;
  ctx->launches = l0;  // nothing ran yet
  if (s || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return s ? s : GPA_ERR_CUDA;
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) { cudaGetLastError(); return GPA_ERR_CUDA; }
  if (R->step_exec) cudaGraphExecDestroy(R->step_exec);
  R->step_exec = ex;
  R->step_launches = kernels;
  return GPA_OK;
}

gpa_status gpa_step_launch(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!R->step_exec) return GPA_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamWaitEvent(st, ctx->scratch_ev, 0));
  CK(cudaGraphLaunch(R->step_exec, st));
  CK(cudaEventRecord(ctx->scratch_ev, st));
  ctx->launches += R->step_launches;
  return GPA_OK;
}

static gpa_status copy_advice(ProgramRec* R, const gpa_advice* out, cudaStream_t st) {
  const Prog& P = R->P;
  const size_t nf = P.nf, no = GPA_NUM_OPT;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return (dst && bytes) ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
  };
  CK(cp(out->totals, P.a_totals, nf * 4 * 8));
  CK(cp(out->matched, P.a_matched, nf * no * 8));
  CK(cp(out->speedup, P.a_speedup, nf * no * 8));
  CK(cp(out->rank, P.a_rank, nf * no * 4));
  CK(cp(out->n_hot, P.a_nhot, nf * no * 4));
  CK(cp(out->hot, P.a_hot, nf * no * 5 * 6 * 8));
  CK(cp(out->loop_active, P.a_loop_active, (size_t)P.nl * 8));
  CK(cp(out->loop_matched, P.a_loop_matched, (size_t)P.nl * 8));
  CK(cp(out->loop_speedup, P.a_loop_speedup, (size_t)P.nl * 8));
  CK(cp(out->line_stall, P.a_line_stall, (size_t)P.n_lines * 8));
  CK(cp(out->line_latency, P.a_line_lat, (size_t)P.n_lines * 8));
  CK(cp(out->par_match, P.a_par_match, nf * 2 * 4));
  CK(cp(out->par_speedup, P.a_par_speedup, nf * 2 * 8));
  CK(cp(out->par_warps, P.a_par_warps, nf * 4 * 8));
  CK(cp(out->par_limit, P.a_par_limit, nf * 4));
  CK(cudaStreamSynchronize(st));
  return GPA_OK;
}

static_assert(sizeof(LaunchRec) == sizeof(gpa_launch_stats) && offsetof(gpa_launch_stats, threads_per_block) == 8 &&
                  offsetof(LaunchRec, threads) == 8 && offsetof(gpa_launch_stats, smem_per_block) == 16 &&
                  offsetof(LaunchRec, smem) == 16,
              "LaunchRec mirrors gpa_launch_stats");

gpa_status gpa_set_launch_stats(gpa_ctx* ctx, gpa_pid pid, const gpa_launch_stats* stats, const gpa_sm_model* sm) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  Prog& P = R->P;
  if (stats) {
    if (!sm || sm->n_sms < 1 || sm->schedulers_per_sm < 1 || sm->max_warps_per_sm < 1 || sm->max_blocks_per_sm < 1 ||
        sm->regs_per_sm < 1 || sm->reg_alloc_unit < 1 || sm->smem_per_sm < 1 || sm->smem_alloc_unit < 1 ||
        sm->smem_reserved_per_block < 0)
      return GPA_ERR_INVALID_ARG;
    for (int f = 0; f < P.nf; ++f) {
      const gpa_launch_stats& L = stats[f];
      if (L.blocks < 1 || L.threads_per_block < 1 || L.threads_per_block > 1024 || L.regs_per_thread < 0 ||
          L.regs_per_thread > 255 || L.smem_per_block < 0 || L.reserved != 0)
        return GPA_ERR_INVALID_ARG;
    }
  }
  // Kernels of earlier calls may read the old statistics; a captured step
  // holds the old ones and is dropped (capture it again).
  CK(cudaDeviceSynchronize());
  if (R->step_exec) {
    cudaGraphExecDestroy(R->step_exec);
    R->step_exec = nullptr;
  }
  if (!stats) {
    P.launch = nullptr;
    return GPA_OK;
  }
  if (!R->launch && cudaMalloc(&R->launch, sizeof(LaunchRec) * (size_t)std::max(P.nf, 1)) != cudaSuccess) {
    R->launch = nullptr;
    return GPA_ERR_OOM;
  }
  CK(cudaMemcpy(R->launch, stats, sizeof(LaunchRec) * (size_t)P.nf, cudaMemcpyHostToDevice));
  P.launch = R->launch;
  P.sm = SmModel{sm->n_sms, sm->schedulers_per_sm, sm->max_warps_per_sm, sm->max_blocks_per_sm, sm->regs_per_sm,
                 sm->reg_alloc_unit, sm->smem_per_sm, sm->smem_alloc_unit, sm->smem_reserved_per_block};
  return GPA_OK;
}

gpa_status gpa_sm_model_of_device(int device, gpa_sm_model* out) {
  if (!out) return GPA_ERR_INVALID_ARG;
  cudaDeviceProp d{};
  CK(cudaGetDeviceProperties(&d, device));
  out->n_sms = d.multiProcessorCount;
  out->schedulers_per_sm = 4;
  out->max_warps_per_sm = d.maxThreadsPerMultiProcessor / 32;
  out->max_blocks_per_sm = d.maxBlocksPerMultiProcessor;
  out->regs_per_sm = d.regsPerMultiprocessor;
  out->reg_alloc_unit = 256;
  out->smem_per_sm = (int32_t)d.sharedMemPerMultiprocessor;
  out->smem_alloc_unit = 128;
  out->smem_reserved_per_block = (int32_t)d.reservedSharedMemPerBlock;
  return GPA_OK;
}

gpa_status gpa_advise(gpa_ctx* ctx, gpa_pid pid, const gpa_advice* out, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  cudaStream_t st = (cudaStream_t)stream;
  launch_advise(R->P, ctx->arch, st, ctx->sms, &ctx->launches);
  CK(cudaGetLastError());
  if (out) return copy_advice(R, out, st);
  return GPA_OK;
}

gpa_status gpa_get_advice(gpa_ctx* ctx, gpa_pid pid, const gpa_advice* out, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!out) return GPA_ERR_INVALID_ARG;
  return copy_advice(R, out, (cudaStream_t)stream);
}

gpa_status gpa_sync_status(gpa_ctx* ctx, gpa_pid pid, gpa_stream stream, int64_t* info) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[SS_N];
  CK(cudaStreamSynchronize(st));
  CK(cudaMemcpy(h, R->P.stats, sizeof h, cudaMemcpyDeviceToHost));
  if (info) {
    info[0] = (int64_t)h[SS_INVALID];
    info[1] = (int64_t)h[SS_GENERAL];
    info[2] = (int64_t)h[SS_MAX_NODES];
    info[3] = (int64_t)h[SS_SWEEPS];
    info[4] = (int64_t)h[SS_OVF_N];
    info[5] = (int64_t)(h[SS_OVF2_N] + h[SS_HINT3_N] + std::min<unsigned long long>(h[SS_LARGE_N], kLargeQueue));
    info[6] = (int64_t)(h[SS_MAX_TASK] & 0x7FFFFFFFull);     // use of the largest search
    info[7] = (int64_t)((h[SS_MAX_TASK] >> 31) & 0x1FFull);  // its resource
  }
  return status_from(h[SS_STATUS]);
}

gpa_status gpa_get_search_profile(gpa_ctx* ctx, gpa_pid pid, uint64_t* out, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!out) return GPA_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(out, R->P.stats + SS_PHASE, 42 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(out + 42, R->P.stats + SS_SIZE_CYC, 16 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(out + 58, R->P.stats + SS_FAILBITS, sizeof(uint64_t), cudaMemcpyDeviceToHost));
  return GPA_OK;
}

gpa_status gpa_get_counts(gpa_ctx* ctx, gpa_pid pid, uint64_t* counts, uint64_t* invalid, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(st));
  if (counts) CK(cudaMemcpy(counts, R->P.cnt, (size_t)R->P.ni * kCnt * 8, cudaMemcpyDeviceToHost));
  if (invalid) CK(cudaMemcpy(invalid, R->P.stats + SS_INVALID, 8, cudaMemcpyDeviceToHost));
  return GPA_OK;
}

gpa_status gpa_get_reaching(gpa_ctx* ctx, gpa_pid pid, uint32_t* rin, uint32_t* rout, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  if (rin) CK(cudaMemcpy(rin, R->P.rin, (size_t)R->P.nb * kWords * 4, cudaMemcpyDeviceToHost));
  if (rout) CK(cudaMemcpy(rout, R->P.rout, (size_t)R->P.nb * kWords * 4, cudaMemcpyDeviceToHost));
  return GPA_OK;
}

gpa_status gpa_get_blame(gpa_ctx* ctx, gpa_pid pid, uint64_t* blame, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!blame) return GPA_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  CK(cudaMemcpy(blame, R->P.blame, (size_t)R->P.ni * kCnt * 8, cudaMemcpyDeviceToHost));
  return GPA_OK;
}

gpa_status gpa_get_edges(gpa_ctx* ctx, gpa_pid pid, int64_t* n_edges, int64_t cap, int32_t* use, int32_t* def,
                         int32_t* dmin, int32_t* dlong, uint32_t* flags, uint64_t* share, gpa_stream stream) {
  ProgramRec* R = find(ctx, pid);
  if (!R) return GPA_ERR_NO_PROGRAM;
  if (!n_edges) return GPA_ERR_INVALID_ARG;
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  int32_t total = 0;
  CK(cudaMemcpy(&total, R->P.edge_off + R->P.ni, 4, cudaMemcpyDeviceToHost));
  if (total > R->P.edge_cap) total = (int32_t)R->P.edge_cap;
  *n_edges = total;
  const size_t m = (size_t)std::min<int64_t>(total, cap < 0 ? 0 : cap);
  if (m) {
    if (use) CK(cudaMemcpy(use, R->P.e_use, m * 4, cudaMemcpyDeviceToHost));
    if (def) CK(cudaMemcpy(def, R->P.e_def, m * 4, cudaMemcpyDeviceToHost));
    if (dmin) CK(cudaMemcpy(dmin, R->P.e_dmin, m * 4, cudaMemcpyDeviceToHost));
    if (dlong) CK(cudaMemcpy(dlong, R->P.e_dlong, m * 4, cudaMemcpyDeviceToHost));
    if (flags) CK(cudaMemcpy(flags, R->P.e_flags, m * 4, cudaMemcpyDeviceToHost));
    if (share) CK(cudaMemcpy(share, R->P.e_share, m * 8 * 8, cudaMemcpyDeviceToHost));
  }
  return GPA_OK;
}

int64_t gpa_launch_count(gpa_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"
