// Layout derivations done once per loaded program (predecessor lists, the
// block of each instruction, loop depths) and a device exclusive scan.
#include "gpa_internal.cuh"

namespace gpa {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-local exclusive scan of a 4096-element tile; writes the tile total.
__global__ void k_scan_tiles(int32_t* buf, int n, int32_t* sums) {
  __shared__ int32_t warp_tot[32];
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t local = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    v[t] = (base + t < n) ? buf[base + t] : 0;
    local += v[t];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int32_t w = warp_tot[lane];
    int32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_tot[lane] = wi - w;
    if (lane == 31) sums[blockIdx.x] = wi;
  }
  __syncthreads();
  int32_t run = warp_tot[warp] + incl - local;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < n) buf[base + t] = run;
    run += v[t];
  }
}

__global__ void k_scan_add(int32_t* buf, int n, const int32_t* offs) {
  const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  const int32_t o = offs[blockIdx.x];
#pragma unroll
  for (int t = 0; t < kScanItems; ++t)
    if (base + t < n) buf[base + t] += o;
}

__global__ void k_instr_block(Prog P) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x)
    for (int x = P.block_instr_off[b]; x < P.block_instr_off[b + 1]; ++x) ((int32_t*)P.instr_block)[x] = b;
}

__global__ void k_block_func(Prog P) {
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < P.nf; f += gridDim.x * blockDim.x)
    for (int b = P.func_block_off[f]; b < P.func_block_off[f + 1]; ++b) ((int32_t*)P.block_func)[b] = f;
}

__global__ void k_pred_count(Prog P, int n_succ, int32_t* pred_cnt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_succ; e += gridDim.x * blockDim.x)
    atomicAdd(&pred_cnt[P.succ[e]], 1);
}

__global__ void k_pred_fill(Prog P, int32_t* cursor) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x)
    for (int e = P.succ_off[b]; e < P.succ_off[b + 1]; ++e) {
      int s = P.succ[e];
      int at = atomicAdd(&cursor[s], 1);
      ((int32_t*)P.pred)[P.pred_off[s] + at] = b;
    }
}

// Predecessor lists in ascending block order (they are short).
__global__ void k_pred_sort(Prog P) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x) {
    int32_t* a = (int32_t*)P.pred + P.pred_off[b];
    const int n = P.pred_off[b + 1] - P.pred_off[b];
    for (int i = 1; i < n; ++i) {
      int v = a[i], k = i - 1;
      while (k >= 0 && a[k] > v) { a[k + 1] = a[k]; --k; }
      a[k + 1] = v;
    }
  }
}

__global__ void k_loop_depth(Prog P) {
  for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < P.nl; l += gridDim.x * blockDim.x) {
    int d = 0;
    for (int q = l; q >= 0 && d <= P.nl; q = P.loop_parent[q]) ++d;
    ((int32_t*)P.loop_depth)[l] = d;
  }
}

// Event lists for the backward scans, one segment per (block, resource bucket
// k = ev_bucket(r)): for each instruction of the block from the last to the
// first, its defs of the bucket's resources (with kind and guard) and, if
// unguarded, its reads of them. A scan for resource r reads only its bucket's
// segment (about 2.6 events on the batched workload, against 21.5 for the
// whole block); the events of r appear in it in the order of a bottom-up walk
// of the block (an instruction's defs before its reads). ev_off is the CSR over
// (block, bucket) pairs: segment (b, k) is [ev_off[b * 16 + k], ev_off[b * 16 + k + 1]).
__global__ void k_ev_count(Prog P, int32_t* cnt) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x) {
    int c[kEvBuckets] = {};
    for (int x = P.block_instr_off[b]; x < P.block_instr_off[b + 1]; ++x) {
      for (int e = P.def_off[x]; e < P.def_off[x + 1]; ++e) ++c[ev_bucket(P.def_res[e] & 0x1FF)];
      if (P.guard[x] == 0)
        for (int e = P.use_off[x]; e < P.use_off[x + 1]; ++e) ++c[ev_bucket(P.use_res[e] & 0x1FF)];
    }
    for (int k = 0; k < kEvBuckets; ++k) cnt[(size_t)b * kEvBuckets + k] = c[k];
  }
}

__global__ void k_ev_fill(Prog P, const int32_t* ev_off, uint32_t* events) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x) {
    const int first = P.block_instr_off[b];
    for (int k = 0; k < kEvBuckets; ++k) {
      int o = ev_off[(size_t)b * kEvBuckets + k];
      const int o_end = ev_off[(size_t)b * kEvBuckets + k + 1];
      for (int x = P.block_instr_off[b + 1] - 1; x >= first && o < o_end; --x) {
        const uint32_t pos = (uint32_t)(x - first) << 16;
        const uint32_t g = P.guard[x];
        for (int e = P.def_off[x]; e < P.def_off[x + 1]; ++e) {
          const uint32_t v = P.def_res[e];
          if (ev_bucket(v & 0x1FFu) == k) events[o++] = (v & 0x1FFu) | 0x200u | (((v >> 12) & 3u) << 10) | (g << 12) | pos;
        }
        if (g == 0)
          for (int e = P.use_off[x]; e < P.use_off[x + 1]; ++e)
            if (ev_bucket(P.use_res[e] & 0x1FFu) == k) events[o++] = (P.use_res[e] & 0x1FFu) | pos;
      }
    }
  }
}

}  // namespace

void launch_build_events(const Prog& P, int32_t* ev_off, uint32_t* events, int32_t* tmp, cudaStream_t st, int sms,
                         int64_t* launches) {
  k_ev_count<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P, ev_off);
  ++*launches;
  scan_exclusive_inplace(ev_off, P.nb * kEvBuckets, tmp, st, launches);
  k_ev_fill<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P, ev_off, events);
  ++*launches;
}

__global__ void k_block_meta(Prog P, int4* meta) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x) {
    meta[2 * (size_t)b] = make_int4(P.block_instr_off[b], P.block_instr_off[b + 1], P.ev_off[(size_t)b * kEvBuckets],
                                    P.ev_off[(size_t)(b + 1) * kEvBuckets]);
    const int q0 = P.pred_off[b], q1 = P.pred_off[b + 1];
    meta[2 * (size_t)b + 1] = make_int4(q0, q1, q1 > q0 ? P.pred[q0] : -1, q1 > q0 + 1 ? P.pred[q0 + 1] : -1);
  }
}

void launch_build_meta(const Prog& P, int4* meta, cudaStream_t st, int sms, int64_t* launches) {
  k_block_meta<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P, meta);
  ++*launches;
}

namespace {
__global__ void k_store_u64(unsigned long long* p, unsigned long long v) { *p = v; }
}  // namespace

void launch_store_u64(unsigned long long* p, unsigned long long v, cudaStream_t st, int64_t* launches) {
  k_store_u64<<<1, 1, 0, st>>>(p, v);
  ++*launches;
}

int grid_for(int64_t n, int threads, int sms) {
  int64_t g = (n + threads - 1) / threads;
  int64_t cap = (int64_t)sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

size_t scan_tmp_ints(int n) {
  size_t total = 0;
  int m = n + 1;
  while (true) {
    int tiles = (m + kScanTile - 1) / kScanTile;
    total += (size_t)tiles + 1;
    if (tiles <= 1) break;
    m = tiles;
  }
  return total + 16;
}

// buf has n + 1 entries; on return buf[k] = sum of the first k inputs and
// buf[n] = the total (the input buf[n] is ignored).
static void scan_rec(int32_t* buf, int m, int32_t* tmp, cudaStream_t st, int64_t* launches) {
  int tiles = (m + kScanTile - 1) / kScanTile;
  int32_t* sums = tmp;
  k_scan_tiles<<<tiles, kScanThreads, 0, st>>>(buf, m, sums);
  ++*launches;
  if (tiles > 1) {
    scan_rec(sums, tiles, tmp + tiles + 1, st, launches);
    k_scan_add<<<tiles, kScanThreads, 0, st>>>(buf, m, sums);
    ++*launches;
  }
}

void scan_exclusive_inplace(int32_t* buf, int n, int32_t* tmp, cudaStream_t st, int64_t* launches) {
  // Scanning n + 1 entries whose last input is 0 puts the total in buf[n].
  cudaMemsetAsync(buf + n, 0, sizeof(int32_t), st);
  scan_rec(buf, n + 1, tmp, st, launches);
}

void launch_build_layout(const Prog& P, cudaStream_t st, int sms, int64_t* launches) {
  k_instr_block<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P);
  k_loop_depth<<<grid_for(P.nl > 0 ? P.nl : 1, 256, sms), 256, 0, st>>>(P);
  k_block_func<<<grid_for(P.nf, 256, sms), 256, 0, st>>>(P);
  *launches += 3;
}

// Predecessor CSR: count, scan, fill, sort. pred_cnt has nb + 1 ints and
// ends up holding pred_off; cursor has nb ints.
void launch_build_preds(const Prog& P, int n_succ, int32_t* pred_off, int32_t* cursor, int32_t* tmp, cudaStream_t st,
                        int sms, int64_t* launches) {
  cudaMemsetAsync(pred_off, 0, sizeof(int32_t) * (P.nb + 1), st);
  cudaMemsetAsync(cursor, 0, sizeof(int32_t) * P.nb, st);
  k_pred_count<<<grid_for(n_succ > 0 ? n_succ : 1, 256, sms), 256, 0, st>>>(P, n_succ, pred_off);
  ++*launches;
  scan_exclusive_inplace(pred_off, P.nb, tmp, st, launches);
  k_pred_fill<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P, cursor);
  k_pred_sort<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P);
  *launches += 2;
}

}  // namespace gpa
