// Step (b), first half: per-block resource summaries and the reaching-
// definitions fixpoint at resource granularity (Sec. 4, backward slicing over
// registers, predicates and virtual barrier registers).
//
// The classic def-site reaching definitions projected on resources reduces to
// reachability of definitions: some def of r reaches the exit of b iff b
// defines r or some def of r reaches its entry (an unpredicated def kills the
// earlier defs of r but itself reaches on), and reaches the entry iff it
// reaches the exit of a predecessor. So
//   RIN[b] = OR over preds p of ROUT[p],   ROUT[b] = DEF[b] | RIN[b],
// 268-bit masks in 9 words. The backward searches use ROUT to skip blocks no
// def of the searched resource can leave.
#include <algorithm>

#include "gpa_internal.cuh"

namespace gpa {

namespace {

// Warp per basic block: lanes over its instructions, one reduce-or per word.
__global__ void k_block_masks(Prog P) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  for (int b = warp; b < P.nb; b += n_warps) {
    uint32_t dm[kWords], um[kWords];
#pragma unroll
    for (int w = 0; w < kWords; ++w) { dm[w] = 0; um[w] = 0; }
    const int x1 = P.block_instr_off[b + 1];
    for (int x = P.block_instr_off[b] + lane; x < x1; x += 32) {
      for (int e = P.def_off[x]; e < P.def_off[x + 1]; ++e) {
        const int r = P.def_res[e] & 0x1FF;
#pragma unroll
        for (int w = 0; w < kWords; ++w) dm[w] |= ((r >> 5) == w) ? (1u << (r & 31)) : 0u;
      }
      if (P.guard[x] == 0) {
        for (int e = P.use_off[x]; e < P.use_off[x + 1]; ++e) {
          const int r = P.use_res[e] & 0x1FF;
#pragma unroll
          for (int w = 0; w < kWords; ++w) um[w] |= ((r >> 5) == w) ? (1u << (r & 31)) : 0u;
        }
      }
    }
#pragma unroll
    for (int w = 0; w < kWords; ++w) {
      const uint32_t d = __reduce_or_sync(0xffffffffu, dm[w]);
      const uint32_t u = __reduce_or_sync(0xffffffffu, um[w]);
      if (lane == w) {
        P.def_mask[(size_t)b * kWords + w] = d;
        P.uuse_mask[(size_t)b * kWords + w] = u;
        P.touch_mask[(size_t)b * kWords + w] = d | u;
        P.rin[(size_t)b * kWords + w] = 0u;
        P.rout[(size_t)b * kWords + w] = d;
      }
    }
  }
}

// Largest latency of any def of each resource in each function (the
// distance beyond which no def of that resource can pass the latency rule),
// and the guard literals its defs carry there.
__global__ void k_res_maxlat(Prog P, Arch A) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < P.ni; x += gridDim.x * blockDim.x) {
    const int f = P.block_func[P.instr_block[x]];
    const int lat = A.lat[P.opclass[x]];
    const int g = P.guard[x];
    for (int e = P.def_off[x]; e < P.def_off[x + 1]; ++e) {
      const size_t k = (size_t)f * kNumRes + (P.def_res[e] & 0x1FF);
      atomicMax(&P.res_maxlat[k], lat);
      if (g) atomicOr(&P.res_guards[k], 1u << (g - 1));
    }
  }
}

// One warp per function, the function staged in shared memory: ROUT (9
// words per block, starting at DEF) and the predecessor lists as local block
// indices. ROUT only grows, so ROUT[b] = ROUT[b] | OR of the predecessors'
// ROUT needs no separate DEF. Each sweep visits the blocks one after another
// in layout order (a topological order of the forward edges, so one sweep
// carries a def along any forward path), lanes 0-8 over the 9 words, with the
// previous block's ROUT kept in a register (the fall-through predecessor);
// sweeps repeat until one changes nothing (back edges). Then RIN = OR of the
// predecessors' ROUT and both go to global memory. Functions needing more
// than P.reach_smem bytes are left to k_reaching.
__global__ void __launch_bounds__(32) k_reaching_smem(Prog P, int max_sweeps) {
  extern __shared__ uint32_t sm[];
  const int lane = threadIdx.x;
  while (true) {
    // Functions are taken largest first, so the long ones start early.
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(&P.stats[SS_REACH_HEAD], 1ull);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= (unsigned long long)P.nf) break;
    const int f = P.reach_order[q];
    const int b0 = P.func_block_off[f], b1 = P.func_block_off[f + 1], nbf = b1 - b0;
    const int e0 = P.pred_off[b0], ne = P.pred_off[b1] - e0;
    if (nbf == 0 || reach_smem_need(nbf, ne) > P.reach_smem) continue;
    uint32_t* so = sm;
    int* spo = reinterpret_cast<int*>(so + (size_t)nbf * kWords);
    int* sp = spo + nbf + 1;
    for (int t = lane; t < nbf * kWords; t += 32) so[t] = P.def_mask[(size_t)b0 * kWords + t];
    for (int t = lane; t <= nbf; t += 32) spo[t] = P.pred_off[b0 + t] - e0;
    for (int t = lane; t < ne; t += 32) sp[t] = P.pred[e0 + t] - b0;
    __syncwarp();
    bool converged = false;
    int sweep = 0;
    for (; sweep < max_sweeps && !converged; ++sweep) {
      bool ch = false;
      if (lane < kWords) {
        uint32_t prev = 0u;
        int e_lo = spo[0];
        for (int b = 0; b < nbf; ++b) {
          const int e_hi = spo[b + 1];
          const uint32_t old = so[b * kWords + lane];
          uint32_t in = 0u;
          for (int e = e_lo; e < e_hi; ++e) {
            const int p = sp[e];
            in |= p == b - 1 ? prev : so[p * kWords + lane];
          }
          const uint32_t o = old | in;
          ch |= o != old;
          so[b * kWords + lane] = o;
          prev = o;
          e_lo = e_hi;
        }
      }
      converged = !__any_sync(0xffffffffu, ch);
    }
    __syncwarp();
    for (int t = lane; t < nbf * kWords; t += 32) {
      const int b = t / kWords, w = t - b * kWords;
      uint32_t in = 0u;
      for (int e = spo[b]; e < spo[b + 1]; ++e) in |= so[sp[e] * kWords + w];
      P.rin[(size_t)b0 * kWords + t] = in;
      P.rout[(size_t)b0 * kWords + t] = so[t];
    }
    if (lane == 0) {
      if (!converged) set_status(P, ST_NOT_CONVERGED);
      atomicMax(&P.stats[SS_SWEEPS], (unsigned long long)sweep);
    }
    __syncwarp();
  }
}

// Warp per function. Blocks are visited in layout order (a topological order
// of the forward edges) 32 at a time, lane per block; inside a window the
// lanes iterate until __ballot_sync reports no change, then move on. A full
// pass without change ends the fixpoint; max_sweeps passes without reaching it
// set ST_NOT_CONVERGED. Monotone OR updates from 0 make the result the least
// fixpoint regardless of the visiting order.
__global__ void k_reaching(Prog P, int max_sweeps) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  for (int f = warp; f < P.nf; f += n_warps) {
    const int b0 = P.func_block_off[f], b1 = P.func_block_off[f + 1];
    if (b1 > b0 && reach_smem_need(b1 - b0, P.pred_off[b1] - P.pred_off[b0]) <= P.reach_smem) continue;
    bool converged = false;
    int sweep = 0;
    for (; sweep < max_sweeps && !converged; ++sweep) {
      bool changed_any = false;
      for (int w0 = b0; w0 < b1; w0 += 32) {
        const int b = w0 + lane;
        const bool mine = b < b1;
        for (int it = 0; it < 64; ++it) {
          bool ch = false;
          if (mine) {
            uint32_t in[kWords];
#pragma unroll
            for (int w = 0; w < kWords; ++w) in[w] = 0u;
            for (int e = P.pred_off[b]; e < P.pred_off[b + 1]; ++e) {
              const volatile uint32_t* ro = P.rout + (size_t)P.pred[e] * kWords;
#pragma unroll
              for (int w = 0; w < kWords; ++w) in[w] |= ro[w];
            }
            volatile uint32_t* ri = P.rin + (size_t)b * kWords;
            volatile uint32_t* ro = P.rout + (size_t)b * kWords;
            const uint32_t* dm = P.def_mask + (size_t)b * kWords;
#pragma unroll
            for (int w = 0; w < kWords; ++w) {
              const uint32_t o = dm[w] | in[w];
              if (in[w] != ri[w] || o != ro[w]) ch = true;
              ri[w] = in[w];
              ro[w] = o;
            }
          }
          __syncwarp();
          if (!__ballot_sync(0xffffffffu, ch)) break;
          changed_any = true;
        }
      }
      converged = !changed_any;
    }
    if (lane == 0) {
      if (!converged) set_status(P, ST_NOT_CONVERGED);
      atomicMax(&P.stats[SS_SWEEPS], (unsigned long long)sweep);
    }
  }
}

}  // namespace

void launch_dataflow(const Prog& P, const Arch& A, int max_sweeps, cudaStream_t st, int sms, int64_t* launches) {
  const int threads = 256;
  int64_t warps_needed = P.nb;
  int blocks = (int)((warps_needed * 32 + threads - 1) / threads);
  if (blocks > sms * 16) blocks = sms * 16;
  if (blocks < 1) blocks = 1;
  k_block_masks<<<blocks, threads, 0, st>>>(P);
  if (P.reach_smem > 0) {
    allow_max_smem(k_reaching_smem);
    int per_sm = (int)((200 * 1024) / (P.reach_smem + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 16) per_sm = 16;
    const int g = std::min(P.nf, sms * per_sm);
    k_reaching_smem<<<g, 32, P.reach_smem, st>>>(P, max_sweeps);
    ++*launches;
  }
  int fblocks = (P.nf * 32 + 127) / 128;
  if (fblocks > sms * 16) fblocks = sms * 16;
  if (fblocks < 1) fblocks = 1;
  k_reaching<<<fblocks, 128, 0, st>>>(P, max_sweeps);
  cudaMemsetAsync(P.res_maxlat, 0, sizeof(int32_t) * (size_t)P.nf * kNumRes, st);
  cudaMemsetAsync(P.res_guards, 0, sizeof(uint32_t) * (size_t)P.nf * kNumRes, st);
  k_res_maxlat<<<grid_for(P.ni, 256, sms), 256, 0, st>>>(P, A);
  *launches += 3;
}

}  // namespace gpa
