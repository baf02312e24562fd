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
// words per block, starting at DEF), and per block a record of its first two
// predecessors other than the block before it, its innermost loop, and flags
// (the block before it is a predecessor; more predecessors in the CSR). ROUT
// only grows, so ROUT[b] = ROUT[b] | OR of the predecessors' ROUT needs no
// separate DEF. A sweep visits the blocks one after another in layout order (a
// topological order of the forward edges, so one sweep carries a def along any
// forward path), lanes 0-8 over the 9 words, with the previous block's ROUT in
// a register and the next block's record and ROUT loaded a block ahead.
// When every loop body of the function is a natural loop (or it has none),
// each block also takes in, from the start, the defs of the bodies of the loops
// around it: every block of a natural loop reaches every other one through the
// back edge, and a def from outside a loop enters it through its header, which
// precedes the body in layout order. With that, the first sweep gives every
// block all the defs that reach it: the least fixpoint, in one sweep. Other
// functions sweep until a sweep changes nothing (max_sweeps at most). Then RIN
// = OR of the predecessors' ROUT and both go to global memory. The launch
// takes reach_order[q_lo, q_hi) from the counter at `head`; functions needing
// more than `cap` bytes are left to another launch.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__global__ void __launch_bounds__(32) k_reaching_smem(Prog P, int max_sweeps, int q_lo, int q_hi, int head, int cap) {
  extern __shared__ __align__(16) uint32_t sm[];
  const int lane = threadIdx.x;
  while (true) {
    // Functions are taken largest first, so the long ones start early.
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(&P.stats[head], 1ull);
    q = __shfl_sync(0xffffffffu, q, 0) + (unsigned long long)q_lo;
    if (q >= (unsigned long long)q_hi) break;
    const int f = P.reach_order[q];
    const int b0 = P.func_block_off[f], b1 = P.func_block_off[f + 1], nbf = b1 - b0;
    const int e0 = P.pred_off[b0], ne = P.pred_off[b1] - e0;
    const int l0 = P.func_loop_off[f], nlf = P.func_loop_off[f + 1] - l0;
    if (nbf == 0 || reach_smem_need(nbf, ne, nlf) > cap) continue;
    const bool exact = P.func_natural[f];  // one seeded sweep is the fixpoint
    const bool seed = exact && nlf > 0;
    uint32_t* so = sm;
    int4* rec = reinterpret_cast<int4*>(so + (size_t)nbf * kWords + ((nbf * kWords) & 3 ? 4 - ((nbf * kWords) & 3) : 0));
    int* spo = reinterpret_cast<int*>(rec + nbf);
    int* sp = spo + nbf + 1;
    int* sloop = sp + ne;
    int* spar = sloop + nbf;
    uint32_t* ldef = reinterpret_cast<uint32_t*>(spar + nlf);
    uint32_t* lin = ldef + (size_t)nlf * kWords;
    // Staging: asynchronous 4-byte copies, all in flight together, then the
    // global indices rebased to the function in place.
    for (int t = lane; t < nbf * kWords; t += 32) cp_async4(so + t, P.def_mask + (size_t)b0 * kWords + t);
    for (int t = lane; t <= nbf; t += 32) cp_async4(spo + t, P.pred_off + b0 + t);
    for (int t = lane; t < ne; t += 32) cp_async4(sp + t, P.pred + e0 + t);
    if (seed) {
      for (int t = lane; t < nbf; t += 32) cp_async4(sloop + t, P.block_loop + b0 + t);
      for (int t = lane; t < nlf; t += 32) cp_async4(spar + t, P.loop_parent + l0 + t);
    }
    cp_async_wait_all();
    __syncwarp();
    for (int t = lane; t <= nbf; t += 32) spo[t] -= e0;
    for (int t = lane; t < ne; t += 32) sp[t] -= b0;
    if (seed) {
      for (int t = lane; t < nbf; t += 32) sloop[t] = sloop[t] >= 0 ? sloop[t] - l0 : -1;
      for (int t = lane; t < nlf; t += 32) spar[t] = spar[t] >= 0 ? spar[t] - l0 : -1;
      for (int t = lane; t < nlf * kWords; t += 32) ldef[t] = 0u;
    }
    __syncwarp();
    for (int b = lane; b < nbf; b += 32) {
      int p1 = -1, p2 = -1, fl = 0;
      for (int e = spo[b]; e < spo[b + 1]; ++e) {
        const int p = sp[e];
        if (p == b - 1) fl |= 1;
        else if (p1 < 0) p1 = p;
        else if (p2 < 0) p2 = p;
        else fl |= 2;
      }
      rec[b] = make_int4(p1, p2, seed ? sloop[b] : -1, fl);
    }
    if (seed) {
      // the defs of each loop's body, nested loops included
      for (int t = lane; t < nbf * kWords; t += 32) {
        const uint32_t v = so[t];
        if (!v) continue;
        const int w = t % kWords;
        for (int l = sloop[t / kWords]; l >= 0; l = spar[l]) atomicOr(&ldef[l * kWords + w], v);
      }
      __syncwarp();
      // and of the enclosing loops' bodies
      for (int t = lane; t < nlf * kWords; t += 32) {
        const int w = t % kWords;
        uint32_t v = 0u;
        for (int l = t / kWords; l >= 0; l = spar[l]) v |= ldef[l * kWords + w];
        lin[t] = v;
      }
    }
    __syncwarp();
    bool converged = false;
    int sweep = 0;
    const int limit = exact ? 1 : max_sweeps;
    for (; sweep < limit && !converged; ++sweep) {
      bool ch = false;
      if (lane < kWords) {
        uint32_t prev = 0u;
        int4 r = rec[0];
        uint32_t old = so[lane];
        for (int b = 0; b < nbf; ++b) {
          const bool more = b + 1 < nbf;
          const int4 rn = more ? rec[b + 1] : r;
          const uint32_t oldn = more ? so[(b + 1) * kWords + lane] : 0u;
          uint32_t in = r.z >= 0 ? lin[r.z * kWords + lane] : 0u;
          if (r.w & 1) in |= prev;
          if (r.x >= 0) in |= so[r.x * kWords + lane];
          if (r.y >= 0) in |= so[r.y * kWords + lane];
          if (r.w & 2)
            for (int e = spo[b]; e < spo[b + 1]; ++e) in |= so[sp[e] * kWords + lane];
          const uint32_t o = old | in;
          ch |= o != old;
          so[b * kWords + lane] = o;
          prev = o;
          r = rn;
          old = oldn;
        }
      }
      converged = exact || !__any_sync(0xffffffffu, ch);
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
// fixpoint regardless of the visiting order. Takes the functions the staged
// kernel does not (every function with `all`).
__global__ void k_reaching(Prog P, int max_sweeps, int all) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  for (int f = warp; f < P.nf; f += n_warps) {
    const int b0 = P.func_block_off[f], b1 = P.func_block_off[f + 1];
    if (!all && b1 > b0 &&
        reach_smem_need(b1 - b0, P.pred_off[b1] - P.pred_off[b0], P.func_loop_off[f + 1] - P.func_loop_off[f]) <=
            P.reach_smem)
      continue;
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

void launch_dataflow(const Prog& P, const Arch& A, int max_sweeps, int schedule, cudaStream_t st, int sms,
                     int64_t* launches) {
  const int threads = 256;
  int64_t warps_needed = P.nb;
  int blocks = (int)((warps_needed * 32 + threads - 1) / threads);
  if (blocks > sms * 16) blocks = sms * 16;
  if (blocks < 1) blocks = 1;
  k_block_masks<<<blocks, threads, 0, st>>>(P);
  if (schedule == 0 && P.reach_smem > 0) {
    // One launch per size class: the larger the functions, the more shared
    // memory each warp stages and the fewer warps per SM.
    allow_max_smem(k_reaching_smem);
    cudaMemsetAsync(&P.stats[SS_REACH_CLS], 0, 4 * sizeof(unsigned long long), st);
    for (int c = 0; c < 4; ++c) {
      const int n = P.reach_cls[c + 1] - P.reach_cls[c];
      if (n <= 0 || P.reach_cls_smem[c] <= 0) continue;
      const int smem = P.reach_cls_smem[c];
      const int per_sm = std::max(1, std::min(32, (int)((200 * 1024) / (smem + 1024))));
      const int g = std::min(n, sms * per_sm);
      k_reaching_smem<<<g, 32, smem, st>>>(P, max_sweeps, P.reach_cls[c], P.reach_cls[c + 1], SS_REACH_CLS + c, smem);
      ++*launches;
    }
  }
  int fblocks = (P.nf * 32 + 127) / 128;
  if (fblocks > sms * 16) fblocks = sms * 16;
  if (fblocks < 1) fblocks = 1;
  k_reaching<<<fblocks, 128, 0, st>>>(P, max_sweeps, schedule == 1 ? 1 : 0);
  cudaMemsetAsync(P.res_maxlat, 0, sizeof(int32_t) * (size_t)P.nf * kNumRes, st);
  cudaMemsetAsync(P.res_guards, 0, sizeof(uint32_t) * (size_t)P.nf * kNumRes, st);
  k_res_maxlat<<<grid_for(P.ni, 256, sms), 256, 0, st>>>(P, A);
  *launches += 3;
}

}  // namespace gpa
