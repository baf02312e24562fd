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

// Thread per basic block (blocks average 7 instructions, so a warp per block
// left most lanes idle): the masks stay in registers, each resource's bit
// added to its word by a compare per word (no indexed register array), then
// the 9 words of each mask stored.
__global__ void k_block_masks(Prog P) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.nb; b += gridDim.x * blockDim.x) {
    uint32_t dm[kWords], um[kWords];
#pragma unroll
    for (int w = 0; w < kWords; ++w) { dm[w] = 0; um[w] = 0; }
    const int x1 = P.block_instr_off[b + 1];
    for (int x = P.block_instr_off[b]; x < x1; ++x) {
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
    const size_t o = (size_t)b * kWords;
#pragma unroll
    for (int w = 0; w < kWords; ++w) {
      P.def_mask[o + w] = dm[w];
      P.uuse_mask[o + w] = um[w];
      P.touch_mask[o + w] = dm[w] | um[w];
      P.rin[o + w] = 0u;
      P.rout[o + w] = dm[w];
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

// One CTA per function, the function staged in shared memory: ROUT (9 words
// per block, starting at DEF), and per block a record of its first two
// predecessors other than the block before it, its innermost loop, and flags
// (the block before it is a predecessor; more predecessors in the CSR). ROUT
// only grows, so ROUT[b] = ROUT[b] | OR of the predecessors' ROUT needs no
// separate DEF. A sweep visits the blocks one after another in layout order (a
// topological order of the forward edges, so one sweep carries a def along any
// forward path), lanes 0-8 of the first warp over the 9 words, with the
// previous block's ROUT in a register. A block's other predecessors are never
// the block just before it, so their words for the next block are loaded
// before this block's ROUT is stored: the sweep's chain per block is an OR and
// a store. The rest (staging, records, loop masks, RIN and the copy-out) is
// spread over the CTA's threads.
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

__global__ void __launch_bounds__(256) k_reaching_smem(Prog P, int max_sweeps, int q_lo, int q_hi, int head, int cap) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ int s_f;
  const int tid = threadIdx.x, nt = blockDim.x;
  while (true) {
    // Functions are taken largest first, so the long ones start early.
    __syncthreads();  // every thread has read s_f and left the previous function's stage
    if (tid == 0) {
      const unsigned long long q = atomicAdd(&P.stats[head], 1ull) + (unsigned long long)q_lo;
      s_f = q < (unsigned long long)q_hi ? P.reach_order[q] : -1;
    }
    __syncthreads();
    const int f = s_f;
    if (f < 0) break;
    const int b0 = P.func_block_off[f], b1 = P.func_block_off[f + 1], nbf = b1 - b0;
    const int e0 = P.pred_off[b0], ne = P.pred_off[b1] - e0;
    const int l0 = P.func_loop_off[f], nlf = P.func_loop_off[f + 1] - l0;
    if (nbf == 0 || reach_smem_need(nbf, ne, nlf) > cap) continue;  // the same for every thread
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
    for (int t = tid; t < nbf * kWords; t += nt) cp_async4(so + t, P.def_mask + (size_t)b0 * kWords + t);
    for (int t = tid; t <= nbf; t += nt) cp_async4(spo + t, P.pred_off + b0 + t);
    for (int t = tid; t < ne; t += nt) cp_async4(sp + t, P.pred + e0 + t);
    if (seed) {
      for (int t = tid; t < nbf; t += nt) cp_async4(sloop + t, P.block_loop + b0 + t);
      for (int t = tid; t < nlf; t += nt) cp_async4(spar + t, P.loop_parent + l0 + t);
    }
    cp_async_wait_all();
    __syncthreads();
    for (int t = tid; t <= nbf; t += nt) spo[t] -= e0;
    for (int t = tid; t < ne; t += nt) sp[t] -= b0;
    if (seed) {
      for (int t = tid; t < nbf; t += nt) sloop[t] = sloop[t] >= 0 ? sloop[t] - l0 : -1;
      for (int t = tid; t < nlf; t += nt) spar[t] = spar[t] >= 0 ? spar[t] - l0 : -1;
      for (int t = tid; t < nlf * kWords; t += nt) ldef[t] = 0u;
    }
    __syncthreads();
    for (int b = tid; b < nbf; b += nt) {
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
      for (int t = tid; t < nbf * kWords; t += nt) {
        const uint32_t v = so[t];
        if (!v) continue;
        const int w = t % kWords;
        for (int l = sloop[t / kWords]; l >= 0; l = spar[l]) atomicOr(&ldef[l * kWords + w], v);
      }
      __syncthreads();
      // and of the enclosing loops' bodies
      for (int t = tid; t < nlf * kWords; t += nt) {
        const int w = t % kWords;
        uint32_t v = 0u;
        for (int l = t / kWords; l >= 0; l = spar[l]) v |= ldef[l * kWords + w];
        lin[t] = v;
      }
    }
    __syncthreads();
    if (tid < 32) {
      const int lane = tid;
      bool converged = false;
      int sweep = 0;
      const int limit = exact ? 1 : max_sweeps;
      for (; sweep < limit && !converged; ++sweep) {
        bool ch = false;
        if (lane < kWords) {
          // words from the record's two predecessors and the enclosing loops
          auto pre = [&](const int4& r) -> uint32_t {
            return (r.z >= 0 ? lin[r.z * kWords + lane] : 0u) | (r.x >= 0 ? so[r.x * kWords + lane] : 0u) |
                   (r.y >= 0 ? so[r.y * kWords + lane] : 0u);
          };
          uint32_t prev = 0u;
          int4 r = rec[0];
          uint32_t old = so[lane];
          uint32_t in_r = pre(r);
          for (int b = 0; b < nbf; ++b) {
            const bool more = b + 1 < nbf;
            const int4 rn = more ? rec[b + 1] : r;
            const uint32_t oldn = more ? so[(b + 1) * kWords + lane] : 0u;
            const uint32_t in_n = more ? pre(rn) : 0u;  // rn.x, rn.y != b: not written below
            uint32_t in = in_r;
            if (r.w & 1) in |= prev;
            if (r.w & 2)
              for (int e = spo[b]; e < spo[b + 1]; ++e) in |= so[sp[e] * kWords + lane];
            const uint32_t o = old | in;
            ch |= o != old;
            so[b * kWords + lane] = o;
            prev = o;
            r = rn;
            old = oldn;
            in_r = in_n;
          }
        }
        converged = exact || !__any_sync(0xffffffffu, ch);
      }
      if (lane == 0) {
        if (!converged) set_status(P, ST_NOT_CONVERGED);
        atomicMax(&P.stats[SS_SWEEPS], (unsigned long long)sweep);
      }
    }
    __syncthreads();
    for (int t = tid; t < nbf * kWords; t += nt) {
      const int b = t / kWords, w = t - b * kWords;
      uint32_t in = 0u;
      for (int e = spo[b]; e < spo[b + 1]; ++e) in |= so[sp[e] * kWords + w];
      P.rin[(size_t)b0 * kWords + t] = in;
      P.rout[(size_t)b0 * kWords + t] = so[t];
    }
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
  k_block_masks<<<grid_for(P.nb, 256, sms), 256, 0, st>>>(P);
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
      // the larger the functions, the more threads share a function's
      // staging, records and copy-out (its sweep is one warp's in any case)
      const int threads = c == 0 ? 256 : c == 1 ? 128 : c == 2 ? 64 : 32;
      k_reaching_smem<<<g, threads, smem, st>>>(P, max_sweeps, P.reach_cls[c], P.reach_cls[c + 1], SS_REACH_CLS + c,
                                               smem);
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
