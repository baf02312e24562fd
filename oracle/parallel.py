"""Parallel optimizers of GPA (Table 2 "Parallel Optimizers") and their
estimator (Sec. 5.2 "Parallel Optimization Estimator", Eqs. 6-10) — TEST
INFRASTRUCTURE ONLY (part of the oracle; the product never imports it).

Plain Python, one function (kernel launch) at a time, in the paper's notation.
The paper leaves three things open; the readings used here:
  * f of Eq. 10 is 1.
  * W (Eqs. 8-9) is the active warps per warp scheduler: the blocks resident
    on an SM times the warps per block, over the SM's schedulers. Blocks per SM
    follow the public occupancy-calculator rules (warp slots, registers
    allocated per warp on one scheduler's share of the register file, shared
    memory with a per-block reserve and an allocation unit, the block-count
    cap), and an SM holds no more of the kernel's blocks than the grid gives it.
  * C_W (Eq. 6) compares the warps a scheduler executes over the run. Block
    Increase spreads the same threads over one block per SM: every SM runs one
    wave, so these are its resident warps, W_new = W * blocks / SMs. Thread
    Increase merges the same threads into larger blocks on the same SMs until
    the warp, register or shared-memory limit (shared memory counted per warp)
    or the grid binds: the warps a scheduler executes over the run are
    unchanged, C_W = 1, and only the issue probability moves (C_I).
Match rules (Table 2): Block Increase when the grid has fewer blocks than the
GPU has SMs; Thread Increase when the block-count cap is the binding occupancy
limit (strictly below the others) and the grid gives an SM at least that many
blocks. Unmatched optimizers, or a launch without issued samples or without a
resident block, keep speedup 1.0.
"""
from __future__ import annotations

import math

import numpy as np

# order of the occupancy limits (ties report the lowest)
LIMIT_WARPS, LIMIT_REGISTERS, LIMIT_SHARED, LIMIT_BLOCKS = 0, 1, 2, 3


def _ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def occupancy(threads: int, regs: int, smem: int, sm: dict) -> dict:
    """Blocks per SM of one launch configuration and which limit binds."""
    warps_per_block = _ceil_div(threads, 32)
    limits = {}
    limits[LIMIT_WARPS] = sm["max_warps_per_sm"] // warps_per_block
    if regs > 0:
        regs_per_warp = _ceil_div(regs * 32, sm["reg_alloc_unit"]) * sm["reg_alloc_unit"]
        per_scheduler = sm["regs_per_sm"] // sm["schedulers_per_sm"]
        warps_by_regs = sm["schedulers_per_sm"] * (per_scheduler // regs_per_warp)
        limits[LIMIT_REGISTERS] = warps_by_regs // warps_per_block
    else:
        warps_by_regs = sm["max_warps_per_sm"]
        limits[LIMIT_REGISTERS] = None
    if smem > 0:
        per_block = _ceil_div(smem + sm["smem_reserved_per_block"], sm["smem_alloc_unit"]) * sm["smem_alloc_unit"]
        limits[LIMIT_SHARED] = sm["smem_per_sm"] // per_block
        warps_by_smem = limits[LIMIT_SHARED] * warps_per_block
    else:
        warps_by_smem = None
        limits[LIMIT_SHARED] = None
    limits[LIMIT_BLOCKS] = sm["max_blocks_per_sm"]
    present = [(v, k) for k, v in limits.items() if v is not None]
    blocks_per_sm, limit = min(present)      # the least limit; equal values: the lower id
    return dict(warps_per_block=warps_per_block, blocks_per_sm=blocks_per_sm, limit=limit, limits=limits,
                warps_by_regs=warps_by_regs, warps_by_smem=warps_by_smem)


def issue_probability(r_i: float, w: float) -> float:
    """Eqs. 8-9: a scheduler issues when at least one of its W warps is ready."""
    return 1.0 - math.pow(1.0 - r_i, w)


def estimate(launch: dict, sm: dict, total_samples: int, issued_samples: int) -> dict:
    """Both parallel optimizers for one function: match flags, S^p (Eq. 10),
    (W, W_new) per optimizer, the binding limit."""
    occ = occupancy(launch["threads_per_block"], launch["regs_per_thread"], launch["smem_per_block"], sm)
    wpb = occ["warps_per_block"]
    blocks = launch["blocks"]
    blocks_given = _ceil_div(blocks, sm["n_sms"])          # blocks the grid gives the busiest SM
    resident = min(occ["blocks_per_sm"], blocks_given)
    W = (resident * wpb) / sm["schedulers_per_sm"]

    match = [blocks < sm["n_sms"],
             occ["limit"] == LIMIT_BLOCKS and blocks_given >= occ["blocks_per_sm"]]

    # Block Increase: one block per SM with the same threads
    w_new_block = W * blocks / sm["n_sms"]
    # Thread Increase: larger blocks, the next limit (or the grid) binds
    candidates = [sm["max_warps_per_sm"], occ["warps_by_regs"], _ceil_div(blocks * wpb, sm["n_sms"])]
    if occ["warps_by_smem"] is not None:
        candidates.append(occ["warps_by_smem"])
    w_new_thread = min(candidates) / sm["schedulers_per_sm"]
    w_new = [w_new_block, w_new_thread]

    speedup = [1.0, 1.0]
    warps = [[0.0, 0.0], [0.0, 0.0]]
    can_estimate = occ["blocks_per_sm"] > 0 and total_samples > 0 and issued_samples > 0
    r_i = issued_samples / total_samples if total_samples else 0.0    # ratio of issued samples
    for k in range(2):
        if not match[k]:
            continue
        warps[k] = [W, w_new[k]]
        if not can_estimate:
            continue
        c_w = w_new[k] / W if k == 0 else 1.0                              # Eq. 6 (reading above)
        c_i = issue_probability(r_i, w_new[k]) / issue_probability(r_i, W)  # Eq. 7
        speedup[k] = (1.0 / c_w) * c_i * 1.0                              # Eq. 10, f = 1
    return dict(match=[int(m) for m in match], speedup=speedup, warps=warps, limit=occ["limit"])


def parallel(stats, sm: dict, totals: np.ndarray) -> dict:
    """stats: records (blocks, threads_per_block, regs_per_thread, smem_per_block)
    per function, or None; totals: [n_functions, 4] = T, A, L, issued.
    Returns par_match [nf, 2], par_speedup [nf, 2], par_warps [nf, 2, 2], par_limit [nf]."""
    nf = totals.shape[0]
    out = dict(par_match=np.zeros((nf, 2), np.int32), par_speedup=np.ones((nf, 2), np.float64),
               par_warps=np.zeros((nf, 2, 2), np.float64), par_limit=np.full(nf, -1, np.int32))
    if stats is None:
        return out
    for f in range(nf):
        launch = {k: int(stats[k][f]) for k in ("blocks", "threads_per_block", "regs_per_thread", "smem_per_block")}
        e = estimate(launch, sm, int(totals[f, 0]), int(totals[f, 3]))
        out["par_match"][f] = e["match"]
        out["par_speedup"][f] = e["speedup"]
        out["par_warps"][f] = e["warps"]
        out["par_limit"][f] = e["limit"]
    return out
