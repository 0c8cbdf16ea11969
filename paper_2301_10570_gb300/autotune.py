"""Plan chooser: leaf capacity, cutoff and expansion order for one workload.

A plan is (leaf_capacity, cutoff, rho_max, p, m2l_min_pairs).  For each
candidate the tuner times whole plasticity steps (tree, attraction,
selection) on the GPU and measures the attraction error against the
all-pairs evaluation of the same GPU (msp_direct).  That reference is
single precision with compensated (Kahan) sums of its tiles; its own error
against double precision brute force is below 1e-6 (5.2e-7 measured at
1,048,576 clustered neurons on 4,096 sampled targets), so a plan is accepted
when its deviation from it stays below tol - ref_err, which keeps the plan
within tol of the exact attraction.  The fastest accepted plan wins.

    from paper_2301_10570_gb300 import autotune, workloads
    best, table = autotune.tune(workloads.clustered_1m())
"""
from __future__ import annotations

import itertools
import statistics
import time

DEFAULT_CANDIDATES = dict(
    leaf_capacity=(64, 128, 192, 256),
    cutoff=(3.0, 3.25, 3.5, 4.0),
    expansions=((0.0, 4, 0), (0.25, 6, 256), (0.3, 6, 1024)),   # (rho_max, p, m2l_min_pairs)
)


def _step_ms(g, dev, reps):
    import torch
    ts = []
    for k in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.build_tree(*dev)
        u = g.attraction()
        g.select_partners(k)
        torch.cuda.synchronize()
        ts.append(1e3 * (time.perf_counter() - t0))
    return statistics.median(ts[1:]) if len(ts) > 1 else ts[0], u


def tune(workload, tol=1e-4, ref_err=1e-6, candidates=None, reps=4, device=0, verbose=False):
    """Return (best plan dict, list of per-candidate results); the plan is
    None when no candidate meets the accuracy target."""
    import torch

    from . import msp
    cand = dict(DEFAULT_CANDIDATES)
    if candidates:
        cand.update(candidates)
    dev = msp.to_device(workload, f"cuda:{device}")
    ref_ctx = msp.MSP(workload.params, device=device)
    ref_ctx.build_tree(*dev)
    ref = ref_ctx.direct()
    torch.cuda.synchronize()
    mask = ref > 1e-6 * ref.max()
    ref_ctx.close()
    results = []
    for C, cut, (rho, p, mp) in itertools.product(cand["leaf_capacity"], cand["cutoff"],
                                                  cand["expansions"]):
        plan = dict(leaf_capacity=C, cutoff=cut, rho_max=rho, p=p, m2l_min_pairs=mp)
        params = dict(workload.params, **plan)
        try:
            g = msp.MSP(params, device=device)
            ms, u = _step_ms(g, dev, reps)
            err = ((u[mask] - ref[mask]).abs() / ref[mask]).max().item()
            st = g.stats()
            g.close()
        except msp.MSPError as e:     # e.g. a plan too large for memory
            results.append(dict(plan=plan, error=str(e)))
            continue
        ok = err <= tol - ref_err
        results.append(dict(plan=plan, step_ms=ms, max_rel_dev=err, accepted=ok,
                            near_field_ms=st["near_field_ms"], far_pairs=st["n_far"],
                            near_pairs=st["n_p2p"], interactions=st["p2p_interactions"]))
        if verbose:
            print(results[-1], flush=True)
    accepted = [r for r in results if r.get("accepted")]
    if not accepted:
        return None, results
    best = min(accepted, key=lambda r: r["step_ms"])
    return best["plan"], results


BATCH_CUTOFFS = (3.25, 3.5, 4.0, 4.5, 5.0)


def tune_batch_cutoffs(workload, tol=1e-4, ref_err=3e-5, cutoffs=BATCH_CUTOFFS, device=0,
                       verbose=False):
    """Per-network cutoffs for a batch of networks in their own frames (a
    workload from Batch.framed with a shared plan; its layout must leave every
    cell wider than the largest candidate).  Every network starts at the
    smallest candidate; a network whose attraction deviates from its own
    all-pairs evaluation (msp_direct of the batch: each target against its own
    network's sources) by more than tol - ref_err moves to the next candidate,
    and the batch is evaluated again, until every network passes or has the
    largest candidate.  ref_err covers the all-pairs path's own deviation
    from the exact sum of the unscaled network (its positions are rounded to
    single precision in sigma units, up to ~133 sigma from the cell's
    corner: a few 1e-5 observed).  Returns (cutoffs per network, report)."""
    import numpy as np
    import torch

    from . import msp
    offsets, level = workload.frames[0], workload.frames[1]
    K = len(offsets) - 1
    dev = msp.to_device(workload, f"cuda:{device}")
    g = msp.MSP(workload.params, device=device, frames=(offsets, level))
    try:
        g.build_tree(*dev)
        ref = g.direct().cpu().numpy().astype(np.float64)
        va = workload.vac_axon
        net = np.repeat(np.arange(K), np.diff(offsets))
        # per-network mask: vacant axons and u >= 1e-6 of the network's largest
        big = np.maximum.reduceat(ref, offsets[:-1])
        mask = (va > 0) & (ref >= 1e-6 * big[net])
        cur = np.zeros(K, np.int64)
        rounds = []
        while True:
            cuts = [float(cutoffs[i]) for i in cur]
            g.set_frames(offsets, level, None, cuts)
            g.build_tree(*dev)
            u = g.attraction().cpu().numpy().astype(np.float64)
            torch.cuda.synchronize()
            rel = np.where(mask, np.abs(u - ref) / np.maximum(ref, 1e-300), 0.0)
            err = np.maximum.reduceat(rel, offsets[:-1])
            fail = (err > tol - ref_err) & (cur < len(cutoffs) - 1)
            rounds.append(dict(max_err=float(err.max()), failing=int((err > tol - ref_err).sum()),
                               interactions=g.stats()["p2p_interactions"]))
            if verbose:
                print(rounds[-1], flush=True)
            if not fail.any():
                break
            cur[fail] += 1
    finally:
        g.close()
    return cuts, dict(rounds=rounds, per_network_max_err=err.tolist(),
                      raised=int((cur > 0).sum()))
