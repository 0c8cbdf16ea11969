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
