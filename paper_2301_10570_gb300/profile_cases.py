"""Small, named workloads for profiling the CUDA path under ncu.

    python -m paper_2301_10570_gb300.profile_cases near_field_131k
    python -m paper_2301_10570_gb300.profile_cases step_1m --steps 2
    python -m paper_2301_10570_gb300.profile_cases graph_1m --steps 4
    python -m paper_2301_10570_gb300.profile_cases neuron_1m --steps 2
    python -m paper_2301_10570_gb300.profile_cases translations_256k --p 4 --centre-mode 1
    python -m paper_2301_10570_gb300.profile_cases gradient_262k --steps 2

Each case builds the library, runs a few plasticity steps (tree, attraction,
selection; graph_1m: the whole step captured as one CUDA graph and replayed;
neuron_1m: calls of 10 neuron steps of the model on the 1M network;
gradient_262k: derivative passes of the attraction on 16 clusters of 16,384)
and prints the library's statistics; it exits non-zero on any error.  The cases are sized for the profiling rules of the pool: the full
capture case holds well under 1 GB on the device.
"""
from __future__ import annotations

import argparse
import sys


def _plan():
    # the benchmark's plan (leaf capacity, cutoff, no translations)
    return dict(leaf_capacity=256, cutoff=3.25, rho_max=0.0, p=4, m2l_min_pairs=0)


def near_field_131k():
    from . import workloads as W
    return W.clustered(8, 16_384, 100_000.0 * (8 / 64) ** (1 / 3), 1500.0, 4500.0, seed=3,
                       name="clustered_131k", **_plan())


def step_1m():
    from . import workloads as W
    return W.clustered_1m(**_plan())


def translations_256k(p=4, centre_mode=0):
    from . import workloads as W
    return W.uniform_256k(leaf_capacity=8, rho_max=0.5, cutoff=4.0, m2l_min_pairs=0, p=p,
                          centre_mode=centre_mode)


def gradient_262k():
    # the derivative benchmark's workload and plan (cutoff 5 sigma, leaf
    # capacity 128, no translations)
    from . import workloads as W
    return W.clustered_small(16, 16_384, seed=15, leaf_capacity=128, cutoff=5.0, rho_max=0.0,
                             p=4, m2l_min_pairs=0)


CASES = {"near_field_131k": near_field_131k, "step_1m": step_1m, "graph_1m": step_1m,
         "neuron_1m": step_1m, "translations_256k": translations_256k,
         "gradient_262k": gradient_262k}


def _neuron_case(w, g, steps):
    # neuron steps on the 1M network with 1.5 random synapses per neuron
    import numpy as np
    import torch

    from . import msp
    n = w.n
    rng = np.random.default_rng(42)
    m = 3 * n // 2
    edges = msp.edge_list(m, pre=rng.integers(0, n, m), post=rng.integers(0, n, m),
                          type_=np.zeros(m, np.uint8))
    state = {k: torch.zeros(n, dtype=t, device="cuda") for k, t in msp.NEURON_STATE}
    state["x"].fill_(0.065)
    state["calcium"].uniform_(0.3, 0.8)
    for k in range(steps):
        g.neuron_steps(10 * k, 10, msp.neuron_params(), edges, state)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--p", type=int, default=4, help="translations_256k: expansion order")
    ap.add_argument("--centre-mode", type=int, default=0,
                    help="translations_256k: 0 centroids, 1 geometric centres")
    args = ap.parse_args(argv)
    import torch

    from . import build, msp
    build.build()
    if args.case == "translations_256k":
        w = translations_256k(args.p, args.centre_mode)
    else:
        w = CASES[args.case]()
    g = msp.MSP(w.params)
    dev = msp.to_device(w)
    if args.case == "neuron_1m":
        _neuron_case(w, g, args.steps)
    elif args.case == "translations_256k":
        # attraction only, timed with CUDA events (median of the steps after the first)
        import statistics
        g.build_tree(*dev)
        ts = []
        for _ in range(max(args.steps, 2)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.attraction()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        print(f"attraction_ms {statistics.median(ts[1:]):.3f}")
    elif args.case == "gradient_262k":
        # geometric lists (every count 1), derivatives at the real counts
        import numpy as np
        pos, typ, va, ve, vi = dev
        ones = torch.ones_like(va)
        g.build_tree(pos, typ, ones, ones, ones)
        g.attraction()
        gv = torch.from_numpy(np.random.default_rng(6).normal(size=w.n)).float().cuda()
        for _ in range(args.steps):
            g.attraction_grad(typ, va, ve, vi, g=gv)
    elif args.case.startswith("graph"):
        # one eager step sizes the graph; then the whole step as graph
        # replays (walk, build, attraction, selection, commit)
        pos, typ, va, ve, vi = dev
        va, ve, vi = va.clone(), ve.clone(), vi.clone()
        g.build_tree(pos, typ, va, ve, vi)
        g.attraction()
        g.step_graph_capture(pos, typ, va, ve, vi, first_step=0)
        g.run_steps(0, args.steps)
    else:
        for k in range(args.steps):
            g.build_tree(*dev)
            g.attraction()
            g.select_partners(k)
    torch.cuda.synchronize()
    print(args.case, g.stats())
    return 0


if __name__ == "__main__":
    sys.exit(main())
