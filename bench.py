#!/usr/bin/env python
"""Plasticity-step throughput of the GB300 synapse search.

One step = the whole hot path on one network: vacancy update (seeded +-1 walk),
Morton keys + sort + octree + box sums, dual traversal, expansions and near
field (the attraction u of every neuron with vacant axons, and the box-pair
attraction table), the Algorithm 1/2 descent to a partner per vacant axonal
element, request resolution, and the consumption of the formed synapses.

Workload: 1,048,576 neurons in 64 isotropic Gaussian clusters (std 1,500 um)
inside a 100,000 um cube, sigma = 750 um, 80/20 excitatory/inhibitory, vacant
counts uniform in {0..3} (synthetic, seeded).

  python bench.py [--gpus N --steps K --warmup W]          # this library
  python bench.py --impl reference [...]                    # the FP64 CPU oracle
  python bench.py --workload batched_256|gradient_262k|simulation_1m
  python bench.py --profile-case NAME [--steps K]           # small named cases for ncu
Multi-GPU runs are independent replicas (one network per GPU, no exchange).
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "plasticity-step neurons/s at 1M neurons, FMM vs direct on GB300, rel.err<=1e-4"
UNIT = "neurons/s"
SM_COUNT = 152
# The near field's unit of work is one target-source interaction.  Its work
# count in the design is 8 FP32 operations (3 differences, 3 products or FMAs
# for r^2, the scale, the accumulate) and 1 EX2; the FP32 pipe takes 128
# operations per SM per clock, the EX2 unit 30.25 results (measured with a
# dedicated kernel, 16 blocks of 128 threads per SM; profiles/sfu_rate_gb300.md),
# so at that count the FP32 pipe binds: 16 interactions per SM per clock.  The
# kernel evaluates an interaction with 4 FP32 operations (the expanded
# exponent), which leaves the EX2 unit as its own binding unit: 30.25 per SM
# per clock.  Both bases are reported.
EX2_PER_SM_CLK = 30.25
FP32_PER_SM_CLK = 128
FP32_PER_INTERACTION = 8
# algorithmic DRAM bytes of one near-field launch: per neuron its packed point
# (16 B) and log-weights (8 B) read once and u (4 B) written; per near-field
# pair its source range (8 B), list entry (4 B) and W slot (8 B)
NF_BYTES_PER_NEURON = 28
NF_BYTES_PER_PAIR = 20
# the fastest plan with translated pairs found for the 1M clustered network
# (profiles/autotune_clustered_1m.md): timed beside the headline
FMM_TRANSLATED_PLAN = dict(leaf_capacity=64, cutoff=3.5, rho_max=0.35, p=6, m2l_min_pairs=256)
FP64_SAMPLE = 4096


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-direct", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the records beside the headline (batched, gradient, translated "
                         "plan, full rebuild)")
    ap.add_argument("--autotune", action="store_true",
                    help="rerun the plan chooser on this workload and bench its plan")
    ap.add_argument("--workload", default="clustered_1m",
                    choices=["clustered_1m", "batched_256", "gradient_262k", "simulation_1m"],
                    help="clustered_1m: the headline network; batched_256: 256 independent "
                         "networks (about 11.7M neurons) in one batched step; gradient_262k: "
                         "the derivatives of the attraction at 262,144 clustered neurons; "
                         "simulation_1m: the model's simulation loop (100 neuron steps and one "
                         "connectivity update per cycle) on the 1M clustered network")
    ap.add_argument("--profile-case", default=None, choices=sorted(PROFILE_CASES),
                    help="run a small named case for a profiler and print the library's "
                         "statistics (no timing)")
    ap.add_argument("--case-p", type=int, default=4, help="translations_256k: expansion order")
    ap.add_argument("--case-centre-mode", type=int, default=0,
                    help="translations_256k: 0 centroids, 1 geometric centres")
    return ap.parse_args()


_PLAN_OVERRIDE = None


def tuned_params():
    """Plan chosen by the plan chooser for this workload (leaf capacity, cutoff,
    expansions; `python bench.py --autotune` reruns it, see
    paper_2301_10570_gb300/autotune.py and profiles/autotune_clustered_1m.md)."""
    if _PLAN_OVERRIDE is not None:
        return dict(_PLAN_OVERRIDE)
    return dict(leaf_capacity=256, cutoff=3.25, rho_max=0.0, p=4, m2l_min_pairs=0)


def workload():
    from paper_2301_10570_gb300 import workloads as W
    return W.clustered_1m(**tuned_params())


BATCH_METRIC = "batched-step neurons/s, 256 independent networks (11.7M neurons) on GB300"
BATCH_DESC = ("batched_256: 256 networks, n log-uniform in [1024, 262144] (11,718,582 neurons), "
              "sigma uniform in [300, 1500] um, uniform or clustered, each scaled to sigma units "
              "in its own octree cell and frame (msp_batch_layout, msp_set_frames), leaf "
              "capacity 256 for all, a cutoff per network from the batch plan chooser")


_BATCH_TUNING = {}


def batched_workload(dev, rank=0, world=1, common_frame=False):
    """The 256-network batch as one problem of kernel width 1, each network in
    its own cell and frame, with the shared plan's leaf capacity and a cutoff
    per network from the batch plan chooser (autotune.tune_batch_cutoffs; the
    workload carries the frames and the cutoffs); with several ranks, rank r
    takes networks r, r + N, r + 2N, ... (the networks are independent: no
    exchange).  common_frame: the same networks moved into one frame instead,
    with the shared plan (for the host-core oracle, which has no frames)."""
    import torch

    from paper_2301_10570_gb300 import autotune, msp, workloads as W
    b = W.batched_256()
    if world > 1:
        b = b.select(range(rank, len(b.sigma), world))
    plan = tuned_params()
    # cells wide enough for the largest candidate cutoff
    local, side, level = msp.batch_layout(torch.from_numpy(b.pos).to(dev), b.offsets, b.sigma,
                                          max(autotune.BATCH_CUTOFFS), plan["leaf_capacity"])
    local = local.cpu().numpy()
    if common_frame:
        return b.placed(local, side, level, **plan)
    w = b.framed(local, side, level, **plan)
    cuts, rep = autotune.tune_batch_cutoffs(w, device=dev.index)
    _BATCH_TUNING.update(cutoffs=cuts, **rep)
    return b.framed(local, side, level, plans=(None, cuts), **plan)


def batch_tuning_summary():
    """The batch plan chooser's result for the benchmark line."""
    import collections
    if not _BATCH_TUNING:
        return None
    hist = collections.Counter(_BATCH_TUNING["cutoffs"])
    return {"cutoffs": {str(k): v for k, v in sorted(hist.items())},
            "networks_raised": _BATCH_TUNING["raised"],
            "rounds": _BATCH_TUNING["rounds"],
            "max_rel_dev_vs_own_all_pairs": max(_BATCH_TUNING["per_network_max_err"])}


def near_field_traffic():
    """DRAM bytes of one near-field launch on this workload, from the ncu
    capture summarised in profiles/ (null once the kernel source changed)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "near_field_traffic_clustered_1m.md")
    src = os.path.join(ROOT, "paper_2301_10570_gb300", "csrc", "msp_nearfield.cu")
    try:
        fields = {}
        with open(path) as f:
            for line in f:
                if ":" in line and line.split(":")[0].strip() in ("dram_bytes_per_launch",
                                                                    "kernel_source_sha256",
                                                                    "plan_leaf_capacity"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        if fields.get("kernel_source_sha256") != sha:
            return None
        if fields.get("plan_leaf_capacity") != str(tuned_params()["leaf_capacity"]):
            return None
        return int(float(fields["dram_bytes_per_launch"]))
    except Exception:
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def near_field_roofline(inter, nf_ms, n, n_p2p, traffic=None):
    """Roofline of the near-field kernel for `inter` interactions in `nf_ms`:
    the design's work count (8 FP32 + 1 EX2 per interaction, FP32 binds) as
    the primary basis, the EX2 unit (the kernel's own ceiling) beside it, and
    the algorithmic bytes over the measured copy bandwidth."""
    peaks = measured_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    hbm = float(peaks.get("hbm_gbs", 6800.0)) * 1e9
    p_fp32 = SM_COUNT * FP32_PER_SM_CLK * clk           # FP32 operations / s
    p_ex2 = SM_COUNT * EX2_PER_SM_CLK * clk              # EX2 results / s
    nbytes = NF_BYTES_PER_NEURON * n + NF_BYTES_PER_PAIR * n_p2p
    t = {"fp32": FP32_PER_INTERACTION * inter / p_fp32, "ex2": inter / p_ex2,
         "hbm": nbytes / hbm}
    bound_t = max(t.values())
    sec = nf_ms / 1e3
    achieved = inter / sec / 1e9 if sec > 0 else 0.0
    peak = p_fp32 / FP32_PER_INTERACTION / 1e9
    peak_ex2 = p_ex2 / 1e9
    return {"kernel": "k_near_field", "bound": "alu", "achieved": round(achieved, 1),
            "peak": round(peak, 1), "unit": "G interactions/s",
            "frac": round(achieved / peak, 4) if peak else 0.0,
            "traffic": traffic, "near_field_ms": round(nf_ms, 3),
            "interactions_per_launch": int(inter),
            "algorithmic_bytes_per_launch": int(nbytes),
            "roofline_ms": {k: round(1e3 * v, 4) for k, v in t.items()},
            "frac_of_roofline_time": round(bound_t / sec, 4) if sec > 0 else 0.0,
            "peak_basis": (f"design work count 8 FP32 + 1 EX2 per interaction: FP32 pipe "
                           f"{SM_COUNT} SMs x {FP32_PER_SM_CLK}/clk x {clk / 1e6:.0f} MHz / 8 "
                           f"(binds: EX2 {EX2_PER_SM_CLK}/clk measured, bytes over the "
                           f"measured copy bandwidth far below)"),
            "ex2_basis": {"peak": round(peak_ex2, 1),
                          "frac": round(achieved / peak_ex2, 4) if peak_ex2 else 0.0,
                          "note": "the kernel's own ceiling: it evaluates an interaction with "
                                  "4 FP32 operations (expanded exponent), so its EX2 unit "
                                  "binds"}}


# -- clocks ------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = None
        self.proc = None
        self.dev = device_index

    def start(self):
        """Start sampling every 20 ms; returns once the sampler has written its
        first line (at most 3 s), so that it is live when the timed region
        begins, and drops that line (taken before the region)."""
        self.skip = 0
        fd, self.path = tempfile.mkstemp(prefix="msp_clocks_", suffix=".csv")
        self.f = os.fdopen(fd, "w")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            self.f.close()
            os.unlink(self.path)
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and self._lines() == 0:
            time.sleep(0.01)
        self.mark()

    def _lines(self) -> int:
        try:
            with open(self.path) as f:
                return f.read().count("\n")
        except OSError:
            return 0

    def mark(self):
        """The timed region begins: samples written before now are dropped."""
        if self.proc is not None:
            self.skip = self._lines()

    def stop(self):
        if self.proc is None:
            return None
        # at least one sample from the timed region or right after it (at most 1 s)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 1.0 and self._lines() <= self.skip:
            time.sleep(0.01)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f.read().splitlines()[self.skip:]:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# -- the derivative pass (config 4) ------------------------------------------------
GRAD_METRIC = "gradient-pass neurons/s (u, du/dsigma, dL/dw) at 262k clustered neurons on GB300"
GRAD_PLAN = dict(leaf_capacity=128, cutoff=5.0, rho_max=0.0, p=4, m2l_min_pairs=0)
GRAD_DESC = ("gradient_262k: 16 Gaussian clusters x 16,384 neurons (std 1500 um, cluster spacing "
             "of clustered_1m), sigma 750 um, cutoff 5 sigma, pair lists from a tree with every "
             "count 1; outputs u, du/dsigma, dL/dw^E, dL/dw^I")


def gradient_passes(steps, warmup, dev, timed_clocks=False):
    """u, du/dsigma and the weight gradient of L = sum g u over the leaf pairs
    of a tree built with every count 1 (cutoff 5 sigma, no translations), at
    the workload's counts; timed per pass with CUDA events, L2 flushed.
    Returns (neurons, per-pass ms list, launches, clocks, interactions)."""
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import msp, replicas, workloads as W
    # leaf capacity 128: fastest of 64 / 128 / 192 for this pass (7.2 ms vs 11.1 / 7.9)
    w = W.clustered_small(16, 16_384, seed=15, **GRAD_PLAN)
    n = w.n
    pos, t, a, e, i = msp.to_device(w, dev)
    ones = torch.ones_like(a)
    g = msp.MSP(w.params, device=dev.index)
    g.build_tree(pos, t, ones, ones, ones)
    g.attraction()
    gv = torch.from_numpy(np.random.default_rng(6).normal(size=n)).float().to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(warmup):
        g.attraction_grad(t, a, e, i, g=gv)
    torch.cuda.synchronize()
    replicas.barrier()
    launches0 = g.stats()["kernel_launches"]
    clocks = Clocks(dev.index) if timed_clocks else None
    if clocks:
        clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record()
        g.attraction_grad(t, a, e, i, g=gv)
        ev[k][1].record()
    torch.cuda.synchronize()
    replicas.barrier()
    clk = clocks.stop() if clocks else None
    launches = g.stats()["kernel_launches"] - launches0
    ms_list = [x.elapsed_time(y) for x, y in ev]
    # exact interaction count: every target with a vacant axon against the
    # sources of its leaf's partner leaves (self excluded), once forward and
    # once transposed
    tr, pr = g.export_tree(), g.export_pairs()
    cnt = tr["count"].astype(np.int64)
    p2p = pr["kind"] == 2
    X, Y = pr["X"][p2p], pr["Y"][p2p]
    act_sorted = (w.vac_axon[tr["perm"]] > 0).astype(np.int64)
    first = tr["first"]
    nact = np.array([act_sorted[first[k]:first[k] + cnt[k]].sum() for k in range(len(cnt))])
    fwd = int((nact[X] * cnt[Y]).sum() - nact[X[X == Y]].sum())
    g.close()
    return n, ms_list, launches, clk, 2 * fwd


def run_gradient(args, rank, world):
    from paper_2301_10570_gb300 import replicas
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n, ms_list, launches, clk, inter = gradient_passes(args.steps, args.warmup, dev, True)
    agg = replicas.aggregate_throughput(n, sum(ms_list) / len(ms_list), dev)
    ms = agg["ms"]
    achieved = inter / (ms / 1e3) / 1e9
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = SM_COUNT * EX2_PER_SM_CLK * sm_max * 1e6 / 1e9
    return {"metric": GRAD_METRIC, "value": agg["per_s"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": GRAD_DESC, "plan": GRAD_PLAN,
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed (256 MB write) between timed passes",
                       "timing": "CUDA events per pass, mean over passes",
                       "median_ms_per_step": round(statistics.median(ms_list), 3)},
            "clocks": clk, "gpu_launches": int(launches),
            "roofline": {"kernel": "k_grad_forward + k_grad_adjoint", "bound": "alu",
                         "achieved": round(achieved, 1), "peak": round(peak, 1),
                         "unit": "G interactions/s", "frac": round(achieved / peak, 4),
                         "traffic": None, "interactions_per_step": inter,
                         "peak_basis": f"EX2 rate: {SM_COUNT} SMs x {EX2_PER_SM_CLK} "
                                       f"results/clk (measured) x {sm_max:.0f} MHz, one EX2 per "
                                       f"interaction; these kernels use the difference form "
                                       f"(about 7 instructions per interaction, paired FP32 "
                                       f"over two sources)"}}


# -- the simulation loop of the model (neuron side + synapse search) ------------
SIM_METRIC = ("MSP simulation neuron-steps/s at 1M neurons (100 activity steps and one "
              "connectivity update per cycle) on GB300")


def run_simulation(args, rank, world):
    """Cycles of the model's simulation (Section 3.1): 100 steps of activity,
    spikes, calcium and element growth, then the update of synapses
    (deletion, vacancies) and the synapse search on those vacancies with the
    formed synapses appended to the network.  Timed per cycle with CUDA
    events, L2 flushed between cycles."""
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import msp, replicas, workloads as W
    dev = torch.device("cuda", torch.cuda.current_device())
    plan = tuned_params()
    w = W.clustered_1m(**plan)
    n = w.n
    rng = np.random.default_rng(41)
    pos, t, a, e, i = msp.to_device(w, dev)
    # activity at rest, calcium spread over the growth curve, elements just
    # above the workload's vacant counts (no synapse yet)
    state = {
        "x": torch.full((n,), 0.065, dtype=torch.float32, device=dev),
        "refractory": torch.zeros(n, dtype=torch.uint8, device=dev),
        "calcium": torch.from_numpy(rng.uniform(0.3, 0.8, n).astype(np.float32)).to(dev),
        "z_axon": a.float() + 0.5, "z_dend_e": e.float() + 0.5, "z_dend_i": i.float() + 0.5,
        "spiked": torch.zeros(n, dtype=torch.uint8, device=dev)}
    params = msp.neuron_params()
    edges = msp.edge_list(12 * n, device=dev)
    vac = [torch.zeros(n, dtype=torch.uint8, device=dev) for _ in range(3)]
    cap = 6 * n
    sel = dict(partner=torch.empty(cap, dtype=torch.int32, device=dev),
               syn_pre=torch.empty(cap, dtype=torch.int32, device=dev),
               syn_post=torch.empty(cap, dtype=torch.int32, device=dev),
               syn_type=torch.empty(cap, dtype=torch.uint8, device=dev),
               n_syn=torch.zeros(1, dtype=torch.int64, device=dev))
    g = msp.MSP(w.params, device=dev.index)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def cycle(k, ev=None):
        if ev is not None:
            ev[0].record()
        g.neuron_steps(100 * k, 100, params, edges, state)
        if ev is not None:
            ev[1].record()
        g.update_synapses(k, state, edges, *vac)
        g.build_tree(pos, t, *vac)
        if g.num_elements() > cap:
            raise RuntimeError("more vacant axonal elements than the selection buffers hold")
        g.attraction()
        g.select_partners(k, out=sel)
        g.append_synapses(sel, edges)
        if ev is not None:
            ev[2].record()

    for k in range(args.warmup):
        cycle(k)
    torch.cuda.synchronize()
    replicas.barrier()
    launches0 = g.stats()["kernel_launches"]
    n_edges = []
    clocks = Clocks(dev.index)
    clocks.start()
    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        n_edges.append(edges["n"].clone())
        cycle(args.warmup + k, evs[k])
    torch.cuda.synchronize()
    replicas.barrier()
    clk = clocks.stop()
    launches = g.stats()["kernel_launches"] - launches0
    cyc = [x.elapsed_time(z) for x, _, z in evs]
    neu = [x.elapsed_time(y) for x, y, _ in evs]
    agg = replicas.aggregate_throughput(100 * n, sum(cyc) / len(cyc), dev)
    # algorithmic bytes of a neuron step: per neuron the state read and
    # written (activity 4+4, refractory 1+1, calcium 4+4, three element
    # counts 12+12, spike flag 1, input count 4+4) = 51 B; per spiking neuron
    # its edge range (8 B) and per outgoing edge the target (4 B) and the
    # input count it adds to (4 B); spikes per step from the last step
    m = float(torch.stack(n_edges).double().mean().item())
    spikes = float(state["spiked"].sum().item())
    bytes_step = 51.0 * n + spikes * (8.0 + 8.0 * m / n)
    nm = statistics.mean(neu)
    achieved = 100 * bytes_step / (nm / 1e3) / 1e9
    peaks = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    g.close()
    return {"metric": SIM_METRIC, "value": agg["per_s"], "unit": "neuron-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(agg["ms"], 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "simulation_1m: clustered_1m positions and types; a step of "
                                   "the cycle is 100 neuron steps (Table 1 parameters), the "
                                   "update of synapses and one synapse search whose synapses "
                                   "join the network",
                       "plan": plan, "parallelism": f"replicas x{world}",
                       "l2": "flushed (256 MB write) between timed cycles",
                       "timing": "CUDA events per cycle, mean over cycles",
                       "median_ms_per_step": round(statistics.median(cyc), 3),
                       "neuron_steps_ms_per_cycle": round(nm, 3),
                       "edges_mean": round(m, 1)},
            "clocks": clk, "gpu_launches": int(launches),
            "roofline": {"kernel": "k_neuron_step", "bound": "hbm",
                         "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "bytes_per_step": round(bytes_step, 1),
                         "spikes_per_step": spikes,
                         "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}}


# -- our arm -------------------------------------------------------------------
def _timed_replays(g, steps, flush):
    """`steps` graph replays, one per CUDA-event pair, L2 flushed between them
    (untimed); a replay that halted is finished eagerly and the steps timed
    again.  Returns (per-step ms, next step index, halt bits)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    halted = 0
    for attempt in range(2):
        for i in range(steps):
            flush.zero_()
            ev[i][0].record()
            g.step_graph_launch(1)
            ev[i][1].record()
        nxt, halted = g.step_graph_finish()
        if not halted:
            break
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], nxt, halted


def _fp64_targets(job):
    """One host core: the oracle's FP64 brute force (Eq. 8) for some targets."""
    arrays, sigma, idx = job
    from oracle import oracle as O
    return O.direct(*arrays, sigma, targets=idx)


def fp64_reference(w, idx, cores=None):
    """FP64 brute force for the targets idx, split over the host cores (one
    spawned process each)."""
    import multiprocessing as mp

    import numpy as np

    from oracle import oracle as O
    O.build()
    cores = cores or max(1, min(os.cpu_count() or 1, 16))
    parts = [p for p in np.array_split(np.asarray(idx), cores) if len(p)]
    jobs = [(w.arrays(), w.params["sigma"], p) for p in parts]
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_fp64_targets, jobs, chunksize=1)
    return np.concatenate(res)


def error_report(u, ref):
    """Accuracy of u against ref (same targets): the bar's masked relative
    error (targets with ref >= 1e-6 max ref), with the count of targets it
    leaves out, the normwise errors, the largest relative error over every
    target with ref > 0, and the targets whose u is 0 while ref > 0."""
    import numpy as np
    u = np.asarray(u, np.float64)
    ref = np.asarray(ref, np.float64)
    pos = ref > 0
    m = ref >= 1e-6 * ref.max()
    d = np.abs(u - ref)
    return {"max_rel_err": float(np.max(d[m] / ref[m])) if m.any() else 0.0,
            "targets": int(len(ref)), "targets_below_mask": int((pos & ~m).sum()),
            "max_abs_err_over_max_ref": float(d.max() / ref.max()) if ref.max() > 0 else 0.0,
            "l2_rel_err": float(np.linalg.norm(u - ref) / np.linalg.norm(ref)) if pos.any() else 0.0,
            "max_rel_err_all_positive": float(np.max(d[pos] / ref[pos])) if pos.any() else 0.0,
            "zero_where_positive": int(((u == 0) & pos).sum())}


def run_ours(args, rank, world):
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import msp, replicas

    dev = torch.device("cuda", torch.cuda.current_device())
    batched = args.workload == "batched_256"
    w = batched_workload(dev, rank, world) if batched else workload()
    n = w.n
    g = msp.MSP(w.params, device=dev.index, frames=w.frames)
    pos, typ, va0, ve0, vi0 = msp.to_device(w, dev)
    va, ve, vi = va0.clone(), ve0.clone(), vi0.clone()
    u = torch.empty(n, dtype=torch.float32, device=dev)
    ne_cap = 5 * n          # vacancies are clamped to [0, 5]
    sel = dict(partner=torch.empty(ne_cap, dtype=torch.int32, device=dev),
               syn_pre=torch.empty(ne_cap, dtype=torch.int32, device=dev),
               syn_post=torch.empty(ne_cap, dtype=torch.int32, device=dev),
               syn_type=torch.empty(ne_cap, dtype=torch.uint8, device=dev),
               n_syn=torch.zeros(1, dtype=torch.int64, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(k):
        # the same step as separate calls (one host synchronisation each)
        g.vacancy_walk(k, va, ve, vi)
        g.build_tree(pos, typ, va, ve, vi)
        g.attraction(out=u)
        g.select_partners(k, out=sel)
        g.commit_synapses(sel, va, ve, vi)

    # eager warm-up: sizes the tree levels and the pair table for the graph
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    # the whole step as one CUDA graph, replayed once per step; its own
    # warm-up replays, then the timed ones
    k0 = args.warmup
    gout = g.step_graph_capture(pos, typ, va, ve, vi, first_step=k0,
                                history_len=args.warmup + 2 * args.steps)
    k0 = g.run_steps(k0, args.warmup)
    torch.cuda.synchronize()
    replicas.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    launches0 = g.stats()["kernel_launches"]
    t_wall = time.perf_counter()
    step_ms, nxt, halted = _timed_replays(g, args.steps, flush)
    replicas.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    # the vacancy state a replay's build sees (the timed replays' last state
    # walked once more, as the next step's walk would): the end-to-end leg
    # below runs on it (the host-buffer call runs steps a1-a12, without the
    # walk and the commit; the runs in between walk and commit further)
    timed_state = [v.clone() for v in (va, ve, vi)]
    g.vacancy_walk(nxt, *timed_state)
    st = g.stats()
    launches = st["kernel_launches"] - launches0
    clk = clocks.stop()
    agg = replicas.aggregate_throughput(n, sum(step_ms) / len(step_ms), dev)
    ms = agg["ms"]
    value = agg["per_s"]
    first_timed = nxt - args.steps
    hist = gout["history"].cpu().numpy()
    synapses = [int(v) for v in hist[first_timed - args.warmup:nxt - args.warmup]]
    nf_ms, inter, n_p2p = st["near_field_ms"], st["p2p_interactions"], st["n_p2p"]

    # the same step with the whole octree rebuilt in every replay (a1-a12 in
    # full: Morton keys, radix sort, subdivision, aggregates)
    full = None
    if not args.no_extras:
        g.build_tree(pos, typ, va, ve, vi)
        g.attraction()
        g.step_graph_set_full_build(True)
        g.step_graph_capture(pos, typ, va, ve, vi, first_step=nxt)
        kf = g.run_steps(nxt, args.warmup)
        fms, nxt, fh = _timed_replays(g, args.steps, flush)
        g.step_graph_set_full_build(False)
        fst = g.stats()
        full = {"ms_per_step": round(statistics.mean(fms), 3),
                "median_ms_per_step": round(statistics.median(fms), 3),
                "neurons_per_s": n / (statistics.mean(fms) / 1e3),
                "near_field_ms": round(fst["near_field_ms"], 3), "graph_halted": int(fh),
                "path": "whole step as one CUDA graph whose replays rebuild the octree "
                        "(Morton keys, radix sort, subdivision, aggregates) from the positions "
                        "every step"}

    # the same steps as separate calls, for comparison
    for k in range(nxt, nxt + 2):
        step(k)                            # fresh build after the graph, and warm
    torch.cuda.synchronize()
    eager_ms = []
    for i in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(nxt + 2 + i)
        e1.record()
        torch.cuda.synchronize()
        eager_ms.append(e0.elapsed_time(e1))

    # End to end through the C ABI's host-buffer call: every step copies the
    # inputs (positions, types, vacant counts) up from pinned host memory, runs
    # steps a1-a12 and copies u, the partners and the synapses back (the call
    # replays its own graph of the step after the first call).  The vacant
    # counts are those a timed replay's build sees (snapshot above).
    pinned = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hp = pinned(w.pos)
    ht = pinned(w.type)
    ha, he, hi = (pinned(v.cpu().numpy()) for v in timed_state)
    ne0 = int(ha.sum(dtype=np.int64))
    hout = dict(u=pinned(np.zeros(n, np.float32)), partner=pinned(np.zeros(ne0, np.int32)),
                syn_pre=pinned(np.zeros(ne0, np.int32)), syn_post=pinned(np.zeros(ne0, np.int32)),
                syn_type=pinned(np.zeros(ne0, np.uint8)), n_syn=pinned(np.zeros(1, np.int64)))
    for k in range(max(2, args.warmup)):
        g.plasticity_step_host(k, hp, ht, ha, he, hi, out=hout)
    torch.cuda.synchronize()
    e2e_t, d2h = [], []
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.plasticity_step_host(100 + i, hp, ht, ha, he, hi, out=hout)
        e2e_t.append(time.perf_counter() - t0)
        d2h.append(8 + 4 * n + 4 * ne0 + 9 * int(hout["n_syn"][0]))
    e2e = replicas.aggregate_throughput(n, 1e3 * sum(e2e_t) / len(e2e_t), dev)

    # the attraction at the vacancy state the timed replays walked to, and of
    # the unwalked inputs (accuracy checks below)
    from paper_2301_10570_gb300 import workloads as W
    g.build_tree(pos, typ, va, ve, vi)
    uw = g.attraction().cpu().numpy()
    walked = (W.Workload(w.name + "_walked", w.pos, w.type, va.cpu().numpy(), ve.cpu().numpy(),
                         vi.cpu().numpy(), dict(w.params)), uw)
    g.build_tree(pos, typ, va0, ve0, vi0)
    uf = g.attraction()
    torch.cuda.synchronize()
    # the attraction alone, near field only (the plan's), for the translated
    # plan's comparison
    att_ms = []
    for _ in range(3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.attraction(out=u)
        e1.record()
        torch.cuda.synchronize()
        att_ms.append(e0.elapsed_time(e1))
    # direct all-pairs evaluation of the attraction on the same GPU
    direct, ud = None, None
    if not args.no_direct and not batched:
        ud = torch.empty(n, dtype=torch.float32, device=dev)
        g.direct(out=ud)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record()
        g.direct(out=ud)
        e1.record()
        torch.cuda.synchronize()
        d_ms = e0.elapsed_time(e1)
        rep = error_report(uf.cpu().numpy(), ud.cpu().numpy())
        direct = {"direct_attraction_ms": round(d_ms, 3),
                  "direct_neurons_per_s": n / (d_ms / 1e3),
                  "speedup_step_vs_direct_attraction": round(d_ms / ms, 2),
                  "max_rel_err_vs_direct_fp32": rep["max_rel_err"],
                  "error_vs_direct_fp32": rep}
    uf_np = uf.cpu().numpy()
    ud_np = ud.cpu().numpy() if ud is not None else None
    g.close()

    traffic = None if batched else near_field_traffic()
    roofline = near_field_roofline(inter, nf_ms, n, n_p2p, traffic)
    roofline["near_field_share_of_step"] = round(nf_ms / ms, 3) if ms > 0 else 0.0

    out = {"metric": BATCH_METRIC if batched else METRIC, "value": value, "unit": UNIT,
           "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           # the batch's networks are split over the ranks (fixed total work);
           # the single network is replicated (fixed work per rank)
           "higher_is_better": True, "scaling": "strong" if batched else "weak",
           "vs_baseline": None, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": BATCH_DESC if batched else
                      "clustered_1m: 1,048,576 neurons, 64 Gaussian clusters (std 1500 um), "
                      "100,000 um cube, sigma 750 um, 80/20 E/I, vacancies U{0..3} + walk",
                      "plan": tuned_params(), "parallelism": f"replicas x{world}",
                      **({"batch_plan_chooser": batch_tuning_summary()} if batched else {}),
                      "l2": "flushed (256 MB write) between timed steps",
                      "timing": "CUDA events per step (one graph replay each), mean over steps",
                      "step_path": "whole step captured as one CUDA graph (msp_step_graph_*); "
                                   "the replays reuse the octree of the fixed positions and "
                                   "refresh its counts and aggregates (full_rebuild_step: the "
                                   "octree rebuilt every replay)",
                      "graph_halted": int(halted),
                      "median_ms_per_step": round(statistics.median(step_ms), 3),
                      "note": "the plan translates no box pair: every pair of leaf boxes within "
                              "the cutoff (3.25 sigma) is evaluated exactly and pairs beyond it "
                              "are dropped (their kernel is below exp(-10.6) = 2.6e-5), so the "
                              "step is itself the cutoff-pruned direct evaluation plus the tree, "
                              "the descent and the resolution; direct_* is the unpruned all-pairs "
                              "evaluation; fmm_translated is the fastest plan with translated "
                              "pairs",
                      "eager_ms_per_step": round(statistics.mean(eager_ms), 3),
                      "attraction_ms": round(statistics.median(att_ms), 3),
                      "wall_s_timed_loop": round(t_wall, 3),
                      "synapses_per_step": int(statistics.mean(synapses)),
                      **(direct or {})},
           "clocks": clk,
           "e2e": {"value": e2e["per_s"], "unit": UNIT,
                   "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": int(statistics.mean(d2h)),
                   "ms_per_step": round(e2e["ms"], 3),
                   "path": "msp_plasticity_step_host (C ABI, host buffers): positions, types and "
                           "vacant counts copied up from pinned memory, steps a1-a12, u, partners "
                           "and synapses copied back, every step; the call replays its own graph "
                           "of the step (the vacancy state a timed replay's build sees: its last "
                           "state walked once more; the walk and the commit, about 40 us of the "
                           "replayed step under ncu, are not part of this call)",
                   "timing": "host wall clock per call, mean over calls, L2 flushed between"},
           "gpu_launches": int(launches),
           "roofline": roofline}
    if full:
        out["full_rebuild_step"] = full
    return out, w, uf_np, ud_np, walked


def accuracy_fp64(w, uf, ud, sample=FP64_SAMPLE):
    """u of the plan and of the all-pairs path against the oracle's FP64 brute
    force on `sample` seeded targets (split over the host cores)."""
    import numpy as np
    idx = np.sort(np.random.default_rng(0).choice(w.n, min(sample, w.n), replace=False))
    ref = fp64_reference(w, idx)
    res = {"targets": int(len(idx)), "plan": error_report(uf[idx], ref)}
    if ud is not None:
        res["direct_fp32"] = error_report(ud[idx], ref)
    return res, idx, ref


def fmm_translated_record(w, dev, idx, ref, reps=3):
    """The fastest plan with translated pairs (Hermite coefficients, their
    translation and the Taylor evaluation, Eq. 6-7) on the same network and
    counts: attraction time and its error against FP64 on the same targets."""
    import torch

    from paper_2301_10570_gb300 import msp
    plan = dict(FMM_TRANSLATED_PLAN)
    params = dict(w.params, **plan)
    g = msp.MSP(params, device=dev.index)
    g.build_tree(*msp.to_device(w, dev))
    u = g.attraction()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.attraction(out=u)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    st = g.stats()
    un = u.cpu().numpy()
    g.close()
    rep = error_report(un[idx], ref)
    return {"plan": plan, "attraction_ms": round(statistics.median(ts), 3),
            "far_pairs": st["n_far"], "near_field_pairs": st["n_p2p"],
            "near_field_interactions": st["p2p_interactions"],
            "expansion_boxes": st["expansion_nodes"],
            "near_field_ms": round(st["near_field_ms"], 3),
            "error_vs_fp64": rep, "meets_1e-4": rep["max_rel_err"] <= 1e-4}


def batched_record(dev, steps, warmup, fp64=True):
    """The 256-network batch as one graph-replayed step (msp_batch_layout and
    msp_set_frames, then the ordinary path): a few timed replays; and the
    attraction of 8 sampled networks, 512 sampled targets each, against the
    FP64 brute force of that network alone at its own width on its own
    unscaled positions."""
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import msp, workloads as W
    w = batched_workload(dev)
    n = w.n
    g = msp.MSP(w.params, device=dev.index, frames=w.frames)
    pos, typ, va, ve, vi = msp.to_device(w, dev)
    g.build_tree(pos, typ, va, ve, vi)
    ub = g.attraction().cpu().numpy()
    b = W.batched_256()
    errs = []
    rng = np.random.default_rng(1)
    # the FP64 checks run the oracle on the host cores: part of the CPU leg
    for k in (sorted(rng.choice(len(b.sigma), 8, replace=False).tolist()) if fp64 else []):
        wk = b.network(k, **tuned_params())
        idx = np.sort(rng.choice(wk.n, min(512, wk.n), replace=False))
        ref = fp64_reference(wk, idx)
        uk = ub[b.offsets[k]:b.offsets[k + 1]][idx]
        errs.append(error_report(uk, ref)["max_rel_err"])
    g.step_graph_capture(pos, typ, va, ve, vi, first_step=0)
    g.run_steps(0, warmup)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ms_list, _, halted = _timed_replays(g, steps, flush)
    st = g.stats()
    g.close()
    ms = statistics.mean(ms_list)
    return {"workload": BATCH_DESC, "neurons": n, "steps": steps,
            "ms_per_step": round(ms, 3), "neurons_per_s": n / (ms / 1e3),
            "graph_halted": int(halted),
            "max_rel_err_sampled_networks_vs_own_fp64": max(errs) if errs else None,
            "plan_chooser": batch_tuning_summary(),
            "accuracy_note": "8 sampled networks x 512 sampled targets, each network against "
                             "the FP64 brute force of that network alone at its own width on "
                             "its own unscaled positions (every network keeps its own frame)",
            "roofline": near_field_roofline(st["p2p_interactions"], st["near_field_ms"], n,
                                            st["n_p2p"])}


def length_loss_passes(steps, warmup, dev, target=1000.0):
    """The loss of the differentiation workload: the expected mean synapse
    length m, (m - target)^2 and its gradient with respect to sigma and the
    dendritic weights (msp_length_loss), timed per pass with CUDA events."""
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import msp, workloads as W
    w = W.clustered_small(16, 16_384, seed=15, **GRAD_PLAN)
    pos, t, a, e, i = msp.to_device(w, dev)
    ones = torch.ones_like(a)
    g = msp.MSP(w.params, device=dev.index)
    g.build_tree(pos, t, ones, ones, ones)
    g.attraction()
    rng = np.random.default_rng(7)
    wE = torch.from_numpy(rng.uniform(0.2, 3.0, w.n)).float().to(dev)
    wI = torch.from_numpy(rng.uniform(0.2, 3.0, w.n)).float().to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(warmup):
        r = g.length_loss(t, a, wE, wI, target)
    ms_list = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = g.length_loss(t, a, wE, wI, target)
        e1.record()
        torch.cuda.synchronize()
        ms_list.append(e0.elapsed_time(e1))
    g.close()
    return w.n, ms_list, r


def _timed_attraction(g, flush, reps):
    import torch
    u = g.attraction()
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.attraction(out=u)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), u


def uniform_records(dev, reps=3, fp64=True):
    """The two uniform workloads: 4,096 neurons in a 10,000 um cube (p = 4,
    leaf capacity 32: a whole eager step, launch-bound; u against the oracle's
    FP64 brute force on every target) and 262,144 neurons at the same density
    in a 40,000 um cube, attraction with translated pairs at p = 3, 4, 6 (leaf
    capacity 8, rho_max 0.5, cutoff 4 sigma), with the near field only, and
    with the plan chooser's plan, each against the all-pairs evaluation of the
    same GPU on every target and the FP64 brute force on 4,096 sampled
    targets."""
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import autotune, msp, workloads as W
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {}
    w = W.uniform_4k()
    g = msp.MSP(w.params, device=dev.index)
    d = msp.to_device(w, dev)
    g.build_tree(*d)
    u4 = g.attraction().cpu().numpy()
    # the FP64 checks run the oracle on the host cores: part of the CPU leg
    ref4 = fp64_reference(w, np.arange(w.n)) if fp64 else None
    ts = []
    for k in range(reps + 2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.build_tree(*d)
        g.attraction()
        g.select_partners(k)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    g.close()
    out["uniform_4k"] = {"what": "eager step (tree, attraction, selection), p = 4, leaf capacity 32; "
                                 "the positions are fixed, so each build keeps the octree and each "
                                 "attraction the lists (counts, aggregates and sums refreshed)",
                         "ms_per_step": round(statistics.median(ts[2:]), 3),
                         "neurons_per_s": w.n / (statistics.median(ts[2:]) / 1e3),
                         "error_vs_fp64_all_targets": error_report(u4, ref4) if fp64 else None}
    rows = []
    ref = None
    w0 = W.uniform_256k()
    idx = np.sort(np.random.default_rng(0).choice(w0.n, FP64_SAMPLE, replace=False))
    ref64 = fp64_reference(w0, idx) if fp64 else None
    chosen, _ = autotune.tune(w0, device=dev.index, candidates=dict(
        leaf_capacity=(16, 32, 64, 128), cutoff=(3.25, 3.5, 4.0),
        expansions=((0.0, 4, 0), (0.5, 4, 0), (0.5, 6, 0))), reps=3)
    plans = [dict(leaf_capacity=8, rho_max=0.5, cutoff=4.0, p=3, m2l_min_pairs=0),
             dict(leaf_capacity=8, rho_max=0.5, cutoff=4.0, p=4, m2l_min_pairs=0),
             dict(leaf_capacity=8, rho_max=0.5, cutoff=4.0, p=6, m2l_min_pairs=0),
             dict(leaf_capacity=64, rho_max=0.0, cutoff=3.5, p=4, m2l_min_pairs=0)]
    if chosen is not None:
        plans.append(dict(chosen))
    for i, plan in enumerate(plans):
        w = W.uniform_256k(**plan)
        g = msp.MSP(w.params, device=dev.index)
        g.build_tree(*msp.to_device(w, dev))
        if ref is None:
            ref = g.direct().cpu().numpy()
        ms, u = _timed_attraction(g, flush, reps)
        st = g.stats()
        g.close()
        un = u.cpu().numpy()
        rep = error_report(un, ref)
        rows.append({"plan": plan, "chosen_by_plan_chooser": chosen is not None and
                     i == len(plans) - 1, "attraction_ms": round(ms, 3), "far_pairs": st["n_far"],
                     "near_field_pairs": st["n_p2p"],
                     "max_rel_err_vs_direct_fp32": rep["max_rel_err"],
                     "l2_rel_err": rep["l2_rel_err"],
                     "max_rel_err_vs_fp64_sampled":
                         error_report(un[idx], ref64)["max_rel_err"] if fp64 else None})
    out["uniform_256k"] = rows
    return out


def simulation_record(steps, warmup):
    """The model's simulation cycle on the 1M clustered network (100 neuron
    steps, the update of synapses and one synapse search whose synapses join
    the network): a few timed cycles."""
    sargs = argparse.Namespace(steps=steps, warmup=warmup)
    r = run_simulation(sargs, 0, 1)
    return {"workload": r["config"]["workload"], "cycles": steps,
            "ms_per_cycle": r["ms_per_step"], "neuron_steps_per_s": r["value"],
            "neuron_steps_ms_per_cycle": r["config"]["neuron_steps_ms_per_cycle"],
            "edges_mean": r["config"]["edges_mean"],
            "neuron_step_hbm_frac": r["roofline"]["frac"]}


def gradient_record(dev, steps, warmup):
    n, ms_list, launches, _, inter = gradient_passes(steps, warmup, dev)
    ms = statistics.mean(ms_list)
    peaks = measured_peaks()
    clk = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    p_ex2 = SM_COUNT * EX2_PER_SM_CLK * clk
    _, lms, r = length_loss_passes(steps, warmup, dev)
    return {"workload": GRAD_DESC, "neurons": n, "steps": steps, "ms_per_pass": round(ms, 3),
            "neurons_per_s": n / (ms / 1e3), "interactions_per_pass": inter,
            "ex2_frac": round(inter / (ms / 1e3) / p_ex2, 4),
            "length_loss": {"ms_per_pass": round(statistics.mean(lms), 3),
                            "neurons_per_s": n / (statistics.mean(lms) / 1e3),
                            "mean_synapse_length_um": round(r["mean"], 3),
                            "loss": r["loss"], "dloss_dsigma": r["dloss_dsigma"],
                            "what": "expected mean synapse length m, (m - 1000 um)^2 and its "
                                    "gradient in sigma and the dendritic weights, uniform "
                                    "weights in [0.2, 3]"}}


def _oracle_steps(job):
    """One host core: the oracle as it stands on one sample (its own cluster of
    the workload), `warmup` untimed then `steps` timed plasticity steps
    (walk, build, attraction, selection, commit).  Returns (neurons, seconds
    of the timed steps)."""
    params, arrays, warmup, steps = job
    from oracle import oracle as O
    pos, typ, a, e, i = arrays
    o = O.Oracle(params)
    t0 = 0.0
    for k in range(warmup + steps):
        if k == warmup:
            t0 = time.perf_counter()
        a, e, i = O.vacancy_walk(params["seed"], k, a, e, i)
        o.build_tree(pos, typ, a, e, i)
        o.attraction()
        r = o.select_partners(k)
        a, e, i = O.commit_synapses(r["syn_pre"], r["syn_post"], r["syn_type"], a, e, i)
    return pos.shape[1], time.perf_counter() - t0


def oracle_on_host_cores(w, warmup, steps, per_core=16_384, cores=None):
    """The oracle on every host core at once, each core on its own block of
    `per_core` neurons of the workload (a cluster of the 1M network; the
    first networks of a batch), one spawned process per core.  Returns
    (neurons/s over all cores, cores, seconds per step of the slowest)."""
    import multiprocessing as mp

    from oracle import oracle as O
    from paper_2301_10570_gb300 import workloads as W
    O.build()
    cores = cores or min(os.cpu_count() or 1, max(1, w.n // per_core))
    jobs = []
    for c in range(cores):
        sub = W.subset(w, range(c * per_core, (c + 1) * per_core), name=f"sample_{c}")
        jobs.append((sub.params, sub.arrays(), warmup, steps))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_steps, jobs, chunksize=1)
    slowest = max(t for _, t in res) / steps
    return sum(n for n, _ in res) / slowest, cores, slowest


def cpu_baseline(w):
    """The FP64 oracle as it stands on every host core (one process per core,
    each on its own 16,384-neuron block of the workload, one full step)."""
    value, cores, dt = oracle_on_host_cores(w, 0, 1)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes, each one full step (walk, tree, attraction, selection, "
                      f"commit) on its own 16,384-neuron block of the workload (a cluster of the "
                      f"1M network, or the first networks of the batch); slowest {dt:.1f} s"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on every host core (one
    process per core, each on its own cluster of the workload, steps with the
    vacancy walk and the commit), bounded in size."""
    w = workload()
    steps = max(1, args.steps)
    value, cores, dt = oracle_on_host_cores(w, args.warmup, steps)
    sample = (f"{cores} processes, each on its own 16,384-neuron cluster of the 1M clustered "
              f"workload, {steps} timed steps (walk, tree, attraction, selection, commit)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "clustered_1m (bounded sample)", "plan": tuned_params()},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# -- small named cases for profilers (ncu) ---------------------------------------
def _profile_plan():
    # the benchmark's plan (leaf capacity, cutoff, no translations)
    return dict(leaf_capacity=256, cutoff=3.25, rho_max=0.0, p=4, m2l_min_pairs=0)


def _case_near_field_131k(args):
    from paper_2301_10570_gb300 import workloads as W
    return W.clustered(8, 16_384, 100_000.0 * (8 / 64) ** (1 / 3), 1500.0, 4500.0, seed=3,
                       name="clustered_131k", **_profile_plan())


def _case_step_1m(args):
    from paper_2301_10570_gb300 import workloads as W
    return W.clustered_1m(**_profile_plan())


def _case_translations_256k(args):
    from paper_2301_10570_gb300 import workloads as W
    return W.uniform_256k(leaf_capacity=8, rho_max=0.5, cutoff=4.0, m2l_min_pairs=0,
                          p=args.case_p, centre_mode=args.case_centre_mode)


def _case_translations_65k(args):
    # the uniform density of translations_256k on a quarter of the neurons
    from paper_2301_10570_gb300 import workloads as W
    return W.uniform_cube(65_536, 40_000.0 * 0.25 ** (1 / 3), seed=2, name="uniform_65k",
                          leaf_capacity=8, rho_max=0.55, cutoff=4.0, m2l_min_pairs=0,
                          p=args.case_p, centre_mode=args.case_centre_mode)


def _case_translated_1m(args):
    from paper_2301_10570_gb300 import workloads as W
    return W.clustered_1m(**FMM_TRANSLATED_PLAN)


def _case_gradient_262k(args):
    from paper_2301_10570_gb300 import workloads as W
    return W.clustered_small(16, 16_384, seed=15, **GRAD_PLAN)


# name -> (workload, what runs): "steps" eager steps (tree, attraction,
# selection); "graph"/"graph_full" the whole step captured and replayed
# (octree reused / rebuilt each replay); "neuron" calls of 10 neuron steps;
# "attraction" attraction calls timed with CUDA events; "gradient"
# derivative passes, then synapse-length losses
PROFILE_CASES = {"near_field_131k": (_case_near_field_131k, "steps"),
                 "step_1m": (_case_step_1m, "steps"),
                 "graph_1m": (_case_step_1m, "graph"),
                 "graph_full_1m": (_case_step_1m, "graph_full"),
                 "neuron_1m": (_case_step_1m, "neuron"),
                 "translations_256k": (_case_translations_256k, "attraction"),
                 "translations_65k": (_case_translations_65k, "attraction"),
                 "translated_1m": (_case_translated_1m, "attraction"),
                 "gradient_262k": (_case_gradient_262k, "gradient")}


def run_profile_case(args):
    """One small named case (a few steps, well under a GB on the device),
    exiting non-zero on any error; prints the library's statistics."""
    import numpy as np
    import torch

    from paper_2301_10570_gb300 import build, msp
    build.build()
    make, kind = PROFILE_CASES[args.profile_case]
    w = make(args)
    g = msp.MSP(w.params)
    dev = msp.to_device(w)
    steps = max(args.steps, 1)
    if kind == "neuron":
        # neuron steps on the 1M network with 1.5 random synapses per neuron
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
    elif kind == "attraction":
        # attraction only, timed with CUDA events (median of the calls after the first)
        g.build_tree(*dev)
        ts = []
        for _ in range(max(steps, 2)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.attraction()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        print(f"attraction_ms {statistics.median(ts[1:]):.3f}")
    elif kind == "gradient":
        # geometric lists (every count 1), derivatives at the real counts
        pos, typ, va, ve, vi = dev
        ones = torch.ones_like(va)
        g.build_tree(pos, typ, ones, ones, ones)
        g.attraction()
        gv = torch.from_numpy(np.random.default_rng(6).normal(size=w.n)).float().cuda()
        for _ in range(steps):
            g.attraction_grad(typ, va, ve, vi, g=gv)
        # then the synapse-length loss with its gradient (k_len_pairs)
        for _ in range(steps):
            g.length_loss(typ, va, ve.float(), vi.float(), 1000.0)
    elif kind in ("graph", "graph_full"):
        # one eager step sizes the graph; then the whole step as graph
        # replays (walk, build, attraction, selection, commit)
        pos, typ, va, ve, vi = dev
        va, ve, vi = va.clone(), ve.clone(), vi.clone()
        g.build_tree(pos, typ, va, ve, vi)
        g.attraction()
        g.step_graph_set_full_build(kind == "graph_full")
        g.step_graph_capture(pos, typ, va, ve, vi, first_step=0)
        g.run_steps(0, steps)
    else:
        for k in range(steps):
            g.build_tree(*dev)
            g.attraction()
            g.select_partners(k)
    torch.cuda.synchronize()
    print(args.profile_case, g.stats())
    return 0


def main():
    args = parse()
    if args.profile_case:
        sys.exit(run_profile_case(args))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)))
        return
    import torch
    if world > 1:
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2301_10570_gb300 import build as B
    B.build()
    if args.autotune:
        global _PLAN_OVERRIDE
        from paper_2301_10570_gb300 import autotune
        best, table = autotune.tune(workload(), device=torch.cuda.current_device())
        for row in table:
            print(json.dumps(row), file=sys.stderr)
        if best is None:
            raise RuntimeError("no candidate plan meets the accuracy target")
        _PLAN_OVERRIDE = best
    if args.workload in ("gradient_262k", "simulation_1m"):
        out = (run_gradient if args.workload == "gradient_262k" else run_simulation)(
            args, rank, world)
        if rank == 0:
            print(json.dumps(out))
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return
    out, w, uf, ud, walked = run_ours(args, rank, world)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0 and world == 1 and args.workload == "clustered_1m":
        idx = ref = None
        if not args.no_cpu_baseline:
            acc, idx, ref = accuracy_fp64(w, uf, ud)
            # the same targets at the vacancy state of the walked replays
            ww, uw = walked
            acc["walked_state"] = {
                "after": "the warm-up, the timed graph replays and the eager steps, every "
                         "step with the vacancy walk and the commit of its synapses",
                "plan": error_report(uw[idx], fp64_reference(ww, idx))}
            out["accuracy_vs_fp64"] = acc
        if not args.no_extras:
            if idx is not None:
                out["fmm_translated"] = fmm_translated_record(w, dev, idx, ref)
            out["batched_256"] = batched_record(dev, 3, 2, fp64=not args.no_cpu_baseline)
            out["gradient_262k"] = gradient_record(dev, 3, 2)
            out["simulation_1m"] = simulation_record(3, 2)
            out.update(uniform_records(dev, fp64=not args.no_cpu_baseline))
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        # the oracle has no frames: the batch's networks in one common frame
        out["cpu_baseline"] = cpu_baseline(batched_workload(dev, common_frame=True)
                                           if args.workload == "batched_256" else w)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
