"""Many independent networks as one problem (the batched step).

The layout scales each network by 1/sigma and gives it its own octree cell,
with an empty cell between networks; each network keeps its own frame
(positions relative to its cell) and the context is told of the frames
(msp_set_frames).  Checks: the layout itself; the whole batch through the
CUDA path against the oracle run on the same problem in one common frame, on
networks whose scaled positions lie on a dyadic grid so that the common frame
holds them exactly (keys bit for bit, the usual bars for u, partners and
synapses); independence and precision: every network's attraction against
the FP64 brute force of that network alone, at its own width, on its own
unscaled positions; the argument checks of the frames.
"""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import msp  # noqa: E402

PLAN = dict(leaf_capacity=16, cutoff=3.25, rho_max=0.0, p=4, m2l_min_pairs=0)
PLANS = {"exact": dict(PLAN), "translations": dict(PLAN, rho_max=0.3, leaf_capacity=8),
         "geo_translations": dict(PLAN, rho_max=0.3, leaf_capacity=8, centre_mode=1),
         "wide": dict(PLAN, cutoff=5.0)}


def _layout(b, **plan):
    pos = torch.from_numpy(b.pos).cuda()
    local, side, level = msp.batch_layout(pos, b.offsets, b.sigma, plan["cutoff"],
                                          plan["leaf_capacity"])
    return local.cpu().numpy(), side, level


def _dyadic(b, grid=256.0):
    """The batch scaled to sigma units by the test, positions rounded to
    multiples of 1/grid, every width 1: the layout then only translates, and
    the common frame of the whole batch holds every position exactly."""
    k = b.network_of()
    pos = np.round(b.pos.astype(np.float64) / b.sigma[k] * grid) / grid
    return W.Batch(b.name + "_dyadic", np.ascontiguousarray(pos, np.float32), b.type,
                   b.vac_axon, b.vac_dend_e, b.vac_dend_i, b.offsets.copy(),
                   np.ones_like(b.sigma), list(b.kinds))


def _gpu(w, step=4):
    g = msp.MSP(w.params, frames=w.frames)
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    ud = g.direct().cpu().numpy()
    sel = g.select_partners(step)
    torch.cuda.synchronize()
    ne = g.num_elements()
    ns = int(sel["n_syn"].item())
    res = dict(u=u, ud=ud, partner=sel["partner"][:ne].cpu().numpy(), n_syn=ns,
               pre=sel["syn_pre"][:ns].cpu().numpy(), post=sel["syn_post"][:ns].cpu().numpy(),
               keys=g.export_tree()["keys"], stats=g.stats())
    g.close()
    return res


_cache = {}


def _run(plan_key, dyadic):
    key = (plan_key, dyadic)
    if key not in _cache:
        plan = PLANS[plan_key]
        b = W.batched_small()
        if dyadic:
            b = _dyadic(b)
        local, side, level = _layout(b, **plan)
        w = b.framed(local, side, level, **plan)
        _cache[key] = (b, w, local, side, level, _gpu(w))
    return _cache[key]


def test_layout_scales_each_network_into_its_own_cell():
    b = W.batched_small()
    local, side, level = _layout(b, **PLAN)
    cell = side / 2.0 ** level
    G = 2 ** (level - 1)
    assert G ** 3 >= len(b.sigma)
    assert cell == 2.0 ** np.round(np.log2(cell))      # a power of two
    assert side == 2 * G * cell
    for k in range(len(b.sigma)):
        a, e = b.offsets[k], b.offsets[k + 1]
        src = b.pos[:, a:e].astype(np.float64)
        lo = src.min(axis=1, keepdims=True)
        want = (src - lo) / b.sigma[k]
        got = local[:, a:e].astype(np.float64)
        assert np.max(np.abs(got - want)) <= 4e-7 * max(1.0, want.max())
        assert np.all(got >= 0) and np.all(got < cell)
        # networks one cell apart: the gap exceeds the cutoff
        assert cell - want.max() > PLAN["cutoff"]


def test_layout_rejects_small_networks_and_bad_widths():
    b = W.batched_small()
    pos = torch.from_numpy(b.pos).cuda()
    with pytest.raises(msp.MSPError):
        msp.batch_layout(pos, b.offsets, b.sigma, 3.25, 1000)      # a network of <= 1000
    bad = b.sigma.copy()
    bad[2] = 0.0
    with pytest.raises(msp.MSPError):
        msp.batch_layout(pos, b.offsets, bad, 3.25, 16)


@pytest.mark.parametrize("plan_key", ["exact", "translations", "geo_translations"])
def test_batch_matches_oracle_on_the_common_frame(plan_key, boundary_report):
    """Frames against the oracle on the networks moved into one frame: on a
    dyadic batch that frame is exact, so the problem is the same one."""
    from oracle import oracle as O
    b, w, local, side, level, res = _run(plan_key, dyadic=True)
    wp = b.placed(local, side, level, **PLANS[plan_key])
    exact = local.astype(np.float64) + b.cell_corners(side, level)
    assert np.array_equal(wp.pos.astype(np.float64), exact)   # the premise: no rounding
    o = O.Oracle(wp.params)
    o.build_tree(*wp.arrays())
    uo = o.attraction()
    ro = o.select_partners(4)
    keys, _ = o.keys()
    assert np.array_equal(res["keys"], keys)
    m = (w.vac_axon > 0) & (uo >= 1e-6 * uo.max())
    assert np.max(np.abs(res["u"][m] - uo[m]) / uo[m]) < 1e-5
    if plan_key != "exact":
        assert res["stats"]["n_far"] > 0
    nb = ro["near_boundary"]
    differ = res["partner"] != ro["partner"]
    st = o.stats()
    boundary_report[f"batch_frames_{plan_key}"] = dict(
        band=1e-5 if PLANS[plan_key]["rho_max"] > 0 else 1e-6, draws=st["draws"],
        boundary_draws=st["boundary_draws"], flagged=int(nb.sum()), elements=len(nb),
        differ=int(differ.sum()), differ_flagged=bool(np.all(nb[differ])))
    assert np.all(nb[differ])
    o.close()
    if not nb.any():
        assert res["n_syn"] == ro["n_syn"]
        assert np.array_equal(res["pre"], ro["syn_pre"])
        assert np.array_equal(res["post"], ro["syn_post"])


def test_each_network_matches_its_own_fp64_evaluation(precision_report):
    """Every network of the batch (its own width, its own unscaled positions)
    against the FP64 all-pairs sum of that network alone: the frames keep
    each network at its own single-precision resolution, however wide the
    batch's domain.  Both the search (cutoff 5 sigma: the dropped attraction
    is below exp(-25) of a neighbour's) and the all-pairs path of the batch."""
    from oracle import oracle as O
    b, w, local, side, level, res = _run("wide", dyadic=False)
    worst_u = worst_d = 0.0
    for k in range(len(b.sigma)):
        a, e = b.offsets[k], b.offsets[k + 1]
        wk = b.network(k)
        exact = O.direct(*wk.arrays(), wk.params["sigma"])
        m = (wk.vac_axon > 0) & (exact >= 1e-6 * exact.max())
        worst_u = max(worst_u, np.max(np.abs(res["u"][a:e][m] - exact[m]) / exact[m]))
        worst_d = max(worst_d, np.max(np.abs(res["ud"][a:e][m] - exact[m]) / exact[m]))
        assert np.all(res["ud"][a:e][wk.vac_axon == 0] == 0)
    precision_report["batch_frames_u_vs_fp64_each_network"] = worst_u
    precision_report["batch_frames_direct_vs_fp64_each_network"] = worst_d
    assert worst_u < 1e-5
    assert worst_d < 1e-5


def test_no_partner_or_synapse_crosses_networks():
    b, w, local, side, level, res = _run("wide", dyadic=False)
    net = b.network_of()
    owner = np.repeat(np.arange(b.n), w.vac_axon)
    part = res["partner"]
    ok = part >= 0
    assert ok.mean() > 0.8
    assert np.all(net[part[ok]] == net[owner[ok]])
    assert res["n_syn"] > 0
    assert np.all(net[res["pre"]] == net[res["post"]])


PER_NET = dict(leaf_capacity=[8, 32, 16, 64, 24], cutoff=[2.5, 3.5, 3.0, 4.0, 3.25])


def _ranges(first, count, sel, base):
    return {(int(f) - base, int(c)) for f, c in zip(first[sel], count[sel])}


def test_per_network_plans_match_each_network_alone(precision_report):
    """Every network with its own leaf capacity and cutoff inside the batch:
    its leaves and its near-field box pairs (as point ranges of its sorted
    points) equal those of the oracle run on that network alone, in its
    frame, with its plan, bit for bit; its u agrees within 1e-5; every
    partner lies within its own network's cutoff."""
    from oracle import oracle as O
    b = W.batched_small()
    caps, cuts = PER_NET["leaf_capacity"], PER_NET["cutoff"]
    plan = dict(PLAN, cutoff=max(cuts), leaf_capacity=max(caps))
    local, side, level = _layout(b, **plan)
    w = b.framed(local, side, level, plans=(caps, cuts), **plan)
    g = msp.MSP(w.params, frames=w.frames)
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    sel = g.select_partners(4)
    torch.cuda.synchronize()
    partner = sel["partner"][:g.num_elements()].cpu().numpy()
    tree, pairs = g.export_tree(), g.export_pairs()
    g.close()
    net = b.network_of()
    net_sorted = net[tree["perm"]]
    cell = side / 2.0 ** level
    leaf = tree["child_first"] < 0
    near = pairs["kind"] == 2
    worst = 0.0
    for k in range(len(b.sigma)):
        a, e = int(b.offsets[k]), int(b.offsets[k + 1])
        base = int(np.argmax(net_sorted == k))
        assert np.all(net_sorted[base:base + e - a] == k)      # contiguous in Morton order
        params = W.default_params(cell, sigma=1.0, leaf_capacity=caps[k], cutoff=cuts[k],
                                  rho_max=0.0, p=4, m2l_min_pairs=0, max_depth=21 - level)
        o = O.Oracle(params)
        o.build_tree(np.ascontiguousarray(local[:, a:e]), b.type[a:e], b.vac_axon[a:e],
                     b.vac_dend_e[a:e], b.vac_dend_i[a:e])
        uo = o.attraction()
        on, op = o.nodes(), o.pairs()
        o.close()
        mine = (tree["first"] >= base) & (tree["first"] < base + e - a) & \
            (tree["level"] >= level)
        assert _ranges(tree["first"], tree["count"], leaf & mine, base) == \
            _ranges(on["first"], on["count"], on["child_first"] < 0, 0), k
        X, Y = pairs["X"][near], pairs["Y"][near]
        inX = (tree["first"][X] >= base) & (tree["first"][X] < base + e - a)
        got = {(int(tree["first"][x]) - base, int(tree["count"][x]), int(tree["first"][y]) - base,
                int(tree["count"][y])) for x, y in zip(X[inX], Y[inX])}
        oX, oY = op["X"][op["kind"] == 2], op["Y"][op["kind"] == 2]
        want = {(int(on["first"][x]), int(on["count"][x]), int(on["first"][y]),
                 int(on["count"][y])) for x, y in zip(oX, oY)}
        assert got == want, k
        m = (b.vac_axon[a:e] > 0) & (uo >= 1e-6 * uo.max())
        worst = max(worst, float(np.max(np.abs(u[a:e][m] - uo[m]) / uo[m])))
    precision_report["batch_per_network_plans_u_vs_oracle_alone"] = worst
    assert worst < 1e-5
    owner = np.repeat(np.arange(b.n), b.vac_axon)
    ok = partner >= 0
    assert ok.mean() > 0.5
    assert np.all(net[partner[ok]] == net[owner[ok]])
    d = np.linalg.norm(local[:, owner[ok]].astype(np.float64) -
                       local[:, partner[ok]].astype(np.float64), axis=0)
    lim = np.asarray(cuts)[net[owner[ok]]]
    assert np.all(d < lim * (1 + 1e-5))
    # the radius is each network's own: the wider networks reach past the
    # narrowest network's radius
    assert np.any(d > min(cuts))


def test_count_rule_on_frames_matches_each_network_alone(precision_report):
    """Algorithm 2's count rule (mac_mode 1) on networks in their frames: the
    boxes above the cell level, which span several networks, are never
    translated, so every network gets the pairs of its own count-rule
    evaluation alone (its cell as the root box): the translated-pair count
    equals the oracle's over the networks run alone, and each network's u
    equals the same library's evaluation of that network alone.  (Against
    the oracle the count rule's translations of adjacent boxes, far from
    convergence at 1.3e-1 of the exact sum, amplify single- against
    double-precision rounding to a few 1e-4; that figure is recorded.)"""
    from oracle import oracle as O
    b = _dyadic(W.batched_small())
    plan = dict(PLAN, mac_mode=1, c1=70, c2=70, p=6, leaf_capacity=8)
    local, side, level = _layout(b, **plan)
    w = b.framed(local, side, level, **plan)
    g = msp.MSP(w.params, frames=w.frames)
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    st = g.stats()
    g.close()
    assert st["n_far"] > 0
    cell = side / 2.0 ** level
    worst_gpu = worst_orc = 0.0
    far_orc = far_gpu = 0
    for k in range(len(b.sigma)):
        a, e = int(b.offsets[k]), int(b.offsets[k + 1])
        params = W.default_params(cell, sigma=1.0, max_depth=21 - level,
                                  **{kk: v for kk, v in plan.items()})
        arrays = (np.ascontiguousarray(local[:, a:e]), b.type[a:e], b.vac_axon[a:e],
                  b.vac_dend_e[a:e], b.vac_dend_i[a:e])
        o = O.Oracle(params)
        o.build_tree(*arrays)
        uo = o.attraction()
        far_orc += o.stats()["far_pairs"]
        o.close()
        gk = msp.MSP(params)
        gk.build_tree(*msp.to_device(W.Workload("alone", *arrays, params)))
        ug = gk.attraction().cpu().numpy()
        far_gpu += gk.stats()["n_far"]
        gk.close()
        m = (b.vac_axon[a:e] > 0) & (ug >= 1e-6 * ug.max())
        worst_gpu = max(worst_gpu, float(np.max(np.abs(u[a:e][m] - ug[m]) / ug[m])))
        m = (b.vac_axon[a:e] > 0) & (uo >= 1e-6 * uo.max())
        worst_orc = max(worst_orc, float(np.max(np.abs(u[a:e][m] - uo[m]) / uo[m])))
    precision_report["batch_frames_count_rule_u_vs_same_path_alone"] = worst_gpu
    precision_report["batch_frames_count_rule_u_vs_oracle_alone"] = worst_orc
    assert far_orc == st["n_far"] and far_gpu == st["n_far"]
    assert worst_gpu < 1e-5
    assert worst_orc < 1e-3


def test_frames_check_their_arguments():
    b = W.batched_small()
    local, side, level = _layout(b, **PLAN)
    w = b.framed(local, side, level, **PLAN)
    g = msp.MSP(w.params)
    off = b.offsets
    for args in [(off, 0), (off, 11), (off, w.params["max_depth"]),
                 (np.array([0, 10, b.n]), level),                  # a network of <= 16
                 (np.array([1, b.n]), level),                      # offsets[0] != 0
                 (np.linspace(0, 9 * 100, 10).astype(np.int64), 2)]:   # 9 networks, 8 cells
        with pytest.raises(msp.MSPError) as ei:
            g.set_frames(*args)
        assert ei.value.code == 1
    nn = len(b.sigma)
    for caps, cuts in [([0] * nn, None), ([400] * nn, None),       # a network of 400
                       (None, [0.0] * nn), (None, [5.5] * nn)]:
        with pytest.raises(msp.MSPError) as ei:
            g.set_frames(off, level, caps, cuts)
        assert ei.value.code == 1
    with pytest.raises(ValueError):
        g.set_frames(off, level, [16] * (nn - 1))
    g.close()
    # a cell no wider than the cutoff radius
    g = msp.MSP(dict(w.params, side=2 ** level * 3.0))
    with pytest.raises(msp.MSPError):
        g.set_frames(off, level)
    g.close()
    # the next build must be given offsets[-1] neurons, inside their cells
    g = msp.MSP(w.params, frames=w.frames)
    dev = msp.to_device(w)
    with pytest.raises(msp.MSPError) as ei:
        g.build_tree(dev[0][:, :-1].contiguous(), *[t[:-1].contiguous() for t in dev[1:]])
    assert ei.value.code == 1
    bad = dev[0].clone()
    bad[0, 3] = side / 2 ** level
    with pytest.raises(msp.MSPError) as ei:
        g.build_tree(bad, *dev[1:])
    assert ei.value.code == 1 and "frame" in str(ei.value)
    g.build_tree(*dev)
    u = g.attraction().cpu().numpy()
    assert np.isfinite(u).all() and u.max() > 0
    # without frames the same context takes one common frame again
    g.set_frames(None, 0)
    wp = b.placed(local, side, level, **PLAN)
    g.build_tree(*msp.to_device(wp))
    g.attraction()
    g.close()


def test_batch_plan_chooser_raises_the_cutoff_only_where_needed():
    """The batch plan chooser against each network's own all-pairs
    evaluation: with a tight bar it raises the cutoff of some networks, never
    lowers one, and every network it leaves below the largest candidate
    meets the bar (checked again here from the chosen cutoffs)."""
    from paper_2301_10570_gb300 import autotune
    b = W.batched_small()
    local, side, level = _layout(b, **dict(PLAN, cutoff=max(autotune.BATCH_CUTOFFS)))
    w = b.framed(local, side, level, **PLAN)
    # a bar between the networks' errors at the smallest cutoff: some meet
    # it there, the others need a larger cutoff
    first, rep0 = autotune.tune_batch_cutoffs(w, tol=1.0, ref_err=0.0)
    assert first == [autotune.BATCH_CUTOFFS[0]] * len(b.sigma)
    errs0 = np.asarray(rep0["per_network_max_err"])
    tol = float(np.median(errs0))
    assert tol > 0
    cuts, rep = autotune.tune_batch_cutoffs(w, tol=tol, ref_err=0.0)
    assert len(cuts) == len(b.sigma)
    assert all(c in autotune.BATCH_CUTOFFS for c in cuts)
    assert rep["raised"] >= 1
    assert rep["rounds"][-1]["max_err"] <= rep["rounds"][0]["max_err"]
    wt = b.framed(local, side, level, plans=(None, cuts), **PLAN)
    g = msp.MSP(wt.params, frames=wt.frames)
    g.build_tree(*msp.to_device(wt))
    u = g.attraction().cpu().numpy()
    ud = g.direct().cpu().numpy()
    g.close()
    for k in range(len(b.sigma)):
        if cuts[k] == max(autotune.BATCH_CUTOFFS):
            continue
        a, e = b.offsets[k], b.offsets[k + 1]
        m = (b.vac_axon[a:e] > 0) & (ud[a:e] >= 1e-6 * ud[a:e].max())
        assert np.max(np.abs(u[a:e][m] - ud[a:e][m]) / ud[a:e][m]) <= tol, k
