"""Many independent networks as one problem (the batched step).

The layout scales each network by 1/sigma and places it in its own octree
cell with an empty cell between networks.  Checks: the placement itself; the
whole batch through the CUDA path against the oracle run on the same placed
problem (the usual parity bars); and independence: every network's
attraction equals its own all-pairs evaluation at its own kernel width, and
no partner or synapse crosses networks.
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


def _placed(b, **plan):
    pos = torch.from_numpy(b.pos).cuda()
    placed, side, level = msp.batch_layout(pos, b.offsets, b.sigma, plan["cutoff"],
                                           plan["leaf_capacity"])
    return b.placed(placed.cpu().numpy(), side, **plan), side, level


_cache = {}


def _run(plan_key="exact"):
    if plan_key in _cache:
        return _cache[plan_key]
    plan = {"exact": dict(PLAN), "translations": dict(PLAN, rho_max=0.3, leaf_capacity=8),
            "wide": dict(PLAN, cutoff=5.0)}[plan_key]
    b = W.batched_small()
    w, side, level = _placed(b, **plan)
    g = msp.MSP(w.params)
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    sel = g.select_partners(4)
    torch.cuda.synchronize()
    ne = g.num_elements()
    ns = int(sel["n_syn"].item())
    res = dict(u=u, partner=sel["partner"][:ne].cpu().numpy(), n_syn=ns,
               pre=sel["syn_pre"][:ns].cpu().numpy(), post=sel["syn_post"][:ns].cpu().numpy(),
               typ=sel["syn_type"][:ns].cpu().numpy(), keys=g.export_tree()["keys"],
               stats=g.stats())
    g.close()
    _cache[plan_key] = (b, w, side, level, res)
    return _cache[plan_key]


def test_layout_scales_and_separates_networks():
    b = W.batched_small()
    w, side, level = _placed(b, **PLAN)
    cell = side / 2.0 ** level
    G = 2 ** (level - 1)
    for k in range(len(b.sigma)):
        a, e = b.offsets[k], b.offsets[k + 1]
        src = b.pos[:, a:e].astype(np.float64)
        lo = src.min(axis=1, keepdims=True)
        c = np.array([k % G, (k // G) % G, k // (G * G)], np.float64)[:, None]
        want = 2 * c * cell + (src - lo) / b.sigma[k]
        got = w.pos[:, a:e].astype(np.float64)
        assert np.max(np.abs(got - want)) < 1e-5 * side
        # inside its own (even) cell
        assert np.all(got >= 2 * c * cell - 1e-6 * side)
        assert np.all(got < (2 * c + 1) * cell)
    # any two networks are more than the cutoff apart (sigma units)
    net = b.network_of()
    cells = np.floor(w.pos / cell).astype(np.int64)
    for k in range(len(b.sigma)):
        assert len(np.unique(cells[:, net == k], axis=1).T) >= 1
        assert np.all(cells[:, net == k] % 2 == 0)


def test_layout_rejects_small_networks_and_bad_widths():
    b = W.batched_small()
    pos = torch.from_numpy(b.pos).cuda()
    with pytest.raises(msp.MSPError):
        msp.batch_layout(pos, b.offsets, b.sigma, 3.25, 1000)      # a network of <= 1000
    bad = b.sigma.copy()
    bad[2] = 0.0
    with pytest.raises(msp.MSPError):
        msp.batch_layout(pos, b.offsets, bad, 3.25, 16)


@pytest.mark.parametrize("plan_key", ["exact", "translations"])
def test_batch_matches_oracle_on_the_placed_problem(plan_key):
    from oracle import oracle as O
    b, w, side, level, res = _run(plan_key)
    o = O.Oracle(w.params)
    o.build_tree(*w.arrays())
    uo = o.attraction()
    ro = o.select_partners(4)
    keys, _ = o.keys()
    assert np.array_equal(res["keys"], keys)
    m = (w.vac_axon > 0) & (uo >= 1e-6 * uo.max())
    assert np.max(np.abs(res["u"][m] - uo[m]) / uo[m]) < 1e-5
    ok = ~ro["near_boundary"]
    assert np.array_equal(res["partner"][ok], ro["partner"][ok])
    if not ro["near_boundary"].any():
        assert res["n_syn"] == ro["n_syn"]
        assert np.array_equal(res["pre"], ro["syn_pre"])
        assert np.array_equal(res["post"], ro["syn_post"])


def test_networks_are_independent():
    # cutoff 5 sigma: the dropped attraction (below exp(-25) of a neighbour's)
    # is far below single precision, so each network's u must equal its own
    # all-pairs evaluation within the library's bar against brute force (both
    # are single-precision sums in different orders: ~3e-5 observed on dense
    # clusters)
    b, w, side, level, res = _run("wide")
    net = b.network_of()
    owner = np.repeat(np.arange(b.n), w.vac_axon)
    part = res["partner"]
    ok = part >= 0
    assert ok.mean() > 0.8
    assert np.all(net[part[ok]] == net[owner[ok]])
    assert np.all(net[res["pre"]] == net[res["post"]])
    # each network's attraction is its own all-pairs evaluation at its own width
    for k in range(len(b.sigma)):
        a, e = b.offsets[k], b.offsets[k + 1]
        wk = b.network(k)
        gk = msp.MSP(wk.params)
        gk.build_tree(*msp.to_device(wk))
        ud = gk.direct().cpu().numpy()
        gk.close()
        ub = res["u"][a:e]
        m = (wk.vac_axon > 0) & (ud >= 1e-6 * ud.max())
        assert np.max(np.abs(ub[m] - ud[m]) / ud[m]) < 1e-4, k
