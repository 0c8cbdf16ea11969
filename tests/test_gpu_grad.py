"""Derivatives of the attraction (the adjoint) through the C ABI.

The pair lists come from a tree built with every count 1 (no box pruned for
being empty), cutoff 5 sigma and no translated pairs; the derivatives are
taken at the workload's real counts.  Bars: against the oracle on the same
lists, single-precision sums vs double (1e-5 relative for u and du/dsigma;
the signed weight gradients 2e-5 of their largest magnitude); against a
central difference of the GPU attraction in sigma (h = 1e-3 relative, so the
difference of two single-precision results carries ~1e-3); against FP64
brute force over all pairs at 16,384 neurons (1e-4).
"""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import msp  # noqa: E402

PLAN = dict(leaf_capacity=32, cutoff=5.0, rho_max=0.0, p=4, m2l_min_pairs=0)


def _gpu_grad(w, g):
    pos, t, a, e, i = msp.to_device(w)
    ones = torch.ones_like(a)
    ctx = msp.MSP(w.params)
    ctx.build_tree(pos, t, ones, ones, ones)
    ctx.attraction()
    out = ctx.attraction_grad(t, a, e, i, g=torch.from_numpy(g).float().cuda())
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items() if v is not None}
    ctx.close()
    return res


def _rel(a, b, floor=1e-6):
    m = np.abs(b) >= floor * np.abs(b).max()
    return np.max(np.abs(a[m] - b[m]) / np.abs(b[m]))


@pytest.mark.parametrize("leaf_capacity", [32, 160])
def test_gradients_match_the_oracle_on_the_same_pairs(leaf_capacity, precision_report):
    # leaves of up to 160 points: passes of more than 32 evaluation points
    # (two per lane) and leaves that take several passes
    from oracle import oracle as O
    w = W.clustered_small(2, 2048, seed=12, **dict(PLAN, leaf_capacity=leaf_capacity))
    g = np.random.default_rng(4).normal(size=w.n)
    r = _gpu_grad(w, g)
    ones = np.ones(w.n, np.uint8)
    o = O.Oracle(w.params)
    o.build_tree(w.pos, w.type, ones, ones, ones)
    o.attraction()
    ro = o.attraction_grad(w.type, w.vac_axon, w.vac_dend_e, w.vac_dend_i, g=g)
    precision_report[f"gradient pass u rel, leaf capacity {leaf_capacity}"] = _rel(r["u"], ro["u"])
    precision_report[f"gradient pass du/dsigma rel, leaf capacity {leaf_capacity}"] = _rel(
        r["du_dsigma"], ro["dudsigma"])
    assert _rel(r["u"], ro["u"]) < 1e-5
    assert _rel(r["du_dsigma"], ro["dudsigma"]) < 1e-5
    for k, ko in (("grad_w_e", "gE"), ("grad_w_i", "gI")):
        e = np.max(np.abs(r[k] - ro[ko])) / np.abs(ro[ko]).max()
        precision_report[f"gradient pass {k} (of largest), leaf capacity {leaf_capacity}"] = e
        assert e < 2e-5, k


def test_dsigma_matches_central_difference_of_the_attraction():
    w = W.clustered_small(1, 4096, seed=13, **PLAN)
    g = np.zeros(w.n)
    r = _gpu_grad(w, g)
    sig, h = w.params["sigma"], 1e-3
    us = []
    for f in (1 + h, 1 - h):
        ctx = msp.MSP(dict(w.params, sigma=sig * f))
        ctx.build_tree(*msp.to_device(w))
        us.append(ctx.attraction().cpu().numpy().astype(np.float64))
        ctx.close()
    fd = (us[0] - us[1]) / (2 * sig * h)
    assert _rel(fd, r["du_dsigma"], floor=1e-3) < 5e-3


def test_gradients_match_fp64_brute_force_at_16k():
    from oracle import oracle as O
    w = W.clustered_small(1, 16_384, seed=14, **PLAN)
    g = np.random.default_rng(5).normal(size=w.n)
    r = _gpu_grad(w, g)
    ref = O.direct_grad(*w.arrays(), w.params["sigma"], g=g)
    assert _rel(r["u"], ref["u"]) < 1e-4
    assert _rel(r["du_dsigma"], ref["dudsigma"]) < 1e-4
    for k, ko in (("grad_w_e", "gE"), ("grad_w_i", "gI")):
        assert np.max(np.abs(r[k] - ref[ko])) < 1e-4 * np.abs(ref[ko]).max(), k


def test_gradients_refuse_translated_pairs_and_missing_g():
    w = W.clustered_small(1, 1536, seed=9, leaf_capacity=8, rho_max=0.3, p=4)
    pos, t, a, e, i = msp.to_device(w)
    ctx = msp.MSP(w.params)
    with pytest.raises(msp.MSPError):
        ctx.attraction_grad(t, a, e, i)                 # no attraction yet
    ctx.build_tree(pos, t, a, e, i)
    ctx.attraction()
    assert ctx.stats()["n_far"] > 0
    with pytest.raises(msp.MSPError):
        ctx.attraction_grad(t, a, e, i)
    ctx.close()
