"""The expected mean synapse length, its loss and gradients through the C ABI
(msp_length_loss), the autograd wrapper and the calibration of sigma.

Pair lists from a tree built with every count 1, cutoff 5 sigma, no
translated pairs.  Bars: against the oracle on the same lists (single
precision sums with compensated chunks against double: 1e-5 relative for the
mean, the loss and the sigma derivatives, 1e-4 of the largest magnitude for
the signed weight gradients); against central differences of the GPU loss
(h = 1e-3 relative: the difference of two single precision results carries
~1e-3 of the derivative); against FP64 brute force over all pairs at 16,384
neurons (1e-4 relative, 2e-4 of the largest weight gradient).
"""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import calibrate, msp  # noqa: E402

PLAN = dict(leaf_capacity=32, cutoff=5.0, rho_max=0.0, p=4, m2l_min_pairs=0)
TARGET = 1000.0


def _weights(w, seed=3):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.2, 3.0, w.n), rng.uniform(0.2, 3.0, w.n)


def _ctx(w):
    pos, t, a, e, i = msp.to_device(w)
    ones = torch.ones_like(a)
    ctx = msp.MSP(w.params)
    ctx.build_tree(pos, t, ones, ones, ones)
    ctx.attraction()
    return ctx, t, a


def _gpu(ctx, t, a, we, wi, grad=True):
    r = ctx.length_loss(t, a, torch.from_numpy(we).float().cuda(),
                        torch.from_numpy(wi).float().cuda(), TARGET, grad=grad)
    if grad:
        r["gE"] = r["gE"].cpu().numpy().astype(np.float64)
        r["gI"] = r["gI"].cpu().numpy().astype(np.float64)
    return r


@pytest.mark.parametrize("leaf_capacity", [32, 160])
def test_length_loss_matches_the_oracle_on_the_same_pairs(leaf_capacity, precision_report):
    from oracle import oracle as O
    w = W.clustered_small(2, 2048, seed=12, **dict(PLAN, leaf_capacity=leaf_capacity))
    we, wi = _weights(w)
    ctx, t, a = _ctx(w)
    r = _gpu(ctx, t, a, we, wi)
    ctx.close()
    ones = np.ones(w.n, np.uint8)
    o = O.Oracle(w.params)
    o.build_tree(w.pos, w.type, ones, ones, ones)
    o.attraction()
    ro = o.length_loss(w.type, w.vac_axon, we.astype(np.float32), wi.astype(np.float32), TARGET)
    for key in ("mean", "loss", "dmean_dsigma", "dloss_dsigma"):
        precision_report[f"length loss {key} rel, leaf capacity {leaf_capacity}"] = abs(
            r[key] - ro[key]) / abs(ro[key])
        assert r[key] == pytest.approx(ro[key], rel=1e-5), key
    for key in ("gE", "gI"):
        e = np.max(np.abs(r[key] - ro[key])) / np.abs(ro[key]).max()
        precision_report[f"length loss {key} (of largest), leaf capacity {leaf_capacity}"] = e
        assert e <= 1e-4, key


def test_length_loss_against_central_differences():
    """dloss/dsigma against the central difference of the GPU loss (the
    lists redone at sigma (1 +- 1e-3)), and the weight gradient along a
    random direction (every weight moved by 1e-3 relative)."""
    w = W.clustered_small(2, 2048, seed=14, **PLAN)
    we, wi = _weights(w, 5)
    ctx, t, a = _ctx(w)
    r = _gpu(ctx, t, a, we, wi)
    sig = w.params["sigma"]
    h = 1e-3
    vals = []
    for f in (1 + h, 1 - h):
        ctx.set_sigma(sig * f)
        ctx.attraction()
        vals.append(_gpu(ctx, t, a, we, wi, grad=False)["mean"])
    fd = (vals[0] - vals[1]) / (2 * h * sig)
    assert fd == pytest.approx(r["dmean_dsigma"], rel=2e-2)
    ctx.set_sigma(sig)
    ctx.attraction()
    dirn = np.random.default_rng(6).choice([-1.0, 1.0], size=(2, w.n))
    dE, dI = 1e-3 * we * dirn[0], 1e-3 * wi * dirn[1]
    up = _gpu(ctx, t, a, we + dE, wi + dI, grad=False)["loss"]
    dn = _gpu(ctx, t, a, we - dE, wi - dI, grad=False)["loss"]
    fd_w = (up - dn) / 2
    pred = float(r["gE"] @ dE + r["gI"] @ dI)
    assert fd_w == pytest.approx(pred, rel=2e-2)
    ctx.close()


def test_length_loss_against_fp64_brute_force_at_16k():
    from oracle import oracle as O
    w = W.clustered_small(1, 16_384, seed=16, **dict(PLAN, leaf_capacity=64))
    we, wi = _weights(w, 7)
    ctx, t, a = _ctx(w)
    r = _gpu(ctx, t, a, we, wi)
    ctx.close()
    ref = O.direct_length_loss(w.pos, w.type, w.vac_axon, we.astype(np.float32),
                               wi.astype(np.float32), w.params["sigma"], TARGET)
    for key in ("mean", "loss", "dmean_dsigma", "dloss_dsigma"):
        assert r[key] == pytest.approx(ref[key], rel=1e-4), key
    for key in ("gE", "gI"):
        assert np.max(np.abs(r[key] - ref[key])) <= 2e-4 * np.abs(ref[key]).max(), key


def test_autograd_function_gives_the_library_gradient():
    w = W.clustered_small(1, 4096, seed=18, **PLAN)
    we, wi = _weights(w, 9)
    ctx, t, a = _ctx(w)
    sigma = torch.tensor(800.0, dtype=torch.float64, requires_grad=True)
    wE = torch.from_numpy(we).float().cuda().requires_grad_(True)
    wI = torch.from_numpy(wi).float().cuda().requires_grad_(True)
    loss = msp.SynapseLengthLoss.apply(sigma, wE, wI, ctx, t, a, TARGET)
    (3.0 * loss).backward()
    ctx.set_sigma(800.0)
    ctx.attraction()
    r = _gpu(ctx, t, a, we, wi)
    assert loss.item() == pytest.approx(r["loss"], rel=1e-12)
    assert sigma.grad.item() == pytest.approx(3.0 * r["dloss_dsigma"], rel=1e-12)
    assert np.allclose(wE.grad.cpu().numpy(), 3.0 * r["gE"], rtol=1e-6, atol=0)
    assert np.allclose(wI.grad.cpu().numpy(), 3.0 * r["gI"], rtol=1e-6, atol=0)
    ctx.close()


def test_sigma_calibration_reaches_the_target_length():
    """Newton steps on m(sigma) - 1000 um from sigma = 750 um: the mean
    synapse length of the calibrated sigma is within 1e-4 of the target, and
    the oracle's all-pairs mean at that sigma agrees."""
    from oracle import oracle as O
    w = W.clustered_small(1, 8192, seed=20, **PLAN)
    we, wi = _weights(w, 11)
    ctx, t, a = _ctx(w)
    wE = torch.from_numpy(we).float().cuda()
    wI = torch.from_numpy(wi).float().cuda()
    sigma, hist = calibrate.calibrate_sigma(ctx, t, a, wE, wI, TARGET, sigma0=750.0)
    ctx.close()
    assert len(hist) <= 8
    assert abs(hist[-1][1] - TARGET) <= 1e-4 * TARGET
    ref = O.direct_length_loss(w.pos, w.type, w.vac_axon, we.astype(np.float32),
                               wi.astype(np.float32), sigma, TARGET, grad=False)
    assert ref["mean"] == pytest.approx(TARGET, rel=3e-4)
