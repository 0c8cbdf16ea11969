"""Pins of the neuron-side oracle (Section 3.1, Table 1): the properties the
paper states for the model, closed forms and invariants, independent of the
oracle's own code.
"""
import numpy as np
import pytest

from oracle import oracle as O

T1 = O.TABLE1


def test_expf_matches_exp_within_a_few_ulp():
    xs = np.concatenate([np.linspace(-87.0, 0.0, 20001), [-1e-8, -0.5, -1.0, -10.0, -86.9]])
    got = np.array([O.expf(float(np.float32(x))) for x in xs])
    want = np.exp(xs.astype(np.float32).astype(np.float64))
    rel = np.abs(got - want) / want
    assert rel.max() < 3e-7, rel.max()
    assert O.expf(0.0) == 1.0
    assert O.expf(-88.0) == 0.0 and O.expf(-1000.0) == 0.0


@pytest.mark.parametrize("eta", [T1["eta_axon"], T1["eta_dend"]])
def test_growth_curve_zeros_and_maximum(eta):
    # Section 3.1: the curve crosses zero at the left intersection eta (where
    # elements start to grow) and at the right intersection eps (the target),
    # and attains its maximum mu in between; far away it retracts at -mu
    eps, mu = T1["eps"], T1["mu"]
    assert abs(O.growth(eta, eta, eps, mu)) < 1e-6 * mu
    assert abs(O.growth(eps, eta, eps, mu)) < 1e-6 * mu
    mid = 0.5 * (eta + eps)
    g = np.array([O.growth(c, eta, eps, mu) for c in np.linspace(0.0, 1.5, 3001)])
    assert abs(g.max() - mu) < 1e-6 * mu
    assert abs(O.growth(mid, eta, eps, mu) - mu) < 1e-6 * mu
    assert g[0] < 0 and g[-1] < 0
    assert abs(O.growth(50.0, eta, eps, mu) + mu) < 1e-6 * mu
    # positive exactly between the intersections
    cs = np.linspace(0.0, 1.5, 3001)
    inside = (cs > eta + 1e-3) & (cs < eps - 1e-3)
    outside = (cs < eta - 1e-3) | (cs > eps + 1e-3)
    assert np.all(g[inside] > 0) and np.all(g[outside] < 0)


def _state(n, **kw):
    st = dict(x=np.zeros(n, np.float32), refractory=np.zeros(n, np.uint8),
              calcium=np.zeros(n, np.float32), z_axon=np.zeros(n, np.float32),
              z_dend_e=np.zeros(n, np.float32), z_dend_i=np.zeros(n, np.float32),
              spiked=np.zeros(n, np.uint8))
    st.update(kw)
    return st


E0 = (np.zeros(0, np.int32), np.zeros(0, np.int32))


def test_activity_relaxes_to_rest_plus_background():
    # without input, x_{k+1} = x_k + (x0 - x_k)/tau + I has the fixed point
    # x0 + tau I; spikes do not reset the activity
    st = O.neuron_steps(1, 0, 400, O.neuron_params(), *E0, _state(64))
    assert np.allclose(st["x"], T1["x0"] + T1["tau_x"] * T1["background"], rtol=1e-6, atol=0)


def test_spike_rate_of_a_renewal_process_with_refractory_period():
    # at constant activity q a neuron spikes with probability q whenever it is
    # not refractory; after a spike it waits `refractory` steps: the mean
    # interval is refractory + 1/q, the rate q / (1 + refractory q)
    n, steps = 4096, 2000
    pre = O.neuron_params()
    st = O.neuron_steps(7, 0, 300, pre, *E0, _state(n))      # activity settles
    q = float(st["x"][0])
    count = np.zeros(n)
    for k in range(steps // 100):
        st = O.neuron_steps(7, 300 + 100 * k, 1, pre, *E0, st)
        count += st["spiked"]
        st = O.neuron_steps(7, 301 + 100 * k, 99, pre, *E0, st)
    # sample one step in every hundred: the stationary spike probability
    rate = count.sum() / (n * (steps // 100))
    want = q / (1 + T1["refractory"] * q)
    assert abs(rate - want) < 0.1 * want, (rate, want)


def test_refractory_period_is_exact_when_the_neuron_always_fires():
    # activity above 1: every draw fires, so a neuron fires exactly every
    # refractory + 1 steps
    p = O.neuron_params(x0=2.0)
    st = _state(8, x=np.full(8, 2.0, np.float32))
    fired = []
    for k in range(30):
        st = O.neuron_steps(3, k, 1, p, *E0, st)
        fired.append(int(st["spiked"][0]))
    assert fired == ([1] + [0] * T1["refractory"]) * 6


def test_calcium_decay_and_spike_increments():
    # no activity (x0 = I = 0): no spike, Ca_k = Ca_0 (1 - d)^k
    p = O.neuron_params(x0=0.0, background=0.0)
    st = O.neuron_steps(1, 0, 100, p, *E0, _state(4, calcium=np.full(4, 0.5, np.float32)))
    assert st["spiked"].sum() == 0
    assert np.allclose(st["calcium"], 0.5 * (1 - T1["decay_ca"]) ** 100, rtol=2e-5)
    # firing at steps 0, 5, ..., 495 from Ca = 0: after 500 steps each spike
    # has decayed over the steps after it, Ca = beta sum_{j<100} (1-d)^(5j + 4)
    p = O.neuron_params(x0=2.0)
    st = O.neuron_steps(1, 0, 500, p, *E0, _state(4, x=np.full(4, 2.0, np.float32)))
    d, b = T1["decay_ca"], T1["beta_ca"]
    want = b * sum((1 - d) ** (5 * j + 4) for j in range(100))
    assert np.allclose(st["calcium"], want, rtol=1e-4)


def test_input_adds_a_fixed_amount_per_spiking_partner():
    # neuron 0 spiked in the previous step; neuron 1 receives m edges from it
    n, m = 4, 5
    pre = np.zeros(m, np.int32)
    post = np.ones(m, np.int32)
    p = O.neuron_params(x0=0.0, background=0.0)
    a = O.neuron_steps(1, 0, 1, p, pre, post, _state(n, spiked=np.array([1, 0, 0, 0], np.uint8)))
    b = O.neuron_steps(1, 0, 1, p, *E0, _state(n, spiked=np.array([1, 0, 0, 0], np.uint8)))
    assert abs(float(a["x"][1]) - float(b["x"][1]) - m * T1["input_per_spike"]) < 1e-9
    assert a["x"][2] == b["x"][2]


def test_elements_grow_at_target_free_calcium():
    # calcium between eta_dend and eta_axon: dendrites grow, axons retract
    # (and stay at zero)
    ca = np.full(4, 0.25, np.float32)
    p = O.neuron_params(x0=0.0, background=0.0, decay_ca=0.0)
    st = O.neuron_steps(1, 0, 100, p, *E0, _state(4, calcium=ca))
    assert np.all(st["z_axon"] == 0)
    assert np.all(st["z_dend_e"] > 0) and np.all(st["z_dend_e"] == st["z_dend_i"])
    g = O.growth(0.25, T1["eta_dend"], T1["eps"], T1["mu"])
    assert np.allclose(st["z_dend_e"], 100 * g, rtol=1e-4)


def _random_edges(rng, n, m):
    pre = rng.integers(0, n, m).astype(np.int32)
    post = rng.integers(0, n, m).astype(np.int32)
    typ = rng.integers(0, 2, m).astype(np.uint8)
    return pre, post, typ


def test_deletion_leaves_no_side_over_its_elements_and_keeps_order():
    rng = np.random.default_rng(3)
    n, m = 200, 3000
    pre, post, typ = _random_edges(rng, n, m)
    z = [rng.uniform(0, 25, n).astype(np.float32) for _ in range(3)]
    (p2, q2, t2), (va, ve, vi) = O.update_synapses(11, 4, *z, pre, post, typ)
    fz = [np.floor(v).astype(np.int64) for v in z]
    out = np.bincount(p2, minlength=n)
    inE = np.bincount(q2[t2 == 0], minlength=n)
    inI = np.bincount(q2[t2 == 1], minlength=n)
    assert np.all(out <= fz[0]) and np.all(inE <= fz[1]) and np.all(inI <= fz[2])
    assert np.array_equal(va, np.clip(fz[0] - out, 0, 255))
    assert np.array_equal(ve, np.clip(fz[1] - inE, 0, 255))
    assert np.array_equal(vi, np.clip(fz[2] - inI, 0, 255))
    # the kept edges are a subsequence of the original list
    keys = list(zip(pre.tolist(), post.tolist(), typ.tolist()))
    j = 0
    for e in zip(p2.tolist(), q2.tolist(), t2.tolist()):
        while keys[j] != e:
            j += 1
        j += 1
    # an edge goes only if one of its sides had too many synapses
    bo = np.bincount(pre, minlength=n)
    bi = np.bincount(2 * post + typ, minlength=2 * n)
    over_out = bo > fz[0]
    over_in = bi > np.stack([fz[1], fz[2]], 1).reshape(-1)
    kept = np.zeros(m, bool)
    j = 0
    for i, e in enumerate(keys):
        if j < len(p2) and e == (int(p2[j]), int(q2[j]), int(t2[j])):
            kept[i] = True
            j += 1
    gone = ~kept
    assert np.all(over_out[pre[gone]] | over_in[2 * post[gone] + typ[gone]])
    # a side with excess keeps exactly floor(z) unless the other side took more
    ok_out = over_out & ~np.isin(np.arange(n), pre[gone & over_in[2 * post + typ]])
    assert np.all(out[ok_out] == fz[0][ok_out])


def test_deletion_chooses_uniformly():
    # one neuron with 10 outgoing synapses and 7 axonal elements deletes 3,
    # each with probability 3/10
    n = 12
    pre = np.zeros(10, np.int32)
    post = np.arange(1, 11, dtype=np.int32)
    typ = np.zeros(10, np.uint8)
    za = np.zeros(n, np.float32)
    za[0] = 7.5
    zd = np.full(n, 5.0, np.float32)
    hits = np.zeros(10)
    trials = 3000
    for s in range(trials):
        (p2, q2, _), _ = O.update_synapses(s, 0, za, zd, zd, pre, post, typ)
        assert len(p2) == 7
        hits[np.setdiff1d(post, q2) - 1] += 1
    freq = hits / trials
    assert np.all(np.abs(freq - 0.3) < 0.04), freq
