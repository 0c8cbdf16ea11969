"""The neuron side of the model (Section 3.1, Table 1) through the C ABI,
against the oracle on the same inputs: activity, spikes, calcium and
elements bit for bit over hundreds of steps; synapse deletion and vacancies
bit for bit; the whole simulation loop (neuron steps, deletion, synapse
search, append) over several connectivity updates; argument errors.
"""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import oracle as O  # noqa: E402
from paper_2301_10570_gb300 import msp  # noqa: E402

PLAN = dict(leaf_capacity=32, cutoff=3.25, rho_max=0.0, p=4, m2l_min_pairs=0)


def _random_state(rng, n):
    return dict(x=rng.uniform(0, 0.3, n).astype(np.float32),
                refractory=rng.integers(0, 5, n).astype(np.uint8),
                calcium=rng.uniform(0, 1.0, n).astype(np.float32),
                z_axon=rng.uniform(0, 10, n).astype(np.float32),
                z_dend_e=rng.uniform(0, 10, n).astype(np.float32),
                z_dend_i=rng.uniform(0, 10, n).astype(np.float32),
                spiked=(rng.random(n) < 0.1).astype(np.uint8))


def _to_dev(st):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in st.items()}


def _same(a, b):
    a, b = np.asarray(a), np.asarray(b)
    if a.dtype == np.float32:
        return np.array_equal(a.view(np.uint32), b.view(np.uint32))
    return np.array_equal(a, b)


def _ctx(**kw):
    w = W.uniform_4k(**PLAN)
    return msp.MSP(dict(w.params, **kw))


def _to_dev_offset(st):
    # views that start one element into a larger buffer (no 16-byte alignment)
    out = {}
    for k, v in st.items():
        buf = torch.zeros(len(v) + 1, dtype=torch.from_numpy(v[:1]).dtype, device="cuda")
        buf[1:] = torch.from_numpy(np.ascontiguousarray(v)).cuda()
        out[k] = buf[1:]
    return out


@pytest.mark.parametrize("input_per_spike,n,aligned", [(5e-4, 5000, True), (0.02, 5000, True),
                                                       (0.02, 5003, True), (0.02, 5000, False)])
def test_neuron_steps_match_the_oracle_bit_for_bit(input_per_spike, n, aligned):
    # four neurons per thread with 16-byte accesses where the arrays allow it,
    # one per thread for the remainder and for unaligned arrays
    rng = np.random.default_rng(31)
    m = 25_000
    pre = rng.integers(0, n, m).astype(np.int32)
    post = rng.integers(0, n, m).astype(np.int32)
    st = _random_state(rng, n)
    kw = dict(input_per_spike=input_per_spike)
    want = O.neuron_steps(17, 40, 300, O.neuron_params(**kw), pre, post, st)
    g = _ctx(seed=17)
    edges = msp.edge_list(m, pre=pre, post=post, type_=np.zeros(m, np.uint8))
    dev = _to_dev(st) if aligned else _to_dev_offset(st)
    g.neuron_steps(40, 300, msp.neuron_params(**kw), edges, dev)
    torch.cuda.synchronize()
    g.close()
    for k, _ in msp.NEURON_STATE:
        assert _same(dev[k].cpu().numpy(), want[k]), k
    assert want["spiked"].sum() > 0


def test_update_synapses_matches_the_oracle_bit_for_bit():
    rng = np.random.default_rng(32)
    n, m = 3000, 40_000
    pre = rng.integers(0, n, m).astype(np.int32)
    post = rng.integers(0, n, m).astype(np.int32)
    typ = rng.integers(0, 2, m).astype(np.uint8)
    st = _random_state(rng, n)
    for k in ("z_axon", "z_dend_e", "z_dend_i"):
        st[k] = rng.uniform(0, 20, n).astype(np.float32)
    (p2, q2, t2), (va, ve, vi) = O.update_synapses(5, 9, st["z_axon"], st["z_dend_e"],
                                                   st["z_dend_i"], pre, post, typ)
    assert 0 < len(p2) < m
    g = _ctx(seed=5)
    edges = msp.edge_list(m + 100, pre=pre, post=post, type_=typ)
    dev = _to_dev(st)
    vac = [torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(3)]
    g.update_synapses(9, dev, edges, *vac)
    torch.cuda.synchronize()
    k = int(edges["n"].item())
    assert k == len(p2)
    assert _same(edges["pre"][:k].cpu().numpy(), p2)
    assert _same(edges["post"][:k].cpu().numpy(), q2)
    assert _same(edges["type"][:k].cpu().numpy(), t2)
    for got, ref in zip(vac, (va, ve, vi)):
        assert _same(got.cpu().numpy(), ref)
    g.close()


def test_empty_edge_list_and_errors():
    rng = np.random.default_rng(33)
    n = 100
    st = _random_state(rng, n)
    g = _ctx(seed=1)
    edges = msp.edge_list(10)
    dev = _to_dev(st)
    g.neuron_steps(0, 5, msp.neuron_params(), edges, dev)
    want = O.neuron_steps(1, 0, 5, O.neuron_params(), np.zeros(0, np.int32),
                          np.zeros(0, np.int32), st)
    assert _same(dev["x"].cpu().numpy(), want["x"])
    vac = [torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(3)]
    g.update_synapses(0, dev, edges, *vac)
    assert int(edges["n"].item()) == 0
    # an edge naming a neuron outside [0, n) is refused and nothing changes
    bad = msp.edge_list(10, pre=[0, 1], post=[2, n], type_=[0, 0])
    with pytest.raises(msp.MSPError) as ei:
        g.update_synapses(0, dev, bad, *vac)
    assert ei.value.code == 1
    assert int(bad["n"].item()) == 2
    # appending beyond the capacity keeps what fits and reports it
    sel = dict(n_syn=torch.tensor([5], dtype=torch.int64, device="cuda"),
               syn_pre=torch.arange(5, dtype=torch.int32, device="cuda"),
               syn_post=torch.arange(5, dtype=torch.int32, device="cuda"),
               syn_type=torch.zeros(5, dtype=torch.uint8, device="cuda"))
    small = msp.edge_list(3)
    with pytest.raises(msp.MSPError) as ei:
        g.append_synapses(sel, small)
    assert ei.value.code == 7
    assert int(small["n"].item()) == 3
    assert small["pre"][:3].tolist() == [0, 1, 2]
    ok = msp.edge_list(8, pre=[7], post=[7], type_=[1])
    g.append_synapses(sel, ok)
    assert int(ok["n"].item()) == 6 and ok["pre"][:6].tolist() == [7, 0, 1, 2, 3, 4]
    with pytest.raises(msp.MSPError):
        g.neuron_steps(0, 1, msp.neuron_params(refractory=300), edges, dev)
    g.close()


def test_simulation_loop_matches_the_oracle():
    # 100 neuron steps, deletion, the synapse search on the resulting
    # vacancies, append; three connectivity updates, compared after each
    w = W.clustered_small(2, 2048, seed=34, **PLAN)
    n = w.n
    rng = np.random.default_rng(35)
    m0 = 2 * n
    pre = rng.integers(0, n, m0).astype(np.int32)
    post = rng.integers(0, n, m0).astype(np.int32)
    typ = w.type[pre].astype(np.uint8)
    st = _random_state(rng, n)
    # elements a little above the bound synapses: some vacant, some in excess
    bo = np.bincount(pre, minlength=n)
    bi = np.bincount(2 * post + typ, minlength=2 * n)
    st["z_axon"] = (bo + rng.uniform(-1.0, 2.5, n)).clip(0).astype(np.float32)
    st["z_dend_e"] = (bi[0::2] + rng.uniform(-1.0, 2.5, n)).clip(0).astype(np.float32)
    st["z_dend_i"] = (bi[1::2] + rng.uniform(-1.0, 2.5, n)).clip(0).astype(np.float32)
    params = dict(input_per_spike=0.01, mu=5e-3)
    # oracle
    o_st = dict(st)
    o_edges = (pre.copy(), post.copy(), typ.copy())
    g = msp.MSP(w.params)
    d_st = _to_dev(st)
    edges = msp.edge_list(20 * n, pre=pre, post=post, type_=typ)
    pos, t_dev = msp.to_device(w)[:2]
    vac = [torch.zeros(n, dtype=torch.uint8, device="cuda") for _ in range(3)]
    compared = 0
    for cycle in range(3):
        o_st = O.neuron_steps(w.params["seed"], 100 * cycle, 100, O.neuron_params(**params),
                              o_edges[0], o_edges[1], o_st)
        o_edges, (va, ve, vi) = O.update_synapses(w.params["seed"], cycle, o_st["z_axon"],
                                                  o_st["z_dend_e"], o_st["z_dend_i"],
                                                  *o_edges)
        o = O.Oracle(w.params)
        o.build_tree(w.pos, w.type, va, ve, vi)
        o.attraction()
        ro = o.select_partners(cycle)
        o_edges = tuple(np.concatenate([a, b]) for a, b in
                        zip(o_edges, (ro["syn_pre"], ro["syn_post"], ro["syn_type"])))
        # GPU
        g.neuron_steps(100 * cycle, 100, msp.neuron_params(**params), edges, d_st)
        g.update_synapses(cycle, d_st, edges, *vac)
        for a, b in zip(vac, (va, ve, vi)):
            assert _same(a.cpu().numpy(), b), cycle
        g.build_tree(pos, t_dev, *vac)
        g.attraction()
        sel = g.select_partners(cycle)
        g.append_synapses(sel, edges)
        torch.cuda.synchronize()
        for k, _ in msp.NEURON_STATE:
            assert _same(d_st[k].cpu().numpy(), o_st[k]), (cycle, k)
        if ro["near_boundary"].any():
            break       # a draw within rounding of a boundary: the runs may part here
        k = int(edges["n"].item())
        assert k == len(o_edges[0]), cycle
        for a, b in zip(("pre", "post", "type"), o_edges):
            assert _same(edges[a][:k].cpu().numpy(), b), (cycle, a)
        compared += 1
    g.close()
    assert compared >= 1


def test_neuron_steps_full_size_bit_exact():
    # the simulation benchmark's size: 1,048,576 neurons, 1.5 synapses each,
    # 20 steps; every state array bit for bit against the oracle
    rng = np.random.default_rng(36)
    n = 1 << 20
    m = 3 * n // 2
    pre = rng.integers(0, n, m).astype(np.int32)
    post = rng.integers(0, n, m).astype(np.int32)
    st = _random_state(rng, n)
    kw = dict(input_per_spike=0.02)
    want = O.neuron_steps(19, 1000, 20, O.neuron_params(**kw), pre, post, st)
    g = _ctx(seed=19)
    edges = msp.edge_list(m, pre=pre, post=post, type_=np.zeros(m, np.uint8))
    dev = _to_dev(st)
    g.neuron_steps(1000, 20, msp.neuron_params(**kw), edges, dev)
    torch.cuda.synchronize()
    g.close()
    for k, _ in msp.NEURON_STATE:
        assert _same(dev[k].cpu().numpy(), want[k]), k
