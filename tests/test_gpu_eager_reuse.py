"""Eager calls on fixed positions keep the octree and the interaction lists.

A context whose next build gets the positions of its last build keeps the
sorted order and the octree (the positions' checksum decides), and an
attraction after such a build keeps the last attraction's lists.  The results
must be those of a fresh context, bit for bit (every sum has a fixed order),
and anything that changes the octree or the lists (a moved neuron, a new
kernel width) must be seen."""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import msp  # noqa: E402


def _fresh(params, dev, step=3):
    g = msp.MSP(params)
    g.build_tree(*dev)
    u = g.attraction().cpu().numpy()
    sel = g.select_partners(step)
    torch.cuda.synchronize()
    part = sel["partner"][:g.num_elements()].cpu().numpy()
    st = g.stats()
    g.close()
    return u, part, st


def _again(g, dev, step=3):
    g.build_tree(*dev)
    u = g.attraction().cpu().numpy()
    sel = g.select_partners(step)
    torch.cuda.synchronize()
    return u, sel["partner"][:g.num_elements()].cpu().numpy(), g.stats()


@pytest.mark.parametrize("plan", [dict(leaf_capacity=32, cutoff=3.25, rho_max=0.0),
                                  dict(leaf_capacity=8, cutoff=4.0, rho_max=0.3, p=4)])
def test_reused_octree_and_lists_equal_a_fresh_context(plan):
    w = W.clustered_small(2, 2048, seed=21, **plan)
    dev = list(msp.to_device(w))
    g = msp.MSP(w.params)
    first = _again(g, dev)
    # new vacancies, same positions: the octree and the lists are kept
    rng = np.random.default_rng(2)
    for k in range(3):
        va = torch.from_numpy(rng.integers(0, 4, w.n).astype(np.uint8)).cuda()
        dev[2] = va
        u, part, st = _again(g, dev, step=10 + k)
        uf, pf, stf = _fresh(w.params, dev, step=10 + k)
        assert np.array_equal(u, uf)
        assert np.array_equal(part, pf)
        assert st["n_pairs"] == stf["n_pairs"] and st["n_p2p"] == stf["n_p2p"]
        assert st["n_far"] == stf["n_far"]
    assert first[2]["n_nodes"] == st["n_nodes"]
    g.close()


def test_a_moved_neuron_rebuilds_the_octree():
    w = W.clustered_small(2, 2048, seed=22, leaf_capacity=32, cutoff=3.25, rho_max=0.0)
    dev = list(msp.to_device(w))
    g = msp.MSP(w.params)
    _again(g, dev)
    moved = w.pos.copy()
    moved[:, 7] = moved[:, 3000]            # onto another neuron's place
    dev[0] = torch.from_numpy(moved).cuda()
    u, part, st = _again(g, dev)
    uf, pf, stf = _fresh(w.params, dev)
    assert np.array_equal(u, uf)
    assert np.array_equal(part, pf)
    g.close()


def test_a_new_kernel_width_drops_the_lists():
    w = W.clustered_small(2, 2048, seed=23, leaf_capacity=32, cutoff=3.25, rho_max=0.0)
    dev = list(msp.to_device(w))
    g = msp.MSP(w.params)
    _again(g, dev)
    g.set_sigma(1.3 * w.params["sigma"])
    u, part, st = _again(g, dev)
    uf, pf, stf = _fresh(dict(w.params, sigma=1.3 * w.params["sigma"]), dev)
    assert np.array_equal(u, uf)
    assert np.array_equal(part, pf)
    assert st["n_pairs"] == stf["n_pairs"]
    g.close()


def test_count_rule_recomputes_its_lists():
    # Algorithm 2's rule depends on the counts: the octree is kept, the
    # traversal redone with the new counts
    w = W.clustered_small(2, 2048, seed=24, leaf_capacity=8, mac_mode=1, c1=70, c2=70, p=4,
                          rho_max=0.0, cutoff=3.25)
    dev = list(msp.to_device(w))
    g = msp.MSP(w.params)
    _again(g, dev)
    dev[3] = torch.zeros_like(dev[3])        # no excitatory dendrites left
    u, part, st = _again(g, dev)
    uf, pf, stf = _fresh(w.params, dev)
    assert np.array_equal(u, uf)
    assert np.array_equal(part, pf)
    assert st["n_far"] == stf["n_far"]
    g.close()
