"""The whole plasticity step as one CUDA graph (walk, build, attraction,
selection, commit) against the same steps issued as separate eager calls.

Both sides run the same kernels; the graph takes its launch shapes from
capacity bounds and its step index from device memory, neither of which
changes a result, so the per-step synapse counts, the final vacancy state
and the last step's partners and synapse lists must be identical.  The halt
test forces a pair-table overflow inside a replay (a capacity far below the
pairs of a step with vacancies) and checks that the halted step is finished
eagerly with the same result.
"""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import msp  # noqa: E402


def _state(w):
    pos, t, a, e, i = msp.to_device(w)
    return pos, t, a.clone(), e.clone(), i.clone()


def _eager(w, first, k_steps):
    """Steps first .. first+k_steps-1 as separate calls; returns per-step
    synapse counts, the final state and the last step's selection."""
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params, frames=w.frames)
    counts = []
    sel = None
    for k in range(first, first + k_steps):
        g.vacancy_walk(k, a, e, i)
        g.build_tree(pos, t, a, e, i)
        g.attraction()
        sel = g.select_partners(k)
        g.commit_synapses(sel, a, e, i)
        counts.append(int(sel["n_syn"].item()))
    ne = g.num_elements()
    last = dict(partner=sel["partner"][:ne].cpu().numpy(), n_syn=counts[-1],
                pre=sel["syn_pre"][:counts[-1]].cpu().numpy(),
                post=sel["syn_post"][:counts[-1]].cpu().numpy(),
                typ=sel["syn_type"][:counts[-1]].cpu().numpy())
    g.close()
    return counts, [v.cpu().numpy() for v in (a, e, i)], last


def _graph(w, first, k_steps, pair_capacity=None, manual=False, full_build=False):
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params, frames=w.frames)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    if pair_capacity is not None:
        g.set_pair_capacity(pair_capacity)
    g.step_graph_set_full_build(full_build)
    out = g.step_graph_capture(pos, t, a, e, i, first_step=first, history_len=k_steps)
    halts = []
    if manual:
        step, end = first, first + k_steps
        while step < end:
            g.step_graph_launch(end - step)
            step, h = g.step_graph_finish()
            halts.append(h)
    else:
        assert g.run_steps(first, k_steps) == first + k_steps
    st = g.stats()
    counts = out["history"].cpu().numpy().tolist()
    ns = counts[-1]
    last = dict(n_syn=ns, pre=out["syn_pre"][:ns].cpu().numpy(),
                post=out["syn_post"][:ns].cpu().numpy(), typ=out["syn_type"][:ns].cpu().numpy(),
                partner_all=out["partner"].cpu().numpy(), n_elem=st["n_elements"])
    res = (counts, [v.cpu().numpy() for v in (a, e, i)], last, st, halts)
    g.close()
    return res


def _workload():
    return W.clustered_small(2, 2048, seed=11, leaf_capacity=32)


def test_graph_replays_equal_eager_steps():
    w = _workload()
    k_steps = 6
    ce, se, le = _eager(w, 3, k_steps)
    cg, sg, lg, st, _ = _graph(w, 3, k_steps)
    assert cg == ce
    for x, y in zip(sg, se):
        assert np.array_equal(x, y)
    assert lg["n_elem"] == len(le["partner"])
    assert np.array_equal(lg["partner_all"][:lg["n_elem"]], le["partner"])
    for key in ("pre", "post", "typ"):
        assert np.array_equal(lg[key], le[key])
    assert st["near_field_ms"] > 0.0 and st["p2p_interactions"] > 0


def test_graph_lists_do_not_depend_on_the_vacancies():
    """No vacant axons when the graph is captured: the pair lists depend on the
    positions only (no pair is dropped for empty counts), so the replays, whose
    walk then creates vacant axons, need no larger table and never halt, and
    they equal the eager steps."""
    w = _workload()
    w.vac_axon[:] = 0
    k_steps = 4
    ce, se, _ = _eager(w, 0, k_steps)
    cg, sg, _, st, halts = _graph(w, 0, k_steps, manual=True)
    assert halts == [0], halts
    assert sum(ce) > 0 and cg == ce
    for x, y in zip(sg, se):
        assert np.array_equal(x, y)


def test_graph_with_moved_positions_halts_and_rebuilds():
    # graph steps reuse the octree of the eager build (neurons do not move);
    # positions changed after the capture are detected by their checksum:
    # the replay halts (the tree bit) and the step is finished eagerly on a
    # new tree, so the run equals eager steps on the new positions
    w = _workload()
    moved = W.clustered_small(2, 2048, seed=11, leaf_capacity=32)
    moved.pos[:, 10] = moved.pos[:, 500]         # one neuron onto another's place
    k_steps = 3
    ce, se, _ = _eager(moved, 0, k_steps)
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    out = g.step_graph_capture(pos, t, a, e, i, first_step=0, history_len=k_steps)
    pos.copy_(torch.from_numpy(moved.pos).cuda())
    step, halts = 0, []
    while step < k_steps:
        g.step_graph_launch(k_steps - step)
        step, h = g.step_graph_finish()
        halts.append(h)
    assert halts[0] & 4, halts
    assert out["history"].cpu().numpy().tolist() == ce
    for x, y in zip([v.cpu().numpy() for v in (a, e, i)], se):
        assert np.array_equal(x, y)
    g.close()


def test_graph_detects_a_move_in_the_leading_bits_of_z():
    # a neuron moved by doubling its z coordinate (same mantissa, next
    # exponent): the positions' checksum covers every bit of every coordinate,
    # so the replay halts and the step is finished on a new tree
    w = _workload()
    moved = W.clustered_small(2, 2048, seed=11, leaf_capacity=32)
    side = moved.params["side"]
    j = int(np.argmax((moved.pos[2] > 0.05 * side) & (moved.pos[2] < 0.45 * side)))
    moved.pos[2, j] = moved.pos[2, j] * np.float32(2.0)
    assert 0 < moved.pos[2, j] < side
    ce, se, _ = _eager(moved, 0, 2)
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    out = g.step_graph_capture(pos, t, a, e, i, first_step=0, history_len=2)
    pos.copy_(torch.from_numpy(moved.pos).cuda())
    step, halts = 0, []
    while step < 2:
        g.step_graph_launch(2 - step)
        step, h = g.step_graph_finish()
        halts.append(h)
    assert halts[0] & 4, halts
    assert out["history"].cpu().numpy().tolist() == ce
    g.close()


def test_graph_counts_its_kernel_launches():
    w = _workload()
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    g.step_graph_capture(pos, t, a, e, i, first_step=0)
    k0 = g.stats()["kernel_launches"]
    g.step_graph_launch(3)
    nxt, halted = g.step_graph_finish()
    assert (nxt, halted) == (3, 0)
    per = (g.stats()["kernel_launches"] - k0) / 3
    # a whole number of launches per replayed step, at least one per kind of
    # work (the walk, the near field, the descent, the draw, the resolution)
    assert per >= 20 and per == int(per)
    g.close()


def test_graph_call_order_errors():
    w = _workload()
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    with pytest.raises(msp.MSPError):
        g.step_graph_capture(pos, t, a, e, i, first_step=0)     # no build yet
    with pytest.raises(msp.MSPError):
        g.step_graph_launch(1)                                  # nothing captured
    with pytest.raises(msp.MSPError):
        g.set_pair_capacity(0)
    g.close()


def test_full_size_graph_replays_equal_eager_steps():
    """The benchmark workload (1,048,576 neurons) in the configuration the
    benchmark times: two graph replays against the same two eager steps."""
    import bench
    w = bench.workload()
    ce, se, le = _eager(w, 5, 2)
    cg, sg, lg, _, _ = _graph(w, 5, 2)
    assert cg == ce
    for x, y in zip(sg, se):
        assert np.array_equal(x, y)
    for key in ("pre", "post", "typ"):
        assert np.array_equal(lg[key], le[key])


def test_graph_refuses_to_replay_after_workspace_reallocation():
    # any workspace (re)allocation after the capture, here the batch
    # layout's scratch, invalidates the graph: launch fails, a new capture works
    from paper_2301_10570_gb300 import workloads as W2
    w = _workload()
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    g.step_graph_capture(pos, t, a, e, i, first_step=0)
    g.run_steps(0, 1)
    b = W2.batched_small()
    msp.batch_layout(torch.from_numpy(b.pos).cuda(), b.offsets, b.sigma, 3.25, 16)
    with pytest.raises(msp.MSPError):
        g.step_graph_launch(1)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    g.step_graph_capture(pos, t, a, e, i, first_step=1)
    assert g.run_steps(1, 2) == 3
    g.close()


@pytest.mark.parametrize("full_build", [False, True])
def test_graph_replays_of_a_batch_equal_eager_steps(full_build):
    # the batched problem (several networks, each in its own frame, as one
    # problem, with a cutoff per network) through the step graph, against the
    # same steps as eager calls; with full_build the replays recompute the
    # frames' Morton keys and the octree every step
    from paper_2301_10570_gb300 import workloads as W2
    b = W2.batched_small()
    plan = dict(leaf_capacity=16, cutoff=3.25, rho_max=0.0, p=4, m2l_min_pairs=0)
    local, side, level = msp.batch_layout(torch.from_numpy(b.pos).cuda(), b.offsets, b.sigma,
                                          4.0, plan["leaf_capacity"])
    w = b.framed(local.cpu().numpy(), side, level, plans=(None, [3.25, 4.0, 3.5, 3.25, 3.5]),
                 **plan)
    ce, se, le = _eager(w, 7, 4)
    cg, sg, lg, _, _ = _graph(w, 7, 4, full_build=full_build)
    assert cg == ce
    for x, y in zip(sg, se):
        assert np.array_equal(x, y)
    for key in ("pre", "post", "typ"):
        assert np.array_equal(lg[key], le[key])


@pytest.mark.parametrize("case", ["clustered_4k_c32", "bench_plan_2x16k"])
def test_graph_replays_equal_the_oracle_steps(case):
    """K replays of the captured step (walk, tree, attraction, selection,
    commit), one at a time, each against the oracle's step from the same
    vacancy state (read back from the GPU before the replay): partners
    identical except draws the oracle flags as within its band of a CDF
    boundary; whenever no partner differs, the step's synapse count (also in
    the graph's history), synapse lists and the vacancy state after the commit
    bit for bit."""
    from oracle import oracle as O
    if case == "clustered_4k_c32":
        w, k_steps = W.clustered_small(1, 4096, seed=21, leaf_capacity=32, cutoff=3.25,
                                       rho_max=0.0), 8
    else:
        w, k_steps = W.clustered_small(2, 16_384, seed=22, leaf_capacity=256, cutoff=3.25,
                                       rho_max=0.0, m2l_min_pairs=0), 4
    first = 5
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    g.build_tree(pos, t, a, e, i)
    g.attraction()
    out = g.step_graph_capture(pos, t, a, e, i, first_step=first, history_len=k_steps)
    o = O.Oracle(w.params)
    exact_steps = 0
    for k in range(first, first + k_steps):
        pre = [v.cpu().numpy() for v in (a, e, i)]
        assert g.run_steps(k, 1) == k + 1
        oa, oe, oi = O.vacancy_walk(w.params["seed"], k, *pre)
        o.build_tree(w.pos, w.type, oa, oe, oi)
        o.attraction()
        r = o.select_partners(k)
        ne = len(r["partner"])
        assert g.stats()["n_elements"] == ne
        gp = out["partner"][:ne].cpu().numpy()
        differ = gp != r["partner"]
        assert np.all(r["near_boundary"][differ])
        if differ.any():
            continue
        ns = r["n_syn"]
        assert int(out["n_syn"].item()) == ns
        assert int(out["history"][k - first].item()) == ns
        assert np.array_equal(out["syn_pre"][:ns].cpu().numpy(), r["syn_pre"])
        assert np.array_equal(out["syn_post"][:ns].cpu().numpy(), r["syn_post"])
        assert np.array_equal(out["syn_type"][:ns].cpu().numpy(), r["syn_type"])
        ref = O.commit_synapses(r["syn_pre"], r["syn_post"], r["syn_type"], oa, oe, oi)
        for got, want in zip((a, e, i), ref):
            assert np.array_equal(got.cpu().numpy(), want)
        exact_steps += 1
    assert exact_steps >= k_steps // 2
    g.close()


def test_full_build_graph_replays_equal_eager_steps():
    """Replays that rebuild the whole octree every step (steps a1-a12 in
    full) give the same steps as the eager calls and as the replays that
    reuse the octree."""
    w = W.clustered_small(2, 4096, seed=4, leaf_capacity=32, rho_max=0.0)
    ec, es, el = _eager(w, 3, 5)
    gc, gs, gl, st, _ = _graph(w, 3, 5, full_build=True)
    assert gc == ec
    for x, y in zip(gs, es):
        assert np.array_equal(x, y)
    assert np.array_equal(gl["pre"], el["pre"]) and np.array_equal(gl["post"], el["post"])
    rc, rs, _, _, _ = _graph(w, 3, 5, full_build=False)
    assert rc == gc


def test_graph_halts_when_another_build_replaced_its_octree():
    """A replay that reuses the octree checks the build it was captured after:
    an eager build of other positions (same n) in between halts the replay,
    which is finished eagerly on its own positions and captured again."""
    w = W.clustered_small(1, 4096, seed=6, leaf_capacity=32, rho_max=0.0)
    other = W.clustered_small(1, 4096, seed=7, leaf_capacity=32, rho_max=0.0)
    ec, es, _ = _eager(w, 2, 3)
    pos, t, a, e, i = _state(w)
    g = msp.MSP(w.params)
    odev = msp.to_device(other)
    g.build_tree(*odev)             # sizes the workspace for both trees first, so that
    g.build_tree(pos, t, a, e, i)   # the later build reallocates nothing (a reallocation
    g.attraction()                  # is refused earlier, by the allocation epoch)
    out = g.step_graph_capture(pos, t, a, e, i, first_step=2, history_len=3)
    g.build_tree(*odev)             # replaces the octree
    g.step_graph_launch(1)
    nxt, halted = g.step_graph_finish()
    assert halted != 0 and nxt == 3
    assert g.run_steps(3, 2) == 5
    assert out["history"].cpu().numpy().tolist() == ec
    for x, y in zip((a, e, i), es):
        assert np.array_equal(x.cpu().numpy(), y)
