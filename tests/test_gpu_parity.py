"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: bit-exact for every integer result (Morton keys, sort permutation,
octree arrays, box sums, traversal pairs); floating point within the
tolerances derived from the arithmetic (single precision sums with
round-to-nearest and the SFU exp2, against double precision):
  - u(t) within 1e-5 relative of the oracle FMM at the same p, tree and lists
    (targets with u >= 1e-6 max u), and within 1e-4 of FP64 brute force where
    the truncation allows (near field only, or p >= 6);
  - box-pair attractions within 1e-5 relative for near-field pairs and
    1e-4 where they come from single precision translations;
  - partner choices identical except elements whose path had a draw within
    the oracle's boundary band (1e-6 of the total when no pair is
    translated, where the single precision sums of exact terms move a
    boundary by a few 1e-7; 1e-5 with translations, whose single precision
    coefficients move W by ~1e-5); the flagged draws are counted and
    reported;
  - synapse lists identical whenever the partners are.
"""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import msp  # noqa: E402


def _coincident():
    w = W.uniform_cube(300, 4000.0, seed=5, leaf_capacity=6, rho_max=0.4)
    w.pos[:, 50:90] = w.pos[:, 50:51]          # 41 points in one grid cell
    return w


CASES = {
    "uniform_4k": lambda: W.uniform_4k(),
    "clustered_far_p4": lambda: W.clustered_small(1, 4096, leaf_capacity=8, rho_max=0.3, p=4),
    "clustered_far_p6": lambda: W.clustered_small(1, 1536, seed=9, leaf_capacity=8, rho_max=0.3,
                                                  p=6),
    "ragged_37": lambda: W.uniform_cube(37, 2000.0, seed=2, leaf_capacity=4, rho_max=0.4),
    "big_leaves": lambda: W.clustered_small(1, 4096, leaf_capacity=64, rho_max=0.0),
    "wide_sparse_leaves": lambda: W.uniform_cube(3000, 60_000.0, seed=6, leaf_capacity=64),
    "coincident": _coincident,
    "single_leaf": lambda: W.uniform_cube(40, 3000.0, seed=31, leaf_capacity=64),
    "one_neuron": lambda: W.uniform_cube(1, 1000.0, seed=1),
    "no_vacancies": lambda: _zero_axons(),
    # every neuron sends 3 axonal elements, 3 neurons have vacant dendrites:
    # groups of thousands of requests at one dendrite, most boxes without
    # attraction (translated pairs included)
    "few_dendrites": lambda: _few_dendrites(),
    # expansions about the geometric centres: translations grouped by offset
    # as matrix products (p <= 5), one pair at a time above
    "geo_far_p4": lambda: W.clustered_small(1, 4096, leaf_capacity=8, rho_max=0.3, p=4,
                                            centre_mode=1),
    "geo_far_p5": lambda: W.clustered_small(2, 2048, seed=17, leaf_capacity=8, rho_max=0.3,
                                            p=5, centre_mode=1),
    "geo_far_p6": lambda: W.clustered_small(1, 1536, seed=9, leaf_capacity=8, rho_max=0.3,
                                            p=6, centre_mode=1),
    # the benchmark's plan (leaf capacity 256, cutoff 3.25 sigma, no
    # translations) on three clusters of the benchmark's size and spacing:
    # near-field rounds of up to 125 targets, leaf-draw slices over leaves of
    # more than 32 sources, leaves above the staged 256 sources
    "bench_plan_3x16k": lambda: W.clustered_small(3, 16_384, seed=3, leaf_capacity=256,
                                                  cutoff=3.25, rho_max=0.0, p=4,
                                                  m2l_min_pairs=0),
    # leaves of up to 512 points: the leaf draw reads leaves of more than 256
    # sources from global memory and walks slices of more than 8 blocks of 32
    "leaf_capacity_512": lambda: W.clustered_small(1, 16_384, seed=5, leaf_capacity=512,
                                                   cutoff=3.25, rho_max=0.0, p=4,
                                                   m2l_min_pairs=0),
    # Algorithm 2's count rule (c1 = c2 = 70): inner pairs expanded by their
    # dendrite counts at every level, boxes of at most ~2 sigma
    "paper_count_rule_p6": lambda: W.uniform_cube(1500, 3000.0, seed=3, leaf_capacity=8, p=6,
                                                  mac_mode=1, cutoff=5.0),
}

# cases whose FP64 brute force runs on sampled targets (all-targets would
# take the oracle tens of seconds)
SAMPLED_DIRECT = {"bench_plan_3x16k": 4096, "leaf_capacity_512": 2048}


def _few_dendrites():
    w = W.uniform_cube(3000, 8000.0, seed=12, leaf_capacity=16)
    w.vac_axon[:] = 3
    w.vac_dend_e[:] = 0
    w.vac_dend_i[:] = 0
    idx = np.array([5, 1200, 2900])
    w.vac_dend_e[idx] = 5
    w.vac_dend_i[idx] = 5
    return w


def _zero_axons():
    w = W.uniform_cube(500, 5000.0, seed=3, leaf_capacity=16)
    w.vac_axon[:] = 0
    return w


_cache = {}


def run(name, step=3):
    if name in _cache:
        return _cache[name]
    from oracle import oracle as O
    w = CASES[name]()
    g = msp.MSP(w.params)
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    sel = g.select_partners(step)
    torch.cuda.synchronize()
    ne = g.num_elements()
    gres = dict(u=u, tree=g.export_tree(), pairs=g.export_pairs(), stats=g.stats(),
                partner=sel["partner"][:ne].cpu().numpy(), n_syn=int(sel["n_syn"].item()),
                syn_pre=sel["syn_pre"].cpu().numpy(), syn_post=sel["syn_post"].cpu().numpy(),
                syn_type=sel["syn_type"].cpu().numpy(), exps=g.export_expansions())
    gres["direct"] = g.direct().cpu().numpy() if w.n > 0 else np.zeros(0)
    g.close()
    o = O.Oracle(w.params)
    o.build_tree(*w.arrays())
    uo = o.attraction()
    ro = o.select_partners(step)
    keys, perm = o.keys()
    ores = dict(u=uo, keys=keys, perm=perm, nodes=o.nodes(), pairs=o.pairs(), sel=ro,
                far_level=o.far_level(), stats=o.stats())
    nd = ores["nodes"]
    ores["exps"] = [o.expansions(i) for i in range(len(nd["level"]))]
    if name in SAMPLED_DIRECT:
        idx = np.sort(np.random.default_rng(8).choice(w.n, SAMPLED_DIRECT[name], replace=False))
    else:
        idx = np.arange(w.n)
    ores["direct_idx"] = idx
    ores["direct"] = (O.direct(*w.arrays(), w.params["sigma"], targets=idx) if w.n > 0
                      else np.zeros(0))
    _cache[name] = (w, gres, ores)
    return _cache[name]


NAMES = list(CASES)


@pytest.mark.parametrize("name", NAMES)
def test_morton_keys_and_permutation_bit_exact(name):
    w, g, o = run(name)
    assert np.array_equal(g["tree"]["keys"], o["keys"])
    assert np.array_equal(g["tree"]["perm"], o["perm"])


@pytest.mark.parametrize("name", NAMES)
def test_octree_bit_exact(name):
    w, g, o = run(name)
    for k in ("level", "prefix", "first", "count", "parent", "child_first", "nchild", "sums"):
        assert np.array_equal(g["tree"][k], o["nodes"][k]), k
    assert g["stats"]["n_nodes"] == len(o["nodes"]["level"])


@pytest.mark.parametrize("name", NAMES)
def test_centroids(name):
    w, g, o = run(name)
    side = w.params["side"]
    np.testing.assert_allclose(g["tree"]["centroids"], o["nodes"]["centroids"], rtol=0,
                               atol=2e-6 * side)


@pytest.mark.parametrize("name", NAMES)
def test_traversal_pairs_bit_exact(name):
    w, g, o = run(name)
    for k in ("X", "Y", "kind", "child_first", "depth_start"):
        assert np.array_equal(g["pairs"][k], o["pairs"][k]), k
    assert g["stats"]["far_level"] == o["far_level"]
    assert g["stats"]["n_far"] == o["stats"]["far_pairs"]
    assert g["stats"]["n_p2p"] == o["stats"]["p2p_pairs"]


@pytest.mark.parametrize("name", NAMES)
def test_pair_attraction_table(name, precision_report):
    w, g, o = run(name)
    gp, op = g["pairs"], o["pairs"]
    has_far = (op["kind"] == 1).any()
    rtol = 1e-4 if has_far else 1e-5
    for k in ("wE", "wI"):
        scale = max(np.abs(op[k]).max(), 1e-300)
        err = np.abs(gp[k] - op[k])
        big = np.abs(op[k]) > 1e-7 * scale
        if big.any():
            precision_report[f"W rel, {name}, {k}"] = float(np.max(err[big] / np.abs(op[k][big])))
        assert np.all(err <= rtol * np.abs(op[k]) + 1e-7 * scale), k


@pytest.mark.parametrize("name", NAMES)
def test_attraction_matches_oracle_fmm(name, precision_report):
    w, g, o = run(name)
    uo, ug = o["u"], g["u"]
    assert np.all(ug[w.vac_axon == 0] == 0)
    if w.n == 0 or uo.max() <= 0:
        assert np.all(ug == 0)
        return
    m = uo >= 1e-6 * uo.max()
    rel = np.max(np.abs(ug[m] - uo[m]) / uo[m])
    precision_report[f"u rel vs oracle FMM, {name}"] = float(rel)
    ref, idx = o["direct"], o["direct_idx"]
    mb = ref >= 1e-6 * ref.max()
    if mb.any():
        precision_report[f"u rel vs FP64 brute force, {name}"] = float(
            np.max(np.abs(ug[idx][mb] - ref[mb]) / ref[mb]))
    assert rel < 1e-5


@pytest.mark.parametrize("name", ["uniform_4k", "clustered_far_p6", "big_leaves",
                                  "wide_sparse_leaves", "single_leaf", "bench_plan_3x16k",
                                  "leaf_capacity_512"])
def test_attraction_within_1e4_of_fp64_brute_force(name):
    """Cases whose truncation allows it: near field only, or p >= 6 (p = 4 with
    boxes of half-width 0.3-0.4 sigma is at the paper's ~1e-3 level)."""
    w, g, o = run(name)
    ref, idx = o["direct"], o["direct_idx"]
    m = ref >= 1e-6 * ref.max()
    assert np.max(np.abs(g["u"][idx][m] - ref[m]) / ref[m]) < 1e-4


@pytest.mark.parametrize("name", NAMES)
def test_direct_path_matches_oracle_brute_force(name):
    w, g, o = run(name)
    ref, idx = o["direct"], o["direct_idx"]
    if w.n == 0 or ref.max() <= 0:
        return
    m = ref >= 1e-6 * ref.max()
    assert np.max(np.abs(g["direct"][idx][m] - ref[m]) / ref[m]) < 1e-5


@pytest.mark.parametrize("name", ["clustered_far_p4", "clustered_far_p6", "ragged_37",
                                  "geo_far_p4", "geo_far_p5", "geo_far_p6",
                                  "paper_count_rule_p6"])
def test_expansions_match_oracle(name, precision_report):
    w, g, o = run(name)
    A, M, B, first = g["exps"]
    assert first == np.searchsorted(o["nodes"]["level"], o["far_level"])
    worst = {"A": 0.0, "M": 0.0, "B": 0.0}
    for i in range(A.shape[0]):
        oA, oM, oB = o["exps"][first + i]
        for key, got, ref, tol in (("A", A[i], oA, 1e-5), ("M", M[i], oM, 1e-5),
                                   ("B", B[i], oB, 1e-4)):
            scale = max(np.abs(ref).max(), 1e-30)
            e = np.max(np.abs(got - ref)) / scale
            worst[key] = max(worst[key], float(e))
            assert e <= tol
    for key, v in worst.items():
        precision_report[f"{key} (of the box's largest coefficient), {name}"] = v


@pytest.mark.parametrize("name", NAMES)
def test_partners_identical_except_boundary_draws(name):
    w, g, o = run(name)
    ro = o["sel"]
    mism = g["partner"] != ro["partner"]
    assert not np.any(mism & ~ro["near_boundary"]), np.nonzero(mism & ~ro["near_boundary"])
    assert g["stats"]["n_elements"] == len(ro["partner"])


@pytest.mark.parametrize("name", NAMES)
def test_boundary_draws_are_counted_and_few(name, boundary_report):
    """The draws the oracle flags as within its band of a CDF boundary are
    counted and reported; every partner that differs is among them, and they
    are a small share of the draws."""
    w, g, o = run(name)
    ro, st = o["sel"], o["stats"]
    differ = g["partner"] != ro["partner"]
    translates = float(w.params["rho_max"]) > 0.0 or int(w.params.get("mac_mode", 0)) == 1
    band = 1e-5 if translates else 1e-6
    boundary_report[name] = dict(band=band, draws=st["draws"],
                                 boundary_draws=st["boundary_draws"],
                                 flagged=int(ro["near_boundary"].sum()),
                                 elements=len(ro["partner"]), differ=int(differ.sum()),
                                 differ_flagged=bool(np.all(ro["near_boundary"][differ])))
    assert np.all(ro["near_boundary"][differ])
    assert st["boundary_draws"] <= max(3, 0.01 * st["draws"])


@pytest.mark.parametrize("name", NAMES)
def test_synapses_identical(name):
    w, g, o = run(name)
    ro = o["sel"]
    if np.array_equal(g["partner"], ro["partner"]):
        ns = ro["n_syn"]
        assert g["n_syn"] == ns
        assert np.array_equal(g["syn_pre"][:ns], ro["syn_pre"])
        assert np.array_equal(g["syn_post"][:ns], ro["syn_post"])
        assert np.array_equal(g["syn_type"][:ns], ro["syn_type"])
    else:
        assert abs(g["n_syn"] - ro["n_syn"]) <= int((g["partner"] != ro["partner"]).sum())


def test_device_philox_known_answer_vectors():
    """The library's device Philox4x32-10 (msp_philox, the generator of every
    draw) reproduces the published known-answer vectors (Salmon et al., SC'11;
    tests/golden/philox4x32_10_kat.json) and the oracle's stream on other
    counters."""
    import json
    import os
    from oracle import oracle as O
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")) as f:
        kat = json.load(f)["vectors"]

    def bits(v):
        return np.array([int(h, 16) for h in v], np.uint32)

    ctr = np.stack([bits(v["counter"]) for v in kat])
    key = np.stack([bits(v["key"]) for v in kat])
    rng = np.random.default_rng(4)
    ctr = np.concatenate([ctr, rng.integers(0, 2 ** 32, (1000, 4), dtype=np.uint32)])
    key = np.concatenate([key, rng.integers(0, 2 ** 32, (1000, 2), dtype=np.uint32)])
    out = msp.philox(torch.from_numpy(ctr.view(np.int32)).cuda(),
                     torch.from_numpy(key.view(np.int32)).cuda())
    got = out.cpu().numpy().view(np.uint32)
    for i, v in enumerate(kat):
        assert np.array_equal(got[i], bits(v["output"]))
    for i in range(len(kat), len(ctr)):
        assert np.array_equal(got[i], O.philox(ctr[i], key[i]))


def _device_calls(w, step):
    g = msp.MSP(w.params)
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    sel = g.select_partners(step)
    ne = g.num_elements()
    ns = int(sel["n_syn"].item())
    out = dict(u=u, partner=sel["partner"][:ne].cpu().numpy(), n_syn=ns,
               pre=sel["syn_pre"][:ns].cpu().numpy(), post=sel["syn_post"][:ns].cpu().numpy(),
               typ=sel["syn_type"][:ns].cpu().numpy())
    g.close()
    return out


@pytest.mark.parametrize("rho_max", [0.0, 0.3])
def test_host_buffer_step_equals_device_calls(rho_max):
    """msp_plasticity_step_host, call after call: the first runs eagerly and
    captures the step, later ones replay the graph (new vacancies each call,
    then moved positions, which the graph detects and runs eagerly again);
    every call equals the separate device calls on the same inputs."""
    from paper_2301_10570_gb300 import workloads as W2
    w = W2.clustered_small(1, 4096, leaf_capacity=16, rho_max=rho_max, p=4)
    g = msp.MSP(w.params)
    rng = np.random.default_rng(9)
    for call in range(5):
        if call in (2, 3):
            for v in (w.vac_axon, w.vac_dend_e, w.vac_dend_i):
                v[:] = rng.integers(0, 4, w.n).astype(np.uint8)
        if call == 4:
            w.pos[:, :50] += np.float32(10.0)
        step = 7 + call
        out = g.plasticity_step_host(step, *w.arrays())
        ref = _device_calls(w, step)
        ne, ns = len(ref["partner"]), ref["n_syn"]
        assert int(out["n_syn"][0]) == ns
        assert np.array_equal(out["partner"][:ne], ref["partner"])
        assert np.array_equal(out["syn_pre"][:ns], ref["pre"])
        assert np.array_equal(out["syn_post"][:ns], ref["post"])
        assert np.array_equal(out["syn_type"][:ns], ref["typ"])
        assert np.array_equal(out["u"][: w.n], ref["u"])
        st = g.stats()
        assert st["n_synapses"] == ns and st["n_elements"] == ne
    g.close()


@pytest.mark.parametrize("p", [4, 6])
def test_repeated_runs_are_deterministic(p):
    """With translated pairs too: each target box's far pairs are summed by
    one warp in a fixed order, so u, the pair table and the choices repeat
    bit for bit."""
    w = W.clustered_small(1, 4096, leaf_capacity=8, rho_max=0.3, p=p)
    res = []
    for _ in range(2):
        g = msp.MSP(w.params)
        g.build_tree(*msp.to_device(w))
        u = g.attraction().cpu().numpy()
        sel = g.select_partners(1)
        assert g.stats()["n_far"] > 0
        res.append((g.export_pairs(), sel["partner"].cpu().numpy(), int(sel["n_syn"].item()), u,
                    g.export_expansions()[2]))
        g.close()
    assert np.array_equal(res[0][1], res[1][1]) and res[0][2] == res[1][2]
    assert np.array_equal(res[0][0]["wE"], res[1][0]["wE"])
    assert np.array_equal(res[0][3], res[1][3])
    assert np.array_equal(res[0][4], res[1][4])


def test_vacancy_walk_and_commit_match_oracle():
    from oracle import oracle as O
    rng = np.random.default_rng(1)
    n = 5000
    a, e, i = (rng.integers(0, 6, n).astype(np.uint8) for _ in range(3))
    w = W.uniform_cube(n, 5000.0, seed=1)
    g = msp.MSP(w.params)
    ta, te, ti = (torch.from_numpy(v.copy()).cuda() for v in (a, e, i))
    g.vacancy_walk(12, ta, te, ti)
    oa, oe, oi = O.vacancy_walk(0, 12, a, e, i)
    for t, r in ((ta, oa), (te, oe), (ti, oi)):
        assert np.array_equal(t.cpu().numpy(), r)
    pre = rng.integers(0, n, 3000).astype(np.int32)
    post = rng.integers(0, n, 3000).astype(np.int32)
    ty = rng.integers(0, 2, 3000).astype(np.uint8)
    sel = dict(n_syn=torch.tensor([2500], dtype=torch.int64).cuda(),
               syn_pre=torch.from_numpy(pre).cuda(), syn_post=torch.from_numpy(post).cuda(),
               syn_type=torch.from_numpy(ty).cuda())
    g.commit_synapses(sel, ta, te, ti)
    ra, re_, ri = O.commit_synapses(pre[:2500], post[:2500], ty[:2500], oa, oe, oi)
    for t, r in ((ta, ra), (te, re_), (ti, ri)):
        assert np.array_equal(t.cpu().numpy(), r)


def test_call_order_and_argument_errors():
    w = W.uniform_4k()
    with pytest.raises(msp.MSPError) as ei:
        msp.MSP(dict(w.params, p=9))
    assert ei.value.code == 1
    g = msp.MSP(w.params)
    with pytest.raises(msp.MSPError) as ei:
        g.attraction(out=torch.empty(1, device="cuda"))
    assert ei.value.code == 5
    g.build_tree(*msp.to_device(w))
    with pytest.raises(msp.MSPError) as ei:
        g.select_partners(0)
    assert ei.value.code == 5
    g.attraction()
    g.select_partners(0)


def test_full_size_clustered_sampled():
    """The benchmark workload at full size (1,048,576 neurons) in the launch
    configuration the benchmark times: u on sampled targets against FP64 brute
    force, against the all-pairs GPU path everywhere, and the model's
    invariants on the formed synapses."""
    from oracle import oracle as O
    import bench
    w = bench.workload()
    g = msp.MSP(w.params)
    dev = msp.to_device(w)
    g.build_tree(*dev)
    u = g.attraction()
    sel = g.select_partners(0)
    ud = g.direct()
    torch.cuda.synchronize()
    m = ud > 1e-6 * ud.max()
    assert ((u[m] - ud[m]).abs() / ud[m]).max().item() < 1e-4
    idx = np.random.default_rng(5).choice(w.n, 128, replace=False)
    ref = O.direct(*w.arrays(), w.params["sigma"], targets=idx)
    un = u.cpu().numpy()[idx]
    k = ref > 0
    assert np.max(np.abs(un[k] - ref[k]) / ref[k]) < 1e-4
    ns = int(sel["n_syn"].item())
    pre = sel["syn_pre"][:ns].cpu().numpy()
    post = sel["syn_post"][:ns].cpu().numpy()
    ty = sel["syn_type"][:ns].cpu().numpy()
    assert np.all(pre != post)
    assert np.all(w.type[pre] == ty)
    assert np.all(np.bincount(pre, minlength=w.n) <= w.vac_axon)
    for ch, dend in ((0, w.vac_dend_e), (1, w.vac_dend_i)):
        assert np.all(np.bincount(post[ty == ch], minlength=w.n) <= dend)
    part = sel["partner"][: g.num_elements()].cpu().numpy()
    owner = np.repeat(np.arange(w.n), w.vac_axon)
    ok = part >= 0
    assert ok.mean() > 0.9
    wt = np.where(w.type[owner[ok]] == 0, w.vac_dend_e[part[ok]], w.vac_dend_i[part[ok]])
    assert np.all(wt > 0) and np.all(part[ok] != owner[ok])
