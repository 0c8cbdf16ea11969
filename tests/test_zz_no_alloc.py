"""msp_direct_noalloc: the all-pairs attraction for callers that cannot let a
library allocate device memory (a loop that must never block on cudaMalloc,
or a framework that owns every device allocation).  It must give the same
attraction as the ordinary entry point (msp_direct, which works from a
context's own workspace), call after call, although every call shares one
fixed scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import msp  # noqa: E402

NOALLOC_MAX = msp.NOALLOC_MAX_N


def _reference(w):
    g = msp.MSP(w.params)
    g.build_tree(*msp.to_device(w))
    u = g.direct().cpu().numpy()
    g.close()
    return u


def test_noalloc_matches_the_direct_entry_point_on_two_calls_in_a_row():
    cases = [W.uniform_cube(5000, 8000.0, seed=11), W.clustered_small(1, 3000, seed=12)]
    refs = [_reference(w) for w in cases]
    torch.cuda.synchronize()
    for w, ref in zip(cases, refs):
        u = msp.direct_noalloc(*msp.to_device(w), w.params["sigma"])
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        assert np.all(got[w.vac_axon == 0] == 0)
        m = ref > 1e-6 * ref.max()
        assert np.max(np.abs(got[m] - ref[m]) / ref[m]) < 1e-5


@pytest.mark.parametrize("n", [NOALLOC_MAX, NOALLOC_MAX - 1])
def test_noalloc_at_its_largest_sizes_matches_fp64_brute_force(n):
    """The whole scratch in use (n = MSP_NOALLOC_MAX_N) and a size one short of
    it (a ragged last tile): the all-pairs attraction within 1e-5 of the
    oracle's FP64 brute force on sampled targets and of msp_direct on all."""
    from oracle import oracle as O
    w = W.clustered_small(4, n // 4 + 1, seed=13)
    w = W.subset(w, np.arange(n), name=f"noalloc_{n}")
    ref = _reference(w)
    for _ in range(2):
        u = msp.direct_noalloc(*msp.to_device(w), w.params["sigma"])
        torch.cuda.synchronize()
        got = u.cpu().numpy()
        m = ref > 1e-6 * ref.max()
        assert np.max(np.abs(got[m] - ref[m]) / ref[m]) < 1e-5
    idx = np.sort(np.random.default_rng(3).choice(n, 1024, replace=False))
    idx = np.union1d(idx, [0, n - 1])
    exact = O.direct(*w.arrays(), w.params["sigma"], targets=idx)
    k = exact >= 1e-6 * exact.max()
    assert np.max(np.abs(got[idx][k] - exact[k]) / exact[k]) < 1e-5
    assert np.all(got[w.vac_axon == 0] == 0)


def test_noalloc_checks_its_arguments():
    """Arguments the entry point cannot use are refused before anything runs:
    host memory, counts of the wrong length or type, an output of the wrong
    size."""
    w = W.uniform_cube(1000, 5000.0, seed=2)
    pos, t, a, e, i = msp.to_device(w)
    with pytest.raises(TypeError):
        msp.direct_noalloc(pos, t[:-1], a, e, i, 750.0)
    with pytest.raises(TypeError):
        msp.direct_noalloc(pos, t.float(), a, e, i, 750.0)
    with pytest.raises(TypeError):
        msp.direct_noalloc(pos, t, a, e, i, 750.0,
                           out=torch.empty(999, dtype=torch.float32, device="cuda"))
    # host memory reaches the C entry point only through a direct call: it
    # answers MSP_ERR_INVALID_ARG without launching
    import ctypes as C
    L = msp.load()
    host = np.zeros(1000, np.float32)
    hp = host.ctypes.data_as(C.c_void_p)
    dev = [C.c_void_p(x.data_ptr()) for x in (pos[0].contiguous(), pos[1].contiguous(),
                                              pos[2].contiguous(), t, a, e, i)]
    rc = L.msp_direct_noalloc(1000, *dev, 750.0, hp, None)
    assert rc == 1 and b"device memory" in L.msp_last_error()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = msp.NOALLOC_MAX_N + 1
    pos = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    z8 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(msp.MSPError) as ei:
        msp.direct_noalloc(pos, z8, z8, z8, z8, 750.0)
    assert ei.value.code == 1
    assert "MSP_NOALLOC_MAX_N" in str(ei.value)
