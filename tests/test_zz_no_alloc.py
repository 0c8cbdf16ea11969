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


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = msp.NOALLOC_MAX_N + 1
    pos = torch.zeros((3, n), dtype=torch.float32, device="cuda")
    z8 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(msp.MSPError) as ei:
        msp.direct_noalloc(pos, z8, z8, z8, z8, 750.0)
    assert ei.value.code == 1
    assert "MSP_NOALLOC_MAX_N" in str(ei.value)
