"""The plan chooser picks the fastest plan within the accuracy target, and
that plan really is within the target against FP64 brute force."""
import numpy as np
import pytest

from paper_2301_10570_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_10570_gb300 import autotune, msp  # noqa: E402


def test_autotune_accepts_only_accurate_plans_and_returns_the_fastest():
    from oracle import oracle as O
    w = W.clustered_small(2, 4096, seed=3)
    best, table = autotune.tune(
        w, candidates=dict(leaf_capacity=(32, 128), cutoff=(2.0, 3.25),
                           expansions=((0.0, 4, 0), (0.3, 4, 0))), reps=2)
    ok = [r for r in table if r.get("accepted")]
    assert ok and best == min(ok, key=lambda r: r["step_ms"])["plan"]
    # a 2-sigma cutoff loses ~1e-2 of the attraction and p = 4 translations of
    # 0.3-sigma boxes ~1e-3: neither may be accepted (a plan whose boxes are
    # too big to carry expansions has no translated pairs and is exact)
    for r in table:
        if r["plan"]["cutoff"] == 2.0 or (r["plan"]["rho_max"] > 0 and r["far_pairs"] > 0):
            assert not r["accepted"], r
    g = msp.MSP(dict(w.params, **best))
    g.build_tree(*msp.to_device(w))
    u = g.attraction().cpu().numpy()
    ref = O.direct(*w.arrays(), w.params["sigma"])
    m = ref >= 1e-6 * ref.max()
    assert np.max(np.abs(u[m] - ref[m]) / ref[m]) < 1e-4
