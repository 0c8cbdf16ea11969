import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def oracle_mod():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def boundary_report(request):
    """Per parity case: partner draws, draws the oracle flags as within its
    band of a CDF boundary, and partners that differ from the oracle's
    (printed in the run's summary)."""
    if not hasattr(request.config, "_msp_boundary"):
        request.config._msp_boundary = {}
    return request.config._msp_boundary


@pytest.fixture(scope="session")
def precision_report(request):
    """Observed errors of the GPU results against the FP64 oracle, per
    quantity and case (printed in the run's summary)."""
    if not hasattr(request.config, "_msp_precision"):
        request.config._msp_precision = {}
    return request.config._msp_precision


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    prec = getattr(config, "_msp_precision", None)
    if prec:
        terminalreporter.write_sep("-", "observed errors against the FP64 oracle")
        for key in sorted(prec):
            terminalreporter.write_line(f"{key}: {prec[key]:.3e}")
    rep = getattr(config, "_msp_boundary", None)
    if not rep:
        return
    terminalreporter.write_sep("-", "boundary draws per parity case (oracle band)")
    for name, r in sorted(rep.items()):
        terminalreporter.write_line(
            f"{name}: band {r['band']:.0e}, draws {r['draws']}, flagged draws "
            f"{r['boundary_draws']}, flagged elements {r['flagged']}/{r['elements']}, "
            f"partners differing {r['differ']} (all flagged: {r['differ_flagged']})")
