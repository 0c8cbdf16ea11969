"""Host-side checks that need no GPU: the C-ABI library builds for sm_103a,
loads, exports every entry point include/msp.h declares, its structs have the
layout the binding assumes, the binding fails loudly without the library, and
the replica bookkeeping works across ranks (gloo, world size 2)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2301_10570_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_symbols():
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(msp_[a-z_]+)\s*\(", text)))


def test_header_declares_the_path(lib):
    names = declared_symbols()
    for need in ("msp_build_tree", "msp_attraction", "msp_select_partners", "msp_create",
                 "msp_destroy", "msp_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing


def test_binding_names_match_header():
    from paper_2301_10570_gb300 import msp
    assert sorted(msp.EXPORTED) == declared_symbols()


def test_struct_layouts_match_header(tmp_path):
    from paper_2301_10570_gb300 import msp
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "msp.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(msp_config),'
        ' sizeof(msp_stats), offsetof(msp_config, seed), offsetof(msp_stats, near_field_ms),'
        ' offsetof(msp_config, m2l_min_pairs), offsetof(msp_config, centre_mode),'
        ' sizeof(msp_neuron_params), offsetof(msp_neuron_params, refractory),'
        ' offsetof(msp_neuron_params, mu)); return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [ctypes.sizeof(msp.Config), ctypes.sizeof(msp.Stats), msp.Config.seed.offset,
                   msp.Stats.near_field_ms.offset, msp.Config.m2l_min_pairs.offset,
                   msp.Config.centre_mode.offset, ctypes.sizeof(msp.NeuronParams),
                   msp.NeuronParams.refractory.offset, msp.NeuronParams.mu.offset]


def test_last_error_is_a_string_and_create_validates(lib):
    from paper_2301_10570_gb300 import msp
    L = msp.load()
    h = ctypes.c_void_p()
    cfg = msp.make_config(dict(sigma=-1.0, p=4, leaf_capacity=8, origin=(0, 0, 0), side=1.0,
                               rho_max=0.1, cutoff=4.0))
    assert L.msp_create(ctypes.byref(h), ctypes.byref(cfg), 0) == 1   # invalid argument
    assert b"range" in L.msp_last_error()
    assert L.msp_destroy(None) == 0
    assert L.msp_build_tree(None, 0, *([None] * 7), None) == 1        # null context


def test_missing_library_fails_loudly(tmp_path):
    from paper_2301_10570_gb300 import msp
    saved = msp._lib
    msp._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            msp.load(str(tmp_path / "nope.so"))
    finally:
        msp._lib = saved


def _replica_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2301_10570_gb300 import replicas
    replicas.barrier()
    agg = replicas.aggregate_throughput(1000 * (rank + 1), 10.0 + 5 * rank)
    q.put((rank, agg, replicas.world()))
    dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, agg, (r, wsize) in res:
        assert wsize == 2 and r == rank
        assert agg["units"] == 3000 and agg["ms"] == 15.0
        assert agg["per_s"] == pytest.approx(3000 / 0.015)


def _batch_worker(rank, world, port, q):
    import os

    import torch.distributed as dist

    from paper_2301_10570_gb300 import replicas
    from paper_2301_10570_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = W.batched_small()
    part = b.select(range(rank, len(b.sigma), world))
    total = replicas.sum_over_ranks(part.n)
    q.put((rank, part.n, int(total), part.sigma.tolist()))
    dist.destroy_process_group()


def test_batched_networks_split_over_two_gloo_ranks():
    # every network on exactly one rank, no exchange; the ranks' neurons add up
    import socket

    import torch.multiprocessing as mp
    from paper_2301_10570_gb300 import workloads as W
    b = W.batched_small()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][2] == res[1][2] == b.n == res[0][1] + res[1][1]
    assert sorted(res[0][3] + res[1][3]) == sorted(b.sigma.tolist())


def test_batch_select_keeps_networks_whole():
    import numpy as np

    from paper_2301_10570_gb300 import workloads as W
    b = W.batched_small()
    even, odd = b.select(range(0, 5, 2)), b.select(range(1, 5, 2))
    assert even.n + odd.n == b.n
    for part, nets in ((even, [0, 2, 4]), (odd, [1, 3])):
        for j, k in enumerate(nets):
            a0, a1 = part.offsets[j], part.offsets[j + 1]
            b0, b1 = b.offsets[k], b.offsets[k + 1]
            assert np.array_equal(part.pos[:, a0:a1], b.pos[:, b0:b1])
            assert np.array_equal(part.vac_axon[a0:a1], b.vac_axon[b0:b1])
            assert part.sigma[j] == b.sigma[k] and part.kinds[j] == b.kinds[k]


def test_clock_sampler_drops_samples_before_the_timed_region(tmp_path, monkeypatch):
    # a stand-in for nvidia-smi that prints one sample line every 20 ms: the
    # first line it writes (before the timed region) is dropped, throttle
    # reasons reported as Active are collected
    import sys
    import time
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/bash\n"
                    "echo '0, 1500, 2070, 100.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                    "sleep 0.2\n"
                    "while true; do\n"
                    "  echo '0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.02\n"
                    "done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.4)
    r = c.stop()
    assert r is not None and r["samples"] >= 1
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    # without nvidia-smi there is no clock record, and no error
    monkeypatch.setenv("PATH", str(tmp_path / "none"))
    c = bench.Clocks(0)
    c.start()
    assert c.stop() is None
