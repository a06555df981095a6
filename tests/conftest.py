import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libcwthf.so")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def gctx():
    """One library context for the GPU tests (grids up to 256^3, 3 scales)."""
    import paper_2501_10622_gb300 as pkg
    c = pkg.Context(0, max_ng=256, max_np=(1 << 24) + (1 << 20), max_scales=3)
    yield c
    c.close()


@pytest.fixture(scope="session")
def work64():
    """The 64^3 clumped box (L = 50 Mpc/h, 200 NFW clumps) and its oracle run at w = 2."""
    import oracle
    from paper_2501_10622_gb300 import synth
    wl = synth.WORKLOADS["clumped-64cube-L50"]
    pos = wl.positions()
    return wl, pos, oracle.find(pos.numpy(), wl.box, wl.ng, 2.0)
