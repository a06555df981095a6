"""cwthf_deposit_noalloc: the CIC deposit for callers that cannot allocate
device memory (work captured into a CUDA graph, hosts whose GPU memory is
owned by another allocator, loops that cannot afford the device sync of
cudaMalloc).  It runs on a fixed scratch array inside the library, so its
result must equal cwthf_deposit's exactly -- on consecutive calls too, since
every call reuses the same scratch.  Collected last (file name) so that a
failure here cannot hide the other tests' results."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth

pytestmark = pytest.mark.gpu


def _noalloc(pos, L, ng, mass=None, mass_unit=1.0):
    grid = torch.full((ng, ng, ng), -7, dtype=torch.int64, device="cuda")
    mtot = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    rc = pkg.lib().cwthf_deposit_noalloc(
        ctypes.c_void_p(pos.data_ptr()), None if mass is None else ctypes.c_void_p(mass.data_ptr()),
        float(mass_unit), pos.shape[0], float(L), int(ng), ctypes.c_void_p(grid.data_ptr()),
        ctypes.c_void_p(mtot.data_ptr()), ctypes.c_void_p(status.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    assert rc == 0, pkg.error_string(rc)
    torch.cuda.synchronize()
    return grid, int(mtot), int(status)


def test_matches_cwthf_deposit_on_consecutive_calls():
    ctx = pkg.Context(0, max_ng=128, max_np=262144, max_scales=1)
    # call 1: the 64^3 clumped box (262,144 particles, the scratch's maximum)
    wl = synth.WORKLOADS["clumped-64cube-L50"]
    pos = wl.positions().cuda()
    ref = ctx.deposit(pos, wl.box, wl.ng).clone()
    ctx.check()
    got, mt, st = _noalloc(pos, wl.box, wl.ng)
    assert st == 0 and mt == pos.shape[0]
    assert torch.equal(got, ref)
    # call 2: another box, ragged grid, variable masses -- nothing may leak from call 1
    rng = np.random.default_rng(11)
    pos2 = torch.as_tensor((rng.random((70001, 3)) * 30.0 - 1.0).astype(np.float32)).cuda()
    mass2 = torch.as_tensor((rng.random(70001) * 4.0).astype(np.float32)).cuda()
    ref2 = ctx.deposit(pos2, 30.0, 96, mass=mass2, mass_unit=1.0 / 64).clone()
    ctx.check()
    got2, mt2, st2 = _noalloc(pos2, 30.0, 96, mass=mass2, mass_unit=1.0 / 64)
    assert st2 == 0
    assert torch.equal(got2, ref2)
    ctx.close()


def test_rejects_sizes_beyond_its_scratch():
    pos = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    grid = torch.empty((1,), dtype=torch.int64, device="cuda")
    L = pkg.lib()
    big_ng = L.cwthf_deposit_noalloc(ctypes.c_void_p(pos.data_ptr()), None, 1.0, 10, 10.0, 192,
                                     ctypes.c_void_p(grid.data_ptr()), None, None, None)
    big_np = L.cwthf_deposit_noalloc(ctypes.c_void_p(pos.data_ptr()), None, 1.0, 262145, 10.0, 64,
                                     ctypes.c_void_p(grid.data_ptr()), None, None, None)
    assert big_ng == big_np == pkg._lib.E_SCRATCH_LIMIT
    assert "scratch" in pkg.error_string(big_ng)
