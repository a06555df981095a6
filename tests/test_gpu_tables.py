"""The FFT and wavelet table slots of a context: sized by cwthf_create, so no
later call allocates device memory.  A call captured into a CUDA graph brings
its own table copies, so a graph can use a (grid, box, scale) that no eager
call has seen; a long stream of distinct boxes keeps device memory constant."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth

pytestmark = pytest.mark.gpu


def _box(ng, seed):
    L = ng * 0.78125
    return synth.clumped_box(ng ** 3, L, max(2, ng ** 3 // 1300), seed=seed).cuda(), L


def _outputs(ns, np_, cap=1 << 12):
    return (torch.full((ns, np_), -7, dtype=torch.int32, device="cuda"),
            torch.zeros((ns, cap, 64), dtype=torch.uint8, device="cuda"),
            torch.full((ns,), -7, dtype=torch.int64, device="cuda"))


def test_capture_with_never_seen_tables_and_no_eager_run():
    ctx = pkg.Context(0, max_ng=64, max_np=1 << 18, max_scales=2)
    try:
        p32, L32 = _box(32, 1)
        ctx.find(p32, L32, 32, [pkg.default_params(2.0)], cat_cap=1 << 12)  # loads the kernels, other tables
        ctx.check()
        pos, L = _box(48, 2)
        params = [pkg.default_params(2.7), pkg.default_params(3.1)]  # a grid, box and scales never seen
        hid, cat, nh = _outputs(2, pos.shape[0])
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ctx.find(pos, L, 48, params, cat_cap=1 << 12, halo_id=hid, cat=cat, n_halo=nh, stream=s)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        ref = pkg.Context(0, max_ng=48, max_np=pos.shape[0], max_scales=2)
        try:
            h2, c2, n2 = ref.find(pos, L, 48, params, cat_cap=1 << 12)
            ref.check()
        finally:
            ref.close()
        assert torch.equal(hid, h2) and torch.equal(nh, n2) and int(nh.min()) > 0
        # an eager call may now read the slots the graph filled
        h3, c3, n3 = ctx.find(pos, L, 48, params, cat_cap=1 << 12)
        ctx.check()
        assert torch.equal(h3, h2)
    finally:
        ctx.close()


def test_distinct_boxes_keep_device_memory_constant():
    # 50 boxes of distinct size and scale (more than the context's 48 table
    # slots, so slots are reused): device memory does not move after the first
    ctx = pkg.Context(0, max_ng=48, max_np=48 ** 3, max_scales=1)
    try:
        pos, _ = _box(48, 3)
        hid, cat, nh = _outputs(1, pos.shape[0])
        ctx.find(pos, 30.0, 48, [pkg.default_params(2.0)], cat_cap=1 << 12, halo_id=hid, cat=cat, n_halo=nh)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        counts = []
        for i in range(50):
            L = 30.0 + 0.37 * i
            ctx.find(pos, L, 48, [pkg.default_params(1.5 + 0.05 * i)], cat_cap=1 << 12, halo_id=hid, cat=cat,
                     n_halo=nh)
            ctx.check()
            counts.append(int(nh[0]))
        assert torch.cuda.mem_get_info()[0] == free0
        assert len(set(counts)) > 1
        # slots reused after eviction still give the eager result of a fresh context
        ref = pkg.Context(0, max_ng=48, max_np=pos.shape[0], max_scales=1)
        try:
            h2, _, n2 = ref.find(pos, 30.0 + 0.37 * 3, 48, [pkg.default_params(1.5 + 0.05 * 3)], cat_cap=1 << 12)
            h1, _, n1 = ctx.find(pos, 30.0 + 0.37 * 3, 48, [pkg.default_params(1.5 + 0.05 * 3)], cat_cap=1 << 12)
            ref.check()
            ctx.check()
            assert torch.equal(h1, h2) and int(n1[0]) == int(n2[0]) == counts[3]
        finally:
            ref.close()
    finally:
        ctx.close()


def test_capture_without_a_free_slot_is_refused():
    # a capture may only fill free slots: with all 48 taken by the graph being
    # captured (one twiddle slot, 47 wavelet slots), the next new scale fails
    # with CWTHF_E_TABLE_CACHE instead of evicting a slot the graph reads
    ctx = pkg.Context(0, max_ng=16, max_np=16, max_scales=1)
    try:
        grid = torch.zeros((16, 16, 16), dtype=torch.int64, device="cuda")
        grid[3, 4, 5] = 1 << 30
        cwt = torch.empty((16, 16, 16), dtype=torch.float32, device="cuda")
        s = torch.cuda.Stream()
        lib = pkg.lib()
        rcs = []
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            g.capture_begin()
            try:
                for i in range(48):
                    rcs.append(lib.cwthf_transform(ctx._h, ctypes.c_void_p(grid.data_ptr()), 16, 12.5, 1.0,
                                                   1.0 + 0.01 * i, ctypes.c_void_p(cwt.data_ptr()),
                                                   ctypes.c_void_p(s.cuda_stream)))
            finally:
                g.capture_end()
        assert rcs[:47] == [0] * 47 and rcs[47] == pkg._lib.E_TABLE_CACHE
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        # outside a capture the same call evicts nothing the graph reads and cannot
        # find a slot either (every slot is kept for the graph)
        assert lib.cwthf_transform(ctx._h, ctypes.c_void_p(grid.data_ptr()), 16, 12.5, 1.0, 9.0,
                                   ctypes.c_void_p(cwt.data_ptr()), None) == pkg._lib.E_TABLE_CACHE
        # a scale the graph already holds still works eagerly
        assert lib.cwthf_transform(ctx._h, ctypes.c_void_p(grid.data_ptr()), 16, 12.5, 1.0, 1.0,
                                   ctypes.c_void_p(cwt.data_ptr()), None) == 0
        torch.cuda.synchronize()
        ctx.check()
        c = cwt.cpu().numpy()
        assert np.isfinite(c).all() and c.max() > 0
    finally:
        ctx.close()
