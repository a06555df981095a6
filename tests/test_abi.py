"""The C-ABI library builds, loads and exports every entry point its header
declares; its host-only calls answer without a GPU."""
import ctypes
import subprocess

import pytest

import paper_2501_10622_gb300 as pkg
from paper_2501_10622_gb300 import synth


def test_library_exports_every_declared_symbol():
    names = pkg.header_symbols()
    assert len(names) >= 12
    L = pkg.lib()
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", str(pkg._lib.LIB_PATH)], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported
    # nothing but the C ABI is exported
    assert all(e.startswith("cwthf_") or e.startswith("_") for e in exported), sorted(exported)[:10]


def test_checked_library_exports_the_same_symbols():
    # the range-checked build (CWTHF_CHECKED) is the same ABI
    path = pkg._lib.LIB_CHECKED_PATH
    assert path.exists(), path
    names = pkg.header_symbols()
    L = ctypes.CDLL(str(path))
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", str(path)], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported
    assert all(e.startswith("cwthf_") or e.startswith("_") for e in exported), sorted(exported)[:10]


def test_supported_grid_sizes():
    # every even size from 8 to 1152 (the paper's largest grid, Int(400 2.5 +
    # 150) = 1150, included): radix stages, or Bluestein passes where the
    # length has a prime factor above 7; odd sizes and sizes out of range are
    # refused
    for n in range(8, 1153, 2):
        assert pkg.check_ng(n), n
    for n in (4, 6, 7, 9, 27, 81, 191, 1023, 1151, 1154, 1156, 2048):
        assert not pkg.check_ng(n), n
    smooth = sorted({2 ** a * 3 ** b for a in range(1, 11) for b in range(0, 7) if 8 <= 2 ** a * 3 ** b <= 1024})
    assert synth.smooth_ng(190) in smooth and synth.smooth_ng(1150) == 1024


def test_workspace_bytes_monotone_and_errors():
    a = pkg.workspace_bytes(64, 1 << 18)
    b = pkg.workspace_bytes(128, 1 << 18)
    c = pkg.workspace_bytes(128, 1 << 20)
    d = pkg.workspace_bytes(128, 1 << 20, 3)
    assert 0 < a < b < c < d
    # the self-boundness check's scratch only when asked for: 28 B per particle + 8 per group
    u = pkg.workspace_bytes(128, 1 << 20, 3, unbind=True)
    assert u - d >= 28 * (1 << 20) + 8 * (128 ** 3 // 8)
    with pytest.raises(pkg.CwthfError):
        pkg.workspace_bytes(191, 10)
    with pytest.raises(pkg.CwthfError):
        pkg.workspace_bytes(64, -1)


def test_error_strings_and_defaults():
    for code in range(0, 10):
        assert pkg.error_string(code)
    assert "unknown" in pkg.error_string(99)
    p = pkg.default_params(2.0)
    assert (p.w, p.cwt_min, p.dens_th, p.particle_th) == (2.0, 0.0, 4.0, 15)


def test_create_reports_instead_of_crashing_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert pkg.lib().cwthf_create(0, 64, 100, 1, ctypes.byref(h)) == 5  # CWTHF_E_CUDA
    assert pkg.lib().cwthf_create(0, 191, 100, 1, ctypes.byref(h)) == 2
    assert pkg.lib().cwthf_create(0, 64, -1, 1, ctypes.byref(h)) == 1
    assert pkg.lib().cwthf_sync(None, None) == 1


def test_radix_five_seven_and_bluestein_sizes():
    # radix-5 and radix-7 stages cover sizes such as 350 = 2 5^2 7 or
    # 750 = 2 3 5^3; sizes with a larger prime factor (190 = 2 5 19,
    # 1022 = 2 7 73) run Bluestein passes, so the paper's grid rule
    # Int(400 k_w + 150) is taken to the nearest even size
    for n in (10, 14, 20, 28, 30, 40, 50, 70, 100, 140, 250, 270, 350, 750, 1000, 22, 26, 190, 230, 1022, 1150):
        assert pkg.check_ng(n), n
    for n in (9, 15, 189, 1151):
        assert not pkg.check_ng(n), n
    sizes = pkg.supported_sizes(8, 1152)
    assert sizes == list(range(8, 1153, 2))
    kws, ws, ngs = pkg.paper_scales(50.0, n=20)
    want = [int(400 * k + 150) for k in kws]
    # within one cell of the rule at every scale, the paper's 190 and 1150 included
    assert all(abs(g - v) <= 1 and g % 2 == 0 for g, v in zip(ngs, want)), (ngs, want)
    assert ngs[0] == 190 and ngs[-1] == 1150
    # a smaller limit caps the grids
    assert max(pkg.paper_scales(50.0, n=20, max_ng=1024)[2]) == 1024
