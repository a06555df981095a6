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


def test_supported_grid_sizes():
    smooth = sorted({2 ** a * 3 ** b for a in range(1, 11) for b in range(0, 7) if 8 <= 2 ** a * 3 ** b <= 1024})
    for n in smooth:
        assert pkg.check_ng(n), n
    for n in (4, 6, 7, 22, 26, 27, 81, 1152, 2048, 190, 1150):
        assert not pkg.check_ng(n), n
    assert synth.smooth_ng(190) in smooth and synth.smooth_ng(1150) == 1024


def test_workspace_bytes_monotone_and_errors():
    a = pkg.workspace_bytes(64, 1 << 18)
    b = pkg.workspace_bytes(128, 1 << 18)
    c = pkg.workspace_bytes(128, 1 << 20)
    d = pkg.workspace_bytes(128, 1 << 20, 3)
    assert 0 < a < b < c < d
    with pytest.raises(pkg.CwthfError):
        pkg.workspace_bytes(190, 10)
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
    assert pkg.lib().cwthf_create(0, 190, 100, 1, ctypes.byref(h)) == 2
    assert pkg.lib().cwthf_create(0, 64, -1, 1, ctypes.byref(h)) == 1
    assert pkg.lib().cwthf_sync(None, None) == 1


def test_radix_five_and_seven_sizes():
    # radix-5 and radix-7 stages: the paper's grid rule Int(400 k_w + 150) lands
    # on sizes such as 350 = 2 5^2 7 or 750 = 2 3 5^3; sizes with a prime factor
    # above 7 (190 = 2 5 19, 1150 = 2 5^2 23) need Bluestein and stay refused
    for n in (10, 14, 20, 28, 30, 40, 50, 70, 100, 140, 250, 270, 350, 750, 1000):
        assert pkg.check_ng(n), n
    for n in (22, 26, 190, 230, 1150, 9, 15):
        assert not pkg.check_ng(n), n
    sizes = pkg.supported_sizes(8, 1024)
    assert 350 in sizes and 190 not in sizes and all(s % 2 == 0 for s in sizes)
