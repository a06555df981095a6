"""ctypes binding of libcwthf.so (see include/cwthf.h).

Argument marshalling only: every step of the halo-finding path runs in the
library's CUDA kernels.  Tensors are PyTorch CUDA tensors (device memory and
streams); host-side scalars go by value.  If the library is missing this
module raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libcwthf.so"
LIB_CHECKED_PATH = _PKG / "libcwthf_checked.so"
HEADER = _PKG.parent / "include" / "cwthf.h"

OK = 0
E_INVALID_ARG, E_UNSUPPORTED_SIZE, E_OVERFLOW, E_OOM, E_CUDA, E_NOT_CONVERGED, E_TIMEOUT, E_CAPACITY, E_BAD_INPUT = range(1, 10)
E_SCRATCH_LIMIT = 10
E_TABLE_CACHE = 11
E_INDEX = 12
CREATE_UNBIND = 1  # cwthf_create_ex: scratch of the self-boundness check
FRAC_BITS = 10
MIN_NG, MAX_NG = 8, 1152
# cwthf_debug_set / cwthf_debug_get keys
DEBUG_JUMP_ROUNDS, DEBUG_CHASE_LIMIT, DEBUG_TMA_NO_COPY, DEBUG_FALLBACK_RAN, DEBUG_TABLE_FILLS = 1, 2, 3, 4, 5
DEBUG_UNBIND_GRID_MIN, DEBUG_CHECKED = 6, 7

HALO_DTYPE = np.dtype([("seed", "<i8"), ("n_part", "<i8"), ("n_cells", "<i8"), ("mass", "<f8"),
                       ("centre", "<f8", (3,)), ("peak", "<f4"), ("reserved", "<i4")])
assert HALO_DTYPE.itemsize == 64


MS_HALO_DTYPE = np.dtype([("seed", "<i8"), ("n_part", "<i8"), ("n_cells", "<i8"), ("mass", "<f8"),
                          ("centre", "<f8", (3,)), ("peak", "<f4"), ("scale", "<i4")])
assert MS_HALO_DTYPE.itemsize == 64


def supported_sizes(lo: int = 8, hi: int = MAX_NG) -> list[int]:
    """Grid sizes the library takes within [lo, hi]: even sizes with an FFT
    plan (radix stages, or a Bluestein pass where the length has a larger
    prime factor)."""
    return [n for n in range(max(lo, 2) + (max(lo, 2) % 2), hi + 1, 2) if check_ng(n)]


def paper_scales(L: float, kw_low: float = 0.1, kw_high: float = 2.5, n: int | None = None, n_ref: int = 400,
                 n_min: int = 150, max_ng: int = MAX_NG):
    """The scale list of the multi-scale loop (Fig. 1, Table 1): n values of
    k_w spaced linearly from kw_low to kw_high (n = Int((kw_high - kw_low) * 8)
    by default), w = k_w * 1000 / L, and the grid Int(n_ref * k_w + n_min) per
    scale rounded to the nearest supported size (an even size, since the real
    transform pairs the x samples; the smaller on a tie), at most max_ng.
    Returns (k_w list, w list, ng list)."""
    if n is None:
        n = int((kw_high - kw_low) * 8)
    kws = [kw_low + (kw_high - kw_low) * i / (n - 1) for i in range(n)] if n > 1 else [kw_low]
    sizes = supported_sizes(8, max_ng)
    ngs = []
    for kw in kws:
        want = int(n_ref * kw + n_min)
        ngs.append(min(sizes, key=lambda s: (abs(s - want), s)))
    return kws, [kw * 1000.0 / L for kw in kws], ngs


class Params(ctypes.Structure):
    _fields_ = [("w", ctypes.c_double), ("cwt_min", ctypes.c_float), ("reserved0", ctypes.c_float),
                ("dens_th", ctypes.c_double), ("particle_th", ctypes.c_int64)]


assert ctypes.sizeof(Params) == 32


class CwthfError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {error_string(code)} (code {code})")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Loads the in-tree libcwthf.so (built by __graft_entry__.build()), or
    its range-checked variant libcwthf_checked.so when the environment sets
    CWTHF_CHECKED=1."""
    global _lib
    if _lib is None:
        path = LIB_CHECKED_PATH if os.environ.get("CWTHF_CHECKED") == "1" else LIB_PATH
        if not path.exists():
            raise ImportError(f"{path} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(str(path))
        P, i64, i32, d, f = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float
        L.cwthf_default_params.argtypes = [d, ctypes.POINTER(Params)]
        L.cwthf_default_params.restype = None
        L.cwthf_create.argtypes = [i32, i32, i64, i32, ctypes.POINTER(P)]
        L.cwthf_create_ex.argtypes = [i32, i32, i64, i32, ctypes.c_uint, ctypes.POINTER(P)]
        L.cwthf_workspace_bytes_ex.argtypes = [i32, i64, i32, ctypes.c_uint, ctypes.POINTER(ctypes.c_size_t)]
        L.cwthf_destroy.argtypes = [P]
        L.cwthf_destroy.restype = None
        L.cwthf_workspace_bytes.argtypes = [i32, i64, i32, ctypes.POINTER(ctypes.c_size_t)]
        L.cwthf_check_ng.argtypes = [i32]
        L.cwthf_deposit.argtypes = [P, P, P, d, i64, d, i32, P, P, P]
        L.cwthf_transform.argtypes = [P, P, i32, d, d, d, P, P]
        L.cwthf_transform_stencil.argtypes = [P, P, i32, d, d, d, i32, P, P]
        L.cwthf_segment.argtypes = [P, P, i32, f, P, P]
        L.cwthf_segment_sizes.argtypes = [P, P, P, i64, P, P]
        L.cwthf_prepare.argtypes = [P, i32, d, ctypes.POINTER(d), i32, P]
        L.cwthf_set_fft_plan.argtypes = [P, i32, i32, i32, ctypes.POINTER(i32), i32]
        L.cwthf_debug_set.argtypes = [P, i32, i64]
        L.cwthf_debug_get.argtypes = [P, i32, ctypes.POINTER(i64), P]
        L.cwthf_assign.argtypes = [P, P, P, d, i64, d, i32, P, P, ctypes.POINTER(Params), P, P, i64, P, P]
        L.cwthf_find.argtypes = [P, P, P, d, i64, d, i32, ctypes.POINTER(Params), i32, P, P, i64, P, P]
        L.cwthf_find_multiscale.argtypes = [P, P, P, d, i64, d, i32, ctypes.POINTER(d), ctypes.POINTER(i32), f, d,
                                            i64, P, d, i32, P, P, i64, P, P]
        L.cwthf_unbind.argtypes = [P, P, P, P, d, i64, d, d, P, i64, i32, P, P, P, P]
        L.cwthf_sync.argtypes = [P, P]
        L.cwthf_error_string.argtypes = [i32]
        L.cwthf_error_string.restype = ctypes.c_char_p
        L.cwthf_launch_count.argtypes = [P]
        L.cwthf_launch_count.restype = i64
        L.cwthf_deposit_noalloc.argtypes = [P, P, d, i64, d, i32, P, P, P, P]
        L.cwthf_profile.argtypes = [P, i32]
        L.cwthf_profile_count.argtypes = [P]
        L.cwthf_profile_read.argtypes = [P, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(d),
                                         ctypes.POINTER(i64)]
        _lib = L
    return _lib


def header_symbols() -> list[str]:
    """Function names declared in include/cwthf.h."""
    text = HEADER.read_text()
    return sorted(set(re.findall(r"CWTHF_API\s+[\w\s\*]+?\b(cwthf_\w+)\s*\(", text)))


def error_string(code: int) -> str:
    return lib().cwthf_error_string(int(code)).decode()


def check_ng(ng: int) -> bool:
    return lib().cwthf_check_ng(int(ng)) == OK


def workspace_bytes(max_ng: int, max_np: int, max_scales: int = 1, unbind: bool = False) -> int:
    out = ctypes.c_size_t(0)
    rc = lib().cwthf_workspace_bytes_ex(int(max_ng), int(max_np), int(max_scales), CREATE_UNBIND if unbind else 0,
                                        ctypes.byref(out))
    if rc:
        raise CwthfError(rc, "cwthf_workspace_bytes_ex")
    return int(out.value)


def default_params(w: float, cwt_min: float = 0.0, dens_th: float = 4.0, particle_th: int = 15) -> Params:
    p = Params()
    lib().cwthf_default_params(float(w), ctypes.byref(p))
    p.cwt_min = cwt_min
    p.dens_th = dens_th
    p.particle_th = particle_th
    return p


def _check(rc: int, what: str):
    if rc != OK:
        raise CwthfError(rc, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """A cwthf_ctx: device scratch sized for grids up to max_ng and up to
    max_np particles (and max_scales scales per find call)."""

    def __init__(self, device: int = 0, max_ng: int = 256, max_np: int = 1 << 24, max_scales: int = 1,
                 unbind: bool = False):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.max_ng, self.max_np, self.max_scales = max_ng, max_np, max_scales
        h = ctypes.c_void_p()
        flags = CREATE_UNBIND if unbind else 0
        _check(lib().cwthf_create_ex(int(device), int(max_ng), int(max_np), int(max_scales), flags, ctypes.byref(h)),
               "cwthf_create_ex")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().cwthf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self, stream):
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        return ctypes.c_void_p(s.cuda_stream)

    def _pos(self, pos):
        t = self.torch
        assert pos.is_cuda and pos.dtype == t.float32 and pos.ndim == 2 and pos.shape[1] == 3
        return pos.contiguous()

    def launch_count(self) -> int:
        return int(lib().cwthf_launch_count(self._h))

    def profile(self, enable: bool = True):
        """Turn per-kernel CUDA-event timing on/off (clears the totals)."""
        _check(lib().cwthf_profile(self._h, 1 if enable else 0), "cwthf_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since profiling was enabled."""
        n = lib().cwthf_profile_count(self._h)
        if n < 0:
            raise CwthfError(-n, "cwthf_profile_count")
        out = {}
        for i in range(n):
            nm, ms, k = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int64()
            _check(lib().cwthf_profile_read(self._h, i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(k)),
                   "cwthf_profile_read")
            out[nm.value.decode()] = (ms.value, k.value)
        return out

    def sync(self, stream=None) -> int:
        return int(lib().cwthf_sync(self._h, self._stream(stream)))

    def check(self, stream=None, what="device status"):
        _check(self.sync(stream), what)

    # -- stages -------------------------------------------------------------
    def deposit(self, pos, L, ng, mass=None, mass_unit=1.0, grid=None, mtot=None, stream=None):
        t = self.torch
        pos = self._pos(pos)
        if grid is None:
            grid = t.empty((ng, ng, ng), dtype=t.int64, device=self.device)
        _check(lib().cwthf_deposit(self._h, _ptr(pos), _ptr(mass), float(mass_unit), pos.shape[0], float(L), int(ng),
                                   _ptr(grid), _ptr(mtot), self._stream(stream)), "cwthf_deposit")
        return grid

    def transform(self, grid, L, w, mass_unit=1.0, cwt=None, stream=None):
        t = self.torch
        ng = grid.shape[0]
        if cwt is None:
            cwt = t.empty((ng, ng, ng), dtype=t.float32, device=self.device)
        _check(lib().cwthf_transform(self._h, _ptr(grid), int(ng), float(L), float(mass_unit), float(w), _ptr(cwt),
                                     self._stream(stream)), "cwthf_transform")
        return cwt

    def transform_stencil(self, grid, L, w, R, mass_unit=1.0, cwt=None, stream=None):
        """The paper's direct-space CWT over the cube of radius R (Sec. 2.1)."""
        t = self.torch
        ng = grid.shape[0]
        if cwt is None:
            cwt = t.empty((ng, ng, ng), dtype=t.float32, device=self.device)
        _check(lib().cwthf_transform_stencil(self._h, _ptr(grid), int(ng), float(L), float(mass_unit), float(w),
                                             int(R), _ptr(cwt), self._stream(stream)), "cwthf_transform_stencil")
        return cwt

    def segment(self, cwt, cwt_min=0.0, label=None, stream=None):
        t = self.torch
        ng = cwt.shape[0]
        if label is None:
            label = t.empty((ng, ng, ng), dtype=t.int32, device=self.device)
        _check(lib().cwthf_segment(self._h, _ptr(cwt.contiguous()), int(ng), float(cwt_min), _ptr(label),
                                   self._stream(stream)), "cwthf_segment")
        return label

    def segment_sizes(self, cap, stream=None):
        """Seeds of the last segmentation and their segments' cell counts:
        (seeds int32 [min(n, cap)], n_cells int64 [min(n, cap)], n) on device / host."""
        t = self.torch
        seeds = t.empty(max(cap, 1), dtype=t.int32, device=self.device)
        n_cells = t.empty(max(cap, 1), dtype=t.int64, device=self.device)
        n = t.zeros(1, dtype=t.int64, device=self.device)
        _check(lib().cwthf_segment_sizes(self._h, _ptr(seeds), _ptr(n_cells), int(cap), _ptr(n),
                                         self._stream(stream)), "cwthf_segment_sizes")
        k = int(n)
        return seeds[:min(k, cap)], n_cells[:min(k, cap)], k

    def prepare(self, ng, L, ws, stream=None):
        """Fill the table slots for grid size ng, box L and scales ws."""
        arr = (ctypes.c_double * max(len(ws), 1))(*ws)
        _check(lib().cwthf_prepare(self._h, int(ng), float(L), arr, len(ws), self._stream(stream)), "cwthf_prepare")

    def set_fft_plan(self, ng: int, which: int, C: int = 0, radices=()) -> bool:
        """Use plan (C, radices) for pass `which` (0: y/z, 1: x) of grid size
        ng; radices=() restores the built-in rule.  False if the kernels
        cannot run that plan."""
        n = len(radices)
        arr = (ctypes.c_int * max(n, 1))(*radices)
        rc = lib().cwthf_set_fft_plan(self._h, int(ng), int(which), int(C), arr, n)
        if rc not in (OK, E_INVALID_ARG):
            raise CwthfError(rc, "cwthf_set_fft_plan")
        return rc == OK

    def table_fills(self) -> int:
        return self.debug_get(DEBUG_TABLE_FILLS)

    def debug_set(self, key: int, value: int):
        _check(lib().cwthf_debug_set(self._h, int(key), int(value)), "cwthf_debug_set")

    def debug_get(self, key: int, stream=None) -> int:
        v = ctypes.c_int64(0)
        _check(lib().cwthf_debug_get(self._h, int(key), ctypes.byref(v), self._stream(stream)), "cwthf_debug_get")
        return int(v.value)

    def assign(self, pos, L, label, cwt=None, mass=None, mass_unit=1.0, dens_th=4.0, particle_th=15,
               cat_cap=None, stream=None):
        """Returns (halo_id, catalogue bytes [cap, 64] on device, n_halo tensor)."""
        t = self.torch
        pos = self._pos(pos)
        ng = label.shape[0]
        if cat_cap is None:
            cat_cap = max(1, ng ** 3 // 8)
        halo_id = t.empty(pos.shape[0], dtype=t.int32, device=self.device)
        cat = t.empty((cat_cap, 64), dtype=t.uint8, device=self.device)
        n_halo = t.zeros(1, dtype=t.int64, device=self.device)
        p = default_params(1.0, 0.0, dens_th, particle_th)
        _check(lib().cwthf_assign(self._h, _ptr(pos), _ptr(mass), float(mass_unit), pos.shape[0], float(L), int(ng),
                                  _ptr(label), _ptr(cwt), ctypes.byref(p), _ptr(halo_id), _ptr(cat), int(cat_cap),
                                  _ptr(n_halo), self._stream(stream)), "cwthf_assign")
        return halo_id, cat, n_halo

    def find(self, pos, L, ng, params, mass=None, mass_unit=1.0, cat_cap=None, halo_id=None, cat=None, n_halo=None,
             stream=None):
        """params: list of Params (one per scale).  Returns (halo_id [n_scales, np],
        catalogue bytes [n_scales, cap, 64], n_halo [n_scales]) on device."""
        t = self.torch
        pos = self._pos(pos)
        ns = len(params)
        if cat_cap is None:
            cat_cap = max(1, ng ** 3 // 8)
        if halo_id is None:
            halo_id = t.empty((ns, pos.shape[0]), dtype=t.int32, device=self.device)
        if cat is None:
            cat = t.empty((ns, cat_cap, 64), dtype=t.uint8, device=self.device)
        if n_halo is None:
            n_halo = t.zeros(ns, dtype=t.int64, device=self.device)
        for name, buf, n in (("halo_id", halo_id, ns * pos.shape[0]), ("cat", cat, ns * cat_cap * 64),
                             ("n_halo", n_halo, ns)):
            if not buf.is_contiguous() or buf.numel() < n:
                raise ValueError(f"{name} must be a contiguous buffer of at least {n} elements")
        arr = (Params * ns)(*params)
        _check(lib().cwthf_find(self._h, _ptr(pos), _ptr(mass), float(mass_unit), pos.shape[0], float(L), int(ng),
                                arr, ns, _ptr(halo_id), _ptr(cat), int(cat_cap), _ptr(n_halo), self._stream(stream)),
               "cwthf_find")
        return halo_id, cat, n_halo

    def find_multiscale(self, pos, L, ws, ngs, mass=None, mass_unit=1.0, cwt_min=0.0, dens_th=4.0, particle_th=15,
                        cat_cap=1 << 20, halo_id=None, cat=None, n_halo=None, stream=None, vel=None,
                        G=4.30091727e-9, max_iter=100):
        """The multi-scale loop over scales ws (largest physical scale first)
        on grids ngs; with velocities, the self-boundness check of every scale's
        kept groups (a context created with unbind=True).  Returns
        (halo_id [np], catalogue bytes [cap, 64], n_halo [1])."""
        t = self.torch
        pos = self._pos(pos)
        if vel is not None:
            vel = self._pos(vel)
        n = len(ws)
        if halo_id is None:
            halo_id = t.empty(pos.shape[0], dtype=t.int32, device=self.device)
        if cat is None:
            cat = t.empty((max(cat_cap, 1), 64), dtype=t.uint8, device=self.device)
        if n_halo is None:
            n_halo = t.zeros(1, dtype=t.int64, device=self.device)
        wa = (ctypes.c_double * n)(*ws)
        na = (ctypes.c_int * n)(*ngs)
        _check(lib().cwthf_find_multiscale(self._h, _ptr(pos), _ptr(mass), float(mass_unit), pos.shape[0], float(L),
                                           n, wa, na, float(cwt_min), float(dens_th), int(particle_th), _ptr(vel),
                                           float(G), int(max_iter), _ptr(halo_id), _ptr(cat), int(cat_cap),
                                           _ptr(n_halo), self._stream(stream)),
               "cwthf_find_multiscale")
        return halo_id, cat, n_halo

    def unbind(self, pos, vel, group, L, G=4.30091727e-9, mass=None, mass_unit=1.0, n_groups=None, max_iter=100,
               group_out=None, n_kept=None, iters=None, stream=None):
        """Sec. 2.3: the self-boundness check of every group (group[i] = its
        index or -1).  G defaults to Mpc/h, km/s, Msun/h.  Returns
        (group after the check [np], members kept [n_groups], rounds [n_groups])."""
        t = self.torch
        pos = self._pos(pos)
        vel = self._pos(vel)
        assert group.is_cuda and group.dtype == t.int32 and group.shape == (pos.shape[0],) and group.is_contiguous()
        if n_groups is None:
            n_groups = int(group.max().item()) + 1 if pos.shape[0] else 0
        if group_out is None:
            group_out = t.empty(pos.shape[0], dtype=t.int32, device=self.device)
        if n_kept is None:
            n_kept = t.zeros(max(n_groups, 1), dtype=t.int64, device=self.device)
        if iters is None:
            iters = t.zeros(max(n_groups, 1), dtype=t.int32, device=self.device)
        _check(lib().cwthf_unbind(self._h, _ptr(pos), _ptr(vel), _ptr(mass), float(mass_unit), pos.shape[0], float(L),
                                  float(G), _ptr(group), int(n_groups), int(max_iter), _ptr(group_out), _ptr(n_kept),
                                  _ptr(iters), self._stream(stream)), "cwthf_unbind")
        return group_out, n_kept[:n_groups], iters[:n_groups]


def ms_catalogue_to_numpy(cat, n) -> np.ndarray:
    """Device multi-scale catalogue bytes -> numpy structured array."""
    n = int(n)
    raw = cat[:n].contiguous().cpu().numpy()
    return raw.view(MS_HALO_DTYPE).reshape(n)


def catalogue_to_numpy(cat, n) -> np.ndarray:
    """Device catalogue bytes -> numpy structured array of the first n halos."""
    n = int(n)
    raw = cat[:n].contiguous().cpu().numpy()
    return raw.view(HALO_DTYPE).reshape(n)
