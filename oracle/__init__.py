"""fp64 CPU oracle of the single-scale CWTHF path (arXiv:2501.10622).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The CUDA library never imports,
links or calls anything here, and nothing here imports the CUDA library.

The arithmetic lives in ``cwthf_oracle.c`` (plain C, fp64, single thread);
this module only compiles it with gcc and marshals numpy arrays through ctypes.
Each wrapper names the part of the paper its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "cwthf_oracle.c"
_LIB = _HERE / "liboracle.so"
_lib = None

OK, E_ARG, E_OVERFLOW, E_INEXACT, E_NOMEM, E_CAPACITY = range(6)
FRAC_BITS = 10


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no FMA contraction, so fp64 results are the
    same on x86-64 and aarch64)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < max(_SRC.stat().st_mtime, (_HERE / "cwthf_oracle.h").stat().st_mtime):
        tmp = _LIB.with_suffix(f".so.{os.getpid()}")
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fno-fast-math", str(_SRC), "-lm", "-o", str(tmp)], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        P = ctypes.c_void_p
        i64, i32, d, f = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_float
        L.orc_quantise.argtypes = [P, i64, d, i32, P]
        L.orc_cic.argtypes = [P, P, d, i64, d, i32, P, P]
        L.orc_wavelet.argtypes = [d, d]
        L.orc_wavelet.restype = d
        L.orc_kernel.argtypes = [i32, d, d, P]
        L.orc_kernel.restype = None
        L.orc_dft1d.argtypes = [P, P, i32, i32]
        L.orc_dft3d.argtypes = [P, P, i32, i32]
        L.orc_cwt.argtypes = [P, i32, d, d, d, P]
        L.orc_cwt_direct.argtypes = [P, i32, d, d, d, P]
        L.orc_cwt_at.argtypes = [P, i32, d, d, d, P, i64, P]
        L.orc_cwt_stencil.argtypes = [P, i32, d, d, d, i32, P]
        L.orc_cwt_stencil_at.argtypes = [P, i32, d, d, d, i32, P, i64, P]
        L.orc_parent.argtypes = [P, i32, P]
        L.orc_segment.argtypes = [P, i32, f, P]
        L.orc_assign.argtypes = [P, P, d, i64, d, i32, P, P, d, i64, P, i64, P, P, P, P, P, P, P]
        L.orc_corrected_peak.argtypes = [P, i32, i64, i32]
        L.orc_corrected_peak.restype = f
        L.orc_cross_scale.argtypes = [P, i32, i64, P, i32]
        L.orc_multiscale.argtypes = [P, P, d, i64, d, i32, P, P, f, d, i64, P, d, i32, P, i64, P, P, P, P, P, P, P, P,
                                     P]
        L.orc_unbind.argtypes = [P, P, P, d, i64, d, d, P, i64, i32, P, P, P, P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


def _pos(pos):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    assert pos.ndim == 2 and pos.shape[1] == 3
    return pos


def _mass(mass):
    return None if mass is None else np.ascontiguousarray(mass, dtype=np.float32)


def quantise(pos, L: float, ng: int) -> np.ndarray:
    """Fixed-point positions floor(x*(N/L)*2^10) mod N*2^10, int64 [np][3]."""
    pos = _pos(pos)
    q = np.empty(pos.shape, dtype=np.int64)
    _check(lib().orc_quantise(_ptr(pos), pos.shape[0], float(L), int(ng), _ptr(q)), "quantise")
    return q


def cic(pos, L: float, ng: int, mass=None, mass_unit: float = 1.0):
    """Sec. 2.1 Eq. 1: CIC mass grid, int64 [ng,ng,ng] in units of mass_unit*2^-30,
    and the integer total mass sum m_q."""
    pos, mass = _pos(pos), _mass(mass)
    grid = np.empty((ng, ng, ng), dtype=np.int64)
    mt = np.zeros(1, dtype=np.int64)
    _check(lib().orc_cic(_ptr(pos), _ptr(mass), float(mass_unit), pos.shape[0], float(L), int(ng),
                         _ptr(grid), _ptr(mt)), "cic")
    return grid, int(mt[0])


def wavelet(w: float, r2: float) -> float:
    """Sec. 2.1 Eq. 4: Psi(w, r) for r^2 = r2."""
    return lib().orc_wavelet(float(w), float(r2))


def kernel(ng: int, L: float, w: float) -> np.ndarray:
    """Psi sampled at minimum-image grid offsets, fp64 [ng,ng,ng]."""
    K = np.empty((ng, ng, ng), dtype=np.float64)
    lib().orc_kernel(int(ng), float(L), float(w), _ptr(K))
    return K


def dft1d(x, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    _check(lib().orc_dft1d(_ptr(re), _ptr(im), x.size, int(sign)), "dft1d")
    return re + 1j * im


def dft3d(x, sign: int = -1) -> np.ndarray:
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[0]
    assert x.shape == (n, n, n)
    re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    _check(lib().orc_dft3d(_ptr(re), _ptr(im), n, int(sign)), "dft3d")
    return re + 1j * im


def cwt(grid, L: float, w: float, mass_unit: float = 1.0) -> np.ndarray:
    """Sec. 2.1 Eq. 2-3: grid CWT through the DFT (circular convolution), fp64."""
    grid = np.ascontiguousarray(grid, dtype=np.int64)
    ng = grid.shape[0]
    C = np.empty(grid.shape, dtype=np.float64)
    _check(lib().orc_cwt(_ptr(grid), ng, float(L), float(mass_unit), float(w), _ptr(C)), "cwt")
    return C


def cwt_direct(grid, L: float, w: float, mass_unit: float = 1.0) -> np.ndarray:
    """Eq. 2 summed literally over all node pairs, O(N^6): tiny grids only."""
    grid = np.ascontiguousarray(grid, dtype=np.int64)
    ng = grid.shape[0]
    C = np.empty(grid.shape, dtype=np.float64)
    _check(lib().orc_cwt_direct(_ptr(grid), ng, float(L), float(mass_unit), float(w), _ptr(C)), "cwt_direct")
    return C


def cwt_at(grid, L: float, w: float, nodes, mass_unit: float = 1.0) -> np.ndarray:
    """Eq. 2 summed literally at the given linear node indices (the wavelet's
    fp64 support only, which is the full sum): full-size spot checks."""
    grid = np.ascontiguousarray(grid, dtype=np.int64)
    ng = grid.shape[0]
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty(nodes.shape[0], dtype=np.float64)
    _check(lib().orc_cwt_at(_ptr(grid), ng, float(L), float(mass_unit), float(w), _ptr(nodes), nodes.shape[0],
                            _ptr(out)), "cwt_at")
    return out


def gdw_resolution(kw: float) -> int:
    """Table 1: stencil size of the sampled wavelet, Int(1.5 / k_w + 5)."""
    return int(1.5 / kw + 5)


def cwt_stencil(grid, L: float, w: float, R: int, mass_unit: float = 1.0) -> np.ndarray:
    """Sec. 2.1 as the paper evaluates it: every node adds its mass times the
    wavelet sampled on the cube of offsets |d_x|, |d_y|, |d_z| <= R around it
    (periodic), fp64 literal sum."""
    grid = np.ascontiguousarray(grid, dtype=np.int64)
    ng = grid.shape[0]
    C = np.empty(grid.shape, dtype=np.float64)
    _check(lib().orc_cwt_stencil(_ptr(grid), ng, float(L), float(mass_unit), float(w), int(R), _ptr(C)),
           "cwt_stencil")
    return C


def cwt_stencil_at(grid, L: float, w: float, R: int, nodes, mass_unit: float = 1.0) -> np.ndarray:
    """cwt_stencil at the given linear node indices only."""
    grid = np.ascontiguousarray(grid, dtype=np.int64)
    ng = grid.shape[0]
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty(nodes.shape[0], dtype=np.float64)
    _check(lib().orc_cwt_stencil_at(_ptr(grid), ng, float(L), float(mass_unit), float(w), int(R), _ptr(nodes),
                                    nodes.shape[0], _ptr(out)), "cwt_stencil_at")
    return out


def parent(C) -> np.ndarray:
    """Best cell of self + 26 periodic neighbours under (value, -index)."""
    C = np.ascontiguousarray(C, dtype=np.float32)
    P = np.empty(C.shape, dtype=np.int32)
    _check(lib().orc_parent(_ptr(C), C.shape[0], _ptr(P)), "parent")
    return P


def segment(C, cwt_min: float = 0.0) -> np.ndarray:
    """Sec. 2.3: steepest-ascent segments; label = seed cell index or -1."""
    C = np.ascontiguousarray(C, dtype=np.float32)
    lab = np.empty(C.shape, dtype=np.int32)
    _check(lib().orc_segment(_ptr(C), C.shape[0], float(cwt_min), _ptr(lab)), "segment")
    return lab


def assign(pos, L: float, label, C=None, mass=None, mass_unit: float = 1.0,
           dens_th: float = 4.0, particle_th: int = 15, cap: int | None = None):
    """Sec. 2 steps 6-7, Sec. 2.3-2.4, Table 1: particle halo ids and the
    catalogue (dict of columns, sorted by seed)."""
    pos, mass = _pos(pos), _mass(mass)
    label = np.ascontiguousarray(label, dtype=np.int32)
    ng = label.shape[0]
    np_ = pos.shape[0]
    if cap is None:
        cap = int((label.ravel() == np.arange(label.size, dtype=np.int64)).sum()) + 1
    Cf = None if C is None else np.ascontiguousarray(C, dtype=np.float32)
    hid = np.empty(np_, dtype=np.int32)
    seed = np.empty(cap, np.int64); npart = np.empty(cap, np.int64); ncell = np.empty(cap, np.int64)
    mass_o = np.empty(cap, np.float64); cen = np.empty((cap, 3), np.float64); peak = np.empty(cap, np.float32)
    nh = np.zeros(1, np.int64)
    rc = lib().orc_assign(_ptr(pos), _ptr(mass), float(mass_unit), np_, float(L), ng, _ptr(label), _ptr(Cf),
                          float(dens_th), int(particle_th), _ptr(hid), int(cap), _ptr(seed), _ptr(npart),
                          _ptr(ncell), _ptr(mass_o), _ptr(cen), _ptr(peak), _ptr(nh))
    _check(rc, "assign")
    n = int(nh[0])
    cat = dict(seed=seed[:n], n_part=npart[:n], n_cells=ncell[:n], mass=mass_o[:n], centre=cen[:n], peak=peak[:n])
    return hid, cat


def find(pos, L: float, ng: int, w: float, mass=None, mass_unit: float = 1.0, cwt_min: float = 0.0,
         dens_th: float = 4.0, particle_th: int = 15):
    """The whole single-scale path in the paper's order (Sec. 2 steps 2-7):
    CIC grid -> CWT (fp64) -> rounded to fp32 -> segments -> halos."""
    grid, _ = cic(pos, L, ng, mass, mass_unit)
    C64 = cwt(grid, L, w, mass_unit)
    C32 = C64.astype(np.float32)
    lab = segment(C32, cwt_min)
    hid, cat = assign(pos, L, lab, C32, mass, mass_unit, dens_th, particle_th)
    return dict(grid=grid, cwt=C64, cwt32=C32, label=lab, halo_id=hid, cat=cat)


# ---- the multi-scale identification loop (Sec. 2, Fig. 1, App. B, Sec. 2.4) ----

def corrected_peak(C, seed: int, ng_next: int = 0) -> float:
    """App. B: the maximum at linear node `seed` plus the per-axis quadratic
    terms l1^2/(16 l2 - 8 l1) (Eq. B1), plus the grid-size term when the next
    scale's grid has ng_next nodes per side (0: none).  fp32, as both sides."""
    C = np.ascontiguousarray(C, dtype=np.float32)
    return float(lib().orc_corrected_peak(_ptr(C), C.shape[0], int(seed), int(ng_next)))


def cross_scale(C, seed: int, C_next=None) -> bool:
    """Sec. 2: the corrected peak exceeds the 2x2x2 nodes of the next scale's
    field enclosing the seed's position (a zero field when C_next is None)."""
    C = np.ascontiguousarray(C, dtype=np.float32)
    Cn = None if C_next is None else np.ascontiguousarray(C_next, dtype=np.float32)
    ngn = 0 if Cn is None else Cn.shape[0]
    return bool(lib().orc_cross_scale(_ptr(C), C.shape[0], int(seed), _ptr(Cn), ngn))


def multiscale_on_fields(pos, L: float, fields, mass=None, mass_unit: float = 1.0, cwt_min: float = 0.0,
                         dens_th: float = 4.0, particle_th: int = 15, cap: int = 1 << 20, vel=None,
                         G: float = None, max_iter: int = 100):
    """The loop of Fig. 1 on given fp32 fields (largest physical scale first):
    final halo ids and the catalogue (dict of columns, in halo-id order).
    With velocities, every scale's kept groups pass the self-boundness check
    (Sec. 2.3) before they get ids; cat["margin"] is then the smallest
    relative distance of any of its decisions from its threshold."""
    pos, mass = _pos(pos), _mass(mass)
    if vel is not None:
        vel = _pos(vel)
    if G is None:
        G = G_MPC_KMS_MSUN
    fs = [np.ascontiguousarray(f, dtype=np.float32) for f in fields]
    n = len(fs)
    ngs = np.array([f.shape[0] for f in fs], dtype=np.int32)
    ptrs = (ctypes.c_void_p * n)(*[f.ctypes.data for f in fs])
    hid = np.empty(pos.shape[0], np.int32)
    sc = np.empty(cap, np.int32); seed = np.empty(cap, np.int64); npart = np.empty(cap, np.int64)
    ncell = np.empty(cap, np.int64); mass_o = np.empty(cap, np.float64); cen = np.empty((cap, 3), np.float64)
    peak = np.empty(cap, np.float32); nh = np.zeros(1, np.int64)
    margin = ctypes.c_double(float("inf"))
    _check(lib().orc_multiscale(_ptr(pos), _ptr(mass), float(mass_unit), pos.shape[0], float(L), n, _ptr(ngs),
                                ctypes.cast(ptrs, ctypes.c_void_p), float(cwt_min), float(dens_th), int(particle_th),
                                _ptr(vel), float(G), int(max_iter), _ptr(hid), int(cap), _ptr(sc), _ptr(seed),
                                _ptr(npart), _ptr(ncell), _ptr(mass_o), _ptr(cen), _ptr(peak), _ptr(nh),
                                ctypes.byref(margin)), "multiscale")
    k = int(nh[0])
    cat = dict(scale=sc[:k], seed=seed[:k], n_part=npart[:k], n_cells=ncell[:k], mass=mass_o[:k], centre=cen[:k],
               peak=peak[:k], margin=margin.value)
    return hid, cat


def find_multiscale(pos, L: float, ws, ngs, mass=None, mass_unit: float = 1.0, cwt_min: float = 0.0,
                    dens_th: float = 4.0, particle_th: int = 15, vel=None, G: float = None, max_iter: int = 100):
    """The whole loop: per scale the CIC grid on its own ng^3 grid and the
    fp64 CWT rounded to fp32, then multiscale_on_fields."""
    fields = []
    for w, ng in zip(ws, ngs):
        grid, _ = cic(pos, L, ng, mass, mass_unit)
        fields.append(cwt(grid, L, w, mass_unit).astype(np.float32))
    hid, cat = multiscale_on_fields(pos, L, fields, mass, mass_unit, cwt_min, dens_th, particle_th, vel=vel, G=G,
                                    max_iter=max_iter)
    return dict(fields=fields, halo_id=hid, cat=cat)


# G in (Mpc/h) (km/s)^2 / (Msun/h): positions in Mpc/h, velocities in km/s,
# masses in Msun/h (the h cancels in G M / r).
G_MPC_KMS_MSUN = 4.30091727e-9


def unbind(pos, vel, group, L: float, G: float = G_MPC_KMS_MSUN, mass=None, mass_unit: float = 1.0,
           n_groups: int | None = None, max_iter: int = 100):
    """Sec. 2.3: the self-boundness check of every group (group[i] = index or
    -1).  Returns (group after the check, members kept per group, rounds per
    group, smallest relative distance of any decision from its threshold)."""
    pos, mass = _pos(pos), _mass(mass)
    vel = _pos(vel)
    group = np.ascontiguousarray(group, dtype=np.int32)
    np_ = pos.shape[0]
    assert vel.shape == pos.shape and group.shape == (np_,)
    if n_groups is None:
        n_groups = int(group.max()) + 1 if np_ else 0
    out = np.empty(np_, dtype=np.int32)
    n_out = np.zeros(max(n_groups, 1), dtype=np.int64)
    it_out = np.zeros(max(n_groups, 1), dtype=np.int32)
    margin = ctypes.c_double()
    _check(lib().orc_unbind(_ptr(pos), _ptr(vel), _ptr(mass), float(mass_unit), np_, float(L), float(G), _ptr(group),
                            int(n_groups), int(max_iter), _ptr(out), _ptr(n_out), _ptr(it_out), ctypes.byref(margin)),
           "unbind")
    return out, n_out[:n_groups], it_out[:n_groups], margin.value
