"""FP64 CPU oracle for the spherical harmonic transform -- TEST INFRASTRUCTURE.

A plain, slow, obviously correct evaluation of the transforms of Reinecke &
Seljebotn 2013 (libsharp), Sect. 2 (Eqs. syn_used, ana_used, syn2, ana2) and
Sect. 4 (spin-s harmonics through Wigner d, adjoint transforms, grids).  The
arithmetic lives in ``sht_oracle.c``; this module only compiles it and
marshals numpy arrays through ctypes.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Parity status per function (see the tests under ``tests/test_oracle_*.py``):
  lambda_      pinned: closed-form Y_lm (l <= 4), Wigner's explicit sum in
               high precision (l <= 20, large-l spot checks), addition theorem.
  synthesis    pinned: brute-force direct summation at lmax <= 8, GL round trip.
  analysis     pinned: GL and ECP round trips, adjoint identity.
  gauss/ecp    pinned: exact integration of polynomials.
  healpix      pinned: pixel count, equal area, symmetry, every pixel centre (Gorski et al. 2005).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sht_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsht_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dpp = ctypes.POINTER(_dp)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no fast-math, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.orc_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
        lib.orc_phase.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dpp, ctypes.c_int, _dp, _dp]
        lib.orc_synthesis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dpp,
                                      ctypes.c_int, _dp, _ip, _dp, _i64p, _dp, ctypes.c_int, _ip, _dpp]
        lib.orc_analysis.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dpp,
                                     ctypes.c_int, _dp, _ip, _dp, _i64p, _dp, ctypes.c_int, _ip, _dpp]
        lib.orc_gauss.argtypes = [ctypes.c_int, _dp, _dp]
        lib.orc_healpix.argtypes = [ctypes.c_int, _dp, _ip, _dp, _dp]
        lib.orc_ecp.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
        for f in (lib.orc_lambda, lib.orc_phase, lib.orc_synthesis, lib.orc_analysis,
                  lib.orc_gauss, lib.orc_healpix, lib.orc_ecp):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _ptrs(arrs):
    return (_dp * len(arrs))(*[_d(a) for a in arrs])


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def nalm(lmax: int, mmax: int) -> int:
    """Number of stored complex a_lm, m = 0..mmax, l = m..lmax."""
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def alm_index(lmax: int, l: int, m: int) -> int:
    """Triangular m-major index m (2 lmax + 1 - m) / 2 + l."""
    return m * (2 * lmax + 1 - m) // 2 + l


# ------------------------------------------------------------------ lambda ---
def lambda_(s: int, m: int, lmax: int, theta: float) -> np.ndarray:
    """sLambda_lm(theta) = (-1)^m sqrt((2l+1)/4pi) d^l_{-m,s}(theta), l = 0..lmax."""
    out = np.zeros(lmax + 1)
    _check(_load().orc_lambda(s, m, lmax, float(theta), _d(out)), "lambda")
    return out


# ------------------------------------------------------------------- grids ---
class Rings:
    """Iso-latitude ring description with unit pixel stride (Sect. 2)."""

    def __init__(self, theta, nphi, phi0, weight, ofs=None):
        self.theta = np.ascontiguousarray(theta, dtype=np.float64)
        self.nphi = np.ascontiguousarray(nphi, dtype=np.int32)
        self.phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
        self.weight = np.ascontiguousarray(weight, dtype=np.float64)
        if ofs is None:
            self.ofs = np.zeros(len(self.theta), dtype=np.int64)
            if len(self.theta) > 1:
                self.ofs[1:] = np.cumsum(self.nphi[:-1], dtype=np.int64)
        else:
            self.ofs = np.ascontiguousarray(ofs, dtype=np.int64)
        self.npix = int(np.max(self.ofs + self.nphi)) if len(self.theta) else 0

    @property
    def nrings(self):
        return len(self.theta)


def gauss_nodes(n: int):
    th = np.zeros(n)
    w = np.zeros(n)
    _check(_load().orc_gauss(n, _d(th), _d(w)), "gauss")
    return th, w


def gauss_rings(nlat: int, nlon: int) -> Rings:
    """GL grid: phi0 = 0, map weight = GL weight * 2 pi / nlon."""
    th, w = gauss_nodes(nlat)
    return Rings(th, np.full(nlat, nlon), np.zeros(nlat), w * 2 * np.pi / nlon)


def healpix_rings(nside: int) -> Rings:
    nr = 4 * nside - 1
    th = np.zeros(nr)
    npf = np.zeros(nr, dtype=np.int32)
    p0 = np.zeros(nr)
    w = np.zeros(nr)
    _check(_load().orc_healpix(nside, _d(th), npf.ctypes.data_as(_ip), _d(p0), _d(w)), "healpix")
    return Rings(th, npf, p0, w)


def ecp_nodes(kind: int, nlat: int):
    th = np.zeros(nlat)
    w = np.zeros(nlat)
    _check(_load().orc_ecp(kind, nlat, _d(th), _d(w)), "ecp")
    return th, w


def ecp_rings(kind: int, nlat: int, nlon: int) -> Rings:
    th, w = ecp_nodes(kind, nlat)
    return Rings(th, np.full(nlat, nlon), np.zeros(nlat), w * 2 * np.pi / nlon)


# -------------------------------------------------------------- transforms ---
def _as_list(x):
    if isinstance(x, np.ndarray) and x.ndim == 1:
        return [x]
    return list(x)


def phase(spin: int, lmax: int, mmax: int, alm, thetas) -> np.ndarray:
    """Legendre stage F_{m,y} of Eq. syn2 for m = -mmax..mmax at the given theta.

    ``alm`` is one complex128 array (spin 0) or an (E, B) pair (spin != 0).
    Returns complex array [len(thetas), 2 mmax + 1].
    """
    al = [np.ascontiguousarray(a, dtype=np.complex128).view(np.float64) for a in _as_list(alm)]
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    out = np.zeros((len(th), 2 * (2 * mmax + 1)))
    _check(_load().orc_phase(spin, lmax, mmax, _ptrs(al), len(th), _d(th), _d(out)), "phase")
    return out.view(np.complex128)


def synthesis(spin: int, lmax: int, mmax: int, alm, rings: Rings, rings_sel=None,
              weighted: bool = False):
    """Eq. syn_used.  Returns a list of real maps (length npix each).

    spin 0: one map per a_lm array.  spin != 0: alm = [E0, B0, E1, B1, ...]
    gives maps [Q0, U0, Q1, U1, ...].  ``rings_sel`` restricts the rings that
    are computed (others stay 0).  ``weighted`` multiplies each ring by its
    weight (adjoint analysis).
    """
    al = [np.ascontiguousarray(a, dtype=np.complex128).view(np.float64) for a in _as_list(alm)]
    maps = [np.zeros(rings.npix) for _ in al]
    sel = None if rings_sel is None else np.ascontiguousarray(rings_sel, dtype=np.int32)
    rc = _load().orc_synthesis(
        spin, lmax, mmax, len(maps), _ptrs(al), rings.nrings, _d(rings.theta),
        rings.nphi.ctypes.data_as(_ip), _d(rings.phi0), rings.ofs.ctypes.data_as(_i64p),
        _d(rings.weight) if weighted else None,
        0 if sel is None else len(sel), None if sel is None else sel.ctypes.data_as(_ip),
        _ptrs(maps))
    _check(rc, "synthesis")
    return maps


def _m_of(lmax: int, mmax: int):
    return np.concatenate([np.full(lmax - m + 1, m) for m in range(mmax + 1)])


def real_to_complex(a, lmax: int, mmax: int):
    """Real-harmonic storage (Sect. 4.5; reading): for m > 0 the two numbers of a
    slot are [a_{l,m}, a_{l,-m}] = sqrt2 (Re a_lm, -Im a_lm), the coefficients of
    the real basis sqrt2 Re Y_lm, sqrt2 Im Y_lm; m = 0 slots are unchanged."""
    a = np.asarray(a, dtype=np.complex128)
    m = _m_of(lmax, mmax)
    c = (a.real - 1j * a.imag) / np.sqrt(2.0)
    return np.where(m > 0, c, a)


def complex_to_real(a, lmax: int, mmax: int):
    """Inverse of real_to_complex."""
    a = np.asarray(a, dtype=np.complex128)
    m = _m_of(lmax, mmax)
    r = np.sqrt(2.0) * (a.real - 1j * a.imag)
    return np.where(m > 0, r, a)


def deriv_synthesis(lmax: int, mmax: int, alm, rings: Rings):
    """Sect. 4.3: maps of df/dtheta and df/(sin(theta) dphi) from spin-0 a_lm.

    Reading: the spin-raising operator gives eth Y_lm = -(d/dtheta + i/sin(theta)
    d/dphi) Y_lm = sqrt(l(l+1)) 1Y_lm, so with the E/B convention of the spin
    synthesis (Q + iU = -sum E_lm 1Y_lm) the spin-1 synthesis of
    E = sqrt(l(l+1)) a_lm, B = 0 returns Q = df/dtheta, U = df/(sin(theta) dphi).
    Returns [dtheta_0, dphi_0, dtheta_1, dphi_1, ...].
    """
    out = []
    for a in _as_list(alm):
        a = np.asarray(a, dtype=np.complex128)
        l = np.concatenate([np.arange(m, lmax + 1) for m in range(mmax + 1)]).astype(np.float64)
        e = a * np.sqrt(l * (l + 1.0))
        out += synthesis(1, lmax, mmax, [e, np.zeros_like(e)], rings)
    return out


def analysis(spin: int, lmax: int, mmax: int, maps, rings: Rings, m_sel=None,
             adjoint: bool = False):
    """Eq. ana_used (adjoint=True: all weights 1, i.e. adjoint synthesis).

    Returns a list of complex128 a_lm arrays (triangular m-major layout).
    ``m_sel`` restricts the m that are computed (others stay 0).
    """
    mp = [np.ascontiguousarray(x, dtype=np.float64) for x in _as_list(maps)]
    n = nalm(lmax, mmax)
    outs = [np.zeros(2 * n) for _ in mp]
    sel = None if m_sel is None else np.ascontiguousarray(m_sel, dtype=np.int32)
    rc = _load().orc_analysis(
        spin, lmax, mmax, len(mp), _ptrs(mp), rings.nrings, _d(rings.theta),
        rings.nphi.ctypes.data_as(_ip), _d(rings.phi0), rings.ofs.ctypes.data_as(_i64p),
        None if adjoint else _d(rings.weight),
        0 if sel is None else len(sel), None if sel is None else sel.ctypes.data_as(_ip),
        _ptrs(outs))
    _check(rc, "analysis")
    return [o.view(np.complex128) for o in outs]
