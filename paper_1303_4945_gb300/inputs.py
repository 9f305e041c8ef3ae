"""Seeded synthetic inputs for the SHT workloads.

This module only draws random numbers; it holds none of the transform's
arithmetic, so both the CUDA path and the CPU oracle can use it.

Conventions (shared by every workload):
  * a_lm are complex128 in triangular m-major order, index m(2 lmax+1-m)/2 + l,
    m = 0..mmax, l = m..lmax.
  * numpy ``default_rng(seed)``; all real parts are drawn first, then all
    imaginary parts, each in storage order.
  * m = 0 coefficients are real (their imaginary part is set to 0), as required
    for a real field (Sect. 5.1.2 of the paper).
"""
from __future__ import annotations

import numpy as np


def nalm(lmax: int, mmax: int) -> int:
    return (mmax + 1) * (lmax + 1) - mmax * (mmax + 1) // 2


def lm_arrays(lmax: int, mmax: int):
    """(l, m) of every stored coefficient, in storage order."""
    ls, ms = [], []
    for m in range(mmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def gaussian_alm(rng, lmax: int, mmax: int, cl=None, lmin: int = 0) -> np.ndarray:
    """Gaussian a_lm.

    cl is None: Re and Im each N(0, 1) (m = 0: Im = 0).
    cl callable: for m > 0 Re, Im ~ N(0, C_l / 2); a_l0 ~ N(0, C_l).
    Coefficients with l < lmin are zero.
    """
    n = nalm(lmax, mmax)
    re = rng.standard_normal(n)
    im = rng.standard_normal(n)
    l, m = lm_arrays(lmax, mmax)
    if cl is not None:
        c = cl(l.astype(np.float64))
        sd = np.where(m == 0, np.sqrt(c), np.sqrt(c / 2.0))
        re = re * sd
        im = im * sd
    im[m == 0] = 0.0
    a = re + 1j * im
    a[l < lmin] = 0.0
    return a


def uniform_alm(rng, lmax: int, mmax: int, lmin: int = 0) -> np.ndarray:
    """Re, Im uniform in [-1, 1) with Im a_l0 = 0 (accuracy test recipe, Sect. 5.1.2)."""
    n = nalm(lmax, mmax)
    re = rng.uniform(-1.0, 1.0, n)
    im = rng.uniform(-1.0, 1.0, n)
    l, m = lm_arrays(lmax, mmax)
    im[m == 0] = 0.0
    a = re + 1j * im
    a[l < lmin] = 0.0
    return a


def cl_inverse_square(l):
    """C_l = 1 / (l + 1)^2."""
    return 1.0 / (l + 1.0) ** 2


def gaussian_map(rng, npix: int) -> np.ndarray:
    return rng.standard_normal(npix)


# ---- named workloads ---------------------------------------------------------

def scalar_gl_small(seed: int = 0, lmax: int = 127):
    """GL nlat = lmax+1, nlon = 2 lmax + 1, spin 0, Re/Im N(0,1)."""
    rng = np.random.default_rng(seed)
    return [gaussian_alm(rng, lmax, lmax)]


def healpix_scalar(seed: int = 1, lmax: int = 1535):
    rng = np.random.default_rng(seed)
    return [gaussian_alm(rng, lmax, lmax, cl=cl_inverse_square)]


def spin2_eb(seed: int = 2, lmax: int = 4095, npairs: int = 1):
    """E, B pairs with C_l = 1/(l+1)^2 and zero monopole and dipole."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(npairs):
        out.append(gaussian_alm(rng, lmax, lmax, cl=cl_inverse_square, lmin=2))
        out.append(gaussian_alm(rng, lmax, lmax, cl=cl_inverse_square, lmin=2))
    return out


def batched_lmax(seed: int = 3, n: int = 64, lo: int = 64, hi: int = 2048):
    """lmax drawn log-uniform in [lo, hi], rounded; drawn before any a_lm."""
    rng = np.random.default_rng(seed)
    lm = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), n))).astype(int)
    return rng, lm
