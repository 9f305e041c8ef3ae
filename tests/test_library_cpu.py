"""CPU tests of the C-ABI library: it loads without a GPU, exports every function
include/sht_gb300.h declares, and its host-only parts (grid builders, ring
pairing, a_lm layouts, argument checks) agree with the oracle / the paper."""
import ctypes
import math
import re

import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import build as libbuild

libbuild.build()
from paper_1303_4945_gb300 import sht  # noqa: E402


def test_exports_every_declared_symbol():
    names = sht.exported_symbols_declared()
    assert len(names) >= 15
    lib = ctypes.CDLL(sht.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and nothing internal leaks out under the sht_ prefix that the header does not declare
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", sht.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sht_\w+)", out))
    assert exported == set(names), exported ^ set(names)


def test_error_strings():
    for code in (0, -1, -2, -3, -4, -5):
        assert sht._lib.sht_strerror(code)
    with pytest.raises(sht.ShtError) as e:
        sht.sht_geom_gauss(0, 10)
    assert e.value.code == sht.SHT_ERR_INVALID_ARG


@pytest.mark.parametrize("nlat", [1, 2, 5, 64, 129, 1024])
def test_gauss_grid_matches_oracle(nlat):
    g = sht.sht_geom_gauss(nlat, 7)
    r = g.rings()
    th, w = oracle.gauss_nodes(nlat)
    np.testing.assert_allclose(r["theta"], th, rtol=0, atol=4e-16 * max(1, nlat / 64))
    np.testing.assert_allclose(r["weight"], w * 2 * np.pi / 7, rtol=2e-14)
    assert np.all(r["nphi"] == 7) and np.all(r["phi0"] == 0) and np.all(r["stride"] == 1)
    np.testing.assert_array_equal(r["ofs"], np.arange(nlat) * 7)
    nr, npix, npairs = g.info()
    assert (nr, npix, npairs) == (nlat, 7 * nlat, (nlat + 1) // 2)


@pytest.mark.parametrize("nside", [1, 2, 8, 64])
def test_healpix_grid_matches_oracle(nside):
    g = sht.sht_geom_healpix(nside)
    r = g.rings()
    o = oracle.healpix_rings(nside)
    np.testing.assert_allclose(r["theta"], o.theta, atol=1e-15)
    np.testing.assert_array_equal(r["nphi"], o.nphi)
    np.testing.assert_allclose(r["phi0"], o.phi0, atol=1e-16)
    np.testing.assert_allclose(r["weight"], o.weight, rtol=1e-15)
    np.testing.assert_array_equal(r["ofs"], o.ofs)
    assert g.info() == (4 * nside - 1, 12 * nside * nside, 2 * nside)


@pytest.mark.parametrize("kind,nlat", [(0, 8), (0, 9), (1, 10), (1, 7), (2, 11), (2, 12)])
def test_ecp_grid_matches_oracle(kind, nlat):
    g = sht.sht_geom_ecp(kind, nlat, 5)
    r = g.rings()
    th, w = oracle.ecp_nodes(kind, nlat)
    np.testing.assert_allclose(r["theta"], th, atol=1e-15)
    np.testing.assert_allclose(r["weight"], w * 2 * np.pi / 5, rtol=1e-13, atol=1e-16)


def test_general_and_subset():
    g = sht.sht_geom_gauss(10, 12)
    sub = sht.sht_geom_subset(g, [0, 3, 9])
    r = sub.rings()
    full = g.rings()
    np.testing.assert_array_equal(r["theta"], full["theta"][[0, 3, 9]])
    np.testing.assert_array_equal(r["ofs"], full["ofs"][[0, 3, 9]])
    assert sub.info()[2] == 2  # rings 0 and 9 mirror each other, 3 is alone
    with pytest.raises(sht.ShtError):
        sht.sht_geom_subset(g, [0, 0])
    with pytest.raises(sht.ShtError):
        sht.sht_geom_subset(g, [10])
    with pytest.raises(sht.ShtError):
        sht.sht_geom_general([4.0], [3], [0.0], [0])  # theta > pi
    with pytest.raises(sht.ShtError):
        sht.sht_geom_general([1.0], [0], [0.0], [0])  # nphi < 1
    # asymmetric ring set: nothing pairs
    g2 = sht.sht_geom_general([0.3, 1.0, 2.0], [4, 4, 4], [0, 0, 0], [0, 4, 8])
    assert g2.info()[2] == 3
    # mirrored rings of different nphi do not pair
    g3 = sht.sht_geom_general([0.3, math.pi - 0.3], [4, 5], [0, 0], [0, 4])
    assert g3.info()[2] == 2


def test_alm_layouts():
    a = sht.sht_alm_create(10, 10)
    assert a.size() == oracle.nalm(10, 10)
    b = sht.sht_alm_create(10, 4)
    assert b.size() == oracle.nalm(10, 4)
    c = sht.sht_alm_create(10, 10, mval=[0, 5, 7])
    assert c.size() == 11 + 6 + 4
    d = sht.sht_alm_create(10, 10, mval=[2], mstart=[100], stride=3)
    assert d.size() == 100 + 30 + 1
    for bad in (dict(lmax=-1, mmax=0), dict(lmax=3, mmax=4), dict(lmax=3, mmax=3, mval=[1, 1]),
                dict(lmax=3, mmax=3, mval=[4]), dict(lmax=3, mmax=3, stride=0)):
        with pytest.raises(sht.ShtError):
            sht.sht_alm_create(**bad)


def _smooth235(n):
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


def test_reduced_gauss_geometry():
    # Sect. 4.4.2: ring y holds the smallest 2^a 3^b 5^c >= 2 m_y + 1 pixels, m_y from
    # Eq. eq_polaropt solved for m; same nodes as the full grid; sum Nphi w = 4 pi
    for lmax, spin in ((2047, 0), (1023, 2), (100, 0)):
        nlat = lmax + 1
        red = sht.sht_geom_reduced_gauss(nlat, lmax, spin).rings()
        full = sht.sht_geom_gauss(nlat, 2 * lmax + 1).rings()
        np.testing.assert_array_equal(red["theta"], full["theta"])
        T = max(100.0, 0.01 * lmax)
        th = red["theta"]
        r = T + lmax * np.sin(th)
        # the larger root (the terms of m and -m): the same on mirrored rings
        m = np.minimum(lmax, np.floor(abs(spin) * np.abs(np.cos(th)) + np.sqrt(r * r - spin * spin * np.sin(th) ** 2)))
        for n, mm in zip(red["nphi"], m):
            lo = int(2 * mm + 1)
            assert n >= lo and _smooth235(int(n))
            assert not any(_smooth235(x) for x in range(lo, int(n)))  # the smallest such length
        assert abs(np.sum(red["nphi"] * red["weight"]) - 4 * np.pi) < 1e-12
        assert np.all(np.diff(red["ofs"]) == red["nphi"][:-1])
        np.testing.assert_array_equal(red["nphi"], red["nphi"][::-1])  # mirrored rings pair up
    red = sht.sht_geom_reduced_gauss(2048, 2047)
    assert red.npix < 0.7 * 2048 * 4095  # more than 30% of the pixels saved at lmax > 1000


def _is_prime(n):
    return n > 1 and all(n % d for d in range(2, int(n ** 0.5) + 1))


def test_fft_plan_choice():
    # the ring-FFT planner (host logic): kind 0 direct mixed radix, 1 Rader, 2 Bluestein
    known = {
        8191: (1, 8190, [2, 3, 3, 5, 7, 13]),     # the bench's rings: prime, Rader over 8190
        4095: (0, 4095, [3, 3, 5, 7, 13]),
        37: (0, 37, [37]),                        # one large radix
        16383: (0, 16383, [3, 43, 127]),          # 3 43 127: the largest radix
        131: (1, 130, [2, 5, 13]),
        149: (1, 148, [4, 37]),
        20011: (1, 20010, [2, 3, 5, 23, 29]),
        20480: (0, 20480, [4, 4, 4, 4, 4, 4, 5]),
        262: (2, 525, [3, 5, 5, 7]),              # 2 131: Bluestein, convolution >= 523
        2367: (2, 4736, [4, 4, 4, 2, 37]),
        14803: (2, 29624, [4, 2, 7, 23, 23]),
        1: (0, 1, []),
    }
    for n, want in known.items():
        assert sht.sht_fft_plan_info(n) == want, n
    allowed = {2, 4} | {p for p in range(3, 128, 2) if _is_prime(p)}
    for n in range(1, 3001):
        kind, ln, rad = sht.sht_fft_plan_info(n)
        assert int(np.prod(rad)) == ln and set(rad) <= allowed, n
        assert rad == sorted(rad, key=lambda r: (r not in (2, 4), r == 2, r)), n  # 4s, a 2, odd ascending
        assert rad.count(2) <= 1
        if kind == 0:
            assert ln == n
        elif kind == 1:
            assert _is_prime(n) and ln == n - 1
            assert any(p > 127 for p in range(2, n + 1) if n % p == 0 and _is_prime(p))  # not direct
        else:
            assert kind == 2 and ln >= 2 * n - 1
            assert not _is_prime(n) or any(p > 127 for p in range(2, n) if (n - 1) % p == 0 and _is_prime(p))
    for bad in (0, -5):
        with pytest.raises(sht.ShtError) as ei:
            sht.sht_fft_plan_info(bad)
        assert ei.value.code == sht.SHT_ERR_INVALID_ARG
    with pytest.raises(sht.ShtError) as ei:  # 2 20011: Bluestein would need more than 65536 points
        sht.sht_fft_plan_info(40022)
    assert ei.value.code == sht.SHT_ERR_UNSUPPORTED


@pytest.mark.parametrize("spin", [0, 2, -3])
def test_polar_cut(spin):
    # Sect. 3.3: (m, pair) is skipped when sqrt(m^2 + s^2 - 2 |m s| |cos theta|) - lmax sin theta > T,
    # T = max(100, 0.01 lmax); pairs run pole -> equator, so the kept pairs of each m are a suffix
    lmax = 1023
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    mval = np.arange(lmax + 1)
    first, th, trip = sht.sht_geom_polar_cut(geom, lmax, spin, mval)
    npairs = geom.info()[2]
    assert len(th) == npairs == (lmax + 1) // 2
    gl = np.sort(geom.rings()["theta"])[:npairs]
    np.testing.assert_array_equal(th, gl)  # GL: pair p holds the p-th ring from the north pole
    T = max(100.0, 0.01 * lmax)
    s = abs(spin)
    for m in (0, 1, 7, 300, 600, 800, 1023):
        v = np.sqrt(np.maximum(0.0, m * m + s * s - 2.0 * m * s * np.abs(np.cos(th)))) - lmax * np.sin(th)
        skipped = v > T
        assert first[m] == (np.argmin(skipped) if not skipped.all() else npairs), m
        assert skipped[:first[m]].all() and not skipped[first[m]:].any(), m  # a prefix
    assert first[0] == 0 and np.all(np.diff(first) >= 0)  # more of the cap skipped as m grows
    l0 = np.maximum(mval, s)
    assert trip == int(np.sum((npairs - first) * (lmax - l0 + 1)))
    full = int(np.sum(npairs * (lmax - l0 + 1)))
    assert 0.6 * full < trip < full  # the cut removes a fifth or so of the steps on GL
    for bad in ([lmax + 1], [-1]):
        with pytest.raises(sht.ShtError):
            sht.sht_geom_polar_cut(geom, lmax, spin, bad)


def _ecp_weights_longdouble(kind, nlat, nodes):
    """The defining cosine / sine sums of the three ECP rules (Sect. 4.4.1), evaluated
    term by term in numpy's long double at the given node indices (weights on [-1, 1])."""
    pi = np.longdouble("3.14159265358979323846264338327950288")
    out = []
    for i in nodes:
        if kind == 0:
            N = nlat
            t = pi * (2 * i + 1) / (2 * N)
            k = np.arange(1, N // 2 + 1, dtype=np.longdouble)
            out.append(2 / N * (1 - 2 * np.sum(np.cos(2 * k * t) / (4 * k * k - 1))))
        elif kind == 1:
            N = nlat + 1
            t = pi * (i + 1) / N
            k = np.arange(1, N // 2 + 1, dtype=np.longdouble)
            out.append(4 * np.sin(t) / N * np.sum(np.sin((2 * k - 1) * t) / (2 * k - 1)))
        else:
            N = nlat - 1
            t = pi * i / N
            k = np.arange(1, N // 2 + 1, dtype=np.longdouble)
            b = np.where(2 * k == N, 1, 2)
            c = 1 if i in (0, N) else 2
            out.append(c / N * (1 - np.sum(b * np.cos(2 * k * t) / (4 * k * k - 1))))
    return np.array(out, dtype=np.longdouble)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("nlat", [2, 3, 17, 128, 1001, 4096, 8192])
def test_ecp_weights_by_fft(kind, nlat):
    # the product builds the weights as one DFT of each rule's moment sequence
    # (Waldvogel 2006); against the rule's sum in long double to 1e-14 of the
    # largest weight (every node up to nlat 1001, a spread sample above), and against
    # the oracle's direct double sums to their own accuracy (~1e-16 per term, so
    # up to ~1e-13 of the largest weight at nlat 8192)
    w = sht.sht_geom_ecp(kind, nlat, 1).rings()["weight"] / (2 * np.pi)
    nodes = np.arange(nlat) if nlat <= 1001 else np.unique(np.r_[0:8, nlat - 8:nlat, np.linspace(0, nlat - 1, 48).astype(int)])
    ref = _ecp_weights_longdouble(kind, nlat, nodes)
    wmax = float(np.max(np.abs(ref)))
    assert float(np.max(np.abs(w[nodes] - ref))) <= 1e-14 * wmax
    _, wo = oracle.ecp_nodes(kind, nlat)
    assert np.max(np.abs(w - wo)) <= 2e-13 * np.max(np.abs(wo))
    # exact integration of x^k, k below the rule's degree of exactness (nlat - 1 here)
    x = np.cos(sht.sht_geom_ecp(kind, nlat, 1).rings()["theta"])
    for k in range(0, min(nlat, 40)):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, (k, np.sum(w * x ** k), exact)
