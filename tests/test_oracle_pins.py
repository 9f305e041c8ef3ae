"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test names the passage of Reinecke & Seljebotn 2013 (libsharp) that
defines what is checked, and the independent ground truth used:
  * closed-form Y_lm (textbook, Condon-Shortley phase)     -> Sect. 2, lambda := sY_lm(theta, 0)
  * Wigner's explicit d-sum in 50-digit arithmetic        -> Sect. 4.1 relation lambda <-> d
  * classic normalised P_lm recursion in mpmath           -> enhanced exponent range, Sect. 4.1
  * addition theorem, spin raising (eth), parity           -> properties of sY_lm
  * Gauss / Fejer / Clenshaw-Curtis exactness on polynomials, numpy leggauss -> grids, Sect. 4.4
  * HEALPix pixel count / symmetry / equal area            -> grids, Sect. 4.4
  * brute-force direct sums at lmax <= 6                  -> Eq. syn_used
  * exact GL and ECP round trips, adjoint identity         -> Eqs. ana_used, Sect. 4.5
"""
import math

import mpmath
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

PI = math.pi


# ---------------------------------------------------------------- helpers ---
def ylm_closed(l, m, th):
    """Y_lm(theta, 0), Condon-Shortley phase, l <= 4 (textbook table)."""
    c, s = math.cos(th), math.sin(th)
    am = abs(m)
    t = {
        (0, 0): 0.5 / math.sqrt(PI),
        (1, 0): math.sqrt(3 / (4 * PI)) * c,
        (1, 1): -math.sqrt(3 / (8 * PI)) * s,
        (2, 0): math.sqrt(5 / (16 * PI)) * (3 * c * c - 1),
        (2, 1): -math.sqrt(15 / (8 * PI)) * s * c,
        (2, 2): math.sqrt(15 / (32 * PI)) * s * s,
        (3, 0): math.sqrt(7 / (16 * PI)) * (5 * c ** 3 - 3 * c),
        (3, 1): -math.sqrt(21 / (64 * PI)) * s * (5 * c * c - 1),
        (3, 2): math.sqrt(105 / (32 * PI)) * s * s * c,
        (3, 3): -math.sqrt(35 / (64 * PI)) * s ** 3,
        (4, 0): 3 / (16 * math.sqrt(PI)) * (35 * c ** 4 - 30 * c * c + 3),
        (4, 1): -3 / 8 * math.sqrt(5 / PI) * s * (7 * c ** 3 - 3 * c),
        (4, 2): 3 / 8 * math.sqrt(5 / (2 * PI)) * s * s * (7 * c * c - 1),
        (4, 3): -3 / 8 * math.sqrt(35 / PI) * s ** 3 * c,
        (4, 4): 3 / 16 * math.sqrt(35 / (2 * PI)) * s ** 4,
    }[(l, am)]
    if m < 0:
        t *= (-1) ** am  # Y_{l,-m} = (-1)^m conj(Y_lm), real at phi = 0
    return t


def wigner_d_explicit(j, mp_, m, beta, dps=50):
    """d^j_{m' m}(beta) from Wigner's explicit sum, in mpmath (independent of any recursion)."""
    with mpmath.workdps(dps):
        b = mpmath.mpf(beta)
        c, s = mpmath.cos(b / 2), mpmath.sin(b / 2)
        f = mpmath.factorial
        pref = mpmath.sqrt(f(j + mp_) * f(j - mp_) * f(j + m) * f(j - m))
        tot = mpmath.mpf(0)
        for k in range(max(0, m - mp_), min(j + m, j - mp_) + 1):
            den = f(j + m - k) * f(k) * f(mp_ - m + k) * f(j - k - mp_)
            tot += (-1) ** (m - mp_ + k) / den * c ** (2 * j + m - mp_ - 2 * k) * s ** (mp_ - m + 2 * k)
        return pref * tot


def lambda_explicit(s, m, l, th):
    """(-1)^m sqrt((2l+1)/4pi) d^l_{-m,s}(theta)  (Sect. 4.1), via the explicit sum."""
    if l < max(abs(m), abs(s)):
        return 0.0
    d = wigner_d_explicit(l, -m, s, th)
    return float((-1) ** (m & 1) * mpmath.sqrt(mpmath.mpf(2 * l + 1) / (4 * mpmath.pi)) * d)


def plm_classic_mp(m, lmax, th, dps=40):
    """Orthonormal Y_lm(theta,0) by the classic two-coefficient Legendre recursion
    in mpmath (unbounded exponent range); a different recursion from the oracle's."""
    with mpmath.workdps(dps):
        x = mpmath.cos(mpmath.mpf(th))
        st = mpmath.sin(mpmath.mpf(th))
        v = mpmath.mpf(1) / (4 * mpmath.pi)
        for k in range(1, m + 1):
            v *= mpmath.mpf(2 * k - 1) / (2 * k)
        lam = {m: (-1) ** m * mpmath.sqrt((2 * m + 1) * v) * st ** m}
        prev = mpmath.mpf(0)
        cur = lam[m]
        for l in range(m, lmax):
            L = l + 1
            alpha = mpmath.sqrt(mpmath.mpf(4 * L * L - 1) / (L * L - m * m))
            beta = mpmath.sqrt(mpmath.mpf(l * l - m * m) / (4 * l * l - 1)) if l > 0 else 0
            nxt = alpha * (x * cur - beta * prev)
            prev, cur = cur, nxt
            lam[L] = cur
        return lam


# ----------------------------------------------------------------- lambda ---
@pytest.mark.parametrize("th", [0.3, 1.1, 2.0, 3.0])
def test_lambda_closed_form_ylm(th):
    for l in range(5):
        for m in range(-l, l + 1):
            lam = oracle.lambda_(0, m, 4, th)
            assert abs(lam[l] - ylm_closed(l, m, th)) < 1e-15, (l, m, th)


@pytest.mark.parametrize("s", [-3, -2, -1, 0, 1, 2, 3])
def test_lambda_wigner_explicit_sum(s):
    lmax = 14
    for th in (0.05, 0.9, 1.7, 3.0):
        for m in range(-lmax, lmax + 1, 3):
            lam = oracle.lambda_(s, m, lmax, th)
            for l in range(lmax + 1):
                ref = lambda_explicit(s, m, l, th)
                assert abs(lam[l] - ref) < 2e-14, (s, m, l, th, lam[l], ref)


def test_lambda_wigner_explicit_sum_high_l():
    # a few entries at l ~ 120 with high-precision explicit sums (heavy cancellation)
    for (s, m, l, th) in [(2, 50, 120, 0.8), (-2, 7, 119, 2.3), (3, 100, 121, 1.4), (0, 60, 118, 0.6)]:
        with mpmath.workdps(120):
            d = wigner_d_explicit(l, -m, s, th, dps=120)
            ref = float((-1) ** (m & 1) * mpmath.sqrt(mpmath.mpf(2 * l + 1) / (4 * mpmath.pi)) * d)
        lam = oracle.lambda_(s, m, l, th)[l]
        assert abs(lam - ref) < 1e-13 * max(1.0, abs(ref)), (s, m, l, th, lam, ref)


def test_lambda_underflow_range_classic_recursion():
    # start values far below the double range (sin^m theta ~ 1e-600): the
    # enhanced-exponent recursion must still produce the O(1) values at high l.
    for (m, th, ls) in [(3000, 0.8, [4300, 4600, 5000]), (1500, 0.25, [5990, 6000]),
                        (5000, 1.2, [5300, 5600])]:
        lmax = max(ls)
        ref = plm_classic_mp(m, lmax, th)
        lam = oracle.lambda_(0, m, lmax, th)
        for l in ls:
            r = float(ref[l])
            # rounding grows about linearly with the number of recursion steps
            # (Sect. 5.1.2 reports rms error ~ lmax); allow 5e-16 per step
            tol = 5e-16 * (l - m) * max(abs(r), 1e-3)
            assert abs(lam[l] - r) <= tol, (m, th, l, lam[l], r)
        # the start value itself: 0 where it underflows double, else accurate
        r0 = float(ref[m])
        assert (lam[m] == 0.0 and abs(r0) < 1e-300) or abs(lam[m] - r0) <= 1e-14 * abs(r0)


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_addition_theorem(s):
    lmax = 40
    for th in (0.2, 1.0, 2.5):
        tot = np.zeros(lmax + 1)
        for m in range(-lmax, lmax + 1):
            tot += oracle.lambda_(s, m, lmax, th) ** 2
        l = np.arange(lmax + 1)
        exp = np.where(l >= s, (2 * l + 1) / (4 * PI), 0.0)
        np.testing.assert_allclose(tot, exp, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_spin_raising(s):
    # eth on spin-s: s+1 lambda = -(d/dth - m/sin th - s cot th) s lambda / sqrt((l-s)(l+s+1))
    # d/dth by an 80-digit central difference (h = 1e-25) of the explicit sum
    th, lmax = 0.9, 9
    for m in (-4, -1, 0, 2, 6):
        lam_s = oracle.lambda_(s, m, lmax, th)
        lam_up = oracle.lambda_(s + 1, m, lmax, th)
        for l in range(max(abs(m), s + 1), lmax + 1):
            with mpmath.workdps(80):
                h = mpmath.mpf("1e-25")
                t0 = mpmath.mpf(th)
                der = (wigner_d_explicit(l, -m, s, t0 + h, dps=80)
                       - wigner_d_explicit(l, -m, s, t0 - h, dps=80)) / (2 * h)
                der *= (-1) ** (m & 1) * mpmath.sqrt(mpmath.mpf(2 * l + 1) / (4 * mpmath.pi))
            val = -(float(der) - m * lam_s[l] / math.sin(th) - s * math.cos(th) / math.sin(th) * lam_s[l])
            val /= math.sqrt((l - s) * (l + s + 1))
            assert abs(val - lam_up[l]) < 1e-13, (s, m, l)


@pytest.mark.parametrize("s", [0, 1, 2, 4])
def test_parity_and_conjugation(s):
    lmax = 30
    for th in (0.3, 1.2):
        for m in range(-lmax, lmax + 1, 5):
            a = oracle.lambda_(s, m, lmax, PI - th)
            b = oracle.lambda_(-s, m, lmax, th)
            l = np.arange(lmax + 1)
            np.testing.assert_allclose(a, (-1.0) ** ((l + m) & 1) * b, atol=1e-13)
            c = oracle.lambda_(-s, -m, lmax, th)
            np.testing.assert_allclose(oracle.lambda_(s, m, lmax, th), (-1.0) ** ((s + m) & 1) * c, atol=1e-13)


# ------------------------------------------------------------------ grids ---
def _gl_mp(n, th0):
    """Gauss node nearest th0 and its weight, Newton in 40-digit arithmetic."""
    with mpmath.workdps(40):
        x = mpmath.cos(mpmath.mpf(th0))
        for _ in range(8):
            p0, p1 = mpmath.mpf(1), x
            for k in range(1, n):
                p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
            dp = n * (x * p1 - p0) / (x * x - 1)
            x -= p1 / dp
        return x, 2 / ((1 - x * x) * dp * dp)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 255, 1024])
def test_gauss_nodes(n):
    th, w = oracle.gauss_nodes(n)
    assert np.all(np.diff(th) > 0)
    x = np.cos(th)
    # library routine: a coarse check only, its pole weights are off by ~1e-9 at n = 1024
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(np.sort(x), np.sort(xr), atol=1e-14)
    np.testing.assert_allclose(w[np.argsort(x)], wr[np.argsort(xr)], rtol=1e-8)
    # 40-digit Newton at the pole-most, a middle and the equator-most node
    for i in sorted({0, n // 3, (n - 1) // 2}):
        xm, wm = _gl_mp(n, th[i])
        assert abs(x[i] - float(xm)) < 2e-16
        assert abs(w[i] - float(wm)) < 1e-14 * float(wm), (i, w[i], float(wm))
    if n <= 255:
        for k in range(0, 2 * n):
            exact = 0.0 if k % 2 else 2.0 / (k + 1)
            assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("kind,nlat", [(0, 9), (0, 16), (1, 10), (1, 15), (2, 11), (2, 20)])
def test_ecp_weights_exact(kind, nlat):
    th, w = oracle.ecp_nodes(kind, nlat)
    x = np.cos(th)
    deg = {0: nlat - 1, 1: nlat - 1, 2: nlat - 1}[kind]
    for k in range(deg + 1):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13, (kind, nlat, k)
    step = {0: PI / nlat, 1: PI / (nlat + 1), 2: PI / (nlat - 1)}[kind]
    np.testing.assert_allclose(np.diff(th), step, rtol=1e-12)


@pytest.mark.parametrize("nside", [1, 2, 4, 16])
def test_healpix_rings(nside):
    r = oracle.healpix_rings(nside)
    assert r.nrings == 4 * nside - 1
    assert r.npix == 12 * nside * nside
    np.testing.assert_allclose(r.theta + r.theta[::-1], PI, atol=1e-14)
    assert np.all(r.nphi == r.nphi[::-1]) and np.all(r.phi0 == r.phi0[::-1])
    np.testing.assert_allclose(np.sum(r.nphi * r.weight), 4 * PI, rtol=1e-14)
    # equal area: cap above ring boundary between polar rings i, i+1 holds
    # 2 i (i+1) pixels, and z_i = 1 - i^2/(3 nside^2) on polar rings
    z = np.cos(r.theta)
    for i in range(1, nside):
        assert abs(z[i - 1] - (1 - i * i / (3.0 * nside * nside))) < 1e-14
    if nside == 1:
        np.testing.assert_allclose(r.phi0, [PI / 4, 0.0, PI / 4])
        np.testing.assert_allclose(z, [2 / 3, 0, -2 / 3], atol=1e-15)


def _healpix_pixel_centre(nside, p):
    """(z, phi) of RING-scheme pixel p from the pixel-centre formulas of Gorski et al.
    2005 (written out here, independently of the oracle's ring builder).  North polar
    cap: ring i (1 <= i < nside) holds 4i pixels after 2i(i-1) earlier ones, pixel j
    (1-based) at z = 1 - i^2/(3 nside^2), phi = pi/(2i) (j - 1/2).  Equatorial belt:
    ring i (nside <= i <= 3 nside) holds 4 nside pixels, z = 4/3 - 2i/(3 nside),
    phi = pi/(2 nside) (j - f) with f = 1 when i + nside is odd, 1/2 when even.
    South polar cap: the mirror image of the north one."""
    ncap = 2 * nside * (nside - 1)
    npix = 12 * nside * nside
    if p < ncap:
        i = 1
        while 2 * i * (i + 1) <= p:
            i += 1
        j = p - 2 * i * (i - 1) + 1
        return 1.0 - i * i / (3.0 * nside * nside), PI / (2 * i) * (j - 0.5)
    if p < npix - ncap:
        q = p - ncap
        i = nside + q // (4 * nside)
        j = q % (4 * nside) + 1
        f = 1.0 if (i + nside) % 2 else 0.5
        return 4.0 / 3.0 - 2.0 * i / (3.0 * nside), PI / (2 * nside) * (j - f)
    q = npix - 1 - p  # counted back from the last pixel: ring i from the south pole
    i = 1
    while 2 * i * (i + 1) <= q:
        i += 1
    j = 4 * i - (q - 2 * i * (i - 1))  # position within the ring, 1-based, in increasing phi
    return -(1.0 - i * i / (3.0 * nside * nside)), PI / (2 * i) * (j - 0.5)


@pytest.mark.parametrize("nside", [4, 8])
def test_healpix_pixel_centres(nside):
    """Every pixel centre of the ring description (theta_y, phi0_y + 2 pi x / Nphi_y at
    map index ofs_y + x) equals the Gorski et al. pixel-centre formula: pins the polar
    rings' phi0 = pi/(4i) and the equatorial alternation (reading R6), which a wrong
    shift or pixel order in the ring builder would break."""
    r = oracle.healpix_rings(nside)
    z_ring = np.cos(r.theta)
    for y in range(r.nrings):
        for x in range(r.nphi[y]):
            p = int(r.ofs[y]) + x
            z, phi = _healpix_pixel_centre(nside, p)
            assert abs(z_ring[y] - z) < 1e-14, (nside, y, x)
            assert abs(r.phi0[y] + 2 * PI * x / r.nphi[y] - phi) < 1e-13, (nside, y, x)


# -------------------------------------------------------------- transforms ---
def _brute_synthesis(s, lmax, alm, rings):
    """Eq. syn_used summed term by term with explicit-sum lambdas (lmax tiny)."""
    lam = {}
    for y, th in enumerate(rings.theta):
        for l in range(lmax + 1):
            for m in range(-l, l + 1):
                lam[(y, l, m)] = lambda_explicit(s, m, l, th)
    nj = len(alm) // (2 if s else 1)
    maps = [np.zeros(rings.npix) for _ in alm]
    for j in range(nj):
        for y in range(rings.nrings):
            N = rings.nphi[y]
            phi = rings.phi0[y] + 2 * PI * np.arange(N) / N
            P = np.zeros(N, dtype=complex)
            for l in range(abs(s), lmax + 1):
                for m in range(-l, l + 1):
                    ix = oracle.alm_index(lmax, l, abs(m))
                    if s == 0:
                        a = alm[j][ix]
                        a = a.real + 0j if m == 0 else a
                        coef = a if m >= 0 else (-1) ** abs(m) * np.conj(a)
                    else:
                        E, B = alm[2 * j][ix], alm[2 * j + 1][ix]
                        if m == 0:
                            E, B = E.real + 0j, B.real + 0j
                        if m < 0:
                            E, B = (-1) ** abs(m) * np.conj(E), (-1) ** abs(m) * np.conj(B)
                        coef = -(E + 1j * B)
                    P += coef * lam[(y, l, m)] * np.exp(1j * m * phi)
            o = rings.ofs[y]
            if s == 0:
                assert np.max(np.abs(P.imag)) < 1e-12  # a real field
                maps[j][o:o + N] = P.real
            else:
                maps[2 * j][o:o + N] = P.real
                maps[2 * j + 1][o:o + N] = P.imag
    return maps


@pytest.mark.parametrize("s", [0, 1, 2])
@pytest.mark.parametrize("grid", ["gauss", "healpix"])
def test_synthesis_brute_force(s, grid):
    lmax = 5
    rng = np.random.default_rng(11 + s)
    rings = oracle.gauss_rings(5, 9) if grid == "gauss" else oracle.healpix_rings(2)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(s)) for _ in range(2 if s else 1)]
    # exercise the "Im a_l0 ignored" rule: put garbage there
    for a in alm:
        for l in range(lmax + 1):
            a[oracle.alm_index(lmax, l, 0)] += 0.37j
    ref = _brute_synthesis(s, lmax, alm, rings)
    got = oracle.synthesis(s, lmax, lmax, alm, rings)
    for r, g in zip(ref, got):
        np.testing.assert_allclose(g, r, atol=1e-13)


def test_spin2_pure_e_and_b_closed_form():
    # E_20 = 1: Q + iU = -2Y_20 = -(1/4) sqrt(15/(2 pi)) sin^2 theta, real.
    lmax = 4
    rings = oracle.gauss_rings(6, 9)
    n = oracle.nalm(lmax, lmax)
    E = np.zeros(n, complex)
    B = np.zeros(n, complex)
    E[oracle.alm_index(lmax, 2, 0)] = 1.0
    Q, U = oracle.synthesis(2, lmax, lmax, [E, B], rings)
    expect = -0.25 * math.sqrt(15 / (2 * PI)) * np.repeat(np.sin(rings.theta) ** 2, 9)
    np.testing.assert_allclose(Q, expect, atol=1e-15)
    np.testing.assert_allclose(U, 0.0, atol=1e-15)
    Q, U = oracle.synthesis(2, lmax, lmax, [B, E], rings)  # B_20 = 1
    np.testing.assert_allclose(Q, 0.0, atol=1e-15)
    np.testing.assert_allclose(U, expect, atol=1e-15)


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_gauss_round_trip_exact(s):
    lmax = 24
    rng = np.random.default_rng(5)
    rings = oracle.gauss_rings(lmax + 1, 2 * lmax + 1)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(s)) for _ in range(2 if s else 1)]
    maps = oracle.synthesis(s, lmax, lmax, alm, rings)
    back = oracle.analysis(s, lmax, lmax, maps, rings)
    for a, b in zip(alm, back):
        err = np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(a) ** 2))
        assert err < 1e-13, err


@pytest.mark.parametrize("kind", [0, 2])
def test_ecp_round_trip_exact(kind):
    lmax, s = 12, 2
    rng = np.random.default_rng(6)
    nlat = 2 * lmax + 2
    rings = oracle.ecp_rings(kind, nlat, 2 * lmax + 2)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
    back = oracle.analysis(s, lmax, lmax, oracle.synthesis(s, lmax, lmax, alm, rings), rings)
    for a, b in zip(alm, back):
        assert np.max(np.abs(a - b)) < 1e-12


@pytest.mark.parametrize("s", [0, 2])
def test_adjoint_identity(s):
    # <Y a, p> = sum_{l, m>=0} (2 - delta_m0) Re(a conj(Y^H p))  (Sect. 4.5)
    lmax, mmax = 10, 8
    rng = np.random.default_rng(8)
    rings = oracle.healpix_rings(2)
    alm = [inputs.gaussian_alm(rng, lmax, mmax, lmin=abs(s)) for _ in range(2 if s else 1)]
    maps = [rng.standard_normal(rings.npix) for _ in alm]
    ya = oracle.synthesis(s, lmax, mmax, alm, rings)
    yhp = oracle.analysis(s, lmax, mmax, maps, rings, adjoint=True)
    lhs = sum(np.dot(a, b) for a, b in zip(ya, maps))
    _, m = inputs.lm_arrays(lmax, mmax)
    wgt = np.where(m == 0, 1.0, 2.0)
    rhs = sum(np.sum(wgt * (a * np.conj(b)).real) for a, b in zip(alm, yhp))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_adjoint_analysis_is_weighted_synthesis():
    lmax = 6
    rng = np.random.default_rng(9)
    rings = oracle.healpix_rings(2)
    alm = [inputs.gaussian_alm(rng, lmax, lmax)]
    a = oracle.synthesis(0, lmax, lmax, alm, rings, weighted=True)[0]
    b = oracle.synthesis(0, lmax, lmax, alm, rings)[0] * np.repeat(rings.weight, rings.nphi)
    np.testing.assert_allclose(a, b, atol=1e-15)


def test_selection_matches_full():
    lmax = 16
    rng = np.random.default_rng(10)
    rings = oracle.gauss_rings(17, 33)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
    full = oracle.synthesis(2, lmax, lmax, alm, rings)
    sel = [0, 5, 16]
    part = oracle.synthesis(2, lmax, lmax, alm, rings, rings_sel=sel)
    for f, p in zip(full, part):
        for y in sel:
            o, n = rings.ofs[y], rings.nphi[y]
            np.testing.assert_array_equal(f[o:o + n], p[o:o + n])
    fa = oracle.analysis(2, lmax, lmax, full, rings)
    pa = oracle.analysis(2, lmax, lmax, full, rings, m_sel=[3, 9])
    l, m = inputs.lm_arrays(lmax, lmax)
    for f, p in zip(fa, pa):
        np.testing.assert_array_equal(f[(m == 3) | (m == 9)], p[(m == 3) | (m == 9)])


def test_phase_stage_matches_synthesis():
    # Eq. syn1 applied to the Legendre stage output reproduces Eq. syn_used
    lmax = 9
    rng = np.random.default_rng(12)
    rings = oracle.gauss_rings(10, 19)
    alm = [inputs.gaussian_alm(rng, lmax, lmax)]
    F = oracle.phase(0, lmax, lmax, alm[0], rings.theta)
    mp = oracle.synthesis(0, lmax, lmax, alm, rings)[0]
    for y in range(rings.nrings):
        x = np.arange(19)
        ms = np.arange(-lmax, lmax + 1)
        p = (F[y][None, :] * np.exp(2j * PI * np.outer(x, ms) / 19)).sum(1)
        np.testing.assert_allclose(p.real, mp[rings.ofs[y]:rings.ofs[y] + 19], atol=1e-13)


def test_deriv_synthesis_matches_finite_differences():
    # Sect. 4.3: the two derivative maps against 4th-order central differences of
    # the spin-0 synthesis, in theta (rings moved by +-h, +-2h) and in phi
    # (phi0 moved); pins the reading E = sqrt(l(l+1)) a, B = 0 and its signs
    lmax = 12
    rng = np.random.default_rng(21)
    a = inputs.gaussian_alm(rng, lmax, lmax)
    theta = np.array([0.3, 0.9, 1.4, 2.0, 2.7])
    nphi = np.full(len(theta), 27)
    phi0 = np.array([0.0, 0.1, 0.2, 0.3, 0.4])
    w = np.ones(len(theta))
    base = oracle.Rings(theta, nphi, phi0, w)
    d_th, d_ph = oracle.deriv_synthesis(lmax, lmax, [a], base)
    h = 1e-3

    def syn(th, p0):
        return oracle.synthesis(0, lmax, lmax, [a], oracle.Rings(th, nphi, p0, w))[0]

    fd_th = (-syn(theta + 2 * h, phi0) + 8 * syn(theta + h, phi0) - 8 * syn(theta - h, phi0)
             + syn(theta - 2 * h, phi0)) / (12 * h)
    fd_ph = (-syn(theta, phi0 + 2 * h) + 8 * syn(theta, phi0 + h) - 8 * syn(theta, phi0 - h)
             + syn(theta, phi0 - 2 * h)) / (12 * h)
    fd_ph /= np.repeat(np.sin(theta), nphi)
    scale = np.max(np.abs(d_th))
    assert np.max(np.abs(d_th - fd_th)) < 1e-7 * scale
    assert np.max(np.abs(d_ph - fd_ph)) < 1e-7 * np.max(np.abs(d_ph))


def test_real_harmonic_basis_is_orthonormal():
    # Sect. 4.5 reading: the basis functions of real-harmonic storage (one per
    # stored number: m = 0 real parts, both numbers for m > 0) are orthonormal
    # under Gauss-Legendre quadrature, which fixes the sqrt2 factors
    lmax = 4
    rings = oracle.gauss_rings(lmax + 1, 2 * lmax + 1)
    n = oracle.nalm(lmax, lmax)
    m = oracle._m_of(lmax, lmax)
    coords = [(i, 0) for i in range(n)] + [(i, 1) for i in range(n) if m[i] > 0]
    assert len(coords) == (lmax + 1) ** 2
    basis = []
    for i, part in coords:
        r = np.zeros(n, dtype=np.complex128)
        r[i] = 1.0 if part == 0 else 1j
        basis.append(oracle.synthesis(0, lmax, lmax, [oracle.real_to_complex(r, lmax, lmax)], rings)[0])
    w = np.repeat(rings.weight, rings.nphi)
    gram = np.array([[np.sum(w * u * v) for v in basis] for u in basis])
    np.testing.assert_allclose(gram, np.eye(len(basis)), atol=1e-13)
    a = inputs.gaussian_alm(np.random.default_rng(3), lmax, lmax)
    np.testing.assert_allclose(oracle.complex_to_real(oracle.real_to_complex(a, lmax, lmax), lmax, lmax), a,
                               atol=1e-15)
