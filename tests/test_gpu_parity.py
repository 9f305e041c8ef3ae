"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Every case runs the library on cuda:0 and the oracle on the same rings
(taken from the library's geometry handle) and the same seeded inputs, and
compares element by element.  Tolerances: FP64 form 1e-12 relative L2 (and
5e-12 of the largest value elementwise); the oracle itself drifts ~5e-16 per
recursion step, so both sides carry rounding of that order.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64_L2 = 1e-12
FP64_MAX = 5e-12


@pytest.fixture(scope="module")
def sht():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht as m

    assert torch.cuda.is_available()
    return m


def rel_l2(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rings_of(geom):
    r = geom.rings()
    assert np.all(r["stride"] == 1)
    return oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])


def gpu_synthesis(sht, plan, alm, npix, type_=None, flags=0, init=None):
    type_ = sht.SHT_SYNTHESIS if type_ is None else type_
    a = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in alm]
    if init is None:
        m = [torch.zeros(npix, dtype=torch.float64, device="cuda") for _ in alm]
    else:
        m = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in init]
    sht.sht_execute(plan, type_, a, m, flags)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in m]


def gpu_analysis(sht, plan, maps, nalm, type_=None, flags=0, init=None):
    type_ = sht.SHT_ANALYSIS if type_ is None else type_
    m = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in maps]
    if init is None:
        a = [torch.full((nalm,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda") for _ in maps]
    else:
        a = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in init]
    sht.sht_execute(plan, type_, a, m, flags)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in a]


def check_pair(sht, geom, lmax, mmax, spin, ncomp=1, seed=0, precision=0, l2=FP64_L2, mx=FP64_MAX,
               flags=0, with_adjoint=False):
    """synthesis and analysis parity for one configuration; returns the errors."""
    rng = np.random.default_rng(seed)
    narr = 2 * ncomp if spin else ncomp
    alm = [inputs.gaussian_alm(rng, lmax, mmax, lmin=abs(spin)) for _ in range(narr)]
    rings = rings_of(geom)
    lay = sht.sht_alm_create(lmax, mmax)
    plan = sht.sht_plan_create(geom, lay, spin, ncomp, precision)
    npix = geom.npix
    got = gpu_synthesis(sht, plan, alm, npix, flags=flags)
    ref = oracle.synthesis(spin, lmax, mmax, alm, rings)
    errs = {}
    for g, r in zip(got, ref):
        errs["syn_l2"] = max(errs.get("syn_l2", 0), rel_l2(g, r))
        errs["syn_max"] = max(errs.get("syn_max", 0), rel_max(g, r))
    maps = [rng.standard_normal(npix) for _ in range(narr)]
    got_a = gpu_analysis(sht, plan, maps, oracle.nalm(lmax, mmax), flags=flags)
    ref_a = oracle.analysis(spin, lmax, mmax, maps, rings)
    for g, r in zip(got_a, ref_a):
        errs["ana_l2"] = max(errs.get("ana_l2", 0), rel_l2(g, r))
        errs["ana_max"] = max(errs.get("ana_max", 0), rel_max(g, r))
    if with_adjoint:
        got_j = gpu_analysis(sht, plan, maps, oracle.nalm(lmax, mmax), type_=sht.SHT_ADJOINT_SYNTHESIS, flags=flags)
        ref_j = oracle.analysis(spin, lmax, mmax, maps, rings, adjoint=True)
        for g, r in zip(got_j, ref_j):
            errs["adj_l2"] = max(errs.get("adj_l2", 0), rel_l2(g, r))
        got_w = gpu_synthesis(sht, plan, alm, npix, type_=sht.SHT_ADJOINT_ANALYSIS, flags=flags)
        ref_w = oracle.synthesis(spin, lmax, mmax, alm, rings, weighted=True)
        for g, r in zip(got_w, ref_w):
            errs["adjw_l2"] = max(errs.get("adjw_l2", 0), rel_l2(g, r))
    for k, v in errs.items():
        lim = l2 if k.endswith("l2") else mx
        assert v <= lim, (k, v, errs)
    return errs


# ------------------------------------------------------------------ cases ---
@pytest.mark.parametrize("spin", [0, 1, 2, 3])
def test_gauss_small(sht, spin):
    # nlon = 81 = 3^4 (mixed radix), nlat even
    check_pair(sht, sht.sht_geom_gauss(42, 81), 40, 40, spin, seed=spin, with_adjoint=True)


@pytest.mark.parametrize("spin", [0, 2, -1])
def test_healpix_aliasing(sht, spin):
    # polar rings have 4i < 2 lmax + 1 pixels: the m sum folds (Eq. syn1); phi0 != 0
    check_pair(sht, sht.sht_geom_healpix(8), 28, 28, spin, seed=10 + abs(spin), with_adjoint=True)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nlon,spin", [(37, 0), (53, 2), (94, 0), (94, 2), (255, 1), (1517, 0), (131, 0), (149, 2),
                                       (3527, 0), (262, 0), (2367, 2), (4199, 0)])
def test_fft_lengths(sht, nlon, spin, precision):
    # direct: 37, 53 (one radix above 31), 94 = 2 47, 255 = 3 5 17, 1517 = 37 41 (a
    # twiddled large-radix pass); Rader: 131 (130 = 2 5 13), 149 (148 = 4 37),
    # 3527 (3526 = 2 41 43: a twiddled large-radix pass in the transposed passes);
    # Bluestein: 262 = 2 131 (convolution of 525), 2367 = 3 3 263 (convolution of
    # 4736 = 4^3 2 37); 4199 = 13 17 19 (radices the double-float engine runs as
    # sweeps).  Both engines: FP64 (precision 0) and double-float (mixed plans).
    lmax = min(30, (nlon - 1) // 2)
    tol = dict(l2=MIX_L2, mx=MIX_MAX) if precision else {}
    check_pair(sht, sht.sht_geom_gauss(lmax + 1 + (nlon % 2), nlon), lmax, lmax, spin, seed=nlon,
               precision=precision, **tol)


@pytest.mark.parametrize("nlat", [1, 3, 33])
def test_odd_rings_and_equator(sht, nlat):
    # odd nlat: the equator ring has no partner
    lmax = max(nlat - 1, 2)
    check_pair(sht, sht.sht_geom_gauss(nlat, 2 * lmax + 1), lmax, lmax, 2 if lmax >= 2 else 0, seed=nlat)


def test_clenshaw_curtis_poles(sht):
    # rings exactly at theta = 0 and pi
    check_pair(sht, sht.sht_geom_ecp(sht.SHT_ECP_CC, 34, 65), 31, 31, 0, seed=3)
    check_pair(sht, sht.sht_geom_ecp(sht.SHT_ECP_CC, 34, 65), 31, 31, 2, seed=4)


def test_mmax_below_lmax_and_ncomp(sht):
    check_pair(sht, sht.sht_geom_gauss(40, 61), 39, 20, 0, ncomp=3, seed=21)
    check_pair(sht, sht.sht_geom_gauss(40, 61), 39, 25, 2, ncomp=2, seed=22)


def test_tiny_lmax(sht):
    for lmax in (0, 1, 2):
        check_pair(sht, sht.sht_geom_gauss(lmax + 2, 2 * lmax + 3), lmax, lmax, 0, seed=lmax)
    check_pair(sht, sht.sht_geom_gauss(4, 7), 2, 2, 2, seed=7)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("grid", ["gauss", "healpix"])
def test_m_subset(sht, grid, precision):
    # an m list other than 0..mmax: the FFTs take e^{i m phi0} per m instead of
    # walking it (HEALPix: phi0 != 0 and aliased polar rings)
    lmax, mmax = 30, 30
    mval = [0, 3, 7, 30]
    geom = sht.sht_geom_gauss(31, 61) if grid == "gauss" else sht.sht_geom_healpix(8)
    rings = rings_of(geom)
    tol = FP64_L2 if precision == 0 else MIX_L2
    lay = sht.sht_alm_create(lmax, mmax, mval=mval)
    n = lay.size()
    rng = np.random.default_rng(5)
    full = inputs.gaussian_alm(rng, lmax, mmax)
    l, m = inputs.lm_arrays(lmax, mmax)
    keep = np.isin(m, mval)
    full[~keep] = 0.0
    packed = full[keep]
    assert len(packed) == n
    plan = sht.sht_plan_create(geom, lay, 0, 1, precision)
    got = gpu_synthesis(sht, plan, [packed], geom.npix)[0]
    ref = oracle.synthesis(0, lmax, mmax, [full], rings)[0]
    assert rel_l2(got, ref) < tol
    mp = rng.standard_normal(geom.npix)
    got_a = gpu_analysis(sht, plan, [mp], n)[0]
    ref_a = oracle.analysis(0, lmax, mmax, [mp], rings)[0][keep]
    assert rel_l2(got_a, ref_a) < tol


def test_partial_coverage(sht):
    g = sht.sht_geom_gauss(40, 79)
    sel = [0, 1, 2, 5, 9, 20, 38, 39]  # an unbalanced subset: some pairs, some single rings
    sub = sht.sht_geom_subset(g, sel)
    check_pair(sht, sub, 39, 39, 0, seed=31)
    check_pair(sht, sub, 39, 39, 2, seed=32)


def test_add_output_and_flags(sht):
    lmax = 24
    geom = sht.sht_geom_gauss(25, 49)
    lay = sht.sht_alm_create(lmax, lmax)
    plan = sht.sht_plan_create(geom, lay, 0, 1, 0)
    rng = np.random.default_rng(41)
    alm = [inputs.gaussian_alm(rng, lmax, lmax)]
    base = [rng.standard_normal(geom.npix)]
    one = gpu_synthesis(sht, plan, alm, geom.npix)[0]
    two = gpu_synthesis(sht, plan, alm, geom.npix, flags=sht.SHT_ADD_OUTPUT, init=base)[0]
    np.testing.assert_allclose(two, base[0] + one, rtol=0, atol=1e-13)
    a0 = [inputs.gaussian_alm(rng, lmax, lmax)]
    a1 = gpu_analysis(sht, plan, base, len(a0[0]))[0]
    a2 = gpu_analysis(sht, plan, base, len(a0[0]), flags=sht.SHT_ADD_OUTPUT, init=a0)[0]
    l, m = inputs.lm_arrays(lmax, lmax)
    exp = a0[0] + a1
    np.testing.assert_allclose(a2.real, exp.real, atol=1e-13)
    np.testing.assert_allclose(a2.imag[m > 0], exp.imag[m > 0], atol=1e-13)


def test_polar_cut_matches_full_sum(sht):
    # lmax 300 > T = 100: pole-most rings are skipped for high m (Sect. 3.3)
    lmax = 300
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    lay = sht.sht_alm_create(lmax, lmax)
    for spin in (0, 2):
        plan = sht.sht_plan_create(geom, lay, spin, 1, 0)
        assert plan.triples(0) < plan.triples(sht.SHT_NO_POLAR_OPT)
        rng = np.random.default_rng(50 + spin)
        alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(2 if spin else 1)]
        cut = gpu_synthesis(sht, plan, alm, geom.npix)
        full = gpu_synthesis(sht, plan, alm, geom.npix, flags=sht.SHT_NO_POLAR_OPT)
        for c, f in zip(cut, full):
            assert rel_l2(c, f) < 1e-13
        # and both against the oracle on a few rings, including the pole-most ones
        rings = rings_of(geom)
        sel = [0, 1, 2, 40, 150]
        ref = oracle.synthesis(spin, lmax, lmax, alm, rings, rings_sel=sel)
        for c, r in zip(cut, ref):
            for y in sel:
                o, n = rings.ofs[y], rings.nphi[y]
                assert rel_l2(c[o:o + n], r[o:o + n]) < FP64_L2 * 10, y


def test_gl127_scalar_round_trip(sht):
    # GL 128 x 255, lmax = mmax = 127, spin 0, a_lm N(0,1) with a_l0 real, seed 0
    geom = sht.sht_geom_gauss(128, 255)
    lay = sht.sht_alm_create(127, 127)
    plan = sht.sht_plan_create(geom, lay, 0, 1, 0)
    alm = inputs.scalar_gl_small(0, 127)
    mp = gpu_synthesis(sht, plan, alm, geom.npix)
    back = gpu_analysis(sht, plan, mp, len(alm[0]))[0]
    assert rel_l2(back, alm[0]) < 1e-13
    ref = oracle.synthesis(0, 127, 127, alm, rings_of(geom))[0]
    assert rel_l2(mp[0], ref) < FP64_L2


def test_plan_errors(sht):
    geom = sht.sht_geom_gauss(8, 15)
    lay = sht.sht_alm_create(7, 7)
    with pytest.raises(sht.ShtError) as e:
        sht.sht_plan_create(geom, lay, 8, 1, 0)  # |spin| > lmax
    assert e.value.code == sht.SHT_ERR_UNSUPPORTED
    with pytest.raises(sht.ShtError):
        sht.sht_plan_create(geom, lay, 0, 17, 0)
    with pytest.raises(sht.ShtError):
        sht.sht_plan_create(geom, lay, 0, 1, 5)
    plan = sht.sht_plan_create(geom, lay, 0, 1, 0)
    with pytest.raises(sht.ShtError):
        sht._lib.sht_execute  # noqa: B018
        sht.sht_execute(plan, 9, [0], [0])
    with pytest.raises(sht.ShtError):
        sht.sht_execute(plan, 0, [0], [0])  # NULL device pointers


# ------------------------------------------------------------- mixed form ---
MIX_L2 = 1e-10
MIX_MAX = 1e-9


@pytest.mark.parametrize("spin", [0, 1, 2, 3])
def test_mixed_gauss_small(sht, spin):
    check_pair(sht, sht.sht_geom_gauss(42, 81), 40, 40, spin, seed=100 + spin, precision=sht.SHT_MIXED,
               l2=MIX_L2, mx=MIX_MAX, with_adjoint=True)


@pytest.mark.parametrize("spin", [0, 2])
def test_mixed_healpix(sht, spin):
    check_pair(sht, sht.sht_geom_healpix(16), 47, 47, spin, seed=110 + spin, precision=sht.SHT_MIXED,
               l2=MIX_L2, mx=MIX_MAX)


def test_mixed_other_grids_and_jobs(sht):
    check_pair(sht, sht.sht_geom_gauss(21, 37), 18, 18, 2, seed=120, precision=sht.SHT_MIXED, l2=MIX_L2, mx=MIX_MAX)
    check_pair(sht, sht.sht_geom_ecp(sht.SHT_ECP_CC, 34, 65), 31, 31, 2, seed=121, precision=sht.SHT_MIXED,
               l2=MIX_L2, mx=MIX_MAX)
    check_pair(sht, sht.sht_geom_gauss(40, 61), 39, 20, 0, ncomp=3, seed=122, precision=sht.SHT_MIXED,
               l2=MIX_L2, mx=MIX_MAX)
    check_pair(sht, sht.sht_geom_gauss(40, 61), 39, 25, 2, ncomp=2, seed=123, precision=sht.SHT_MIXED,
               l2=MIX_L2, mx=MIX_MAX)


def test_mixed_large_lmax_against_fp64(sht):
    # lmax 1023: long recursions, deep polar growth phases; mixed vs the FP64 GPU form (which is
    # itself pinned to the oracle above) on the full output, plus the oracle on sampled rings
    lmax = 1023
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    lay = sht.sht_alm_create(lmax, lmax)
    rings = rings_of(geom)
    for spin in (0, 2):
        rng = np.random.default_rng(130 + spin)
        alm = [inputs.gaussian_alm(rng, lmax, lmax, cl=inputs.cl_inverse_square, lmin=abs(spin))
               for _ in range(2 if spin else 1)]
        p64 = sht.sht_plan_create(geom, lay, spin, 1, sht.SHT_FP64)
        pmx = sht.sht_plan_create(geom, lay, spin, 1, sht.SHT_MIXED)
        m64 = gpu_synthesis(sht, p64, alm, geom.npix)
        mmx = gpu_synthesis(sht, pmx, alm, geom.npix)
        for a_, b_ in zip(mmx, m64):
            assert rel_l2(a_, b_) < MIX_L2
        b64 = gpu_analysis(sht, p64, m64, len(alm[0]))
        bmx = gpu_analysis(sht, pmx, m64, len(alm[0]))
        for a_, b_ in zip(bmx, b64):
            assert rel_l2(a_, b_) < MIX_L2
        sel = [0, 3, 200, 511]
        ref = oracle.synthesis(spin, lmax, lmax, alm, rings, rings_sel=sel)
        for g_, r_ in zip(mmx, ref):
            idx = np.concatenate([np.arange(rings.ofs[y], rings.ofs[y] + rings.nphi[y]) for y in sel])
            assert rel_l2(g_[idx], r_[idx]) < MIX_L2


def test_mixed_gl127_scalar_round_trip(sht):
    geom = sht.sht_geom_gauss(128, 255)
    lay = sht.sht_alm_create(127, 127)
    plan = sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_MIXED)
    alm = inputs.scalar_gl_small(0, 127)
    mp = gpu_synthesis(sht, plan, alm, geom.npix)
    back = gpu_analysis(sht, plan, mp, len(alm[0]))[0]
    assert rel_l2(back, alm[0]) < MIX_L2


@pytest.mark.parametrize("scale", [1e-25, 1e-12, 1e20])
def test_mixed_scale_range(sht, scale):
    # The mixed form converts between FP64 and FP32 pairs from the numbers' bit
    # fields; a transform of scaled inputs must equal the scaled transform over
    # FP32's range (1e-25: low words below 2^-64, the two-step scaling path).
    # 1517 = 37 41 (large-radix passes), 131 (Rader), 262 (Bluestein).
    for nlon in (1517, 131, 262):
        lmax = min(30, (nlon - 1) // 2)
        geom = sht.sht_geom_gauss(lmax + 1 + (nlon % 2), nlon)
        rings = rings_of(geom)
        rng = np.random.default_rng(nlon)
        alm = [inputs.gaussian_alm(rng, lmax, lmax) * scale]
        plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 0, 1, sht.SHT_MIXED)
        got = gpu_synthesis(sht, plan, alm, geom.npix)[0]
        ref = oracle.synthesis(0, lmax, lmax, alm, rings)[0]
        assert rel_l2(got, ref) <= MIX_L2, (nlon, scale, rel_l2(got, ref))
        maps = [rng.standard_normal(geom.npix) * scale]
        got_a = gpu_analysis(sht, plan, maps, oracle.nalm(lmax, lmax))[0]
        ref_a = oracle.analysis(0, lmax, lmax, maps, rings)[0]
        assert rel_l2(got_a, ref_a) <= MIX_L2, (nlon, scale, rel_l2(got_a, ref_a))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nlon", [14803, 16383, 20011, 20480])
def test_long_rings(sht, nlon, precision):
    # rings longer than one CTA's shared memory holds run from a global scratch
    # slot: 14803 = 113 131 (Bluestein at 29624), 16383 = 3 43 127 (radices 43
    # and 127), 20011 prime (Rader over 20010 = 2 3 5 23 29), 20480 = 2^12 5
    tol = dict(l2=MIX_L2, mx=MIX_MAX) if precision else {}
    check_pair(sht, sht.sht_geom_gauss(30, nlon), 28, 28, 0, seed=nlon, with_adjoint=True, precision=precision, **tol)
    check_pair(sht, sht.sht_geom_gauss(23, nlon), 20, 20, 2, seed=nlon + 1, precision=precision, **tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_deriv_synthesis(sht, precision):
    # Sect. 4.3: spin-0 a_lm -> df/dtheta, df/(sin theta dphi) through a spin-1 plan
    l2, mx = (FP64_L2, FP64_MAX) if precision == 0 else (MIX_L2, MIX_MAX)
    for geom, lmax, ncomp in ((sht.sht_geom_gauss(42, 81), 40, 1), (sht.sht_geom_healpix(16), 47, 2)):
        rings = rings_of(geom)
        plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 1, ncomp, precision)
        rng = np.random.default_rng(400 + ncomp)
        alm = [inputs.gaussian_alm(rng, lmax, lmax) for _ in range(ncomp)]
        a_d = [torch.from_numpy(a).cuda() for a in alm]
        out = [torch.full((geom.npix,), np.nan, dtype=torch.float64, device="cuda") for _ in range(2 * ncomp)]
        sht.sht_execute(plan, sht.SHT_DERIV_SYNTHESIS, a_d, out)
        base = [torch.from_numpy(rng.standard_normal(geom.npix)).cuda() for _ in range(2 * ncomp)]
        acc = [b.clone() for b in base]
        sht.sht_execute(plan, sht.SHT_DERIV_SYNTHESIS, a_d, acc, sht.SHT_ADD_OUTPUT)
        torch.cuda.synchronize()
        ref = oracle.deriv_synthesis(lmax, lmax, alm, rings)
        for g, r, b, c in zip(out, ref, base, acc):
            g = g.cpu().numpy()
            assert rel_l2(g, r) <= l2 and rel_max(g, r) <= mx, (rel_l2(g, r), rel_max(g, r))
            assert rel_l2(c.cpu().numpy() - b.cpu().numpy(), r) <= l2
    p0 = sht.sht_plan_create(sht.sht_geom_gauss(10, 19), sht.sht_alm_create(8, 8), 0, 1, precision)
    z = torch.zeros(oracle.nalm(8, 8), dtype=torch.complex128, device="cuda")
    with pytest.raises(sht.ShtError):
        sht.sht_execute(p0, sht.SHT_DERIV_SYNTHESIS, [z], [torch.zeros(10 * 19, dtype=torch.float64, device="cuda")])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("spin", [0, 2])
def test_real_harmonic_storage(sht, precision, spin):
    # Sect. 4.5: a_lm stored as real-harmonic coefficients (reading in oracle.real_to_complex)
    l2, mx = (FP64_L2, FP64_MAX) if precision == 0 else (MIX_L2, MIX_MAX)
    lmax = 40
    geom = sht.sht_geom_gauss(42, 81)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, precision)
    narr = plan.narrays
    rng = np.random.default_rng(500 + spin)
    ar = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(narr)]  # real storage
    ac = [oracle.real_to_complex(a, lmax, lmax) for a in ar]
    maps = [rng.standard_normal(geom.npix) for _ in range(narr)]
    R = sht.SHT_REAL_HARMONICS
    # synthesis reads real storage
    a_d = [torch.from_numpy(a).cuda() for a in ar]
    out = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(narr)]
    sht.sht_execute(plan, sht.SHT_SYNTHESIS, a_d, out, R)
    ref = oracle.synthesis(spin, lmax, lmax, ac, rings)
    # analysis and adjoint synthesis write real storage
    m_d = [torch.from_numpy(x).cuda() for x in maps]
    n = oracle.nalm(lmax, lmax)
    ana = [torch.full((n,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda") for _ in range(narr)]
    sht.sht_execute(plan, sht.SHT_ANALYSIS, ana, m_d, R)
    adj = [torch.full((n,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda") for _ in range(narr)]
    sht.sht_execute(plan, sht.SHT_ADJOINT_SYNTHESIS, adj, m_d, R)
    # accumulation in real storage, and the no-alloc entry
    acc = [torch.from_numpy(a).cuda() for a in ar]
    sht.sht_execute(plan, sht.SHT_ANALYSIS, acc, m_d, R | sht.SHT_ADD_OUTPUT)
    out2 = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(narr)]
    sht.sht_execute_noalloc(plan, sht.SHT_SYNTHESIS, a_d, out2, R)
    torch.cuda.synchronize()
    ref_a = [oracle.complex_to_real(x, lmax, lmax) for x in oracle.analysis(spin, lmax, lmax, maps, rings)]
    ref_j = [oracle.complex_to_real(x, lmax, lmax) for x in
             oracle.analysis(spin, lmax, lmax, maps, rings, adjoint=True)]
    for g, r in zip(out, ref):
        assert rel_l2(g.cpu().numpy(), r) <= l2 and rel_max(g.cpu().numpy(), r) <= mx
    for g, r in zip(out2, ref):
        assert rel_l2(g.cpu().numpy(), r) <= l2
    for g, r in zip(ana, ref_a):
        assert rel_l2(g.cpu().numpy(), r) <= l2
    for g, r in zip(adj, ref_j):
        assert rel_l2(g.cpu().numpy(), r) <= l2
    for g, a0, r in zip(acc, ar, ref_a):
        assert rel_l2(g.cpu().numpy() - a0, r) <= l2
    # in real storage the adjoint synthesis is the plain transpose: <S a, p> = <a, S^T p>
    lhs = sum(float(torch.dot(o, m)) for o, m in zip(out, m_d))
    _, mm = inputs.lm_arrays(lmax, lmax)
    rhs = 0.0
    for a, j in zip(ar, adj):
        j = j.cpu().numpy()
        rhs += float(np.sum(a.real * j.real) + np.sum((a.imag * j.imag)[mm > 0]))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_real_harmonic_deriv_and_batch(sht):
    lmax = 30
    geom = sht.sht_geom_gauss(32, 61)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 1, 1, 0)
    ar = inputs.gaussian_alm(np.random.default_rng(510), lmax, lmax)
    out = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    sht.sht_execute(plan, sht.SHT_DERIV_SYNTHESIS, [torch.from_numpy(ar).cuda()], out, sht.SHT_REAL_HARMONICS)
    torch.cuda.synchronize()
    ref = oracle.deriv_synthesis(lmax, lmax, [oracle.real_to_complex(ar, lmax, lmax)], rings)
    for g, r in zip(out, ref):
        assert rel_l2(g.cpu().numpy(), r) <= FP64_L2
    batch = sht.sht_batch_create([plan])
    with pytest.raises(sht.ShtError) as ei:
        sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, [[torch.from_numpy(ar).cuda()] * 2], [out],
                              sht.SHT_REAL_HARMONICS)
    assert ei.value.code == sht.SHT_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", [0, 1])
def test_high_spin(sht, precision):
    # Sect. 4.1: spins well above 2 (the paper repeats its accuracy test at s = 37);
    # plans accept |s| <= 64
    l2, mx = (FP64_L2, FP64_MAX) if precision == 0 else (MIX_L2, MIX_MAX)
    check_pair(sht, sht.sht_geom_gauss(72, 141), 70, 70, 37, seed=600, precision=precision, l2=l2, mx=mx)
    check_pair(sht, sht.sht_geom_gauss(82, 161), 80, 80, 64, seed=601, precision=precision, l2=l2, mx=mx)
    check_pair(sht, sht.sht_geom_healpix(16), 40, 40, -5, seed=602, precision=precision, l2=l2, mx=mx)
    # exact Gauss-Legendre round trip at s = 37
    lmax = 90
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 37, 1, precision)
    rng = np.random.default_rng(603)
    alm = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, lmin=37)).cuda() for _ in range(2)]
    maps = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    back = [torch.empty_like(a) for a in alm]
    sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm, maps)
    sht.sht_execute(plan, sht.SHT_ANALYSIS, back, maps)
    torch.cuda.synchronize()
    for a, b in zip(alm, back):
        assert float(torch.linalg.norm(a - b) / torch.linalg.norm(a)) <= 10 * l2


def test_join_records_skip_only_negligible_steps(sht):
    # a mixed plan's kernels skip each pair's steps before its join block; the
    # count of steps left is below the polar-cut count, the FP64 plan reports the
    # polar-cut count, and the mixed synthesis with the skip matches the oracle on
    # the pole-most rings, where the skipped stretches are longest
    lmax = 600
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    lay = sht.sht_alm_create(lmax, lmax)
    rings = rings_of(geom)
    sel = [0, 1, 3, 20, 150, 300]
    for spin in (0, 2):
        mixed = sht.sht_plan_create(geom, lay, spin, 1, sht.SHT_MIXED)
        fp64 = sht.sht_plan_create(geom, lay, spin, 1, sht.SHT_FP64)
        assert fp64.triples_joined() == fp64.triples(0)
        assert 0 < mixed.triples_joined() < mixed.triples(0)
        rng = np.random.default_rng(60 + spin)
        alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(2 if spin else 1)]
        got = gpu_synthesis(sht, mixed, alm, geom.npix)
        ref = oracle.synthesis(spin, lmax, lmax, alm, rings, rings_sel=sel)
        for c, r in zip(got, ref):
            for y in sel:
                o, n = rings.ofs[y], rings.nphi[y]
                assert rel_l2(c[o:o + n], r[o:o + n]) < 1e-10, (spin, y)
