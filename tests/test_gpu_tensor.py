"""The mixed form's synthesis with the contraction on the tensor cores (tcgen05).

The same transforms as the double-float kernels, checked element by element
against the FP64 oracle at the mixed tolerance (1e-10 relative L2, 1e-9 of the
largest value) and against the double-float contraction of the same plan:
spins 0, 1, 2, 3, -2 and 37; one to eight maps (padded job counts); degrees
spanning several 256-degree windows with a ragged last K-step; ring-pair counts
that leave a partial CTA; Gauss-Legendre, HEALPix (aliased rings, phi0 != 0)
and Clenshaw-Curtis grids; the synthesis, the adjoint analysis and the
derivative synthesis; m subsets; forced FP64 columns; the no-alloc entry point;
inputs scaled far from 1; and the device status word after every run.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIX_L2, MIX_MAX = 1e-10, 1e-9


@pytest.fixture(scope="module")
def sht():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht as m

    assert torch.cuda.is_available()
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rings_of(geom):
    r = geom.rings()
    return oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])


def run_synthesis(sht, plan, alm, npix, nout, type_=None, flags=0, noalloc=False):
    type_ = sht.SHT_SYNTHESIS if type_ is None else type_
    a = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in alm]
    m = [torch.full((npix,), np.nan, dtype=torch.float64, device="cuda") for _ in range(nout)]
    (sht.sht_execute_noalloc if noalloc else sht.sht_execute)(plan, type_, a, m, flags)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return [x.cpu().numpy() for x in m]


def both_forms(sht, plan, alm, npix, nout, **kw):
    """(tensor-core result, double-float result) of the same plan."""
    plan.tensor_cores = True
    tcr = run_synthesis(sht, plan, alm, npix, nout, **kw)
    plan.tensor_cores = False
    dfr = run_synthesis(sht, plan, alm, npix, nout, **kw)
    plan.tensor_cores = True
    return tcr, dfr


def check(got, ref, dfr=None, l2=MIX_L2, mx=MIX_MAX):
    for k, (g, r) in enumerate(zip(got, ref)):
        assert rel_l2(g, r) <= l2 and rel_max(g, r) <= mx, (k, rel_l2(g, r), rel_max(g, r))
    if dfr is not None:  # both contractions of the same recursion values
        for g, d in zip(got, dfr):
            assert rel_l2(g, d) <= 1e-11, rel_l2(g, d)


@pytest.mark.parametrize("spin,ncomp", [(0, 1), (0, 2), (0, 3), (0, 8), (1, 1), (2, 1), (2, 2), (2, 4), (3, 1),
                                        (-2, 1)])
def test_tensor_synthesis_matches_oracle(sht, spin, ncomp):
    # lmax 300: two 256-degree windows for small m, a ragged last K-step; GL 302 x
    # 601 has 151 ring pairs (one full CTA of 128 and a partial one)
    lmax = 300
    geom = sht.sht_geom_gauss(lmax + 2, 2 * lmax + 1)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, ncomp, sht.SHT_MIXED)
    narr = plan.narrays
    rng = np.random.default_rng(700 + 10 * abs(spin) + ncomp)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(narr)]
    got, dfr = both_forms(sht, plan, alm, geom.npix, narr)
    check(got, oracle.synthesis(spin, lmax, lmax, alm, rings), dfr)
    # the adjoint analysis runs the same synthesis stage, then the weights
    got, dfr = both_forms(sht, plan, alm, geom.npix, narr, type_=sht.SHT_ADJOINT_ANALYSIS)
    check(got, oracle.synthesis(spin, lmax, lmax, alm, rings, weighted=True), dfr)


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("flags", [0, 2])
def test_tensor_healpix_and_cc(sht, spin, flags):
    # HEALPix: aliased polar rings, phi0 != 0; Clenshaw-Curtis: poles on the grid;
    # flags 2 = SHT_NO_POLAR_OPT (every term evaluated)
    for geom, lmax in ((sht.sht_geom_healpix(64), 191), (sht.sht_geom_ecp(sht.SHT_ECP_CC, 130, 259), 128)):
        rings = rings_of(geom)
        plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, sht.SHT_MIXED)
        narr = plan.narrays
        rng = np.random.default_rng(800 + spin + flags)
        alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(narr)]
        got, dfr = both_forms(sht, plan, alm, geom.npix, narr, flags=flags)
        check(got, oracle.synthesis(spin, lmax, lmax, alm, rings), dfr)


def test_tensor_high_spin_and_deriv(sht):
    # spin 37 (Sect. 4.1's high-spin case) and the derivative synthesis (Sect. 4.3)
    lmax = 120
    geom = sht.sht_geom_gauss(122, 241)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 37, 1, sht.SHT_MIXED)
    rng = np.random.default_rng(900)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=37) for _ in range(2)]
    got, dfr = both_forms(sht, plan, alm, geom.npix, 2)
    check(got, oracle.synthesis(37, lmax, lmax, alm, rings), dfr)
    for ncomp in (1, 2):
        plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 1, ncomp, sht.SHT_MIXED)
        alm = [inputs.gaussian_alm(rng, lmax, lmax) for _ in range(ncomp)]
        got, dfr = both_forms(sht, plan, alm, geom.npix, 2 * ncomp, type_=sht.SHT_DERIV_SYNTHESIS)
        check(got, oracle.deriv_synthesis(lmax, lmax, alm, rings), dfr)


def test_tensor_m_subset_fp64_columns_noalloc(sht):
    lmax = 280
    geom = sht.sht_geom_healpix(48)
    rings = rings_of(geom)
    # an m list other than 0..mmax, mmax < lmax
    mval = [0, 1, 5, 64, 200]
    lay = sht.sht_alm_create(lmax, 200, mval=mval)
    rng = np.random.default_rng(901)
    full = [inputs.gaussian_alm(rng, lmax, 200, lmin=2) for _ in range(2)]
    _, m = inputs.lm_arrays(lmax, 200)
    keep = np.isin(m, mval)
    for f in full:
        f[~keep] = 0.0
    plan = sht.sht_plan_create(geom, lay, 2, 1, sht.SHT_MIXED)
    got, dfr = both_forms(sht, plan, [f[keep] for f in full], geom.npix, 2)
    check(got, oracle.synthesis(2, lmax, 200, full, rings), dfr)
    # forced FP64 columns (their items keep running in the FP64 kernels), and the
    # same through the no-alloc entry point
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    plan.fp64_columns = 20
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
    ref = oracle.synthesis(2, lmax, lmax, alm, rings)
    got, dfr = both_forms(sht, plan, alm, geom.npix, 2)
    check(got, ref, dfr)
    got = run_synthesis(sht, plan, alm, geom.npix, 2, noalloc=True)
    check(got, ref)


@pytest.mark.parametrize("scale", [1e-20, 1e15])
def test_tensor_scaled_inputs(sht, scale):
    # the digit grids follow the a_lm's own magnitude per window
    lmax = 200
    geom = sht.sht_geom_gauss(202, 401)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    rng = np.random.default_rng(902)
    alm = [scale * inputs.gaussian_alm(rng, lmax, lmax, lmin=2, cl=inputs.cl_inverse_square) for _ in range(2)]
    plan.tensor_cores = True
    got = run_synthesis(sht, plan, alm, geom.npix, 2)
    check(got, oracle.synthesis(2, lmax, lmax, alm, rings))


def test_tensor_setting_errors(sht):
    geom = sht.sht_geom_gauss(10, 19)
    lay = sht.sht_alm_create(8, 8)
    fp = sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_FP64)
    with pytest.raises(sht.ShtError) as e:
        fp.tensor_cores = True
    assert e.value.code == sht.SHT_ERR_INVALID_ARG
    wide = sht.sht_plan_create(geom, lay, 2, 8, sht.SHT_MIXED)  # 64 columns
    with pytest.raises(sht.ShtError) as e:
        wide.tensor_cores = True
    assert e.value.code == sht.SHT_ERR_UNSUPPORTED
    # the default: the tensor cores for every supported shape but a single spin-0 map
    ok = sht.sht_plan_create(geom, lay, 2, 1, sht.SHT_MIXED)
    assert ok.tensor_cores
    assert not sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_MIXED).tensor_cores
    assert sht.sht_plan_create(geom, lay, 0, 2, sht.SHT_MIXED).tensor_cores
    assert not sht.sht_plan_create(geom, lay, 0, 16, sht.SHT_MIXED).tensor_cores
    ok.tensor_cores = False
    assert not ok.tensor_cores and ok.device_status() == 0
