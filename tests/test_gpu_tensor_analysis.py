"""The mixed form's analysis with the contraction over ring pairs on the tensor
cores (tcgen05).

The same transforms as the double-float analysis, checked element by element
against the FP64 oracle at the mixed tolerance (1e-10 relative L2, 1e-9 of the
largest value) and against the double-float contraction of the same plan:
spins 0, 1, 2, 3, -2 and 37; one and two jobs; ring-pair counts that leave a
partial tile; Gauss-Legendre, HEALPix (aliased rings, phi0 != 0) and
Clenshaw-Curtis grids, with and without the polar cut; the analysis and the
adjoint synthesis; m subsets; forced FP64 columns; the no-alloc entry point;
inputs scaled far from 1; work items that walk several tiles into one slot of
partial sums; the Sect. 4.2 stage calls, CUDA-graph capture and a batch (bit for
bit against the plan's own call); and the device status word after every run.
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


def run_analysis(sht, plan, maps, nalm, type_=None, flags=0, noalloc=False):
    type_ = sht.SHT_ANALYSIS if type_ is None else type_
    m = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in maps]
    a = [torch.full((nalm,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda") for _ in maps]
    (sht.sht_execute_noalloc if noalloc else sht.sht_execute)(plan, type_, a, m, flags)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    return [x.cpu().numpy() for x in a]


def both_forms(sht, plan, maps, nalm, **kw):
    """(tensor-core result, double-float result) of the same plan."""
    plan.tensor_core_analysis = True
    tcr = run_analysis(sht, plan, maps, nalm, **kw)
    plan.tensor_core_analysis = False
    dfr = run_analysis(sht, plan, maps, nalm, **kw)
    plan.tensor_core_analysis = True
    return tcr, dfr


def check(got, ref, dfr=None, l2=MIX_L2, mx=MIX_MAX, sel=None):
    sel = slice(None) if sel is None else sel
    for k, (g, r) in enumerate(zip(got, ref)):
        assert rel_l2(g[sel], r[sel]) <= l2 and rel_max(g[sel], r[sel]) <= mx, (k, rel_l2(g[sel], r[sel]),
                                                                                rel_max(g[sel], r[sel]))
    if dfr is not None:  # both contractions of the same recursion values
        for g, d in zip(got, dfr):
            assert rel_l2(g, d) <= 1e-11, rel_l2(g, d)


@pytest.mark.parametrize("spin,ncomp", [(0, 1), (0, 2), (1, 1), (2, 1), (2, 2), (3, 1), (-2, 1)])
def test_tensor_analysis_matches_oracle(sht, spin, ncomp):
    # lmax 300, GL 302 x 601: 151 ring pairs (one full tile of 128 and a partial
    # one); degrees in blocks of 8 with a ragged last block
    lmax = 300
    geom = sht.sht_geom_gauss(lmax + 2, 2 * lmax + 1)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, ncomp, sht.SHT_MIXED)
    narr = plan.narrays
    rng = np.random.default_rng(1700 + 10 * abs(spin) + ncomp)
    maps = [inputs.gaussian_map(rng, geom.npix) for _ in range(narr)]
    nalm = oracle.nalm(lmax, lmax)
    got, dfr = both_forms(sht, plan, maps, nalm)
    check(got, oracle.analysis(spin, lmax, lmax, maps, rings), dfr)
    # the adjoint synthesis runs the same analysis stage without the weights
    got, dfr = both_forms(sht, plan, maps, nalm, type_=sht.SHT_ADJOINT_SYNTHESIS)
    check(got, oracle.analysis(spin, lmax, lmax, maps, rings, adjoint=True), dfr)


@pytest.mark.parametrize("spin", [0, 2])
@pytest.mark.parametrize("flags", [0, 2])
def test_tensor_analysis_healpix_and_cc(sht, spin, flags):
    # HEALPix: aliased polar rings, phi0 != 0; Clenshaw-Curtis: poles on the grid;
    # flags 2 = SHT_NO_POLAR_OPT (every term evaluated)
    for geom, lmax in ((sht.sht_geom_healpix(64), 191), (sht.sht_geom_ecp(sht.SHT_ECP_CC, 130, 259), 128)):
        rings = rings_of(geom)
        plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, sht.SHT_MIXED)
        narr = plan.narrays
        rng = np.random.default_rng(1800 + spin + flags)
        maps = [inputs.gaussian_map(rng, geom.npix) for _ in range(narr)]
        got, dfr = both_forms(sht, plan, maps, oracle.nalm(lmax, lmax), flags=flags)
        check(got, oracle.analysis(spin, lmax, lmax, maps, rings), dfr)


def test_tensor_analysis_high_spin_band_limited(sht):
    # spin 37 (Sect. 4.1's high-spin case); and a band-limited spin-2 map with a
    # decaying spectrum, whose a_lm span orders of magnitude across l
    lmax = 120
    geom = sht.sht_geom_gauss(122, 241)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 37, 1, sht.SHT_MIXED)
    rng = np.random.default_rng(1900)
    maps = [inputs.gaussian_map(rng, geom.npix) for _ in range(2)]
    got, dfr = both_forms(sht, plan, maps, oracle.nalm(lmax, lmax))
    check(got, oracle.analysis(37, lmax, lmax, maps, rings), dfr)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2, cl=inputs.cl_inverse_square) for _ in range(2)]
    maps = oracle.synthesis(2, lmax, lmax, alm, rings)
    got, dfr = both_forms(sht, plan, maps, oracle.nalm(lmax, lmax))
    check(got, oracle.analysis(2, lmax, lmax, maps, rings), dfr)
    for g, a in zip(got, alm):  # Gauss-Legendre quadrature is exact: the input comes back
        assert rel_l2(g, a) <= MIX_L2


@pytest.mark.parametrize("spin", [0, 2])
def test_tensor_analysis_m_subset_fp64_columns_noalloc(sht, spin):
    lmax = 280
    geom = sht.sht_geom_healpix(48)
    rings = rings_of(geom)
    rng = np.random.default_rng(1901 + spin)
    narr = 2 if spin else 1
    maps = [inputs.gaussian_map(rng, geom.npix) for _ in range(narr)]
    # an m list other than 0..mmax, mmax < lmax
    mval = [0, 1, 5, 64, 200]
    lay = sht.sht_alm_create(lmax, 200, mval=mval)
    _, m = inputs.lm_arrays(lmax, 200)
    keep = np.isin(m, mval)
    plan = sht.sht_plan_create(geom, lay, spin, 1, sht.SHT_MIXED)
    got, dfr = both_forms(sht, plan, maps, int(keep.sum()))
    ref = oracle.analysis(spin, lmax, 200, maps, rings, m_sel=mval)
    check(got, [r[keep] for r in ref], dfr)
    # forced FP64 columns: their tiles next to the poles run in the FP64 kernels on
    # the tensor-core analysis' tiling (one pair per thread); the same through the
    # no-alloc entry point
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, sht.SHT_MIXED)
    plan.fp64_columns = 20
    ref = oracle.analysis(spin, lmax, lmax, maps, rings)
    got, dfr = both_forms(sht, plan, maps, oracle.nalm(lmax, lmax))
    check(got, ref, dfr)
    got = run_analysis(sht, plan, maps, oracle.nalm(lmax, lmax), noalloc=True)
    check(got, ref)


@pytest.mark.parametrize("scale", [1e-20, 1e15])
def test_tensor_analysis_scaled_inputs(sht, scale):
    # the G digits' grid follows each tile's own magnitude
    lmax = 200
    geom = sht.sht_geom_gauss(202, 401)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    rng = np.random.default_rng(1902)
    maps = [scale * inputs.gaussian_map(rng, geom.npix) for _ in range(2)]
    plan.tensor_core_analysis = True
    got = run_analysis(sht, plan, maps, oracle.nalm(lmax, lmax))
    check(got, oracle.analysis(2, lmax, lmax, maps, rings))


def test_tensor_analysis_tile_groups(sht):
    # lmax 2047, GL 2048 x 4095: 8 tiles of 128 pairs per m, about 12000 tiles after
    # the polar cut, so an item walks a group of tiles (about 3) into one slot of
    # partial sums; the oracle on sampled m, the double-float form on all
    lmax, ms = 2047, [0, 1, 2, 3, 700, 1500, 2047]
    geom = sht.sht_geom_gauss(2048, 4095)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    rng = np.random.default_rng(1903)
    maps = [inputs.gaussian_map(rng, geom.npix) for _ in range(2)]
    got, dfr = both_forms(sht, plan, maps, oracle.nalm(lmax, lmax))
    _, m = inputs.lm_arrays(lmax, lmax)
    check(got, oracle.analysis(2, lmax, lmax, maps, rings, m_sel=ms), dfr, sel=np.isin(m, ms))


def test_tensor_analysis_settings(sht):
    geom = sht.sht_geom_gauss(40, 79)
    lay = sht.sht_alm_create(38, 38)
    fp = sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_FP64)
    with pytest.raises(sht.ShtError) as e:
        fp.tensor_core_analysis = True
    assert e.value.code == sht.SHT_ERR_INVALID_ARG
    wide = sht.sht_plan_create(geom, lay, 2, 3, sht.SHT_MIXED)  # 4 jobs padded
    with pytest.raises(sht.ShtError) as e:
        wide.tensor_core_analysis = True
    assert e.value.code == sht.SHT_ERR_UNSUPPORTED
    ok = sht.sht_plan_create(geom, lay, 2, 1, sht.SHT_MIXED)
    ok.tensor_core_analysis = True
    assert ok.tensor_core_analysis and ok.tiling()[0] == 1  # one ring pair per thread
    with pytest.raises(sht.ShtError) as e:
        ok.set_tiling(2)
    assert e.value.code == sht.SHT_ERR_UNSUPPORTED
    # the autotuner times the tensor-core analysis beside the tilings and keeps the fastest
    tune = ok.autotune(torch.cuda.current_stream())
    assert "tensor_cores" in tune and tune["tensor_cores"] > 0
    assert ok.tensor_core_analysis == (min(tune, key=tune.get) == "tensor_cores")
    assert "tensor_cores" not in wide.autotune(torch.cuda.current_stream())
    ok.tensor_core_analysis = False
    assert not ok.tensor_core_analysis and ok.device_status() == 0


def test_tensor_analysis_stage_calls_graph_and_batch(sht):
    from paper_1303_4945_gb300 import distributed as D

    lmax = 200
    geom = sht.sht_geom_gauss(lmax + 2, 2 * lmax + 1)
    rings = rings_of(geom)
    r = geom.rings()
    rng = np.random.default_rng(1904)
    maps = [inputs.gaussian_map(rng, geom.npix) for _ in range(2)]
    nalm = oracle.nalm(lmax, lmax)
    # the stage calls of the Sect. 4.2 decomposition (two tasks emulated on this GPU),
    # each task's Legendre plan on the tensor-core analysis
    part = D.Partition.round_robin(lmax, r["theta"], 2)
    stages = [D.LibraryStages(sht, geom, lmax, lmax, 2, 1, sht.SHT_MIXED, part, k) for k in range(2)]
    for st in stages:
        st.plan_m.tensor_core_analysis = True
    maps_loc = [[torch.from_numpy(p[D.ring_pixels(r["ofs"], r["nphi"], part.rings[k])]).cuda() for p in maps]
                for k in range(2)]
    back = D.analysis_emulated(part, stages, maps_loc)
    torch.cuda.synchronize()
    got = [np.zeros(nalm, dtype=np.complex128) for _ in range(2)]
    for k in range(2):
        assert stages[k].plan_m.device_status() == 0
        for c in range(2):
            D.alm_unpack(back[k][c].cpu().numpy(), lmax, lmax, part.m[k], got[c])
    check(got, oracle.analysis(2, lmax, lmax, maps, rings))
    # captured in a CUDA graph after one call outside the capture, replayed with new maps
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    plan.tensor_core_analysis = True
    m_d = [torch.from_numpy(x).cuda() for x in maps]
    a_d = [torch.zeros(nalm, dtype=torch.complex128, device="cuda") for _ in range(2)]
    sht.sht_execute(plan, sht.SHT_ANALYSIS, a_d, m_d)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sht.sht_execute(plan, sht.SHT_ANALYSIS, a_d, m_d, 0, torch.cuda.current_stream())
    maps2 = [inputs.gaussian_map(rng, geom.npix) for _ in range(2)]
    for x, y in zip(m_d, maps2):
        x.copy_(torch.from_numpy(y))
    g.replay()
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    check([a.cpu().numpy() for a in a_d], oracle.analysis(2, lmax, lmax, maps2, rings))
    # a batch of that plan (with a double-float one beside it) runs the tensor-core
    # analysis too: the same items and arithmetic, the same bits
    other = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    batch = sht.sht_batch_create([plan, other])
    b_d = [torch.zeros_like(a) for a in a_d]
    o_d = [torch.zeros_like(a) for a in a_d]
    sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, [b_d, o_d], [m_d, m_d])
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    for x, y in zip(b_d, a_d):
        assert torch.equal(x, y)
    check([x.cpu().numpy() for x in o_d], oracle.analysis(2, lmax, lmax, maps2, rings))
    del batch
