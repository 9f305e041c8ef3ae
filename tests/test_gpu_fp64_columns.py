"""Mixed-form plans whose small-m columns run in the FP64 kernels.

The default threshold is 0 below lmax 2000, so these tests force one on small
plans: results must match the oracle for every transform type (those columns
to the FP64 tolerance, the plan as a whole to the mixed one), inside a batch
and through the no-alloc entry point; the threshold's default and its error
cases are checked too.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sht():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht as m

    assert torch.cuda.is_available()
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rings_of(geom):
    r = geom.rings()
    return oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])


@pytest.mark.parametrize("spin,make", [(0, lambda s: s.sht_geom_gauss(50, 99)),
                                       (2, lambda s: s.sht_geom_gauss(50, 99)),
                                       (0, lambda s: s.sht_geom_healpix(16)),
                                       (1, lambda s: s.sht_geom_healpix(16))])
@pytest.mark.parametrize("flags", [0, 2])
def test_forced_fp64_columns_match_oracle(sht, spin, make, flags):
    lmax = 47
    geom = make(sht)
    rings = rings_of(geom)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, sht.SHT_MIXED)
    assert plan.fp64_columns == 0
    plan.fp64_columns = 9
    assert plan.fp64_columns == 9
    narr = plan.narrays
    rng = np.random.default_rng(300 + spin)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(narr)]
    maps = [rng.standard_normal(geom.npix) for _ in range(narr)]
    _, m = inputs.lm_arrays(lmax, lmax)
    n = oracle.nalm(lmax, lmax)
    cases = [
        (sht.SHT_SYNTHESIS, alm, oracle.synthesis(spin, lmax, lmax, alm, rings), True),
        (sht.SHT_ADJOINT_ANALYSIS, alm, oracle.synthesis(spin, lmax, lmax, alm, rings, weighted=True), True),
        (sht.SHT_ANALYSIS, maps, oracle.analysis(spin, lmax, lmax, maps, rings), False),
        (sht.SHT_ADJOINT_SYNTHESIS, maps, oracle.analysis(spin, lmax, lmax, maps, rings, adjoint=True), False),
    ]
    for type_, inp, ref, to_map in cases:
        src = [torch.from_numpy(x).cuda() for x in inp]
        if to_map:
            out = [torch.full((geom.npix,), np.nan, dtype=torch.float64, device="cuda") for _ in range(narr)]
            sht.sht_execute(plan, type_, src, out, flags)
        else:
            out = [torch.full((n,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
                   for _ in range(narr)]
            sht.sht_execute(plan, type_, out, src, flags)
        torch.cuda.synchronize()
        for g, r in zip(out, ref):
            g = g.cpu().numpy()
            assert rel_l2(g, r) <= 1e-10, (type_, rel_l2(g, r))
            if not to_map:  # the FP64 columns to the FP64 tolerance
                lo = m < 9
                assert rel_l2(g[lo], r[lo]) <= 1e-12, (type_, rel_l2(g[lo], r[lo]))


def test_fp64_columns_in_batch_and_noalloc(sht):
    lmax = 40
    geom = sht.sht_geom_gauss(42, 81)
    rings = rings_of(geom)
    lay = sht.sht_alm_create(lmax, lmax)
    mixed = sht.sht_plan_create(geom, lay, 2, 1, sht.SHT_MIXED)
    mixed.fp64_columns = 6
    other = sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_FP64)
    rng = np.random.default_rng(310)
    alm_m = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
    alm_o = [inputs.gaussian_alm(rng, lmax, lmax)]
    ref_m = oracle.synthesis(2, lmax, lmax, alm_m, rings)
    ref_o = oracle.synthesis(0, lmax, lmax, alm_o, rings)
    batch = sht.sht_batch_create([mixed, other])
    a_in = [[torch.from_numpy(x).cuda() for x in alm_m], [torch.from_numpy(x).cuda() for x in alm_o]]
    m_out = [[torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)],
             [torch.zeros(geom.npix, dtype=torch.float64, device="cuda")]]
    sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_in, m_out)
    torch.cuda.synchronize()
    for g, r in zip(m_out[0], ref_m):
        assert rel_l2(g.cpu().numpy(), r) <= 1e-10
    assert rel_l2(m_out[1][0].cpu().numpy(), ref_o[0]) <= 1e-12
    with pytest.raises(sht.ShtError):
        mixed.fp64_columns = 3  # locked while the batch exists
    del batch
    # the no-alloc entry point uses both converted a_lm tables for such a plan
    out = [torch.full((geom.npix,), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
    sht.sht_execute_noalloc(mixed, sht.SHT_SYNTHESIS, a_in[0], out)
    torch.cuda.synchronize()
    for g, r in zip(out, ref_m):
        assert rel_l2(g.cpu().numpy(), r) <= 1e-10


def test_default_and_errors(sht):
    lay = sht.sht_alm_create(8, 8)
    geom = sht.sht_geom_gauss(10, 17)
    fp = sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_FP64)
    with pytest.raises(sht.ShtError):
        fp.fp64_columns = 2  # FP64 plans have no mixed columns
    mx = sht.sht_plan_create(geom, lay, 0, 1, sht.SHT_MIXED)
    with pytest.raises(sht.ShtError):
        mx.fp64_columns = -1
    big = sht.sht_plan_create(sht.sht_geom_gauss(4097, 5), sht.sht_alm_create(4095, 2), 0, 1, sht.SHT_MIXED)
    assert big.fp64_columns == 24  # lmax / 170 from lmax 2000 on
    small = sht.sht_plan_create(sht.sht_geom_gauss(1025, 5), sht.sht_alm_create(1023, 2), 0, 1, sht.SHT_MIXED)
    assert small.fp64_columns == 0


def test_fp64_items_under_graph_capture(sht):
    # the FP64 items run on a side stream forked and joined by events: a captured
    # synthesis + analysis must replay to the same bits as direct calls
    lmax = 60
    geom = sht.sht_geom_gauss(62, 121)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
    plan.fp64_columns = 12
    rng = np.random.default_rng(320)
    a_in = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, lmin=2)).cuda() for _ in range(2)]
    maps = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    out = [torch.zeros_like(a) for a in a_in]
    sht.sht_execute(plan, sht.SHT_SYNTHESIS, a_in, maps)  # warm
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = torch.cuda.current_stream()
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, a_in, maps, 0, st)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, out, maps, 0, st)
    for rep in range(2):
        for a in a_in:
            a.copy_(torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, lmin=2)).cuda())
        g.replay()
        torch.cuda.synchronize()
        m_ref = [torch.zeros_like(m) for m in maps]
        o_ref = [torch.zeros_like(o) for o in out]
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, a_in, m_ref)
        sht.sht_execute(plan, sht.SHT_ANALYSIS, o_ref, m_ref)
        torch.cuda.synchronize()
        for x, y in zip(maps + out, m_ref + o_ref):
            assert torch.equal(x, y), rep


def test_fft_precision_setting(sht):
    """A mixed plan's ring FFTs run in double-float by default; the FP64 engine is
    selectable per plan.  Both match the oracle, agree with each other far inside
    the mixed tolerance, and run side by side in one batch."""
    lmax = 30
    rng = np.random.default_rng(77)
    cases = []
    for nlon in (1517, 131, 262):  # large radices, Rader, Bluestein
        geom = sht.sht_geom_gauss(lmax + 2, nlon)
        alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
        maps = [rng.standard_normal(geom.npix) for _ in range(2)]
        cases.append((geom, alm, maps))
    n = oracle.nalm(lmax, lmax)
    results = {}
    for fftp in (sht.SHT_MIXED, sht.SHT_FP64):
        plans = []
        for geom, alm, maps in cases:
            plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, sht.SHT_MIXED)
            assert plan.fft_precision == sht.SHT_MIXED
            plan.fft_precision = fftp
            assert plan.fft_precision == fftp
            m_d = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
            sht.sht_execute(plan, sht.SHT_SYNTHESIS, [torch.from_numpy(a).cuda() for a in alm], m_d)
            a_d = [torch.zeros(n, dtype=torch.complex128, device="cuda") for _ in range(2)]
            sht.sht_execute(plan, sht.SHT_ANALYSIS, a_d, [torch.from_numpy(m).cuda() for m in maps])
            torch.cuda.synchronize()
            ref_s = oracle.synthesis(2, lmax, lmax, alm, rings_of(geom))
            ref_a = oracle.analysis(2, lmax, lmax, maps, rings_of(geom))
            got_s = [x.cpu().numpy() for x in m_d]
            got_a = [x.cpu().numpy() for x in a_d]
            for g, r in zip(got_s + got_a, ref_s + ref_a):
                assert rel_l2(g, r) <= 1e-10
            results.setdefault(fftp, []).append((got_s, got_a))
            plans.append(plan)
        if fftp == sht.SHT_FP64:
            fp64_plans = plans
        else:
            df_plans = plans
    for (s1, a1), (s2, a2) in zip(results[sht.SHT_MIXED], results[sht.SHT_FP64]):
        for g, r in zip(s1 + a1, s2 + a2):
            assert rel_l2(g, r) <= 1e-12
    # one batch holding plans of both engines: two FFT launches per stage
    mixed = [df_plans[0], fp64_plans[1], df_plans[2]]
    batch = sht.sht_batch_create(mixed)
    with pytest.raises(sht.ShtError):
        mixed[1].fft_precision = sht.SHT_MIXED  # locked while in a batch
    alms = [[torch.from_numpy(a).cuda() for a in c[1]] for c in cases]
    outs = [[torch.zeros(c[0].npix, dtype=torch.float64, device="cuda") for _ in range(2)] for c in cases]
    sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, alms, outs)
    torch.cuda.synchronize()
    for (geom, alm, _), o in zip(cases, outs):
        ref = oracle.synthesis(2, lmax, lmax, alm, rings_of(geom))
        for g, r in zip(o, ref):
            assert rel_l2(g.cpu().numpy(), r) <= 1e-10
    del batch
    # errors: FP64 plans have no double-float engine; only the two precisions exist
    p64 = sht.sht_plan_create(cases[0][0], sht.sht_alm_create(lmax, lmax), 0, 1, sht.SHT_FP64)
    assert p64.fft_precision == sht.SHT_FP64
    with pytest.raises(sht.ShtError):
        p64.fft_precision = sht.SHT_MIXED
    with pytest.raises(sht.ShtError):
        df_plans[0].fft_precision = 7
