"""GPU parity of sht_batch_execute: many distinct plans through merged launches.

Three layers of evidence:
- a heterogeneous batch of small plans (both precisions, spins 0..3, ncomp up
  to 8, Gauss-Legendre / HEALPix / Clenshaw-Curtis / partial grids, mmax <
  lmax) against the FP64 oracle, for all four transform types, with and
  without the polar cut, and with SHT_ADD_OUTPUT;
- the uneven batched workload at full size (64 scalar Gauss-Legendre problems,
  lmax log-uniform in [64, 2048], nlat = lmax+1, nlon = 2 lmax+1, plus 8 maps
  at lmax 2047, seed 3): the batched results equal per-plan sht_execute bit
  for bit (same items, same arithmetic), every plan's synthesis-analysis round
  trip recovers a_lm (Gauss-Legendre quadrature is exact there), and the
  smallest plan matches the oracle;
- CUDA-graph capture and replay of the batch and of a single plan.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: (1e-12, 5e-12), 1: (1e-10, 1e-9)}  # (relative L2, relative max) per precision


@pytest.fixture(scope="module")
def sht():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht as m

    assert torch.cuda.is_available()
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rings_of(geom):
    r = geom.rings()
    return oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])


def cuda(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# (geometry, lmax, mmax, spin, ncomp, precision)
def small_cases(sht):
    return [
        (sht.sht_geom_gauss(34, 67), 33, 33, 0, 1, sht.SHT_FP64),
        (sht.sht_geom_gauss(21, 37), 18, 18, 2, 2, sht.SHT_FP64),
        (sht.sht_geom_healpix(8), 23, 23, 0, 3, sht.SHT_FP64),  # 3 maps padded to 4 jobs
        (sht.sht_geom_ecp(sht.SHT_ECP_CC, 18, 35), 15, 12, 1, 1, sht.SHT_MIXED),
        (sht.sht_geom_gauss(40, 61), 31, 31, 0, 8, sht.SHT_FP64),
        (sht.sht_geom_gauss(26, 51), 24, 24, 0, 1, sht.SHT_MIXED),
        (sht.sht_geom_subset(sht.sht_geom_gauss(30, 59), np.arange(4, 26)), 28, 28, 2, 1, sht.SHT_MIXED),
        (sht.sht_geom_healpix(4), 11, 11, 3, 1, sht.SHT_FP64),
        (sht.sht_geom_gauss(34, 67), 33, 20, 0, 2, sht.SHT_MIXED),
    ]


def test_batch_heterogeneous_vs_oracle(sht):
    cases = small_cases(sht)
    plans, data = [], []
    rng = np.random.default_rng(50)
    for geom, lmax, mmax, spin, ncomp, prec in cases:
        plans.append(sht.sht_plan_create(geom, sht.sht_alm_create(lmax, mmax), spin, ncomp, prec))
        narr = 2 * ncomp if spin else ncomp
        rings = rings_of(geom)
        alm = [inputs.gaussian_alm(rng, lmax, mmax, lmin=abs(spin)) for _ in range(narr)]
        maps = [rng.standard_normal(geom.npix) for _ in range(narr)]
        cover = np.zeros(geom.npix, bool)
        for o, n in zip(rings.ofs, rings.nphi):
            cover[o:o + n] = True
        data.append(dict(
            alm=alm, maps=maps, npix=geom.npix, nalm=oracle.nalm(lmax, mmax), prec=prec, cover=cover,
            syn=oracle.synthesis(spin, lmax, mmax, alm, rings),
            syn_w=oracle.synthesis(spin, lmax, mmax, alm, rings, weighted=True),
            ana=oracle.analysis(spin, lmax, mmax, maps, rings),
            ana_adj=oracle.analysis(spin, lmax, mmax, maps, rings, adjoint=True)))
    batch = sht.sht_batch_create(plans)
    assert len(batch) == len(plans)
    for flags in (0, sht.SHT_NO_POLAR_OPT):
        for type_, key in ((sht.SHT_SYNTHESIS, "syn"), (sht.SHT_ADJOINT_ANALYSIS, "syn_w")):
            a_in = [[cuda(x) for x in d["alm"]] for d in data]
            m_out = [[torch.full((d["npix"],), np.nan, dtype=torch.float64, device="cuda") for _ in d["alm"]]
                     for d in data]
            sht.sht_batch_execute(batch, type_, a_in, m_out, flags)
            torch.cuda.synchronize()
            for k, d in enumerate(data):
                l2, mx = TOL[d["prec"]]
                c = d["cover"]
                for g, r in zip(m_out[k], d[key]):
                    g = g.cpu().numpy()
                    assert np.isnan(g[~c]).all()  # pixels outside the rings are not touched
                    g, r = g[c], r[c]
                    assert rel_l2(g, r) <= l2 and rel_max(g, r) <= mx, (k, key, flags, rel_l2(g, r))
        for type_, key in ((sht.SHT_ANALYSIS, "ana"), (sht.SHT_ADJOINT_SYNTHESIS, "ana_adj")):
            m_in = [[cuda(x) for x in d["maps"]] for d in data]
            a_out = [[torch.full((d["nalm"],), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
                      for _ in d["maps"]] for d in data]
            sht.sht_batch_execute(batch, type_, a_out, m_in, flags)
            torch.cuda.synchronize()
            for k, d in enumerate(data):
                l2, mx = TOL[d["prec"]]
                for g, r in zip(a_out[k], d[key]):
                    g = g.cpu().numpy()
                    assert rel_l2(g, r) <= l2 and rel_max(g, r) <= mx, (k, key, flags, rel_l2(g, r))
    # accumulation into existing outputs
    a_in = [[cuda(x) for x in d["alm"]] for d in data]
    base = [[np.random.default_rng(k).standard_normal(d["npix"]) for _ in d["alm"]] for k, d in enumerate(data)]
    m_out = [[cuda(b) for b in bs] for bs in base]
    sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_in, m_out, sht.SHT_ADD_OUTPUT)
    m_in = [[cuda(x) for x in d["maps"]] for d in data]
    abase = [[x.copy() for x in d["alm"]] for d in data]
    a_out = [[cuda(x) for x in bs] for bs in abase]
    sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, a_out, m_in, sht.SHT_ADD_OUTPUT)
    torch.cuda.synchronize()
    for k, d in enumerate(data):
        l2, _ = TOL[d["prec"]]
        for g, b, r in zip(m_out[k], base[k], d["syn"]):
            assert rel_l2(g.cpu().numpy() - b, r) <= l2
        for g, b, r in zip(a_out[k], abase[k], d["ana"]):
            assert rel_l2(g.cpu().numpy() - b, r) <= l2


def uneven_batch(sht, precision):
    """The 64 log-uniform scalar problems plus the 8-map instance at lmax 2047."""
    rng, lmaxes = inputs.batched_lmax(seed=3)
    specs = [(int(l), 1) for l in lmaxes] + [(2047, 8)]
    plans, alms = [], []
    for lmax, ncomp in specs:
        geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
        plans.append(sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 0, ncomp, precision))
        alms.append([inputs.gaussian_alm(rng, lmax, lmax) for _ in range(ncomp)])
    return specs, plans, alms


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_uneven_full_size(sht, precision):
    specs, plans, alms = uneven_batch(sht, precision)
    batch = sht.sht_batch_create(plans)
    a_dev = [[cuda(a) for a in al] for al in alms]
    maps_b = [[torch.empty(p.geom.npix, dtype=torch.float64, device="cuda") for _ in al] for p, al in zip(plans, alms)]
    sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_dev, maps_b)
    back_b = [[torch.empty_like(a) for a in al] for al in a_dev]
    sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, back_b, maps_b)
    torch.cuda.synchronize()
    # per-plan calls: identical items and arithmetic, so identical bits
    for k, p in enumerate(plans):
        maps_1 = [torch.empty_like(m) for m in maps_b[k]]
        sht.sht_execute(p, sht.SHT_SYNTHESIS, a_dev[k], maps_1)
        back_1 = [torch.empty_like(a) for a in a_dev[k]]
        sht.sht_execute(p, sht.SHT_ANALYSIS, back_1, maps_b[k])
        torch.cuda.synchronize()
        for x, y in zip(maps_b[k], maps_1):
            assert torch.equal(x, y), k
        for x, y in zip(back_b[k], back_1):
            assert torch.equal(x, y), k
        # round trip: Gauss-Legendre with nlat = lmax+1 integrates the products exactly
        tol = 1e-11 if precision == 0 else 2e-10
        for x, a in zip(back_b[k], a_dev[k]):
            err = float(torch.linalg.norm(x - a) / torch.linalg.norm(a))
            assert err <= tol, (k, specs[k], err)
    # the smallest problem against the oracle
    k = int(np.argmin([l for l, _ in specs]))
    lmax = specs[k][0]
    rings = rings_of(plans[k].geom)
    ref = oracle.synthesis(0, lmax, lmax, alms[k], rings)
    l2, mx = TOL[precision]
    got = maps_b[k][0].cpu().numpy()
    assert rel_l2(got, ref[0]) <= l2 and rel_max(got, ref[0]) <= mx


def test_batch_graph_capture(sht):
    rng = np.random.default_rng(60)
    specs = [(70, 0, 1, 0), (150, 0, 2, 0), (200, 2, 1, 0), (96, 0, 1, 1), (128, 2, 1, 1), (300, 0, 3, 0)]
    plans, npix, nalm = [], [], []
    for lmax, spin, ncomp, prec in specs:
        geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
        plans.append(sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, ncomp, prec))
        npix.append(geom.npix)
        nalm.append(oracle.nalm(lmax, lmax))
    batch = sht.sht_batch_create(plans)
    narr = [p.narrays for p in plans]
    a_in = [[torch.zeros(nalm[k], dtype=torch.complex128, device="cuda") for _ in range(narr[k])] for k in range(len(plans))]
    m_mid = [[torch.zeros(npix[k], dtype=torch.float64, device="cuda") for _ in range(narr[k])] for k in range(len(plans))]
    a_out = [[torch.zeros_like(a) for a in al] for al in a_in]
    single_out = torch.zeros(npix[0], dtype=torch.float64, device="cuda")

    def fill():
        for k, (lmax, spin, _, _) in enumerate(specs):
            for a in a_in[k]:
                a.copy_(cuda(inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin))))

    fill()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        st = torch.cuda.current_stream()
        sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_in, m_mid, 0, st)
        sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, a_out, m_mid, 0, st)
        sht.sht_execute(plans[0], sht.SHT_SYNTHESIS, a_in[0], [single_out], 0, st)
    for rep in range(2):
        fill()  # new inputs in the captured buffers
        g.replay()
        torch.cuda.synchronize()
        m_ref = [[torch.zeros_like(m) for m in ms] for ms in m_mid]
        a_ref = [[torch.zeros_like(a) for a in al] for al in a_out]
        sht.sht_batch_execute(batch, sht.SHT_SYNTHESIS, a_in, m_ref)
        sht.sht_batch_execute(batch, sht.SHT_ANALYSIS, a_ref, m_ref)
        torch.cuda.synchronize()
        for k in range(len(plans)):
            for x, y in zip(m_mid[k], m_ref[k]):
                assert torch.equal(x, y), (rep, k)
            for x, y in zip(a_out[k], a_ref[k]):
                assert torch.equal(x, y), (rep, k)
        assert torch.equal(single_out, m_ref[0][0])


def test_batch_errors(sht):
    geom = sht.sht_geom_gauss(6, 11)
    lay = sht.sht_alm_create(5, 5)
    p = sht.sht_plan_create(geom, lay, 0, 1, 0)
    with pytest.raises(sht.ShtError):
        sht.sht_batch_create([p, p])  # a plan twice would race on its workspace
    many = [sht.sht_plan_create(geom, lay, 0, 16, 0) for _ in range(65)]  # 1040 arrays per side
    with pytest.raises(sht.ShtError) as ei:
        sht.sht_batch_create(many)
    assert ei.value.code == sht.SHT_ERR_UNSUPPORTED
    b = sht.sht_batch_create([p])
    a = [torch.zeros(oracle.nalm(5, 5), dtype=torch.complex128, device="cuda")]
    m = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda")]
    with pytest.raises(sht.ShtError):
        sht.sht_batch_execute(b, 99, [a], [m])
    with pytest.raises(ValueError):
        sht.sht_batch_execute(b, sht.SHT_SYNTHESIS, [a, a], [m, m])
