"""Parity at the full size of the timed workload, in the launch configuration
the bench times: spin 2, Gauss-Legendre 4096 x 8191 (8191-point rings, Rader),
lmax = mmax = 4095, the bench's seeded E/B a_lm (C_l = 1/(l+1)^2), plans
autotuned as the bench does, the mixed plan with its default FP64 columns and
double-float ring FFTs.  The oracle computes sampled outputs one by one:
syntheses on rings spread over latitude (both poles, the equator), analyses on
m values that include the FP64-column boundary and mmax.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LMAX, NLAT, NLON, SPIN = 4095, 4096, 8191, 2
# 17 rings evenly spaced (both poles and the equator included): the sample's
# relative L2 estimates that of the whole map; the polar rings are also checked alone
RINGS = sorted(set(np.linspace(0, 4095, 17).round().astype(int).tolist()) | {1, 37, 4058, 4094})
EVEN = np.linspace(0, 4095, 17).round().astype(int).tolist()
MS = [0, 1, 2, 3, 4, 700, 2048, 4000, 4095]
TOL = {0: 1e-12, 1: 1e-10}


@pytest.fixture(scope="module")
def setup():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht

    assert torch.cuda.is_available()
    th, w = oracle.gauss_nodes(NLAT)
    rings = oracle.Rings(th, np.full(NLAT, NLON), np.zeros(NLAT), w * 2 * np.pi / NLON)
    alm = inputs.spin2_eb(2, LMAX)
    rng = np.random.default_rng(9)
    maps_in = [inputs.gaussian_map(rng, rings.npix) for _ in range(2)]
    ref_syn = oracle.synthesis(SPIN, LMAX, LMAX, alm, rings, rings_sel=RINGS)
    ref_ana = oracle.analysis(SPIN, LMAX, LMAX, maps_in, rings, m_sel=MS)
    return sht, rings, alm, maps_in, ref_syn, ref_ana


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", [0, 1])
def test_headline_workload_against_oracle(setup, precision):
    sht, rings, alm, maps_in, ref_syn, ref_ana = setup
    geom = sht.sht_geom_gauss(NLAT, NLON)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(LMAX, LMAX), SPIN, 1, precision)
    # the plan's work (the bench's roofline counts it) is the polar cut's host count
    assert plan.triples(0) == sht.sht_geom_polar_cut(geom, LMAX, SPIN, np.arange(LMAX + 1))[2]
    stream = torch.cuda.current_stream()
    plan.autotune(stream)
    a_d = [torch.from_numpy(a).cuda() for a in alm]
    m_d = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    sht.sht_execute(plan, sht.SHT_SYNTHESIS, a_d, m_d, 0, stream)
    out = [torch.empty_like(a) for a in a_d]
    sht.sht_execute(plan, sht.SHT_ANALYSIS, out, [torch.from_numpy(m).cuda() for m in maps_in], 0, stream)
    torch.cuda.synchronize()
    maps = [x.cpu().numpy() for x in m_d]
    per_ring = {y: max(rel_l2(g[rings.ofs[y]:rings.ofs[y] + NLON], r[rings.ofs[y]:rings.ofs[y] + NLON])
                       for g, r in zip(maps, ref_syn)) for y in RINGS}
    print("precision", precision, "per-ring rel L2:", {y: f"{e:.2e}" for y, e in per_ring.items()})
    # each ring on its own too: the mixed form to its tolerance, the FP64 form to
    # 1e-11 (its polar rings differ from the oracle's by a few 1e-12, the paper's
    # maximum error growing like lmax^(3/2); the map as a whole is within 1e-12)
    assert max(per_ring.values()) <= (1e-11 if precision == 0 else TOL[1])
    idx = np.concatenate([np.arange(rings.ofs[y], rings.ofs[y] + NLON) for y in EVEN])
    for got, ref in zip(maps, ref_syn):  # Q, U on the evenly spaced rings
        err = rel_l2(got[idx], ref[idx])
        print("precision", precision, "evenly spaced rings rel L2", f"{err:.2e}")
        assert err <= TOL[precision]
    _, m = inputs.lm_arrays(LMAX, LMAX)
    sel = np.isin(m, MS)
    for got, ref in zip(out, ref_ana):  # E, B at the sampled m
        err = rel_l2(got.cpu().numpy()[sel], ref[sel])
        print("precision", precision, "sampled m rel L2", f"{err:.2e}")
        assert err <= TOL[precision]


def test_headline_analysis_tensor_cores(setup):
    # the mixed analysis with its contraction on the tensor cores, whichever the
    # autotuner would pick: the sampled m against the oracle
    sht, rings, alm, maps_in, ref_syn, ref_ana = setup
    geom = sht.sht_geom_gauss(NLAT, NLON)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(LMAX, LMAX), SPIN, 1, 1)
    plan.tensor_core_analysis = True
    out = [torch.empty(len(a), dtype=torch.complex128, device="cuda") for a in alm]
    sht.sht_execute(plan, sht.SHT_ANALYSIS, out, [torch.from_numpy(m).cuda() for m in maps_in], 0)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    _, m = inputs.lm_arrays(LMAX, LMAX)
    sel = np.isin(m, MS)
    for got, ref in zip(out, ref_ana):
        err = rel_l2(got.cpu().numpy()[sel], ref[sel])
        print("tensor-core analysis, sampled m rel L2", f"{err:.2e}")
        assert err <= TOL[1]
