"""Analysis tilings (ring pairs per thread) and the autotuner, through the C ABI.

Every tiling a plan offers runs the analysis against the FP64 oracle (and the
adjoint synthesis, which shares the kernel), for both precisions, spin 0 and
spin 2, one and two jobs; the grid has more ring pairs than one tile of the
widest tiling (kAnaThreads x 8 = 1024) so that several tiles and a ragged last
tile occur.  The autotuner must pick one of the candidates and leave results
unchanged; a plan inside a batch keeps its tiling.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}


@pytest.fixture(scope="module")
def sht():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht as m

    assert torch.cuda.is_available()
    return m


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def grid(sht):
    # 2301 rings (1150 pairs + equator), lmax 60: cheap for the oracle, many pairs
    lmax = 60
    geom = sht.sht_geom_gauss(2301, 2 * lmax + 1)
    r = geom.rings()
    rings = oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])
    return lmax, geom, rings


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("spin,ncomp", [(0, 1), (0, 2), (2, 1), (2, 2)])
def test_every_tiling_matches_oracle(sht, grid, precision, spin, ncomp):
    lmax, geom, rings = grid
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, ncomp, precision)
    cur, cands = plan.tiling()
    assert cur == cands[0] and len(cands) >= 2
    narr = plan.narrays
    rng = np.random.default_rng(200 + 10 * spin + ncomp)
    maps = [rng.standard_normal(geom.npix) for _ in range(narr)]
    ref = oracle.analysis(spin, lmax, lmax, maps, rings)
    ref_adj = oracle.analysis(spin, lmax, lmax, maps, rings, adjoint=True)
    m_dev = [torch.from_numpy(m).cuda() for m in maps]
    n = oracle.nalm(lmax, lmax)
    for ppt in cands:
        plan.set_tiling(ppt)
        assert plan.tiling()[0] == ppt
        for type_, r in ((sht.SHT_ANALYSIS, ref), (sht.SHT_ADJOINT_SYNTHESIS, ref_adj)):
            out = [torch.full((n,), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda") for _ in range(narr)]
            sht.sht_execute(plan, type_, out, m_dev)
            torch.cuda.synchronize()
            for g, rr in zip(out, r):
                assert rel_l2(g.cpu().numpy(), rr) <= TOL[precision], (ppt, type_)
    with pytest.raises(sht.ShtError) as ei:
        plan.set_tiling(3)
    assert ei.value.code == sht.SHT_ERR_UNSUPPORTED


def test_autotune_and_batch_lock(sht, grid):
    lmax, geom, rings = grid
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 2, 1, 1)
    _, cands = plan.tiling()
    times = plan.autotune()
    # the tilings with the double-float analysis, and the tensor-core analysis
    assert set(times) == set(cands) | {"tensor_cores"} and all(t > 0 for t in times.values())
    chosen = plan.tiling()[0]
    best = "tensor_cores" if plan.tensor_core_analysis else chosen
    assert chosen in cands and times[best] == min(times.values())
    rng = np.random.default_rng(7)
    maps = [rng.standard_normal(geom.npix) for _ in range(2)]
    ref = oracle.analysis(2, lmax, lmax, maps, rings)
    out = [torch.zeros(oracle.nalm(lmax, lmax), dtype=torch.complex128, device="cuda") for _ in range(2)]
    sht.sht_execute(plan, sht.SHT_ANALYSIS, out, [torch.from_numpy(m).cuda() for m in maps])
    torch.cuda.synchronize()
    for g, r in zip(out, ref):
        assert rel_l2(g.cpu().numpy(), r) <= TOL[1]
    batch = sht.sht_batch_create([plan])
    other = [c for c in cands if c != chosen][0]
    with pytest.raises(sht.ShtError):
        plan.set_tiling(other)
    with pytest.raises(sht.ShtError):
        plan.autotune()
    del batch
    plan.tensor_core_analysis = False  # free again once the batch is gone
    plan.set_tiling(other)
    assert plan.tiling()[0] == other
