"""The stage calls behind the distributed decomposition of Sect. 4.2, on one GPU.

sht_execute_legendre and sht_execute_rings run through the drivers of
paper_1303_4945_gb300.distributed with one to three tasks emulated in one
process (each task its own m-list plan and ring-subset plan, the all-to-all done
in device memory): the assembled maps and a_lm must equal sht_execute on the
whole problem and the oracle.  Spin 0 and 2, both precisions, Gauss-Legendre and
HEALPix (aliased rings, an unpaired equator ring); the stage calls' own flag
and argument checks too.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import distributed as D
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("ntasks", [1, 2, 3])
@pytest.mark.parametrize("spin,precision,grid", [(0, 0, "gauss"), (2, 0, "healpix"), (0, 1, "healpix"),
                                                 (2, 1, "gauss")])
def test_emulated_tasks_match_whole_transform(sht, ntasks, spin, precision, grid):
    lmax = 60
    geom = sht.sht_geom_gauss(62, 121) if grid == "gauss" else sht.sht_geom_healpix(16)
    r = geom.rings()
    rings = oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])
    part = D.Partition.round_robin(lmax, r["theta"], ntasks)
    stages = [D.LibraryStages(sht, geom, lmax, lmax, spin, 1, precision, part, k) for k in range(ntasks)]
    narr = 2 if spin else 1
    rng = np.random.default_rng(500 + ntasks + 10 * spin)
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(narr)]
    pmap = [rng.standard_normal(geom.npix) for _ in range(narr)]
    # the whole transform through sht_execute, and the oracle
    whole = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, precision)
    w_maps = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(narr)]
    sht.sht_execute(whole, sht.SHT_SYNTHESIS, [torch.from_numpy(a).cuda() for a in alm], w_maps)
    w_alm = [torch.zeros(len(alm[0]), dtype=torch.complex128, device="cuda") for _ in range(narr)]
    sht.sht_execute(whole, sht.SHT_ANALYSIS, w_alm, [torch.from_numpy(p).cuda() for p in pmap])
    ref_maps = oracle.synthesis(spin, lmax, lmax, alm, rings)
    ref_alm = oracle.analysis(spin, lmax, lmax, pmap, rings)
    # distributed synthesis: each task's a_lm of its m values in, its rings' pixels out
    alm_loc = [[torch.from_numpy(D.alm_pack(a, lmax, lmax, part.m[k])).cuda() for a in alm] for k in range(ntasks)]
    maps = D.synthesis_emulated(part, stages, alm_loc)
    torch.cuda.synchronize()
    got = [np.zeros(geom.npix) for _ in range(narr)]
    for k in range(ntasks):
        pix = D.ring_pixels(r["ofs"], r["nphi"], part.rings[k])
        for c in range(narr):
            got[c][pix] = maps[k][c].cpu().numpy()
    for c in range(narr):
        assert rel(got[c], w_maps[c].cpu().numpy()) <= TOL[precision]
        assert rel(got[c], ref_maps[c]) <= TOL[precision]
    # distributed analysis: each task's pixels in, its m values' a_lm out
    maps_loc = [[torch.from_numpy(p[D.ring_pixels(r["ofs"], r["nphi"], part.rings[k])]).cuda() for p in pmap]
                for k in range(ntasks)]
    back = D.analysis_emulated(part, stages, maps_loc)
    torch.cuda.synchronize()
    got_a = [np.zeros(len(alm[0]), dtype=np.complex128) for _ in range(narr)]
    for k in range(ntasks):
        for c in range(narr):
            D.alm_unpack(back[k][c].cpu().numpy(), lmax, lmax, part.m[k], got_a[c])
    for c in range(narr):
        assert rel(got_a[c], w_alm[c].cpu().numpy()) <= TOL[precision]
        assert rel(got_a[c], ref_alm[c]) <= TOL[precision]


def test_stage_call_checks(sht):
    geom = sht.sht_geom_gauss(10, 19)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(8, 8), 0, 1, 0)
    a = [torch.zeros(45, dtype=torch.complex128, device="cuda")]
    ph = torch.zeros(9 * 10, dtype=torch.complex128, device="cuda")
    m = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda")]
    for call, args in ((sht.sht_execute_legendre, (plan, sht.SHT_SYNTHESIS, a, ph, sht.SHT_ADD_OUTPUT)),
                       (sht.sht_execute_rings, (plan, sht.SHT_ANALYSIS, ph, m, sht.SHT_ADD_OUTPUT)),
                       (sht.sht_execute_rings, (plan, sht.SHT_SYNTHESIS, ph, m, sht.SHT_NO_POLAR_OPT)),
                       (sht.sht_execute_legendre, (plan, sht.SHT_DERIV_SYNTHESIS, a, ph, 0))):
        with pytest.raises(sht.ShtError) as e:
            call(*args)
        assert e.value.code == sht.SHT_ERR_INVALID_ARG
