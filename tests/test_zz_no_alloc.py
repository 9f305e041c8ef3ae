"""sht_execute_noalloc: the transform entry point that allocates nothing.

It serves callers that must not allocate device memory while transforming
(stream capture, memory owned by another allocator, latency-bound loops).
The test runs it through the C ABI next to sht_execute on the same plan and
inputs, twice in a row (the static working area keeps the previous call's
contents, which must not leak into the next result), in both precisions and
for synthesis and analysis, and checks the size limit is enforced.  It lives
in a file of its own, collected last.
"""
import numpy as np
import pytest

from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-10}  # relative L2 of the FP64 and mixed parity tests


@pytest.fixture(scope="module")
def sht():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import sht as m

    return m


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("precision,spin", [(0, 0), (0, 2), (1, 0), (1, 2)])
def test_noalloc_matches_execute(sht, precision, spin):
    lmax = 95
    geom = sht.sht_geom_healpix(32)  # aliasing rings, phi0 != 0, Nphi 4..128
    lay = sht.sht_alm_create(lmax, lmax)
    plan = sht.sht_plan_create(geom, lay, spin, 1, precision)
    narr = 2 if spin else 1
    for call in range(2):  # two calls in a row, different inputs
        rng = np.random.default_rng(1000 + 10 * call + spin)
        alm = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin))).cuda() for _ in range(narr)]
        ref = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(narr)]
        got = [torch.full((geom.npix,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(narr)]
        sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm, ref)
        sht.sht_execute_noalloc(plan, sht.SHT_SYNTHESIS, alm, got)
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert _rel(g, r) <= TOL[precision]
        maps = [torch.from_numpy(rng.standard_normal(geom.npix)).cuda() for _ in range(narr)]
        aref = [torch.zeros_like(a) for a in alm]
        agot = [torch.full_like(a, complex(float("nan"), float("nan"))) for a in alm]
        sht.sht_execute(plan, sht.SHT_ANALYSIS, aref, maps)
        sht.sht_execute_noalloc(plan, sht.SHT_ANALYSIS, agot, maps)
        torch.cuda.synchronize()
        for g, r in zip(agot, aref):
            assert _rel(g, r) <= TOL[precision]


def test_noalloc_rejects_oversized_work(sht):
    geom = sht.sht_geom_gauss(2048, 4095)  # phase array 2048 x 1024 pairs x 32 B = 64 MiB + partials
    lay = sht.sht_alm_create(2047, 2047)
    plan = sht.sht_plan_create(geom, lay, 0, 1, 0)
    a = [torch.zeros(lay.size(), dtype=torch.complex128, device="cuda")]
    m = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda")]
    with pytest.raises(sht.ShtError) as e:
        sht.sht_execute_noalloc(plan, sht.SHT_ANALYSIS, a, m)
    assert e.value.code == sht.SHT_ERR_UNSUPPORTED
