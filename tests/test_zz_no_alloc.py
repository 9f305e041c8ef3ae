"""sht_execute_noalloc: the transform entry point that allocates nothing.

It serves callers that must not allocate device memory while transforming:
code recorded under CUDA stream capture (cudaMalloc cannot be captured),
processes whose GPU memory belongs to another allocator's pool, and
latency-bound loops that cannot take an allocation's device synchronisation.
The tests run it through the C ABI next to sht_execute on the same plan and
inputs, twice in a row (the static working area keeps the previous call's
contents, which must not leak into the next result), for every transform type
it accepts, in both precisions, with the mixed form's FP64 columns forced on
(their items run on a side stream and read a second converted a_lm table),
with SHT_ADD_OUTPUT and real-harmonic storage, against the oracle, inside a
captured CUDA graph, and with the device's free memory unchanged across calls.
The size limit is checked too.  The file is collected last.
"""
import numpy as np
import pytest

import oracle
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


def _rings(geom):
    r = geom.rings()
    return oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])


def _nan_maps(geom, n):
    return [torch.full((geom.npix,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(n)]


def _nan_alm(lay, n):
    return [torch.full((lay.size(),), complex(float("nan"), float("nan")), dtype=torch.complex128, device="cuda")
            for _ in range(n)]


@pytest.mark.parametrize("precision,spin,fp64_cols", [(0, 0, 0), (0, 2, 0), (1, 0, 0), (1, 2, 0), (1, 0, 9), (1, 2, 9)])
def test_noalloc_matches_execute(sht, precision, spin, fp64_cols):
    lmax = 95
    geom = sht.sht_geom_healpix(32)  # aliasing rings, phi0 != 0, Nphi 4..128, pairs within 0.05 rad of the poles
    lay = sht.sht_alm_create(lmax, lmax)
    plan = sht.sht_plan_create(geom, lay, spin, 1, precision)
    if fp64_cols:
        plan.fp64_columns = fp64_cols
    narr = 2 if spin else 1
    for call in range(2):  # two calls in a row, different inputs
        rng = np.random.default_rng(1000 + 10 * call + spin + fp64_cols)
        alm = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin))).cuda() for _ in range(narr)]
        maps = [torch.from_numpy(rng.standard_normal(geom.npix)).cuda() for _ in range(narr)]
        for type_ in (sht.SHT_SYNTHESIS, sht.SHT_ADJOINT_ANALYSIS):
            ref = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda") for _ in range(narr)]
            got = _nan_maps(geom, narr)
            sht.sht_execute(plan, type_, alm, ref)
            sht.sht_execute_noalloc(plan, type_, alm, got)
            torch.cuda.synchronize()
            for g, r in zip(got, ref):
                assert _rel(g, r) <= TOL[precision], (type_, _rel(g, r))
        for type_ in (sht.SHT_ANALYSIS, sht.SHT_ADJOINT_SYNTHESIS):
            aref = [torch.zeros_like(a) for a in alm]
            agot = _nan_alm(lay, narr)
            sht.sht_execute(plan, type_, aref, maps)
            sht.sht_execute_noalloc(plan, type_, agot, maps)
            torch.cuda.synchronize()
            for g, r in zip(agot, aref):
                assert _rel(g, r) <= TOL[precision], (type_, _rel(g, r))


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_against_oracle_with_add_output(sht, precision):
    """Adjoint synthesis accumulated onto existing a_lm (SHT_ADD_OUTPUT) and a
    synthesis of real-harmonic a_lm, both against the oracle; the mixed plan runs
    with FP64 columns."""
    lmax, spin = 40, 2
    geom = sht.sht_geom_healpix(16)
    rings = _rings(geom)
    lay = sht.sht_alm_create(lmax, lmax)
    plan = sht.sht_plan_create(geom, lay, spin, 1, precision)
    if precision == 1:
        plan.fp64_columns = 6
    rng = np.random.default_rng(1200 + precision)
    maps = [rng.standard_normal(geom.npix) for _ in range(2)]
    base = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
    ref = oracle.analysis(spin, lmax, lmax, maps, rings, adjoint=True)
    out = [torch.from_numpy(b).cuda() for b in base]
    sht.sht_execute_noalloc(plan, sht.SHT_ADJOINT_SYNTHESIS, out, [torch.from_numpy(m).cuda() for m in maps],
                            sht.SHT_ADD_OUTPUT)
    torch.cuda.synchronize()
    for g, b, r in zip(out, base, ref):
        want = b + r
        assert np.linalg.norm(g.cpu().numpy() - want) / np.linalg.norm(want) <= TOL[precision]
    # real-harmonic storage in, maps out
    alm = [inputs.gaussian_alm(rng, lmax, lmax, lmin=2) for _ in range(2)]
    real = [oracle.complex_to_real(a, lmax, lmax) for a in alm]
    want = oracle.synthesis(spin, lmax, lmax, alm, rings)
    got = _nan_maps(geom, 2)
    sht.sht_execute_noalloc(plan, sht.SHT_SYNTHESIS, [torch.from_numpy(a).cuda() for a in real], got,
                            sht.SHT_REAL_HARMONICS)
    torch.cuda.synchronize()
    for g, w in zip(got, want):
        assert np.linalg.norm(g.cpu().numpy() - w) / np.linalg.norm(w) <= TOL[precision]


def test_noalloc_in_cuda_graph_and_free_memory(sht):
    """After a warm call (which looks up the area's address), the call is captured in
    a CUDA graph -- capture in global mode fails on any allocation -- and its replay
    equals sht_execute; uncaptured calls leave the device's free memory unchanged."""
    lmax, spin = 63, 2
    geom = sht.sht_geom_healpix(16)
    lay = sht.sht_alm_create(lmax, lmax)
    plan = sht.sht_plan_create(geom, lay, spin, 1, sht.SHT_MIXED)
    plan.fp64_columns = 8  # the fork to the side stream is captured too
    rng = np.random.default_rng(1300)
    alm = [torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, lmin=2)).cuda() for _ in range(2)]
    maps = [torch.empty(geom.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    back = [torch.empty_like(a) for a in alm]
    ref_maps = [torch.empty_like(m) for m in maps]
    ref_back = [torch.empty_like(a) for a in alm]
    sht.sht_execute(plan, sht.SHT_SYNTHESIS, alm, ref_maps)
    sht.sht_execute(plan, sht.SHT_ANALYSIS, ref_back, ref_maps)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # warm-up outside the capture
        sht.sht_execute_noalloc(plan, sht.SHT_SYNTHESIS, alm, maps, 0, s)
        sht.sht_execute_noalloc(plan, sht.SHT_ANALYSIS, back, maps, 0, s)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    used0 = torch.cuda.memory_allocated()
    for _ in range(3):
        sht.sht_execute_noalloc(plan, sht.SHT_SYNTHESIS, alm, maps)
        sht.sht_execute_noalloc(plan, sht.SHT_ANALYSIS, back, maps)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == used0
    for t in maps + back:
        t.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        cs = torch.cuda.current_stream()
        sht.sht_execute_noalloc(plan, sht.SHT_SYNTHESIS, alm, maps, 0, cs)
        sht.sht_execute_noalloc(plan, sht.SHT_ANALYSIS, back, maps, 0, cs)
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        for g, r in zip(maps, ref_maps):
            assert _rel(g, r) <= 1e-10
        for g, r in zip(back, ref_back):
            assert _rel(g, r) <= 1e-10


def test_noalloc_rejects_oversized_work_and_deriv(sht):
    geom = sht.sht_geom_gauss(2048, 4095)  # phase array 2048 x 1024 pairs x 32 B = 64 MiB + partials
    lay = sht.sht_alm_create(2047, 2047)
    plan = sht.sht_plan_create(geom, lay, 0, 1, 0)
    a = [torch.zeros(lay.size(), dtype=torch.complex128, device="cuda")]
    m = [torch.zeros(geom.npix, dtype=torch.float64, device="cuda")]
    with pytest.raises(sht.ShtError) as e:
        sht.sht_execute_noalloc(plan, sht.SHT_ANALYSIS, a, m)
    assert e.value.code == sht.SHT_ERR_UNSUPPORTED
    small = sht.sht_geom_gauss(10, 19)
    dplan = sht.sht_plan_create(small, sht.sht_alm_create(8, 8), 1, 1, 0)
    a = [torch.zeros(45, dtype=torch.complex128, device="cuda") for _ in range(2)]
    m = [torch.zeros(small.npix, dtype=torch.float64, device="cuda") for _ in range(2)]
    with pytest.raises(sht.ShtError) as e:
        sht.sht_execute_noalloc(dplan, sht.SHT_DERIV_SYNTHESIS, a, m)
    assert e.value.code == sht.SHT_ERR_INVALID_ARG
