"""torch.autograd wrappers: backward passes through the adjoint kernels.

The scalar loss of the differentiable high-resolution workload,
L = ||synthesis(a_lm) - d||^2 (a_lm with C_l = 1/(l+1)^2 drawn first from
rng(4), then d ~ N(0, 1) per pixel), is differentiated at lmax 63 and checked
against the oracle's adjoint synthesis (dL/da = (2 - delta_m0) Y^H 2(S a - d),
the reading of Sect. 4.5) and against central finite differences; gradcheck
runs at small sizes for synthesis and analysis, spin 0 and 2; the full-size
workload (lmax 8191, Gauss-Legendre 8192 x 16383) runs forward and backward in
both forms, checked by a directional finite difference and by the mixed
gradient against the FP64 one.
"""
import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_1303_4945_gb300 import build

    build.build()
    from paper_1303_4945_gb300 import autograd, sht

    assert torch.cuda.is_available()
    return sht, autograd


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def workload(lmax, geom, rng):
    a = inputs.gaussian_alm(rng, lmax, lmax, cl=inputs.cl_inverse_square)
    d = rng.standard_normal(geom.npix)
    return a, d


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-10)])
def test_gradient_against_oracle_adjoint(mods, precision, tol):
    sht, ag = mods
    lmax = 63
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 0, 1, precision)
    a, d = workload(lmax, geom, np.random.default_rng(4))
    at = torch.from_numpy(a).cuda().reshape(1, -1).requires_grad_(True)
    dt = torch.from_numpy(d).cuda().reshape(1, -1)
    loss = ((ag.synthesis(plan, at) - dt) ** 2).sum()
    loss.backward()
    got = at.grad[0].cpu().numpy()
    r = geom.rings()
    rings = oracle.Rings(r["theta"], r["nphi"], r["phi0"], r["weight"], ofs=r["ofs"])
    p = oracle.synthesis(0, lmax, lmax, [a], rings)[0]
    yh = oracle.analysis(0, lmax, lmax, [2.0 * (p - d)], rings, adjoint=True)[0]
    _, m = inputs.lm_arrays(lmax, lmax)
    ref = np.where(m == 0, yh.real + 0j, 2.0 * yh)
    assert rel_l2(got, ref) <= tol
    assert np.all(got[m == 0].imag == 0)
    assert abs(loss.item() - np.sum((p - d) ** 2)) <= tol * np.sum((p - d) ** 2)


def test_gradient_finite_differences(mods):
    sht, ag = mods
    lmax = 63
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), 0, 1, 0)
    rng = np.random.default_rng(4)
    a, d = workload(lmax, geom, rng)
    dt = torch.from_numpy(d).cuda().reshape(1, -1)
    at = torch.from_numpy(a).cuda().reshape(1, -1).requires_grad_(True)

    def L(x):
        return float(((ag.synthesis(plan, x) - dt) ** 2).sum())

    ((ag.synthesis(plan, at) - dt) ** 2).sum().backward()
    g = at.grad.detach()
    _, m = inputs.lm_arrays(lmax, lmax)
    for trial in range(3):
        v = inputs.gaussian_alm(rng, lmax, lmax)
        v = torch.from_numpy(v).cuda().reshape(1, -1)
        h = 1e-2  # L is quadratic in a: central differences are exact up to rounding
        fd = (L(at.detach() + h * v) - L(at.detach() - h * v)) / (2 * h)
        an = float(torch.sum((g.conj() * v).real))
        assert abs(fd - an) <= 1e-8 * max(1.0, abs(an)), (trial, fd, an)


@pytest.mark.parametrize("spin", [0, 2])
def test_gradcheck_synthesis_and_analysis(mods, spin):
    sht, ag = mods
    lmax = 6
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    plan = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, lmax), spin, 1, 0)
    rng = np.random.default_rng(11)
    narr = plan.narrays
    a = np.stack([inputs.gaussian_alm(rng, lmax, lmax, lmin=abs(spin)) for _ in range(narr)])
    # entries the transform ignores (Im of m = 0, l < |spin|) carry no gradient
    # information; keep the check to the coefficients that act on the maps
    at = torch.from_numpy(a).cuda().requires_grad_(True)
    _, m = inputs.lm_arrays(lmax, lmax)
    l, _ = inputs.lm_arrays(lmax, lmax)
    live = torch.from_numpy((l >= abs(spin)).astype(np.float64)).cuda()
    real0 = torch.from_numpy(m == 0).cuda()

    def f(x):
        x = torch.where(real0, torch.complex(x.real, torch.zeros_like(x.real)), x) * live
        return ag.synthesis(plan, x)

    assert torch.autograd.gradcheck(f, (at,), eps=1e-6, atol=1e-8, rtol=1e-6)
    mp = torch.from_numpy(rng.standard_normal((narr, geom.npix))).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: ag.analysis(plan, x), (mp,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_full_size_forward_backward(mods):
    # lmax 8191 on Gauss-Legendre 8192 x 16383 (rings beyond shared memory)
    sht, ag = mods
    lmax = 8191
    geom = sht.sht_geom_gauss(lmax + 1, 2 * lmax + 1)
    lay = sht.sht_alm_create(lmax, lmax)
    rng = np.random.default_rng(4)
    a, d = workload(lmax, geom, rng)
    dt = torch.from_numpy(d).cuda().reshape(1, -1)
    grads = {}
    for prec in (0, 1):
        plan = sht.sht_plan_create(geom, lay, 0, 1, prec)
        at = torch.from_numpy(a).cuda().reshape(1, -1).requires_grad_(True)
        loss = ((ag.synthesis(plan, at) - dt) ** 2).sum()
        loss.backward()
        grads[prec] = at.grad.detach()
        if prec == 0:
            v = torch.from_numpy(inputs.gaussian_alm(rng, lmax, lmax, cl=inputs.cl_inverse_square)).cuda()
            v = v.reshape(1, -1)
            h = 0.5  # L is quadratic in a: no truncation error

            def L(x):
                return float(((ag.synthesis(plan, x) - dt) ** 2).sum())

            fd = (L(at.detach() + h * v) - L(at.detach() - h * v)) / (2 * h)
            an = float(torch.sum((grads[0].conj() * v).real))
            assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
        del plan
        torch.cuda.empty_cache()
    err = float(torch.linalg.norm(grads[1] - grads[0]) / torch.linalg.norm(grads[0]))
    assert err <= 1e-10, err
