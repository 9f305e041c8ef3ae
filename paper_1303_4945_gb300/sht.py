"""ctypes binding of the C ABI in include/sht_gb300.h (libsht_gb300.so).

Argument marshalling only: every step of a transform runs in the library's
CUDA kernels.  Function names follow the C ABI; handles are wrapped in small
classes that call the matching *_destroy when collected.  Device buffers may
be given as torch CUDA tensors (complex128 a_lm, float64 maps) or as raw
integer device addresses.

Importing this module loads the library and raises if it has not been built
(``python -m paper_1303_4945_gb300.build``); there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

SHT_OK = 0
SHT_ERR_INVALID_ARG = -1
SHT_ERR_UNSUPPORTED = -2
SHT_ERR_OOM = -3
SHT_ERR_CUDA = -4
SHT_ERR_TIMEOUT = -5

SHT_ECP_FEJER1, SHT_ECP_FEJER2, SHT_ECP_CC = 0, 1, 2
SHT_FP64, SHT_MIXED = 0, 1
SHT_SYNTHESIS, SHT_ANALYSIS, SHT_ADJOINT_SYNTHESIS, SHT_ADJOINT_ANALYSIS = 0, 1, 2, 3
SHT_DERIV_SYNTHESIS = 4  # spin-1 plans: ncomp spin-0 a_lm -> (df/dtheta, df/(sin theta dphi)) per component
SHT_ADD_OUTPUT, SHT_NO_POLAR_OPT, SHT_REAL_HARMONICS, SHT_GRADIENT = 1, 2, 4, 8
SHT_NSTAGES = 6
STAGE_NAMES = ("legendre_synthesis", "fft_synthesis", "fft_analysis", "legendre_analysis", "analysis_reduce",
               "fp64_polar_items")

LIB_PATH = _build.LIB
HEADER = os.path.join(_build.ROOT, "include", "sht_gb300.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1303_4945_gb300.build.build()")
_lib = ctypes.CDLL(LIB_PATH)

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_i64p = ctypes.POINTER(ctypes.c_int64)
_sig = {
    "sht_geom_general": [ctypes.c_int, _dp, _ip, _dp, _i64p, _ip, _dp, ctypes.POINTER(_vp)],
    "sht_geom_gauss": [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "sht_geom_reduced_gauss": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "sht_geom_ecp": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "sht_geom_healpix": [ctypes.c_int, ctypes.POINTER(_vp)],
    "sht_geom_subset": [_vp, ctypes.c_int, _ip, ctypes.POINTER(_vp)],
    "sht_geom_info": [_vp, _ip, _i64p, _ip],
    "sht_geom_rings": [_vp, _dp, _ip, _dp, _i64p, _ip, _dp],
    "sht_geom_destroy": [_vp],
    "sht_alm_create": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _i64p, ctypes.c_int, ctypes.POINTER(_vp)],
    "sht_alm_size": [_vp, _i64p],
    "sht_alm_destroy": [_vp],
    "sht_plan_create": [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)],
    "sht_execute": [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, _vp],
    "sht_plan_workspace": [_vp, _i64p],
    "sht_plan_triples": [_vp, ctypes.c_int, _i64p],
    "sht_plan_triples_joined": [_vp, _i64p],
    "sht_plan_destroy": [_vp],
    "sht_execute_noalloc": [_vp, ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, _vp],
    "sht_execute_legendre": [_vp, ctypes.c_int, ctypes.POINTER(_vp), _vp, ctypes.c_int, _vp],
    "sht_execute_rings": [_vp, ctypes.c_int, _vp, ctypes.POINTER(_vp), ctypes.c_int, _vp],
    "sht_plan_profile": [_vp, ctypes.c_int],
    "sht_plan_get_tiling": [_vp, _ip, _ip, _ip],
    "sht_plan_set_tiling": [_vp, ctypes.c_int],
    "sht_plan_autotune": [_vp, _vp, ctypes.POINTER(ctypes.c_float)],
    "sht_plan_set_fp64_columns": [_vp, ctypes.c_int],
    "sht_plan_get_fp64_columns": [_vp, _ip],
    "sht_plan_set_fft_precision": [_vp, ctypes.c_int],
    "sht_measure_pipe_peaks": [ctypes.c_int, _dp],
    "sht_fft_plan_info": [ctypes.c_int, _ip, _ip, _ip, _ip],
    "sht_geom_polar_cut": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, _i64p],
    "sht_plan_get_fft_precision": [_vp, _ip],
    "sht_plan_set_tensor_cores": [_vp, ctypes.c_int],
    "sht_plan_get_tensor_cores": [_vp, _ip],
    "sht_plan_set_tensor_core_analysis": [_vp, ctypes.c_int],
    "sht_plan_get_tensor_core_analysis": [_vp, _ip],
    "sht_plan_device_status": [_vp, _ip],
    "sht_batch_create": [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "sht_batch_execute": [_vp, ctypes.c_int, ctypes.POINTER(ctypes.POINTER(_vp)), ctypes.POINTER(ctypes.POINTER(_vp)),
                          ctypes.c_int, _vp],
    "sht_batch_size": [_vp],
    "sht_batch_destroy": [_vp],
    "sht_plan_profile_read": [_vp, _dp, _i64p],
    "sht_strerror": [ctypes.c_int],
    "sht_last_error": [],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
for _name in ("sht_geom_destroy", "sht_alm_destroy", "sht_plan_destroy", "sht_batch_destroy"):
    getattr(_lib, _name).restype = None
_lib.sht_strerror.restype = ctypes.c_char_p
_lib.sht_last_error.restype = ctypes.c_char_p


def exported_symbols_declared():
    """Names of the functions include/sht_gb300.h declares."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(sht_\w+)\s*\(", txt)))


class ShtError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.sht_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.sht_strerror(code).decode()} ({code}): {msg}")


def _check(rc, where):
    if rc != SHT_OK:
        raise ShtError(rc, where)


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ct)


class _Handle:
    _destroy = None

    def __init__(self, h):
        self._h = h

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and self._destroy is not None:
            getattr(_lib, self._destroy)(h)


class Geometry(_Handle):
    _destroy = "sht_geom_destroy"

    def info(self):
        nr, npix, npairs = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        _check(_lib.sht_geom_info(self._h, ctypes.byref(nr), ctypes.byref(npix), ctypes.byref(npairs)),
               "sht_geom_info")
        return nr.value, npix.value, npairs.value

    @property
    def nrings(self):
        return self.info()[0]

    @property
    def npix(self):
        return self.info()[1]

    def rings(self):
        n = self.nrings
        th, p0, w = np.zeros(n), np.zeros(n), np.zeros(n)
        nphi, st = np.zeros(n, np.int32), np.zeros(n, np.int32)
        ofs = np.zeros(n, np.int64)
        _check(_lib.sht_geom_rings(self._h, _ptr(th, _dp), _ptr(nphi, _ip), _ptr(p0, _dp), _ptr(ofs, _i64p),
                                   _ptr(st, _ip), _ptr(w, _dp)), "sht_geom_rings")
        return dict(theta=th, nphi=nphi, phi0=p0, ofs=ofs, stride=st, weight=w)


class AlmLayout(_Handle):
    _destroy = "sht_alm_destroy"

    def __init__(self, h, lmax, mmax):
        super().__init__(h)
        self.lmax, self.mmax = lmax, mmax

    def size(self):
        n = ctypes.c_int64()
        _check(_lib.sht_alm_size(self._h, ctypes.byref(n)), "sht_alm_size")
        return n.value


class Plan(_Handle):
    _destroy = "sht_plan_destroy"

    def __init__(self, h, geom, alm, spin, ncomp, precision):
        super().__init__(h)
        self.geom, self.alm, self.spin, self.ncomp, self.precision = geom, alm, spin, ncomp, precision

    @property
    def narrays(self):
        return 2 * self.ncomp if self.spin else self.ncomp

    def workspace(self):
        n = ctypes.c_int64()
        _check(_lib.sht_plan_workspace(self._h, ctypes.byref(n)), "sht_plan_workspace")
        return n.value

    def profile(self, enable=True):
        _check(_lib.sht_plan_profile(self._h, 1 if enable else 0), "sht_plan_profile")

    def profile_read(self):
        """{stage name: (total ms, launches)} recorded since profile(True)."""
        ms = np.zeros(SHT_NSTAGES)
        cnt = np.zeros(SHT_NSTAGES, np.int64)
        _check(_lib.sht_plan_profile_read(self._h, _ptr(ms, _dp), _ptr(cnt, _i64p)), "sht_plan_profile_read")
        return {STAGE_NAMES[i]: (float(ms[i]), int(cnt[i])) for i in range(SHT_NSTAGES)}

    def tiling(self):
        """(current ring pairs per analysis thread, candidates)."""
        cur, n = ctypes.c_int(), ctypes.c_int()
        c = (ctypes.c_int * 4)()
        _check(_lib.sht_plan_get_tiling(self._h, ctypes.byref(cur), ctypes.byref(n), c), "sht_plan_get_tiling")
        return cur.value, [c[i] for i in range(n.value)]

    def set_tiling(self, pairs_per_thread):
        _check(_lib.sht_plan_set_tiling(self._h, pairs_per_thread), "sht_plan_set_tiling")

    def autotune(self, stream=None):
        """Times every candidate tiling (and, for mixed plans of up to two jobs, the
        tensor-core analysis), keeps the fastest; returns {candidate: ms per run},
        the tensor-core analysis under "tensor_cores"."""
        _, cands = self.tiling()
        ms = (ctypes.c_float * 5)()
        st = None if stream is None else _vp(_devptr_stream(stream))
        _check(_lib.sht_plan_autotune(self._h, st, ms), "sht_plan_autotune")
        out = {c: float(ms[i]) for i, c in enumerate(cands)}
        if ms[len(cands)] > 0:
            out["tensor_cores"] = float(ms[len(cands)])
        return out

    @property
    def fp64_columns(self):
        """Mixed form: columns m below this run in the FP64 kernels."""
        n = ctypes.c_int()
        _check(_lib.sht_plan_get_fp64_columns(self._h, ctypes.byref(n)), "sht_plan_get_fp64_columns")
        return n.value

    @fp64_columns.setter
    def fp64_columns(self, m_below):
        _check(_lib.sht_plan_set_fp64_columns(self._h, m_below), "sht_plan_set_fp64_columns")

    @property
    def fft_precision(self):
        """Ring FFT engine: SHT_MIXED (double-float, mixed plans' default) or SHT_FP64."""
        n = ctypes.c_int()
        _check(_lib.sht_plan_get_fft_precision(self._h, ctypes.byref(n)), "sht_plan_get_fft_precision")
        return n.value

    @fft_precision.setter
    def fft_precision(self, precision):
        _check(_lib.sht_plan_set_fft_precision(self._h, precision), "sht_plan_set_fft_precision")

    @property
    def tensor_cores(self):
        """Mixed plans: True when the synthesis contraction runs on the tensor cores."""
        n = ctypes.c_int()
        _check(_lib.sht_plan_get_tensor_cores(self._h, ctypes.byref(n)), "sht_plan_get_tensor_cores")
        return bool(n.value)

    @tensor_cores.setter
    def tensor_cores(self, on):
        _check(_lib.sht_plan_set_tensor_cores(self._h, 1 if on else 0), "sht_plan_set_tensor_cores")

    @property
    def tensor_core_analysis(self):
        """Mixed plans: True when the analysis contraction runs on the tensor cores."""
        n = ctypes.c_int()
        _check(_lib.sht_plan_get_tensor_core_analysis(self._h, ctypes.byref(n)), "sht_plan_get_tensor_core_analysis")
        return bool(n.value)

    @tensor_core_analysis.setter
    def tensor_core_analysis(self, on):
        _check(_lib.sht_plan_set_tensor_core_analysis(self._h, 1 if on else 0), "sht_plan_set_tensor_core_analysis")

    def device_status(self):
        """Synchronises; raises ShtError (SHT_ERR_TIMEOUT) if a bounded device-side wait gave up."""
        n = ctypes.c_int()
        _check(_lib.sht_plan_device_status(self._h, ctypes.byref(n)), "sht_plan_device_status")
        return n.value

    def triples(self, flags=0):
        n = ctypes.c_int64()
        _check(_lib.sht_plan_triples(self._h, flags, ctypes.byref(n)), "sht_plan_triples")
        return n.value

    def triples_joined(self):
        n = ctypes.c_int64()
        _check(_lib.sht_plan_triples_joined(self._h, ctypes.byref(n)), "sht_plan_triples_joined")
        return n.value


def sht_geom_general(theta, nphi, phi0, ofs, stride=None, weight=None) -> Geometry:
    th = _arr(theta, np.float64)
    n = len(th)
    npf, p0, o = _arr(nphi, np.int32), _arr(phi0, np.float64), _arr(ofs, np.int64)
    st = None if stride is None else _arr(stride, np.int32)
    w = None if weight is None else _arr(weight, np.float64)
    h = _vp()
    _check(_lib.sht_geom_general(n, _ptr(th, _dp), _ptr(npf, _ip), _ptr(p0, _dp), _ptr(o, _i64p),
                                 _ptr(st, _ip), _ptr(w, _dp), ctypes.byref(h)), "sht_geom_general")
    return Geometry(h.value)


def sht_geom_gauss(nlat, nlon) -> Geometry:
    h = _vp()
    _check(_lib.sht_geom_gauss(nlat, nlon, ctypes.byref(h)), "sht_geom_gauss")
    return Geometry(h.value)


def sht_geom_reduced_gauss(nlat, lmax, spin=0) -> Geometry:
    h = _vp()
    _check(_lib.sht_geom_reduced_gauss(nlat, lmax, spin, ctypes.byref(h)), "sht_geom_reduced_gauss")
    return Geometry(h.value)


def sht_geom_ecp(kind, nlat, nlon) -> Geometry:
    h = _vp()
    _check(_lib.sht_geom_ecp(kind, nlat, nlon, ctypes.byref(h)), "sht_geom_ecp")
    return Geometry(h.value)


def sht_geom_healpix(nside) -> Geometry:
    h = _vp()
    _check(_lib.sht_geom_healpix(nside, ctypes.byref(h)), "sht_geom_healpix")
    return Geometry(h.value)


def sht_geom_subset(geom: Geometry, rings) -> Geometry:
    r = _arr(rings, np.int32)
    h = _vp()
    _check(_lib.sht_geom_subset(geom.handle, len(r), _ptr(r, _ip), ctypes.byref(h)), "sht_geom_subset")
    return Geometry(h.value)


def sht_alm_create(lmax, mmax, mval=None, mstart=None, stride=1) -> AlmLayout:
    mv = None if mval is None else _arr(mval, np.int32)
    ms = None if mstart is None else _arr(mstart, np.int64)
    h = _vp()
    _check(_lib.sht_alm_create(lmax, mmax, 0 if mv is None else len(mv), _ptr(mv, _ip), _ptr(ms, _i64p),
                               stride, ctypes.byref(h)), "sht_alm_create")
    lay = AlmLayout(h.value, lmax, mmax)
    lay.custom = mval is not None or mstart is not None or stride != 1  # not the default triangular layout
    return lay


def sht_plan_create(geom: Geometry, alm: AlmLayout, spin=0, ncomp=1, precision=SHT_FP64) -> Plan:
    h = _vp()
    _check(_lib.sht_plan_create(geom.handle, alm.handle, spin, ncomp, precision, ctypes.byref(h)),
           "sht_plan_create")
    return Plan(h.value, geom, alm, spin, ncomp, precision)


def _devptr(x):
    if isinstance(x, int):
        return x
    return int(x.data_ptr())  # torch tensor


def sht_execute(plan: Plan, type_, alm, maps, flags=0, stream=None):
    """alm, maps: sequences of device buffers (torch tensors or addresses)."""
    n = plan.narrays
    na = plan.ncomp if type_ == SHT_DERIV_SYNTHESIS else n
    if len(alm) != na or len(maps) != n:
        raise ValueError(f"expected {na} a_lm and {n} map buffers")
    ap = (_vp * na)(*[_devptr(a) for a in alm])
    mp = (_vp * n)(*[_devptr(m) for m in maps])
    st = None if stream is None else _vp(_devptr_stream(stream))
    _check(_lib.sht_execute(plan.handle, type_, ap, mp, flags, st), "sht_execute")


def sht_execute_legendre(plan: Plan, type_, alm, phase, flags=0, stream=None):
    """The Legendre stage alone (see include/sht_gb300.h): alm is a sequence of
    device buffers, phase one complex128 device buffer of nmaps x nm x nrings."""
    n = plan.narrays
    if len(alm) != n:
        raise ValueError(f"expected {n} a_lm buffers")
    ap = (_vp * n)(*[_devptr(a) for a in alm])
    st = None if stream is None else _vp(_devptr_stream(stream))
    _check(_lib.sht_execute_legendre(plan.handle, type_, ap, _devptr(phase), flags, st), "sht_execute_legendre")


def sht_execute_rings(plan: Plan, type_, phase, maps, flags=0, stream=None):
    """The ring-FFT stage alone (see include/sht_gb300.h): phase one complex128
    device buffer of nmaps x nm x nrings, maps a sequence of device buffers."""
    n = plan.narrays
    if len(maps) != n:
        raise ValueError(f"expected {n} map buffers")
    mp = (_vp * n)(*[_devptr(m) for m in maps])
    st = None if stream is None else _vp(_devptr_stream(stream))
    _check(_lib.sht_execute_rings(plan.handle, type_, _devptr(phase), mp, flags, st), "sht_execute_rings")


def sht_execute_noalloc(plan: Plan, type_, alm, maps, flags=0, stream=None):
    """As sht_execute, but the working memory comes from the library's static
    area: the call allocates nothing (see include/sht_gb300.h)."""
    n = plan.narrays
    if len(alm) != n or len(maps) != n:
        raise ValueError(f"expected {n} a_lm and {n} map buffers")
    ap = (_vp * n)(*[_devptr(a) for a in alm])
    mp = (_vp * n)(*[_devptr(m) for m in maps])
    st = None if stream is None else _vp(_devptr_stream(stream))
    _check(_lib.sht_execute_noalloc(plan.handle, type_, ap, mp, flags, st), "sht_execute_noalloc")


class Batch(_Handle):
    """Distinct plans run through merged launches (see include/sht_gb300.h).
    Holds references to its plans so they outlive it."""
    _destroy = "sht_batch_destroy"

    def __init__(self, h, plans):
        super().__init__(h)
        self.plans = list(plans)

    def __len__(self):
        return _lib.sht_batch_size(self._h)


def sht_measure_pipe_peaks(device=-1):
    """Measured pipe throughput (see include/sht_gb300.h): FP64 FMA TFLOP/s, FP32 FMA and add T op/s."""
    out = (ctypes.c_double * 3)()
    _check(_lib.sht_measure_pipe_peaks(device, out), "sht_measure_pipe_peaks")
    return {"fp64_fma_tflops": out[0], "fp32_fma_tops": out[1], "fp32_add_tops": out[2]}


def sht_fft_plan_info(n):
    """(kind, transform length, radices) for a ring of n points: kind 0 mixed radix, 1 Rader, 2 Bluestein."""
    kind, ln, nrad = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rad = (ctypes.c_int * 24)()
    _check(_lib.sht_fft_plan_info(n, ctypes.byref(kind), ctypes.byref(ln), ctypes.byref(nrad), rad), "sht_fft_plan_info")
    return kind.value, ln.value, [rad[i] for i in range(nrad.value)]


def sht_geom_polar_cut(geom: Geometry, lmax, spin, mval):
    """(first kept ring pair per m, each pair's northern theta, triples) of the polar optimisation."""
    mv = np.ascontiguousarray(mval, dtype=np.int32)
    first = np.empty(len(mv), np.int32)
    th = np.empty(geom.info()[2], np.float64)
    trip = ctypes.c_int64()
    _check(_lib.sht_geom_polar_cut(geom.handle, lmax, spin, len(mv), _ptr(mv, _ip), _ptr(first, _ip), _ptr(th, _dp),
                                   ctypes.byref(trip)), "sht_geom_polar_cut")
    return first, th, trip.value


def sht_batch_create(plans) -> Batch:
    plans = list(plans)
    hp = (_vp * len(plans))(*[p.handle for p in plans])
    h = _vp()
    _check(_lib.sht_batch_create(len(plans), hp, ctypes.byref(h)), "sht_batch_create")
    return Batch(h.value, plans)


def sht_batch_execute(batch: Batch, type_, alm, maps, flags=0, stream=None):
    """alm[k], maps[k]: plan k's device buffers, as sht_execute takes them."""
    if len(alm) != len(batch.plans) or len(maps) != len(batch.plans):
        raise ValueError(f"expected buffer lists for {len(batch.plans)} plans")
    keep = []
    ap = (ctypes.POINTER(_vp) * len(alm))()
    mp = (ctypes.POINTER(_vp) * len(maps))()
    for k, p in enumerate(batch.plans):
        n = p.narrays
        if len(alm[k]) != n or len(maps[k]) != n:
            raise ValueError(f"plan {k}: expected {n} a_lm and {n} map buffers")
        a = (_vp * n)(*[_devptr(x) for x in alm[k]])
        m = (_vp * n)(*[_devptr(x) for x in maps[k]])
        keep += [a, m]
        ap[k] = ctypes.cast(a, ctypes.POINTER(_vp))
        mp[k] = ctypes.cast(m, ctypes.POINTER(_vp))
    st = None if stream is None else _vp(_devptr_stream(stream))
    _check(_lib.sht_batch_execute(batch.handle, type_, ap, mp, flags, st), "sht_batch_execute")


def _devptr_stream(stream):
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream
