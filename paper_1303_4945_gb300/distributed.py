"""Distributed transforms: the m / ring decomposition of Sect. 4.2 (Figs. 3 and 4).

Each of N tasks holds the a_lm of its own m values and the pixels of its own
rings, assigned round robin as the paper suggests: task i holds m = i, i + N,
i + 2N, ... and the ring pairs i, i + N, i + 2N, ... counted from the north pole
(each pair being a northern ring and its mirror on the other hemisphere, so a
task's rings still pair up for the ring FFTs).

A synthesis runs the Legendre stage of the task's m values over every ring,
giving the phase array F[c][i][y] (map c, the task's i-th m, ring y of the whole
grid); one all-to-all sends every task the F of its rings for every m; the task
assembles F[c][m][y'] (all m, its rings y') and runs the ring FFTs into its
pixels.  An analysis runs the ring FFTs of the task's rings into G[c][m][y'],
one all-to-all gives every task the G of its m values on every ring, and the
task runs the Legendre stage into its a_lm.  The single exchange per transform
moves the phase array, nmaps * (mmax + 1) * nrings complex values in all.

The arithmetic is pluggable: `stages` supplies the four stage functions and
`exchange` the all-to-all, so the same driver runs the library's stage calls
(sht_execute_legendre / sht_execute_rings) with torch.distributed on GPUs, or a
plain CPU data plane for tests.  On one GPU several tasks can be emulated in
one process with `local_exchange`.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Partition", "round_robin_m", "ring_pairs", "round_robin_rings", "synthesis", "analysis",
           "local_exchange", "torch_exchange", "LibraryStages"]


def round_robin_m(mmax: int, ntasks: int, rank: int) -> np.ndarray:
    """The m values task `rank` holds: rank, rank + N, rank + 2N, ... <= mmax."""
    return np.arange(rank, mmax + 1, ntasks, dtype=np.int64)


def ring_pairs(theta: np.ndarray, tol: float = 1e-12) -> list[tuple[int, int]]:
    """Rings as (north, south) pairs ordered from the north pole to the equator;
    south is -1 for a ring without a mirror (the equator, or partial coverage)."""
    theta = np.asarray(theta, dtype=np.float64)
    order = np.argsort(theta, kind="stable")
    used = np.zeros(len(theta), bool)
    pairs = []
    for y in order:
        if used[y]:
            continue
        used[y] = True
        mate = -1
        if theta[y] < 0.5 * np.pi - tol:
            cand = np.nonzero(~used & (np.abs(theta - (np.pi - theta[y])) <= tol))[0]
            if len(cand):
                mate = int(cand[0])
                used[mate] = True
        pairs.append((int(y), mate))
    return pairs


def round_robin_rings(theta: np.ndarray, ntasks: int, rank: int) -> np.ndarray:
    """Ring indices (ascending) of the pairs rank, rank + N, rank + 2N, ..."""
    pairs = ring_pairs(theta)
    rings = [r for k, pr in enumerate(pairs) if k % ntasks == rank for r in pr if r >= 0]
    return np.array(sorted(rings), dtype=np.int64)


@dataclass
class Partition:
    """Who holds what: m lists and ring lists of every task."""
    mmax: int
    nrings: int
    m: list
    rings: list

    @classmethod
    def round_robin(cls, mmax: int, theta: np.ndarray, ntasks: int) -> "Partition":
        return cls(mmax, len(theta), [round_robin_m(mmax, ntasks, r) for r in range(ntasks)],
                   [round_robin_rings(theta, ntasks, r) for r in range(ntasks)])

    @property
    def ntasks(self) -> int:
        return len(self.m)


def local_exchange(send_per_task: list, split_per_task: list) -> list:
    """All-to-all among tasks emulated in one process: send_per_task[r] is task
    r's flat send buffer, cut into split_per_task[r][q] values for task q; returns
    every task's receive buffer (the pieces from tasks 0, 1, ... in order)."""
    n = len(send_per_task)
    pieces = []
    for r in range(n):
        offs = np.concatenate([[0], np.cumsum(split_per_task[r])]).astype(int)
        pieces.append([send_per_task[r][offs[q]:offs[q + 1]] for q in range(n)])
    out = []
    for q in range(n):
        chunks = [pieces[r][q] for r in range(n)]
        out.append(_cat(chunks))
    return out


def torch_exchange(send, send_splits, recv_splits):
    """One all-to-all through torch.distributed (NCCL for CUDA tensors, gloo on the
    CPU), on the float64 view of complex buffers."""
    import torch
    import torch.distributed as dist

    real = torch.view_as_real(send).reshape(-1) if send.is_complex() else send
    out = torch.empty(2 * sum(recv_splits) if send.is_complex() else sum(recv_splits), dtype=real.dtype,
                      device=real.device)
    f = 2 if send.is_complex() else 1
    dist.all_to_all_single(out, real.contiguous(), [f * s for s in recv_splits], [f * s for s in send_splits])
    return torch.view_as_complex(out.reshape(-1, 2)) if send.is_complex() else out


def _cat(chunks):
    if hasattr(chunks[0], "is_cuda"):
        import torch

        return torch.cat(chunks)
    return np.concatenate(chunks)


def _zeros_like_shape(ref, shape):
    if hasattr(ref, "is_cuda"):
        import torch

        return torch.zeros(shape, dtype=ref.dtype, device=ref.device)
    return np.zeros(shape, dtype=ref.dtype)


def _index(a, idx):
    if hasattr(a, "is_cuda"):
        import torch

        return torch.as_tensor(idx, device=a.device)
    return idx


# ---- synthesis: the task's m -> every ring (Legendre) -> all-to-all -> its rings (FFT)
def synthesis_send(part: Partition, rank: int, F_local):
    """Pack F[c][i][y] (task's m, all rings) for the all-to-all: the block of task q
    is F[:, :, rings_q], in task order.  Returns (flat buffer, splits)."""
    blocks = [F_local[:, :, _index(F_local, part.rings[q])].reshape(-1) for q in range(part.ntasks)]
    return _cat(blocks), [int(b.shape[0]) for b in blocks]


def synthesis_recv_splits(part: Partition, rank: int, ncomp_maps: int):
    return [ncomp_maps * len(part.m[q]) * len(part.rings[rank]) for q in range(part.ntasks)]


def synthesis_assemble(part: Partition, rank: int, recv, ncomp_maps: int):
    """F_full[c][m][y'] (every m 0..mmax, the task's rings) from the received blocks."""
    nr = len(part.rings[rank])
    F = _zeros_like_shape(recv, (ncomp_maps, part.mmax + 1, nr))
    off = 0
    for q in range(part.ntasks):
        n = ncomp_maps * len(part.m[q]) * nr
        F[:, _index(recv, part.m[q]), :] = recv[off:off + n].reshape(ncomp_maps, len(part.m[q]), nr)
        off += n
    return F


# ---- analysis: the task's rings (FFT) -> all-to-all -> the task's m (Legendre) over every ring
def analysis_send(part: Partition, rank: int, G_rings):
    """Pack G[c][m][y'] (every m, the task's rings): the block of task q is
    G[:, m_q, :], in task order."""
    blocks = [G_rings[:, _index(G_rings, part.m[q]), :].reshape(-1) for q in range(part.ntasks)]
    return _cat(blocks), [int(b.shape[0]) for b in blocks]


def analysis_recv_splits(part: Partition, rank: int, ncomp_maps: int):
    return [ncomp_maps * len(part.m[rank]) * len(part.rings[q]) for q in range(part.ntasks)]


def analysis_assemble(part: Partition, rank: int, recv, ncomp_maps: int):
    """G_local[c][i][y] (the task's m, every ring) from the received blocks."""
    nm = len(part.m[rank])
    G = _zeros_like_shape(recv, (ncomp_maps, nm, part.nrings))
    off = 0
    for q in range(part.ntasks):
        n = ncomp_maps * nm * len(part.rings[q])
        G[:, :, _index(recv, part.rings[q])] = recv[off:off + n].reshape(ncomp_maps, nm, len(part.rings[q]))
        off += n
    return G


def synthesis(part: Partition, rank: int, stages, exchange, alm_local):
    """Distributed synthesis on task `rank`: its a_lm (its m values) -> its pixels.
    stages.legendre_synthesis(alm_local) -> F[c][i][y]; exchange(send, send_splits,
    recv_splits) -> recv; stages.ring_synthesis(F_full) -> the task's maps."""
    F = stages.legendre_synthesis(alm_local)
    C = F.shape[0]
    send, splits = synthesis_send(part, rank, F)
    recv = exchange(send, splits, synthesis_recv_splits(part, rank, C))
    return stages.ring_synthesis(synthesis_assemble(part, rank, recv, C))


def analysis(part: Partition, rank: int, stages, exchange, maps_local):
    """Distributed analysis on task `rank`: its pixels -> its a_lm (its m values)."""
    G = stages.ring_analysis(maps_local)
    C = G.shape[0]
    send, splits = analysis_send(part, rank, G)
    recv = exchange(send, splits, analysis_recv_splits(part, rank, C))
    return stages.legendre_analysis(analysis_assemble(part, rank, recv, C))


class LibraryStages:
    """The four stages of one task through the C ABI (sht_execute_legendre /
    sht_execute_rings) on the current CUDA device.  The task's a_lm arrays hold
    its m values in the triangular layout over that m list; its maps hold only its
    rings, stored one after another in ascending ring order."""

    def __init__(self, sht, geom, lmax, mmax, spin, ncomp, precision, part: Partition, rank: int, stream=None):
        import torch

        self.sht, self.stream = sht, stream
        r = geom.rings()
        mloc = part.m[rank]
        self.plan_m = sht.sht_plan_create(geom, sht.sht_alm_create(lmax, mmax, mval=mloc), spin, ncomp, precision)
        rings = part.rings[rank]
        nphi = r["nphi"][rings]
        ofs = np.concatenate([[0], np.cumsum(nphi)[:-1]]).astype(np.int64)
        self.geom_r = sht.sht_geom_general(r["theta"][rings], nphi, r["phi0"][rings], ofs, weight=r["weight"][rings])
        self.plan_r = sht.sht_plan_create(self.geom_r, sht.sht_alm_create(lmax, mmax), spin, ncomp, precision)
        self.npix_local = int(np.sum(nphi))
        self.nalm_local = self.plan_m.alm.size()
        self.C = self.plan_m.narrays
        self.nm, self.mmax = len(mloc), mmax
        self.nrings, self.nrings_local = geom.nrings, len(rings)
        self.torch = torch

    def legendre_synthesis(self, alm_local):
        F = self.torch.empty((self.C, self.nm, self.nrings), dtype=self.torch.complex128, device="cuda")
        self.sht.sht_execute_legendre(self.plan_m, self.sht.SHT_SYNTHESIS, alm_local, F, 0, self.stream)
        return F

    def ring_synthesis(self, F_full):
        F_full = F_full.contiguous()
        maps = [self.torch.empty(self.npix_local, dtype=self.torch.float64, device="cuda") for _ in range(self.C)]
        self.sht.sht_execute_rings(self.plan_r, self.sht.SHT_SYNTHESIS, F_full, maps, 0, self.stream)
        return maps

    def ring_analysis(self, maps_local):
        G = self.torch.empty((self.C, self.mmax + 1, self.nrings_local), dtype=self.torch.complex128, device="cuda")
        self.sht.sht_execute_rings(self.plan_r, self.sht.SHT_ANALYSIS, G, maps_local, 0, self.stream)
        return G

    def legendre_analysis(self, G_local):
        G_local = G_local.contiguous()
        alm = [self.torch.empty(self.nalm_local, dtype=self.torch.complex128, device="cuda") for _ in range(self.C)]
        self.sht.sht_execute_legendre(self.plan_m, self.sht.SHT_ANALYSIS, alm, G_local, 0, self.stream)
        return alm


# ---- several tasks in one process (tests, and one GPU standing in for several) ----
def synthesis_emulated(part: Partition, stages_per_task, alm_per_task):
    """The distributed synthesis of every task, the all-to-all emulated in memory."""
    F = [stages_per_task[r].legendre_synthesis(alm_per_task[r]) for r in range(part.ntasks)]
    C = F[0].shape[0]
    packed = [synthesis_send(part, r, F[r]) for r in range(part.ntasks)]
    recv = local_exchange([p[0] for p in packed], [p[1] for p in packed])
    return [stages_per_task[r].ring_synthesis(synthesis_assemble(part, r, recv[r], C)) for r in range(part.ntasks)]


def analysis_emulated(part: Partition, stages_per_task, maps_per_task):
    """The distributed analysis of every task, the all-to-all emulated in memory."""
    G = [stages_per_task[r].ring_analysis(maps_per_task[r]) for r in range(part.ntasks)]
    C = G[0].shape[0]
    packed = [analysis_send(part, r, G[r]) for r in range(part.ntasks)]
    recv = local_exchange([p[0] for p in packed], [p[1] for p in packed])
    return [stages_per_task[r].legendre_analysis(analysis_assemble(part, r, recv[r], C)) for r in range(part.ntasks)]


def alm_pack(full: np.ndarray, lmax: int, mmax: int, mval) -> np.ndarray:
    """The entries of the listed m values from a triangular (all-m) a_lm array, in
    the triangular layout over that m list (m-major, l = m..lmax)."""
    starts = {m: m * (2 * lmax + 1 - m) // 2 for m in range(mmax + 1)}
    return np.concatenate([full[starts[m] + m: starts[m] + lmax + 1] for m in mval])


def alm_unpack(packed: np.ndarray, lmax: int, mmax: int, mval, out: np.ndarray) -> None:
    """Inverse of alm_pack into a triangular (all-m) array."""
    o = 0
    for m in mval:
        s = m * (2 * lmax + 1 - m) // 2
        n = lmax - m + 1
        out[s + m: s + lmax + 1] = packed[o:o + n]
        o += n


def ring_pixels(ofs: np.ndarray, nphi: np.ndarray, rings) -> np.ndarray:
    """Pixel indices of the given rings of a map, one ring after another."""
    return np.concatenate([np.arange(ofs[y], ofs[y] + nphi[y]) for y in rings]).astype(np.int64)
