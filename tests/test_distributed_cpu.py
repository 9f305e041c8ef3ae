"""The m / ring decomposition of Sect. 4.2 on the CPU.

The partition (round robin over m and over ring pairs, mirrored rings kept
together) is checked for coverage; the distributed synthesis and analysis
drivers of paper_1303_4945_gb300.distributed run with a CPU data plane built from
the oracle's Legendre stage (Eq. syn2) and direct ring sums (Eqs. syn1, ana2),
first with three tasks emulated in one process, then as two gloo ranks
exchanging through torch.distributed.all_to_all_single; either way every task's
pixels and a_lm must equal the oracle's single-process transform.
"""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1303_4945_gb300 import distributed as dist_mod
from paper_1303_4945_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PI = np.pi


class OracleStages:
    """The four stages of one task, spin 0, in plain numpy on the oracle's
    Legendre values: F[0][i][y] for the task's m over every ring, the ring sums of
    Eq. syn1 (real maps: F_{-m} = conj F_m) and of Eq. ana2 (ring weights), and
    the Legendre contraction of Eq. ana1."""

    def __init__(self, lmax, mmax, rings, part, rank, as_torch=False):
        self.lmax, self.mmax, self.rings = lmax, mmax, rings
        self.m = part.m[rank]
        self.my_rings = part.rings[rank]
        self.as_torch = as_torch

    def _out(self, a):
        if self.as_torch:
            import torch

            return torch.from_numpy(np.ascontiguousarray(a))
        return a

    def _np(self, a):
        return a.numpy() if hasattr(a, "numpy") else a

    def legendre_synthesis(self, alm_local):
        full = np.zeros(oracle.nalm(self.lmax, self.mmax), dtype=np.complex128)
        dist_mod.alm_unpack(self._np(alm_local[0]), self.lmax, self.mmax, self.m, full)
        F = oracle.phase(0, self.lmax, self.mmax, full, self.rings.theta)  # [ring][m = -mmax..mmax]
        return self._out(F[:, self.mmax + np.asarray(self.m)].T[None, :, :].copy())

    def ring_synthesis(self, F_full):
        F = self._np(F_full)[0]  # [m][ring']
        out = []
        for j, y in enumerate(self.my_rings):
            N = self.rings.nphi[y]
            phi = self.rings.phi0[y] + 2 * PI * np.arange(N) / N
            m = np.arange(self.mmax + 1)
            e = np.exp(1j * np.outer(phi, m))
            w = np.where(m == 0, 1.0, 2.0)
            out.append((e * (w * F[:, j])[None, :]).sum(axis=1).real)
        return [self._out(np.concatenate(out))]

    def ring_analysis(self, maps_local):
        p = self._np(maps_local[0])
        G = np.zeros((1, self.mmax + 1, len(self.my_rings)), dtype=np.complex128)
        o = 0
        for j, y in enumerate(self.my_rings):
            N = self.rings.nphi[y]
            phi = self.rings.phi0[y] + 2 * PI * np.arange(N) / N
            m = np.arange(self.mmax + 1)
            G[0, :, j] = self.rings.weight[y] * (np.exp(-1j * np.outer(m, phi)) * p[o:o + N][None, :]).sum(axis=1)
            o += N
        return self._out(G)

    def legendre_analysis(self, G_local):
        G = self._np(G_local)[0]  # [i][ring]
        parts = []
        for i, m in enumerate(self.m):
            lam = np.array([oracle.lambda_(0, int(m), self.lmax, th) for th in self.rings.theta])  # [ring][l]
            parts.append((G[i][:, None] * lam).sum(axis=0)[m:])
        return [self._out(np.concatenate(parts))]


def _problem(grid):
    if grid == "gauss":
        lmax = 20
        th, w = oracle.gauss_nodes(lmax + 2)
        rings = oracle.Rings(th, np.full(lmax + 2, 2 * lmax + 1), np.zeros(lmax + 2), w * 2 * PI / (2 * lmax + 1))
    else:
        lmax = 14
        rings = oracle.healpix_rings(4)  # aliased polar rings, phi0 != 0, an equator ring without a mirror
    rng = np.random.default_rng(77)
    return lmax, rings, inputs.gaussian_alm(rng, lmax, lmax), rng.standard_normal(rings.npix)


def test_partition_round_robin():
    rings = oracle.healpix_rings(8)
    for n in (1, 2, 3, 5):
        part = dist_mod.Partition.round_robin(40, rings.theta, n)
        assert sorted(np.concatenate(part.m).tolist()) == list(range(41))
        assert sorted(np.concatenate(part.rings).tolist()) == list(range(rings.nrings))
        # every task holds both rings of each of its pairs
        for r in range(n):
            mine = set(part.rings[r].tolist())
            for a, b in dist_mod.ring_pairs(rings.theta):
                if b >= 0:
                    assert (a in mine) == (b in mine)
        # round robin: pair k and m = k go to task k mod n
        assert all(int(m) % n == r for r in range(n) for m in part.m[r])


@pytest.mark.parametrize("grid", ["gauss", "healpix"])
def test_emulated_tasks_match_oracle(grid):
    lmax, rings, alm, pmap = _problem(grid)
    part = dist_mod.Partition.round_robin(lmax, rings.theta, 3)
    stages = [OracleStages(lmax, lmax, rings, part, r) for r in range(3)]
    alm_loc = [[dist_mod.alm_pack(alm, lmax, lmax, part.m[r])] for r in range(3)]
    maps = dist_mod.synthesis_emulated(part, stages, alm_loc)
    ref = oracle.synthesis(0, lmax, lmax, [alm], rings)[0]
    got = np.zeros(rings.npix)
    for r in range(3):
        got[dist_mod.ring_pixels(rings.ofs, rings.nphi, part.rings[r])] = maps[r][0]
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
    maps_loc = [[pmap[dist_mod.ring_pixels(rings.ofs, rings.nphi, part.rings[r])]] for r in range(3)]
    back = dist_mod.analysis_emulated(part, stages, maps_loc)
    ref_a = oracle.analysis(0, lmax, lmax, [pmap], rings)[0]
    got_a = np.zeros_like(ref_a)
    for r in range(3):
        dist_mod.alm_unpack(back[r][0], lmax, lmax, part.m[r], got_a)
    assert np.linalg.norm(got_a - ref_a) <= 1e-12 * np.linalg.norm(ref_a)


CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import numpy as np, torch, torch.distributed as dist
import oracle
from paper_1303_4945_gb300 import distributed as D
from test_distributed_cpu import OracleStages, _problem
dist.init_process_group("gloo")
rank, world = dist.get_rank(), dist.get_world_size()
lmax, rings, alm, pmap = _problem(sys.argv[2])
part = D.Partition.round_robin(lmax, rings.theta, world)
st = OracleStages(lmax, lmax, rings, part, rank, as_torch=True)
mine = D.ring_pixels(rings.ofs, rings.nphi, part.rings[rank])
maps = D.synthesis(part, rank, st, D.torch_exchange, [torch.from_numpy(D.alm_pack(alm, lmax, lmax, part.m[rank]))])
ref = oracle.synthesis(0, lmax, lmax, [alm], rings)[0][mine]
e1 = np.linalg.norm(maps[0].numpy() - ref) / np.linalg.norm(ref)
back = D.analysis(part, rank, st, D.torch_exchange, [torch.from_numpy(pmap[mine])])
ref_a = D.alm_pack(oracle.analysis(0, lmax, lmax, [pmap], rings)[0], lmax, lmax, part.m[rank])
e2 = np.linalg.norm(back[0].numpy() - ref_a) / np.linalg.norm(ref_a)
print("rank", rank, "errors", e1, e2, flush=True)
assert e1 <= 1e-12 and e2 <= 1e-12, (e1, e2)
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("grid", ["gauss", "healpix"])
def test_two_gloo_ranks_match_oracle(grid):
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE="2",
                   LOCAL_RANK=str(rank), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD, ROOT, grid], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, (o, e[-2000:])
        assert "errors" in o
