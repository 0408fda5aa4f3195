"""The paper's m/latitude decomposition over several ranks, on host (gloo) ranks.

Two (and three) gloo processes each own a share of the wavenumbers and of the
ring pairs (paper_1908_06097_gb300.dist.partition) and run the decomposed
inverse and direct transforms through dist.Distributed with ONE
all_to_all_single per direction.  On the CPU the half-transforms are a numpy
stand-in built from the oracle's Legendre functions and plain DFTs (the CUDA
kernels of the halves are checked on one GPU in test_decomposition_gpu.py);
what is tested here is the partition, the exchange pattern, the byte split
sizes and the orchestration: the assembled grid and spectra must equal the
oracle's undecomposed transforms.
"""

import os
import socket

import numpy as np
import pytest

from paper_1908_06097_gb300 import dist, inputs

torch = pytest.importorskip("torch")


class NumpyEngine:
    """The half-transforms of one rank in numpy, with the exchange rows in the
    order the library documents (per destination rank; inverse: rings
    ascending, then m; direct: m ascending, parity, then ring)."""

    def __init__(self, orc, T, N, nfld, nranks, rank, m_owner, ring_owner):
        self.T, self.N, self.nfld, self.nranks, self.rank = T, N, nfld, nranks, rank
        self.mo, self.ro = m_owner, ring_owner
        nl, mmax, npts = orc.grid(0, N, T)
        self.nlon, self.mmax, self.npts = nl, mmax, npts
        self.off = np.concatenate([[0], np.cumsum(nl)])
        self.x, self.w = orc.gauss(2 * N)
        self.nlat = 2 * N
        self.P = {}  # (m, k) -> P_n^m(x_k), n = m..T
        for m in range(T + 1):
            for k in range(self.nlat):
                if m <= mmax[k]:
                    self.P[(m, k)] = orc.plm(m, T, self.x[k])
        self.four = np.zeros((self.nlat, T + 1, nfld), dtype=complex)  # F_m(ring k) per field
        self.gop = {}  # (m, p, north ring) -> folded, weighted operand [nfld] complex
        self.coff = np.array([m * (2 * T + 3 - m) // 2 for m in range(T + 1)])

    def pair(self, k):
        return k if k < self.N else self.nlat - 1 - k

    # -- exchange rows --------------------------------------------------
    def _rows(self, d, frm, to):
        if d == 0:
            return [(k, m) for k in range(self.nlat) if self.ro[self.pair(k)] == to
                    for m in range(self.mmax[k] + 1) if self.mo[m] == frm]
        return [(m, p, kN) for m in range(self.T + 1) if self.mo[m] == to for p in (0, 1)
                for kN in range(self.N) if self.mmax[kN] >= m and self.ro[kN] == frm]

    def counts(self, d):
        send = [len(self._rows(d, self.rank, r)) for r in range(self.nranks)]
        recv = [len(self._rows(d, r, self.rank)) for r in range(self.nranks)]
        return send, recv, 16 * self.nfld

    def pack(self, d):
        vals = []
        for r in range(self.nranks):
            for row in self._rows(d, self.rank, r):
                v = self.four[row[0], row[1]] if d == 0 else self.gop[row]
                vals.append(np.stack([v.real, v.imag], axis=1).ravel())
        flat = np.concatenate(vals) if vals else np.zeros(0)
        return torch.from_numpy(np.ascontiguousarray(flat).view(np.uint8).copy())

    def unpack(self, d, recv):
        vals = recv.numpy().view(np.float64).reshape(-1, self.nfld, 2)
        i = 0
        for r in range(self.nranks):
            for row in self._rows(d, r, self.rank):
                v = vals[i, :, 0] + 1j * vals[i, :, 1]
                if d == 0:
                    self.four[row[0], row[1]] = v
                else:
                    self.gop[row] = v
                i += 1

    # -- half-transforms --------------------------------------------------
    def inv_legendre(self, spec):
        for m in range(self.T + 1):
            if self.mo[m] != self.rank:
                continue
            a = spec[:, self.coff[m]:self.coff[m] + self.T + 1 - m]
            a = a[..., 0] + 1j * (a[..., 1] if m else 0)
            for k in range(self.nlat):
                if m <= self.mmax[k]:
                    self.four[k, m] = a @ self.P[(m, k)]

    def inv_fourier(self, grid):
        for k in range(self.nlat):
            if self.ro[self.pair(k)] != self.rank:
                continue
            n, K = self.nlon[k], self.mmax[k] + 1
            lam = 2 * np.pi * np.arange(n) / n
            E = np.exp(1j * np.outer(np.arange(K), lam))
            F = self.four[k, :K].T.copy()
            F[:, 0] = F[:, 0].real
            c = np.ones(K)
            c[1:] = 2
            grid[:, self.off[k]:self.off[k + 1]] = ((F * c) @ E).real

    def dir_fourier(self, grid):
        for kN in range(self.N):
            if self.ro[kN] != self.rank:
                continue
            kS = self.nlat - 1 - kN
            n, K = self.nlon[kN], self.mmax[kN] + 1
            lam = 2 * np.pi * np.arange(n) / n
            E = np.exp(-1j * np.outer(lam, np.arange(K)))
            FN = grid[:, self.off[kN]:self.off[kN + 1]] @ E / n
            FS = grid[:, self.off[kS]:self.off[kS + 1]] @ E / n
            for m in range(K):
                self.gop[(m, 0, kN)] = self.w[kN] * (FN[:, m] + FS[:, m])
                self.gop[(m, 1, kN)] = self.w[kN] * (FN[:, m] - FS[:, m])

    def dir_legendre(self, spec):
        for m in range(self.T + 1):
            if self.mo[m] != self.rank:
                continue
            acc = np.zeros((self.nfld, self.T + 1 - m), dtype=complex)
            for kN in range(self.N):
                if self.mmax[kN] < m:
                    continue
                P = self.P[(m, kN)]
                par = (np.arange(m, self.T + 1) - m) & 1
                for p in (0, 1):
                    acc[:, par == p] += np.outer(self.gop[(m, p, kN)], P[par == p])
            spec[:, self.coff[m]:self.coff[m] + self.T + 1 - m, 0] = acc.real
            spec[:, self.coff[m]:self.coff[m] + self.T + 1 - m, 1] = acc.imag if m else 0.0


def _rank_main(rank, nranks, port, T, nfld, out_dir):
    import torch.distributed as tdist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    tdist.init_process_group("gloo", rank=rank, world_size=nranks)
    N = T + 1
    mo, ro = dist.partition(T, N, nranks)
    eng = NumpyEngine(oracle, T, N, nfld, nranks, rank, mo, ro)
    d = dist.Distributed(eng, dist.torch_exchange())
    a = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 70)
    g = np.full((nfld, eng.npts), np.nan)
    d.inverse(a, g)
    g_ref = oracle.inverse(T, 0, N, a)
    s = np.full_like(a, np.nan)
    d.direct(g_ref, s)
    np.save(os.path.join(out_dir, f"g{rank}.npy"), g)
    np.save(os.path.join(out_dir, f"s{rank}.npy"), s)
    tdist.barrier()
    tdist.destroy_process_group()


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def test_partition_covers_everything_once():
    for T, nranks in [(79, 2), (79, 3), (159, 4), (1279, 8)]:
        N = T + 1
        mo, ro = dist.partition(T, N, nranks)
        assert mo.shape == (T + 1,) and ro.shape == (N,)
        assert set(mo) == set(range(nranks)) and set(ro) == set(range(nranks))
        assert np.all(np.diff(ro) >= 0)  # ring pairs in contiguous blocks
        mmax, nlon = dist.northern_mmax(T, N)
        L = np.array([(mmax >= m).sum() for m in range(T + 1)])
        work = (T + 2 - np.arange(T + 1)) * L
        per = np.array([work[mo == r].sum() for r in range(nranks)])
        assert per.max() <= 1.05 * per.mean()  # Legendre work balanced within 5 %
        pts = np.array([(2 * nlon)[ro == r].sum() for r in range(nranks)])
        assert pts.max() <= pts.mean() + 2 * nlon.max()


@pytest.mark.parametrize("nranks", [2, 3])
def test_decomposed_transforms_on_gloo_ranks(orc, tmp_path, nranks):
    import torch.multiprocessing as mp

    T, nfld = 23, 3
    mp.spawn(_rank_main, args=(nranks, _free_port(), T, nfld, str(tmp_path)), nprocs=nranks, join=True)
    N = T + 1
    mo, ro = dist.partition(T, N, nranks)
    nl, _, npts = orc.grid(0, N, T)
    off = np.concatenate([[0], np.cumsum(nl)])
    a = inputs.spectral_fields(T, nfld, inputs.SEED_BASE + 70)
    g_ref = orc.inverse(T, 0, N, a)
    s_ref = orc.direct(T, 0, N, g_ref)
    g = np.full((nfld, npts), np.nan)
    s = np.full_like(a, np.nan)
    ns, ms = inputs.coef_nm(T)
    for r in range(nranks):
        gr = np.load(tmp_path / f"g{r}.npy")
        sr = np.load(tmp_path / f"s{r}.npy")
        for k in range(2 * N):
            kp = k if k < N else 2 * N - 1 - k
            if ro[kp] == r:
                assert np.isfinite(gr[:, off[k]:off[k + 1]]).all()
                g[:, off[k]:off[k + 1]] = gr[:, off[k]:off[k + 1]]
            else:
                assert np.isnan(gr[:, off[k]:off[k + 1]]).all()  # only own rings written
        own = mo[ms] == r
        assert np.isfinite(sr[:, own]).all() and np.isnan(sr[:, ~own]).all()
        s[:, own] = sr[:, own]
    assert np.abs(g - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
    assert np.abs(s - s_ref).max() <= 1e-12 * np.abs(s_ref).max()
