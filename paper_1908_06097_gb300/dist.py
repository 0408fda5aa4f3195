"""The paper's decomposition of the transform over several GPUs.

Sec. 3.1.1 of the ESCAPE report distributes the spectral transform so that
every GPU owns some zonal wavenumbers m (its Legendre transforms) and some
latitudes (its ring FFTs), and every GPU exchanges data with every other GPU
once per transform direction; Sec. 3.1.3 moves the buffer packing onto the
GPU and overlaps the per-destination messages.  Here:

  partition()   wavenumbers dealt longest-first to the least-loaded rank
                (the Legendre work of m is (T+2-m) L_m), ring pairs in
                contiguous blocks of about equal grid points;
  Distributed   the transform of one rank: its half-transforms, the pack of
                its outgoing rows, ONE all-to-all, the unpack, the other half;
  LibEngine     the half-transforms and the pack/unpack of a partitioned plan
                (the library's st_inv_legendre, st_exchange_pack, ...);
  torch_exchange the all-to-all over torch.distributed (NCCL for device
                buffers, gloo for host buffers).

The exchange is pluggable so that the same orchestration runs on host ranks
(gloo) in the tests.  No part of it computes the transform itself.
"""

import ctypes

import numpy as np


def northern_mmax(T, N, kind=0):
    """mmax of the northern rings (octahedral: ring i has 4i+16 points)."""
    nlon = 4 * np.arange(1, N + 1) + 16 if kind == 0 else np.full(N, 4 * N)
    return np.minimum(T, nlon // 2 - 1), nlon


def partition(T, N, nranks, kind=0):
    """(m_owner[T+1], ring_owner[N]) for nranks ranks."""
    mmax, nlon = northern_mmax(T, N, kind)
    L = np.array([(mmax >= m).sum() for m in range(T + 1)])
    work = (T + 2 - np.arange(T + 1)) * L
    m_owner = np.zeros(T + 1, dtype=np.int32)
    load = np.zeros(nranks)
    for m in np.argsort(-work, kind="stable"):
        r = int(np.argmin(load))
        m_owner[m] = r
        load[r] += work[m]
    pts = np.cumsum(2 * nlon)
    ring_owner = np.minimum((pts - 1) * nranks // pts[-1], nranks - 1).astype(np.int32)
    return m_owner, ring_owner


class Distributed:
    """One rank's transforms: engine = the half-transforms and the exchange
    buffers of this rank; exchange(send, send_bytes, recv_bytes) -> recv is the
    all-to-all (split sizes in bytes, one per rank)."""

    def __init__(self, engine, exchange):
        self.engine = engine
        self.exchange = exchange

    def _swap(self, direction):
        send_rows, recv_rows, row_bytes = self.engine.counts(direction)
        send = self.engine.pack(direction)
        recv = self.exchange(send, [int(n) * row_bytes for n in send_rows], [int(n) * row_bytes for n in recv_rows])
        self.engine.unpack(direction, recv)

    def inverse(self, spec, grid):
        """spec holds this rank's wavenumbers (the others are not read); grid
        receives this rank's ring pairs (the others are not written)."""
        self.engine.inv_legendre(spec)
        self._swap(0)
        self.engine.inv_fourier(grid)

    def direct(self, grid, spec):
        """grid holds this rank's ring pairs; spec receives this rank's
        wavenumbers."""
        self.engine.dir_fourier(grid)
        self._swap(1)
        self.engine.dir_legendre(spec)


class LibEngine:
    """The half-transforms of a plan partitioned with st_plan_set_partition."""

    def __init__(self, plan, nranks, rank, m_owner, ring_owner, stream=None):
        import torch

        from . import st

        self.plan, self.nranks, self.rank, self.stream = plan, nranks, rank, stream
        self.lib = st.load()
        mo = np.ascontiguousarray(m_owner, dtype=np.int32)
        ro = np.ascontiguousarray(ring_owner, dtype=np.int32)
        st._check(self.lib.st_plan_set_partition(plan.handle, nranks, rank, mo.ctypes.data_as(ctypes.c_void_p),
                                                 ro.ctypes.data_as(ctypes.c_void_p)))
        self._counts = {}
        self._bufs = {}
        for d in (0, 1):
            s = (ctypes.c_long * nranks)()
            r = (ctypes.c_long * nranks)()
            rb = ctypes.c_int()
            st._check(self.lib.st_exchange_counts(plan.handle, d, s, r, ctypes.byref(rb)))
            self._counts[d] = (list(s), list(r), rb.value)
            self._bufs[d] = torch.empty(max(sum(s) * rb.value, 1), dtype=torch.uint8, device="cuda")

    def _s(self):
        from . import st

        return st._stream(self.stream)

    def counts(self, d):
        return self._counts[d]

    def pack(self, d):
        from . import st

        buf = self._bufs[d]
        st._check(self.lib.st_exchange_pack(self.plan.handle, d, ctypes.c_void_p(buf.data_ptr()), self._s()))
        return buf

    def unpack(self, d, recv):
        from . import st

        st._check(self.lib.st_exchange_unpack(self.plan.handle, d, ctypes.c_void_p(recv.data_ptr()), self._s()))

    def inv_legendre(self, spec):
        from . import st

        st._check(self.lib.st_inv_legendre(self.plan.handle, st._ptr(spec), self._s()))

    def inv_fourier(self, grid):
        from . import st

        st._check(self.lib.st_inv_fourier(self.plan.handle, st._ptr(grid), self._s()))

    def dir_fourier(self, grid):
        from . import st

        st._check(self.lib.st_dir_fourier(self.plan.handle, st._ptr(grid), self._s()))

    def dir_legendre(self, spec):
        from . import st

        st._check(self.lib.st_dir_legendre(self.plan.handle, st._ptr(spec), self._s()))


def torch_exchange(group=None):
    """All-to-all over torch.distributed (byte buffers, byte split sizes).  The
    messages are ordered by the collective itself, which is the overlapped
    per-destination pattern of the paper's Sec. 3.1.3.2."""

    def exchange(send, send_bytes, recv_bytes):
        import torch
        import torch.distributed as dist

        recv = torch.empty(max(sum(recv_bytes), 1), dtype=torch.uint8, device=send.device)
        dist.all_to_all_single(recv[: sum(recv_bytes)], send[: sum(send_bytes)], output_split_sizes=recv_bytes,
                               input_split_sizes=send_bytes, group=group)
        return recv

    return exchange
