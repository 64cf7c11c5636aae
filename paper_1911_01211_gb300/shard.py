"""k-point sharding over ranks: the exchange that ng_run_2b_sharded calls (Sec. "MPI
parallelization", Eq. dyson_kspace).

Each rank owns whole blocks of 32 consecutive k-points (``ng_shard_plan``) and calls
``Context.run_2b_sharded`` with an exchange object.  The library asks the exchange for one
operation only: an allgather of the first ``bytes`` of every rank's send buffer into the
receive buffer, rank by rank.  This module provides it in two forms; neither does any of the
method's arithmetic, they only move bytes between the ranks' device buffers.

``DistExchange``   torch.distributed (NCCL between GPUs, gloo between CPU processes); the
                   collective is issued on torch's current stream, which must be the stream
                   the run was given (the binding's default).
``ThreadExchange`` several ranks as host threads of one process sharing one GPU, for tests:
                   each rank's call synchronises its stream, meets the others at a barrier,
                   copies every rank's send buffer and synchronises again.  No kernel waits on
                   another; only the host threads wait.
"""
import ctypes
import threading

import torch

from . import EXCHANGE_FN, ng_shard, shard_plan


class _ExchangeBase:
    def __init__(self, nk, rank, nranks, grid, device):
        self.nk, self.rank, self.nranks = nk, rank, nranks
        self.k_begin, self.k_count, nbytes = shard_plan(nk, rank, nranks, grid)
        n = (nbytes + 15) // 16 * 2              # float64 elements, 16-byte multiple
        self.send = torch.zeros(n, dtype=torch.float64, device=device)
        self.recv = torch.zeros(nranks * n, dtype=torch.float64, device=device)
        self.send_bytes = n * 8
        self.error = None
        self._cb = EXCHANGE_FN(self._callback)

    def _callback(self, user, nbytes):
        try:
            self.allgather(nbytes)
            return 0
        except Exception as e:       # reported to the caller after the run returns
            self.error = e
            return 1

    def c(self):
        return ng_shard(self.nk, self.rank, self.nranks, ctypes.c_void_p(self.send.data_ptr()), self.send_bytes,
                        ctypes.c_void_p(self.recv.data_ptr()), self._cb, None)

    def allgather(self, nbytes):
        raise NotImplementedError


class DistExchange(_ExchangeBase):
    """Allgather through the default torch.distributed process group."""

    def __init__(self, nk, grid, device, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        super().__init__(nk, dist.get_rank(group), dist.get_world_size(group), grid, device)

    def allgather(self, nbytes):
        n = nbytes // 8
        out = self.recv[:self.nranks * n]
        inp = self.send[:n]
        try:
            self.dist.all_gather_into_tensor(out, inp, group=self.group)
        except (RuntimeError, AttributeError, NotImplementedError):
            # process groups without the fused form: gather into the chunks of the same buffer
            self.dist.all_gather(list(out.view(self.nranks, n).unbind(0)), inp, group=self.group)


class ThreadExchange(_ExchangeBase):
    """One rank of a group of host threads sharing a device (see the module docstring)."""

    class Group:
        def __init__(self, nranks, timeout=600.0):
            self.nranks = nranks
            self.barrier = threading.Barrier(nranks, timeout=timeout)
            self.members = [None] * nranks

    def __init__(self, group, nk, rank, grid, device="cuda"):
        super().__init__(nk, rank, group.nranks, grid, device)
        self.group = group
        group.members[rank] = self

    def allgather(self, nbytes):
        n = nbytes // 8
        try:
            torch.cuda.current_stream().synchronize()
            self.group.barrier.wait()
            for r, m in enumerate(self.group.members):
                self.recv[r * n:(r + 1) * n].copy_(m.send[:n])
            torch.cuda.current_stream().synchronize()
            self.group.barrier.wait()
        except Exception:
            self.group.barrier.abort()      # the other ranks' waits end with BrokenBarrierError
            raise
