"""Many independent fields advanced together through the batched C ABI.

Every field keeps its own buffers and workspace (field.Problem).  One epoch
of the batch is serbf_epoch_batched: a fixed number of launches for all
fields, the fused forward + adjoint of every field being one persistent
launch that takes (field, work item) pairs from a single counter.  An epoch
is captured as one CUDA graph.  A field's results are the same bits as its
single-field epochs with the same warps per item (no floating-point atomics
on the path).
"""
import ctypes as C

import torch

from . import _native as N


class Batch:
    def __init__(self, problems, fwd_warps=0):
        self.pbs = list(problems)
        self.dev = self.pbs[0].dev
        self.graph = None
        self._init(fwd_warps)

    def _init(self, fwd_warps):
        """(Re)records every field's arguments; needed again after a field is re-binned."""
        fields = []
        for pb in self.pbs:
            n = pb.n
            fields.append(N.Field(pb.pts, C.c_void_p(pb.sb[:n].data_ptr()), C.c_void_p(pb.psi.data_ptr()),
                                  C.c_void_p(pb.err.data_ptr()), C.c_void_p(pb.mask.data_ptr()), pb.prm,
                                  C.c_void_p(pb.grad.data_ptr()), C.c_void_p(pb.adam_m.data_ptr()),
                                  C.c_void_p(pb.adam_v.data_ptr()), C.c_void_p(pb.state.data_ptr()),
                                  C.c_void_p(pb.stats.data_ptr()), C.pointer(pb.cfg), C.addressof(pb.ws)))
        nbytes = N.serbf_batch_bytes(len(fields))
        self.tables = torch.zeros(nbytes + 256, dtype=torch.uint8, device=self.dev)
        off = (-self.tables.data_ptr()) % 256
        self.b = N.batch_struct()
        N.serbf_batch_init(self.b, fields, fwd_warps, self.tables[off:off + nbytes])
        self.fwd_warps = N.serbf_batch_warps(self.b)
        self.graph = None

    def epoch(self):
        """One Algorithm 3 epoch of every field."""
        N.serbf_epoch_batched(self.b)

    def capture(self):
        """Capture one batch epoch as a CUDA graph (runs one epoch first)."""
        self.epoch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.epoch()
        torch.cuda.synchronize()
        self.graph = g
        return g

    def epoch_graph(self):
        self.graph.replay()

    def autotune(self, reps=5):
        """Times the batched epoch with 1, 2, 4 and 8 warps per forward work
        item (parameters restored after each) and keeps the fastest.
        Returns {warps: ms per epoch}."""
        snap = self.snapshot()
        times = {}
        for g in (1, 2, 4, 8):
            self._init(g)
            self.epoch()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                self.epoch()
            e1.record()
            torch.cuda.synchronize()
            times[g] = e0.elapsed_time(e1) / reps
            self.restore(snap)
        self._init(min(times, key=times.get))
        return times

    def snapshot(self):
        return [pb.snapshot() for pb in self.pbs]

    def restore(self, snaps):
        for pb, s in zip(self.pbs, snaps):
            pb.restore(s)

    def rmse(self):
        return [pb.rmse() for pb in self.pbs]
