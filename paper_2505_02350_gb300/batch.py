"""Many independent fields advanced together.

Every field keeps its own buffers and workspace (field.Problem); one epoch of
the batch runs each field's epoch as a parallel branch on its own stream, and
the whole batch epoch is captured as one CUDA graph, so advancing all fields
is one graph launch per optimiser step.  Fields share nothing, so the results
of each field are the same bits as when it is fitted alone (no floating-point
atomics anywhere on the path).
"""
import torch


class Batch:
    def __init__(self, problems):
        self.pbs = list(problems)
        self.streams = [torch.cuda.Stream(device=pb.dev) for pb in self.pbs]
        self.graph = None

    def _fan_out(self, fn):
        main = torch.cuda.current_stream()
        for st in self.streams:
            st.wait_stream(main)
        for pb, st in zip(self.pbs, self.streams):
            with torch.cuda.stream(st):
                fn(pb)
        for st in self.streams:
            main.wait_stream(st)

    def epoch(self):
        """One Algorithm 3 epoch of every field, the fields concurrently."""
        self._fan_out(lambda pb: pb.epoch())

    def capture(self):
        """Capture one batch epoch as a single CUDA graph (runs one epoch first)."""
        self.epoch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._fan_out(lambda pb: pb.epoch())
        torch.cuda.synchronize()
        self.graph = g
        return g

    def epoch_graph(self):
        self.graph.replay()

    def snapshot(self):
        return [pb.snapshot() for pb in self.pbs]

    def restore(self, snaps):
        for pb, s in zip(self.pbs, snaps):
            pb.restore(s)

    def rmse(self):
        return [pb.rmse() for pb in self.pbs]
