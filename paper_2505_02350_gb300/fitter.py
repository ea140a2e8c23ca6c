"""Algorithm 3 host driver (full batch).

Every epoch is one launch sequence (neighbour rebuild, forward, adjoint,
optimiser step with the gates, deletion, addition) that never waits for the
host; the state machine of Algorithm 3 lives on the device.  The host only
schedules the coarse-to-fine refinement (Sec. 3.4.2: next layer appended at
fixed epochs) and, optionally, reads the per-epoch statistics.
"""
import numpy as np
import torch

from . import _native as N


class Fitter:
    def __init__(self, problem, layers=(), refine_at=(), use_graphs=True):
        """layers: list of (x, y, z, S, t, spacing) appended in order at the epochs in refine_at."""
        self.pb = problem
        self.layers = list(layers)
        self.refine_at = list(refine_at)
        self.use_graphs = use_graphs
        self.history = []
        self._captured = False

    def _refine_if_due(self, epoch):
        if self.layers and self.refine_at and epoch == self.refine_at[0]:
            self.refine_at.pop(0)
            x, y, z, S, t, spacing = self.layers.pop(0)
            self.pb.refine(x, y, z, S, t, spacing=spacing)
            self._captured = False  # the tile layout changed: graphs must be captured again

    def run(self, epochs, log_every=0):
        pb = self.pb
        for e in range(1, epochs + 1):
            self._refine_if_due(e)
            if self.use_graphs:
                if not self._captured:
                    pb.capture()  # also runs this epoch once
                    self._captured = True
                else:
                    pb.epoch_graph()
            else:
                pb.epoch()
            if log_every and e % log_every == 0:
                self.history.append(self.snapshot(e))
        torch.cuda.synchronize()
        return self.history

    def snapshot(self, epoch):
        s = self.pb.stats.cpu().numpy()
        return dict(epoch=epoch, l2=float(s[N.STAT_L2]), count=int(s[N.STAT_COUNT]),
                    max_e=float(s[N.STAT_MAXE]), pairs_fwd=int(s[N.STAT_PAIRS_FWD]),
                    pairs_bwd=int(s[N.STAT_PAIRS_BWD]), alpha=float(s[N.STAT_ALPHA]),
                    b_f=int(s[N.STAT_BF]), m=self.pb.m())

    def rmse(self):
        """Root mean square of E over id_all (Eq. 3-18 filter) after the last forward."""
        s = self.pb.stats.cpu().numpy()
        c = max(float(s[N.STAT_COUNT]), 1.0)
        return float(np.sqrt(s[N.STAT_L2] / c))
