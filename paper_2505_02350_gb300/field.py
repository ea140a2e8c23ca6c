"""Device-resident fitting problem: the buffers of one SDF field and the calls
of one optimisation epoch (Algorithm 3, full batch).

PyTorch is only used for device memory and the stream; every step of the
path runs in libserbf.so.  Point arrays are kept twice: in the caller's order
(for refinement) and in binned order (for the kernels).
"""
import math

import numpy as np
import torch

from . import _native as N


def grid_for(spacing, lo=-1.0, hi=1.0, points_per_cell=4):
    """Binning grid whose cells hold points_per_cell^3 points of a vertex grid
    with the given spacing (cell faces fall half-way between grid planes)."""
    h = points_per_cell * spacing
    origin = lo - 0.5 * spacing
    n = int(math.ceil((hi - lo + spacing) / h - 1e-6))
    g = N.Grid()
    for k in range(3):
        g.origin[k] = origin
        g.n[k] = n
    g.h = h
    return g


def normalize_layers(S_layers, device="cuda", mh_out=None):
    """Eq. 3-10 targets of several grid layers from one map (m and h over all
    of them, as the hierarchical training needs).  Returns float32 numpy
    arrays, one per layer; mh_out (a 2-double device tensor) receives (m, h)."""
    sizes = [len(S) for S in S_layers]
    S = torch.as_tensor(np.concatenate([np.asarray(v, np.float32) for v in S_layers]), device=device)
    t = torch.zeros_like(S)
    mh = torch.zeros(2, dtype=torch.float64, device=device)
    N.serbf_normalize_sdf_noalloc(S, t, mh)
    if mh_out is not None:
        mh_out.copy_(mh)
    t = t.cpu().numpy()
    return list(np.split(t, np.cumsum(sizes)[:-1]))


class Problem:
    """One field: training points, targets, kernels, optimiser state and scratch."""

    def __init__(self, x, y, z, S, P, m, spacing, cfg=None, cap=None, max_points=None, t=None,
                 super_cap=8192, super_factor=4, max_cells=None, device="cuda", fused=True):
        dev = torch.device(device)
        self.dev = dev
        self.fused = fused  # epochs use the one-pass forward + adjoint
        self.cfg = cfg if cfg is not None else N.config_default()
        if self.cfg.add_radius == 0.0:
            self.cfg.add_radius = 2.0 * spacing
        if self.cfg.dbar_min == 0.0:
            self.cfg.dbar_min = 0.5 * spacing
        n = int(len(x))
        self.cap = int(cap if cap is not None else max(P.shape[1], m))
        self.max_points = int(max_points if max_points is not None else n)
        self.spacing = spacing
        self.grid = grid_for(spacing)
        f32 = dict(dtype=torch.float32, device=dev)
        self.x_all = torch.zeros(self.max_points, **f32)
        self.y_all = torch.zeros(self.max_points, **f32)
        self.z_all = torch.zeros(self.max_points, **f32)
        self.t_all = torch.zeros(self.max_points, **f32)
        self.s_all = torch.zeros(self.max_points, **f32)
        self.n = n
        self.x_all[:n] = torch.as_tensor(np.asarray(x, np.float32), device=dev)
        self.y_all[:n] = torch.as_tensor(np.asarray(y, np.float32), device=dev)
        self.z_all[:n] = torch.as_tensor(np.asarray(z, np.float32), device=dev)
        self.s_all[:n] = torch.as_tensor(np.asarray(S, np.float32), device=dev)
        self.mh = torch.zeros(2, dtype=torch.float64, device=dev)
        self.perm = torch.zeros(self.max_points, dtype=torch.int32, device=dev)
        # binned x, y, z, t, S_raw as rows of one block (rows 256-byte
        # aligned), so that one copy can move the training points of a step
        stride = -(-self.max_points // 64) * 64
        self.binned = torch.zeros(5, stride, **f32)
        self.xb, self.yb, self.zb, self.tb, self.sb = self.binned[:, :self.max_points].unbind(0)
        self.psi = torch.zeros(self.max_points, **f32)
        self.err = torch.zeros(self.max_points, **f32)
        self.mask = torch.zeros(self.max_points, dtype=torch.uint8, device=dev)
        Pp = np.zeros((10, self.cap), np.float32)
        Pp[:, :m] = np.asarray(P, np.float32)[:, :m]
        self.p = torch.as_tensor(Pp, device=dev).contiguous()
        self.m_dev = torch.tensor([m], dtype=torch.int32, device=dev)
        self.adam_m = torch.zeros(10, self.cap, **f32)
        self.adam_v = torch.zeros(10, self.cap, **f32)
        self.grad = torch.zeros(10, self.cap, **f32)
        self.state = torch.zeros(N.STATE_BYTES, dtype=torch.uint8, device=dev)
        self.stats = torch.zeros(N.NSTATS, dtype=torch.float64, device=dev)
        ncell = self.grid.n[0] * self.grid.n[1] * self.grid.n[2]
        ncell = max(ncell, int(max_cells or 0))
        self.sizes = N.WsSizes(self.max_points, self.cap, ncell, 0, super_cap, super_factor, 0)
        nbytes = N.serbf_workspace_bytes(self.sizes)
        self.ws_dev = torch.zeros(nbytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.ws_dev.data_ptr()) % 256
        self.ws_view = self.ws_dev[off:off + nbytes]
        self.ws = N.workspace_struct()
        N.serbf_workspace_init(self.ws, self.ws_view, self.sizes)
        N.serbf_state_init(self.state, self.cfg)
        if t is None:
            N.serbf_normalize_sdf(self.s_all[:n], self.t_all[:n], self.mh, self.ws)
        else:
            self.t_all[:n] = torch.as_tensor(np.asarray(t, np.float32), device=dev)
        self.bin()

    def close(self):
        """Release the workspace's CUDA objects (the device buffers are torch's)."""
        if getattr(self, "ws", None) is not None and self.ws_dev is not None:
            torch.cuda.synchronize(self.dev)
            N.serbf_workspace_release(self.ws)
            self.ws_dev = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ structure
    def bin(self):
        n = self.n
        N.serbf_bin_points(self.x_all[:n], self.y_all[:n], self.z_all[:n], self.grid, self.perm[:n],
                           self.xb[:n], self.yb[:n], self.zb[:n], self.ws)
        N.serbf_gather(self.t_all, self.perm[:n], self.tb, n)
        N.serbf_gather(self.s_all, self.perm[:n], self.sb, n)

    def refine(self, x, y, z, S, t, spacing=None):
        """Sec. 3.4.2: append the next layer (its targets t from the global Eq. 3-10 map)."""
        n_new = int(len(x))
        if spacing is not None and spacing < self.spacing:
            self.spacing = spacing
            g = grid_for(spacing)
            ncell = g.n[0] * g.n[1] * g.n[2]
            if ncell > self.sizes.max_cells:
                raise ValueError("refined grid needs a workspace with max_cells >= %d" % ncell)
            self.grid = g
        dev = self.dev
        tt = lambda a: torch.as_tensor(np.asarray(a, np.float32), device=dev)
        N.serbf_refine(self.x_all, self.y_all, self.z_all, self.t_all, self.s_all, self.n, tt(x), tt(y), tt(z),
                       tt(t), tt(S), self.grid, self.perm, self.xb, self.yb, self.zb, self.tb, self.sb, self.ws)
        self.n += n_new

    @property
    def pts(self):
        n = self.n
        return N.points(self.xb[:n], self.yb[:n], self.zb[:n], self.tb[:n], n)

    @property
    def prm(self):
        return N.params(self.p, self.m_dev)

    def init_kernels(self, gamma=1e-3):
        """Replace the kernels by Algorithm 1 + Eq. 3-12 on the current training
        points (fresh Adam moments).  Returns the number of centres found
        (kernels beyond the capacity are dropped)."""
        n = self.n
        _rc, found = N.serbf_init_kernels(self.pts, self.sb[:n], gamma, self.prm, self.ws)
        self.adam_m.zero_()
        self.adam_v.zero_()
        return found

    # ------------------------------------------------------------ hot path
    def build_neighbors(self, kmajor=None, pmajor=None):
        return N.serbf_build_neighbors(self.pts, self.prm, self.cfg, self.ws, kmajor, pmajor)

    def forward(self):
        n = self.n
        N.serbf_forward(self.pts, self.prm, self.cfg, self.psi[:n], self.err[:n], self.mask[:n], self.stats,
                        self.ws)

    def forward_backward(self):
        """Forward and the adjoint of its own residual in one pass."""
        n = self.n
        N.serbf_forward_backward(self.pts, self.prm, self.cfg, self.psi[:n], self.err[:n], self.mask[:n],
                                 self.grad, self.stats, self.ws)

    def backward(self, err=None):
        n = self.n
        N.serbf_backward(self.pts, self.prm, self.cfg, self.err[:n] if err is None else err, self.grad,
                         self.stats, self.ws)

    def step(self):
        N.serbf_step(self.prm, self.grad, self.adam_m, self.adam_v, self.state, self.stats, self.cfg, self.ws)

    def prune(self):
        N.serbf_prune(self.prm, self.adam_m, self.adam_v, self.state, self.cfg)

    def add(self, force=False):
        n = self.n
        N.serbf_add_kernels(self.pts, self.sb[:n], self.err[:n], self.mask[:n], self.prm, self.adam_m,
                            self.adam_v, self.state, self.stats, self.cfg, self.ws, force=force)

    def autotune(self, reps=5):
        """Times the forward (+ adjoint when fused) with 1, 2, 4 and 8 warps per
        work item on the current parameters and keeps the fastest in
        cfg.fwd_warps.  Returns {warps: ms per call}.  Parameters are not
        changed; the outputs of the last call are left in psi/err/grad."""
        fn = self.forward_backward if self.fused else self.forward
        self.build_neighbors()
        times = {}
        for g in (1, 2, 4, 8):
            self.cfg.fwd_warps = g
            fn()  # files the work costs for this configuration's order
            torch.cuda.synchronize(self.dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize(self.dev)
            times[g] = e0.elapsed_time(e1) / reps
        self.cfg.fwd_warps = min(times, key=times.get)
        return times

    def launches_per_epoch(self):
        """Kernel launches of one fused full-batch epoch: item order (2, side
        stream), rebuild (1; 2 when the library builds the candidate lists
        in two levels: cfg.rebuild_levels >= 2, or 0 with super cells x
        kernel capacity >= 2^25 on a grid whose blocks of 2 x 2 x 2 super
        cells fit the workspace; 3 in three levels: cfg.rebuild_levels == 3,
        or 0 with those blocks x capacity >= 2^25 as well), forward + finish
        (2), step (2), deletion (1), addition (3)."""
        sf = self.sizes.super_factor
        ns = [(self.grid.n[k] + sf - 1) // sf for k in range(3)]
        nsuper = ns[0] * ns[1] * ns[2]
        ncoarse = ((ns[0] + 1) // 2) * ((ns[1] + 1) // 2) * ((ns[2] + 1) // 2)
        ntop = ((ns[0] + 3) // 4) * ((ns[1] + 3) // 4) * ((ns[2] + 3) // 4)
        lv = self.cfg.rebuild_levels
        two = (lv >= 2 or (lv == 0 and nsuper * self.cap >= 1 << 25)) and ncoarse <= nsuper // 4 + 16
        three = two and (lv == 3 or (lv == 0 and ncoarse * self.cap >= 1 << 25)) and ntop <= nsuper
        return 11 + (1 if two else 0) + (1 if three else 0)

    def epoch(self):
        """One Algorithm 3 epoch with the full batch: no host synchronisation."""
        self.build_neighbors()
        if self.fused:
            self.forward_backward()
        else:
            self.forward()
            self.backward()
        self.step()
        self.prune()
        self.add()

    def capture(self, split=True):
        """Capture one epoch as CUDA graphs: three (neighbour rebuild | forward
        and adjoint | step, deletion, addition) with split=True, else one, so
        that a step is one to three graph launches.  Re-capture after binning
        changes (refinement)."""
        self.epoch()  # warm up: lazy attribute setup happens outside capture
        torch.cuda.synchronize()
        if not split:
            parts = [self.epoch]
        elif self.fused:
            parts = [self.build_neighbors, self.forward_backward, lambda: (self.step(), self.prune(), self.add())]
        else:
            parts = [self.build_neighbors, self.forward,
                     lambda: (self.backward(), self.step(), self.prune(), self.add())]
        self.graphs = []
        for fn in parts:
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                fn()
            self.graphs.append(g)
        torch.cuda.synchronize()
        return self.graphs

    # ------------------------------------------------------------ snapshots
    def snapshot(self):
        """Device copies of everything an epoch changes (parameters, Adam
        moments, optimiser state, kernel count)."""
        return [t.clone() for t in (self.p, self.adam_m, self.adam_v, self.state, self.m_dev)]

    def restore(self, snap):
        for dst, src in zip((self.p, self.adam_m, self.adam_v, self.state, self.m_dev), snap):
            dst.copy_(src)

    def rmse(self):
        """Root mean square of E over id_all after the last forward."""
        s = self.stats.cpu().numpy()
        return float(np.sqrt(s[N.STAT_L2] / max(float(s[N.STAT_COUNT]), 1.0)))

    def epoch_graph(self):
        for g in self.graphs:
            g.replay()

    # ------------------------------------------------------------ host views
    def status(self, clear=False):
        return N.serbf_status(self.ws, clear=clear)

    def m(self):
        return int(self.m_dev.item())

    def params_host(self):
        return self.p[:, :self.m()].cpu().numpy()

    def state_host(self):
        st = N.State()
        b = self.state.cpu().numpy().tobytes()
        import ctypes
        ctypes.memmove(ctypes.addressof(st), b, len(b))
        return st

    def binned_host(self):
        n = self.n
        return dict(x=self.xb[:n].cpu().numpy(), y=self.yb[:n].cpu().numpy(), z=self.zb[:n].cpu().numpy(),
                    t=self.tb[:n].cpu().numpy(), S=self.sb[:n].cpu().numpy(),
                    perm=self.perm[:n].cpu().numpy().astype(np.int64))


class MiniBatch:
    """Algorithm 3 with mini-batches of training points (the paper's B_s).

    Every epoch the training points are shuffled (seeded permutation) and cut
    into batches of `batch_size`; each batch is gathered, binned into a small
    workspace of its own, and taken through the fused forward + adjoint and
    one optimiser step on the parent problem's parameters, Adam moments and
    state (cfg.epoch_steps = batches per epoch, so the gates run after the
    epoch's last batch on the summed batch L2).  After the epoch: deletion
    and, when due, the addition, whose residuals come from a forward over all
    training points with the epoch's final parameters.
    """

    def __init__(self, problem, batch_size, seed=0):
        pb = problem
        self.pb = pb
        self.bs = int(batch_size)
        self.rng = np.random.default_rng(seed)
        dev = pb.dev
        f32 = dict(dtype=torch.float32, device=dev)
        B = self.bs
        self.idx = torch.zeros(pb.max_points, dtype=torch.int32, device=dev)
        self.raw = [torch.zeros(B, **f32) for _ in range(4)]  # x, y, z, t in batch order
        self.perm = torch.zeros(B, dtype=torch.int32, device=dev)
        self.xb, self.yb, self.zb, self.tb = (torch.zeros(B, **f32) for _ in range(4))
        self.psi, self.err = torch.zeros(B, **f32), torch.zeros(B, **f32)
        self.mask = torch.zeros(B, dtype=torch.uint8, device=dev)
        sz = N.WsSizes(B, pb.cap, pb.sizes.max_cells, 0, pb.sizes.super_cap, pb.sizes.super_factor, 0)
        nbytes = N.serbf_workspace_bytes(sz)
        self.ws_dev = torch.zeros(nbytes + 256, dtype=torch.uint8, device=dev)
        off = (-self.ws_dev.data_ptr()) % 256
        self.ws = N.workspace_struct()
        N.serbf_workspace_init(self.ws, self.ws_dev[off:off + nbytes], sz)
        self.cfg = N.Config.from_buffer_copy(pb.cfg)
        self.batches = []  # host copies of the last epoch's batches (binned indices of the parent)

    def close(self):
        if self.ws_dev is not None:
            torch.cuda.synchronize(self.pb.dev)
            N.serbf_workspace_release(self.ws)
            self.ws_dev = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def epoch(self):
        pb, B = self.pb, self.bs
        n = pb.n
        order = self.rng.permutation(n).astype(np.int32)
        self.idx[:n] = torch.as_tensor(order, device=pb.dev)
        nb = (n + B - 1) // B
        self.batches = [order[b * B:min(n, (b + 1) * B)] for b in range(nb)]
        cfg = self.cfg
        cfg.epoch_steps = nb
        for b in range(nb):
            i0, k = b * B, min(n, (b + 1) * B) - b * B
            sel = self.idx[i0:i0 + k]
            for src, dst in zip((pb.xb, pb.yb, pb.zb, pb.tb), self.raw):
                N.serbf_gather(src, sel, dst, k)
            N.serbf_bin_points(self.raw[0][:k], self.raw[1][:k], self.raw[2][:k], pb.grid, self.perm[:k],
                               self.xb[:k], self.yb[:k], self.zb[:k], self.ws)
            N.serbf_gather(self.raw[3], self.perm[:k], self.tb, k)
            pts = N.points(self.xb[:k], self.yb[:k], self.zb[:k], self.tb[:k], k)
            N.serbf_build_neighbors(pts, pb.prm, cfg, self.ws)
            N.serbf_forward_backward(pts, pb.prm, cfg, self.psi[:k], self.err[:k], self.mask[:k], pb.grad,
                                     pb.stats, self.ws)
            N.serbf_step(pb.prm, pb.grad, pb.adam_m, pb.adam_v, pb.state, pb.stats, cfg, pb.ws)
        pb.prune()
        if pb.state_host().do_add:
            pb.build_neighbors()
            pb.forward()
            pb.add()


def surface_metrics(problem, sdf, n=129, samples=100000, seed=0, mh=None):
    """Sec. 4 evaluation of a fit against a closed-form SDF: the fitted field
    on an n^3 vertex grid over [-1, 1]^3 mapped back to distances (inverse of
    Eq. 3-10 with the training map (m, h)), the zero level sets of it and of
    the true SDF on the same grid (marching tetrahedra), `samples` area-
    weighted points on each, and (HD, CD, CS).  sdf maps float64 arrays
    (x, y, z) to distances."""
    import synth
    dev = problem.dev
    mh = problem.mh if mh is None else mh
    x, y, z = synth.grid(n)
    S_true = np.asarray(sdf(x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)), np.float32)
    m = problem.m()
    ev = Problem(x, y, z, S_true, problem.p[:, :m].cpu().numpy(), m, synth.spacing(n), cap=max(m, 1), device=dev)
    ev.build_neighbors()
    ev.forward()
    N_ = ev.n
    psi = torch.zeros(N_, dtype=torch.float32, device=dev)
    N.serbf_scatter(ev.psi[:N_], ev.perm[:N_], psi, N_)
    S_pred = torch.zeros_like(psi)
    N.serbf_denormalize_sdf(psi, S_pred, N_, mh)
    ev.close()
    out = []
    rng = np.random.default_rng(seed)
    dims, origin, h = (n, n, n), (-1.0, -1.0, -1.0), float(synth.spacing(n))
    scratch = torch.zeros((n - 1) ** 3 + 1, dtype=torch.int64, device=dev)
    for field_ in (torch.as_tensor(S_true, device=dev), S_pred):
        _rc, nt = N.serbf_marching_tets(field_, dims, origin, h, 0.0, None, 0, scratch)
        tri = torch.zeros(max(nt, 1), 9, dtype=torch.float32, device=dev)
        N.serbf_marching_tets(field_, dims, origin, h, 0.0, tri, nt, scratch)
        u = torch.as_tensor(rng.uniform(size=(samples, 3)), device=dev)
        pts = torch.zeros(samples, 3, dtype=torch.float32, device=dev)
        nrm = torch.zeros_like(pts)
        cum = torch.zeros(nt + 1, dtype=torch.int64, device=dev)
        N.serbf_sample_surface(tri, nt, u, samples, pts, nrm, cum)
        out.append((pts, nrm))
    scr = torch.zeros(4 * samples + 6, dtype=torch.float64, device=dev)
    (A, nA), (B, nB) = out
    return N.serbf_surface_metrics(A, nA, samples, B, nB, samples, scr)
