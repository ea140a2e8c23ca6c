"""Algorithm 3 trajectories (parity unpinned: FP32 and FP64 runs drift apart,
so only the outcome is compared).  The device-side driver on the sphere
workload must reduce the loss the way the FP64 oracle's Algorithm 3 does."""
import math

import numpy as np
import pytest

import synth
from gpu_util import oracle_view, torch_cuda

pytestmark = pytest.mark.gpu


def _oracle_run(orc, x, y, z, t, S, P0, m, epochs, cfg_dev):
    cap = P0.shape[1]
    P = P0.astype(np.float64).copy()
    mo = np.zeros_like(P)
    v = np.zeros_like(P)
    cfg = orc.default_cfg()
    st = orc.state_init(cfg)
    hist = []
    r2 = np.float32(cfg_dev.add_radius * cfg_dev.add_radius)
    for e in range(epochs):
        Pf = P[:, :m].astype(np.float32).astype(np.float64)
        psi, err, mask, s = orc.forward(x, y, z, t, Pf, m)
        g, _ = orc.backward(x, y, z, err, Pf, m)
        hist.append(s[0] / max(s[3], 1))
        orc.step(P, m, g, mo, v, s[0], s[2], cfg, st)
        if st.do_prune:
            m = orc.prune(P, m, cfg.tau_d, mo=mo, v=v)
            st.do_prune = 0
        if st.do_add:
            Ef = err.astype(np.float32)
            k = math.ceil(0.01 * s[3])
            cand = orc.select_topk(Ef, mask, cfg.tau_m / 2, k)
            ext = orc.local_max(x, y, z, Ef, mask, cand, r2)
            for i in ext:
                if m >= cap:
                    break
                dbar = max(abs(float(S[i])), cfg_dev.dbar_min)
                P[:, m] = orc.new_kernel((x[i], y[i], z[i]), Ef[i], dbar)
                m += 1
            mo[:] = 0
            v[:] = 0
            st.adam_t = 0
            st.do_add = 0
    return np.array(hist), m


def test_sphere_fit_tracks_oracle(orc):
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build, field
    from paper_2505_02350_gb300.fitter import Fitter
    build.build()
    cfg, lay, P = synth.workload("c1")
    x, y, z, S = lay[0]
    pb = field.Problem(x, y, z, S, P, cfg["m"], synth.spacing(32), cap=256)
    pb.test_src = (x, y, z, S, np.asarray(P, np.float64))
    fit = Fitter(pb)
    hist = fit.run(200, log_every=1)
    msq_gpu = np.array([h["l2"] / max(h["count"], 1) for h in hist])
    assert np.all(np.isfinite(msq_gpu))
    h = oracle_view(pb, orc)
    P0 = np.zeros((10, 256))
    P0[:, :cfg["m"]] = P[:, :cfg["m"]]
    ref, m_or = _oracle_run(orc, h["x"], h["y"], h["z"], h["t"], h["S"], P0, cfg["m"], 200, pb.cfg)
    # the loss falls by the same order of magnitude on both sides; additions
    # make the loss jump for a few epochs at slightly different times, so the
    # best value of the last 40 epochs is compared
    assert msq_gpu[-40:].min() < 0.01 * msq_gpu[0]
    assert ref[-40:].min() < 0.01 * ref[0]
    ratio = msq_gpu[-40:].min() / ref[-40:].min()
    assert 1 / 3 < ratio < 3.0, (msq_gpu[-40:].min(), ref[-40:].min())
    # before the gates fire the two runs agree closely (FP32 vs FP64 drift)
    np.testing.assert_allclose(msq_gpu[:40], ref[:40], rtol=1e-4)


def test_octree_layers_fit():
    """Sec. 3.4.2 on an adaptive octree: initial kernels from the coarsest layer
    (Algorithm 1), finer layers appended at fixed epochs."""
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build, field
    from paper_2505_02350_gb300.fitter import Fitter
    build.build()
    sphere = lambda x, y, z: np.sqrt(x * x + y * y + z * z) - 0.5
    layers = synth.octree_layers(sphere, 4, 6)
    ts = field.normalize_layers([l[3] for l in layers])
    total = sum(l[0].size for l in layers)
    finest = layers[-1][4]
    g = field.grid_for(finest)
    x, y, z, S, _ = layers[0]
    pb = field.Problem(x, y, z, S, np.zeros((10, 2048), np.float32), 0, finest, max_points=total, t=ts[0],
                       cap=2048, max_cells=g.n[0] * g.n[1] * g.n[2])
    found = pb.init_kernels()
    assert 0 < found <= 2048
    more = [(l[0], l[1], l[2], l[3], t, finest) for l, t in zip(layers[1:], ts[1:])]
    fit = Fitter(pb, layers=more, refine_at=[10, 20])
    hist = fit.run(40, log_every=1)
    assert pb.n == total
    msq = [h["l2"] / max(h["count"], 1) for h in hist]
    assert np.isfinite(msq).all() and min(msq[-5:]) < msq[0]


def test_octree_layers_match_oracle_after_each_append(orc):
    """Each octree layer appended to the training set (Sec. 3.4.2): the
    binning of the grown set, its targets and the first forward after the
    append against the oracle -- its own binning, its own Eq. 3-10 map over
    all layers, its own forward with the GPU's current parameters."""
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build, field
    build.build()
    sphere = lambda x, y, z: np.sqrt(x * x + y * y + z * z) - 0.5
    layers = synth.octree_layers(sphere, 4, 6)
    ts = field.normalize_layers([l[3] for l in layers])
    t_or_all, _, _ = orc.normalize(np.concatenate([l[3] for l in layers]))
    t_or_all = t_or_all.astype(np.float32)
    np.testing.assert_allclose(np.concatenate(ts), t_or_all, rtol=2 ** -23, atol=0)
    total = sum(l[0].size for l in layers)
    finest = layers[-1][4]
    g = field.grid_for(finest)
    x, y, z, S, _ = layers[0]
    pb = field.Problem(x, y, z, S, np.zeros((10, 2048), np.float32), 0, finest, max_points=total, t=ts[0],
                       cap=2048, max_cells=g.n[0] * g.n[1] * g.n[2])
    pb.init_kernels()
    for k in range(1, len(layers)):
        for _ in range(10):
            pb.epoch()
        l = layers[k]
        pb.refine(l[0], l[1], l[2], l[3], ts[k], spacing=finest)
        pb.build_neighbors()
        pb.forward()
        torch.cuda.synchronize()
        n, m = pb.n, pb.m()
        xs, ys, zs = (np.concatenate([layers[q][c] for q in range(k + 1)]) for c in range(3))
        perm = orc.bin_points(xs, ys, zs, tuple(pb.grid.origin), pb.grid.h, tuple(pb.grid.n),
                              pb.sizes.super_factor).astype(np.int64)
        np.testing.assert_array_equal(pb.perm[:n].cpu().numpy().astype(np.int64), perm)
        t_or = t_or_all[:n][perm]
        np.testing.assert_allclose(pb.tb[:n].cpu().numpy(), t_or, rtol=2 ** -23, atol=0)
        P = pb.p[:, :m].cpu().numpy().astype(np.float64)
        psi_o, _E, _mask, st = orc.forward(xs[perm], ys[perm], zs[perm], t_or, P, m)
        assert pb.stats[4].item() == st[4]
        assert np.abs(pb.psi[:n].cpu().numpy() - psi_o).max() <= 1e-5 * np.abs(t_or).max()
