"""Algorithm 3 with mini-batches: the GPU driver against the oracle taking
the same batches (the seeded permutation is drawn on the host and handed to
both)."""
import numpy as np
import pytest

from gpu_util import host_params, oracle_view, problem, torch_cuda

pytestmark = pytest.mark.gpu


def test_minibatch_epochs_track_oracle(orc):
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build, field
    build.build()
    pb = problem("c1")
    mb = field.MiniBatch(pb, 8192, seed=5)
    h = oracle_view(pb, orc)
    m, cap = pb.m(), pb.cap
    Po = pb.p.cpu().numpy().astype(np.float64)
    mo, v = np.zeros((10, cap)), np.zeros((10, cap))
    ocfg = orc.default_cfg(epoch_steps=4)
    ost = orc.state_init(ocfg)
    for e in range(3):
        mb.epoch()
        torch.cuda.synchronize()
        assert len(mb.batches) == 4 and sum(len(b) for b in mb.batches) == pb.n
        for bidx in mb.batches:
            x, y, z, t = (h[k][bidx] for k in ("x", "y", "z", "t"))
            _psi, err, _mask, st = orc.forward(x, y, z, t, Po, m)
            g, _ = orc.backward(x, y, z, err, Po, m)
            orc.step(Po, m, g, mo, v, st[0], st[2], ocfg, ost)
        s = pb.state_host()
        assert (s.epoch, s.adam_t, s.step, s.l1_optim) == (ost.epoch, ost.adam_t, ost.step, ost.l1_optim) == \
            (e + 1, 4 * (e + 1), 0, 0)
        # centres, axis parameters and weights; the angles of these isotropic
        # kernels have an exactly zero gradient, which Adam turns into unit
        # steps of rounding noise on the GPU, and they do not change Psi
        rows = [0, 1, 2, 3, 4, 5, 9]
        P = host_params(pb)
        np.testing.assert_allclose(P[rows], Po[rows, :m], rtol=2e-4, atol=2e-6)
        assert s.l2_hist[e] == pytest.approx(ost.l2_hist[e], rel=1e-3)
    mb.close()
