"""Algorithm 1 + Eq. 3-12 on the GPU against the oracle (same interior set,
same centres in the same order, shapes to float rounding)."""
import numpy as np
import pytest

from gpu_util import oracle_view, problem, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,layers", [("c1", None), ("c2", [32])])
def test_init_kernels_match_oracle(orc, name, layers):
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build
    build.build()
    pb = problem(name, layers=layers, cap=4096)
    found = pb.init_kernels(gamma=1e-3)
    torch.cuda.synchronize()
    h = oracle_view(pb, orc)
    idx, n = orc.inscribed(h["x"], h["y"], h["z"], h["t"], h["S"])
    assert found == n and pb.m() == n and n > 1
    P = pb.p[:, :n].cpu().numpy()
    np.testing.assert_array_equal(P[0], h["x"][idx])
    np.testing.assert_array_equal(P[1], h["y"][idx])
    np.testing.assert_array_equal(P[2], h["z"][idx])
    np.testing.assert_allclose(P[9], h["t"][idx], rtol=2 ** -23, atol=0)
    assert np.all(P[6:9] == 0)
    c = np.stack([h["x"][idx], h["y"][idx], h["z"][idx]], 1).astype(np.float64)
    d_o = orc.init_shape(c, h["t"][idx].astype(np.float64), np.abs(h["S"][idx]).astype(np.float64), 1e-3)
    for k in (3, 4, 5):
        np.testing.assert_allclose(P[k], d_o, rtol=2e-6)


def test_init_capacity_and_fit(orc):
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build
    build.build()
    pb = problem("c1")  # capacity 64
    found = pb.init_kernels()
    torch.cuda.synchronize()
    assert found > 64 and pb.m() == 64  # the first 64 centres are kept
    pb2 = problem("c1", cap=1024)
    pb2.init_kernels()
    l2 = []
    for _ in range(60):
        pb2.epoch()
        l2.append(pb2.stats[0].item())
    # the fit starts from these kernels (the paper runs 2000 epochs from here)
    assert np.isfinite(l2).all() and min(l2[-10:]) < l2[0]
