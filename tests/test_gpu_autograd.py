"""torch.autograd.Function around the forward and adjoint kernels (torus
workload, anisotropic rotated kernels): gradients against central finite
differences (h = 1e-3) of the GPU forward, and against the FP64 oracle."""
import numpy as np
import pytest

from gpu_util import host_params, oracle_view, problem, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build
    build.build()
    pb = problem("c2", layers=[32])
    return torch, pb


def _upstream(torch, pb, seed=0):
    g = np.random.default_rng(seed).normal(0, 1, pb.n).astype(np.float32)
    return torch.as_tensor(g, device="cuda")


def test_autograd_matches_oracle(setup, orc):
    torch, pb = setup
    from paper_2505_02350_gb300.autograd import erbf_field
    m = pb.m()
    p = pb.p.clone().requires_grad_(True)
    w = _upstream(torch, pb)
    psi = erbf_field(pb, p)
    (psi * w).sum().backward()
    h = oracle_view(pb, orc)
    P = host_params(pb)
    g_o, _ = orc.backward(h["x"], h["y"], h["z"], 0.5 * w.cpu().numpy().astype(np.float64), P, m)
    g = p.grad[:, :m].cpu().numpy()
    for sl in (slice(0, 3), slice(3, 6), slice(6, 9), slice(9, 10)):
        assert rel_l2(g[sl], g_o[sl]) <= 1e-4


def test_autograd_matches_central_differences(setup):
    torch, pb = setup
    from paper_2505_02350_gb300.autograd import erbf_field
    p0 = pb.p.clone()
    p = p0.clone().requires_grad_(True)
    w = _upstream(torch, pb, seed=1)
    (erbf_field(pb, p) * w).sum().backward()
    grad = p.grad.clone()
    wd = w.double()
    hstep = 1e-3
    rng = np.random.default_rng(2)
    js = rng.choice(pb.m(), 6, replace=False)
    for r in range(10):
        for j in js:
            pp = p0.clone()
            pp[r, j] += hstep
            fp = erbf_field(pb, pp).double()
            pm = p0.clone()
            pm[r, j] -= hstep
            fm = erbf_field(pb, pm).double()
            fd = float(((fp - fm) * wd).sum()) / (2 * hstep)
            an = float(grad[r, j])
            assert abs(an - fd) <= 2e-2 * max(abs(fd), 1.0), (r, int(j), an, fd)
    pb.p.copy_(p0)
