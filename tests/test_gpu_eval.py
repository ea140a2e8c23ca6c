"""Surface extraction, sampling and the Sec. 4 metrics on the GPU against the
oracle (bit-exact triangles and samples, metrics to summation rounding),
and an end-to-end evaluation of a fit."""
import numpy as np
import pytest

import synth
from gpu_util import problem, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = torch_cuda()
    from paper_2505_02350_gb300 import build
    build.build()
    return t


def _torus(x, y, z):
    q = np.sqrt(x * x + y * y) - 0.5
    return np.sqrt(q * q + z * z) - 0.2


def _extract(torch, N, f, n):
    dims, origin, h = (n, n, n), (-1.0, -1.0, -1.0), float(synth.spacing(n))
    fd = torch.as_tensor(f, device="cuda")
    scratch = torch.zeros((n - 1) ** 3 + 1, dtype=torch.int64, device="cuda")
    _rc, nt = N.serbf_marching_tets(fd, dims, origin, h, 0.0, None, 0, scratch)
    tri = torch.zeros(nt, 9, dtype=torch.float32, device="cuda")
    rc, nt2 = N.serbf_marching_tets(fd, dims, origin, h, 0.0, tri, nt, scratch)
    assert rc == N.SERBF_OK and nt2 == nt
    return tri


def test_marching_tets_sampling_metrics_match_oracle(torch, orc):
    from paper_2505_02350_gb300 import _native as N
    n = 33
    x, y, z = synth.grid(n)
    f = _torus(x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)).astype(np.float32)
    g = f + np.float32(0.01) * np.sin(7 * x).astype(np.float32)  # a perturbed copy
    tri = _extract(torch, N, f, n)
    tri_o = orc.marching_tets(f, (n, n, n), (-1, -1, -1), 2.0 / (n - 1))
    np.testing.assert_array_equal(tri.cpu().numpy(), tri_o)
    tri2 = _extract(torch, N, g, n)
    ns = 3000
    rng = np.random.default_rng(3)
    res = []
    for t_dev, t_host in ((tri, tri_o), (tri2, tri2.cpu().numpy())):
        u = rng.uniform(size=(ns, 3))
        ud = torch.as_tensor(u, device="cuda")
        pts = torch.zeros(ns, 3, dtype=torch.float32, device="cuda")
        nrm = torch.zeros_like(pts)
        cum = torch.zeros(t_dev.shape[0] + 1, dtype=torch.int64, device="cuda")
        N.serbf_sample_surface(t_dev, t_dev.shape[0], ud, ns, pts, nrm, cum)
        p_o, n_o = orc.sample_surface(t_host, u)
        np.testing.assert_array_equal(pts.cpu().numpy(), p_o)
        np.testing.assert_array_equal(nrm.cpu().numpy(), n_o)
        res.append((pts, nrm, p_o, n_o))
    (A, nA, Ao, nAo), (B, nB, Bo, nBo) = res
    scr = torch.zeros(4 * ns + 6, dtype=torch.float64, device="cuda")
    hd, cd, cs = N.serbf_surface_metrics(A, nA, ns, B, nB, ns, scr)
    hd_o, cd_o, cs_o = orc.surface_metrics(Ao, nAo, Bo, nBo)
    assert hd == hd_o
    assert cd == pytest.approx(cd_o, rel=1e-12) and cs == pytest.approx(cs_o, rel=1e-12)
    assert 0 < cd < hd < 0.2 and 0.9 < cs <= 1.0  # sparse samples: HD is dominated by their spacing


def test_denormalize_inverts_eq3_10(torch, orc):
    from paper_2505_02350_gb300 import _native as N
    S = np.linspace(-0.4, 0.6, 1001).astype(np.float32)
    t, m, h = orc.normalize(S)
    td = torch.as_tensor(t.astype(np.float32), device="cuda")
    Sd = torch.zeros_like(td)
    mh = torch.tensor([m, h], dtype=torch.float64, device="cuda")
    N.serbf_denormalize_sdf(td, Sd, S.size, mh)
    back = Sd.cpu().numpy()
    keep = S > m + 0.05  # away from the flat top of the map at S = m
    np.testing.assert_allclose(back[keep], S[keep], atol=2e-5)


def test_fit_surface_metrics(torch):
    from paper_2505_02350_gb300 import field
    pb = problem("c1", cap=256)
    for _ in range(150):
        pb.epoch()
    torch.cuda.synchronize()
    sphere = lambda x, y, z: np.sqrt(x * x + y * y + z * z) - 0.5
    hd, cd, cs = field.surface_metrics(pb, sphere, n=65, samples=20000)
    assert np.isfinite([hd, cd, cs]).all()
    assert cd < 0.05 and cs > 0.8
