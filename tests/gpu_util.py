"""Helpers shared by the GPU parity tests: build problems from the seeded
synthetic inputs, and give the oracle its own copy of those inputs in the
binned order (binned by the oracle, targets normalised by the oracle), so
that no oracle input comes from the GPU path."""
import numpy as np

import synth


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def problem(name, layers=None, cap=None, **kw):
    """A Problem on the union of the requested layers of a named workload."""
    from paper_2505_02350_gb300 import field
    cfg, lay, P = synth.workload(name, layers=layers)
    x = np.concatenate([l[0] for l in lay])
    y = np.concatenate([l[1] for l in lay])
    z = np.concatenate([l[2] for l in lay])
    S = np.concatenate([l[3] for l in lay])
    grids = cfg["grids"] if layers is None else layers
    spacing = synth.spacing(max(grids))
    m = cfg["m"]
    pb = field.Problem(x, y, z, S, P, m, spacing, cap=cap or m, **kw)
    pb.test_src = (x, y, z, S, np.asarray(P, np.float64))
    return pb


def oracle_view(pb, orc):
    """The problem's inputs as the oracle sees them: binned with the oracle's
    binning (which must give the GPU's permutation -- checked), targets from
    the oracle's Eq. 3-10.  Returns dict(x, y, z, t, S) in binned order."""
    x, y, z, S, _ = pb.test_src
    g = pb.grid
    perm = orc.bin_points(x, y, z, tuple(g.origin), g.h, tuple(g.n), pb.sizes.super_factor).astype(np.int64)
    gpu_perm = pb.perm[:pb.n].cpu().numpy().astype(np.int64)
    assert np.array_equal(perm, gpu_perm), "binning differs from the oracle's"
    t, _, _ = orc.normalize(S)
    t = t.astype(np.float32)
    return dict(x=x[perm], y=y[perm], z=z[perm], t=t[perm], S=S[perm])


def host_params(pb):
    return pb.p[:, :pb.m()].detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def per_kernel_errors(g, g_o, groups=((0, 3), (3, 6), (6, 9), (9, 10)), rel=1e-3, abs_frac=1e-5, floor=0.0):
    """Kernel-by-kernel gradient check, one number per parameter group; each
    must be <= 1.  Kernel j passes when ||g_j - g_o,j|| <= rel * ||g_o,j||
    + abs_frac * scale, the scale being the group's largest kernel norm (or
    `floor`, for a group that is all rounding, e.g. the rotation gradient of
    isotropic kernels).  The absolute term covers the fused adjoint's
    fixed-point accumulation: each work item's partial is rounded to 2^-36,
    which leaves an absolute error (about 1e-9 of the largest kernel on the
    torus field) on kernels at the fringe of the band whose gradient nearly
    vanishes.  A wrong kernel whose gradient is above abs_frac of the largest
    cannot hide under a group norm."""
    g = np.asarray(g, np.float64)
    g_o = np.asarray(g_o, np.float64)
    out = []
    for a, b in groups:
        num = np.linalg.norm(g[a:b] - g_o[a:b], axis=0)
        den = np.linalg.norm(g_o[a:b], axis=0)
        scale = max(den.max(), floor, 1e-300)
        out.append(float((num / (rel * den + abs_frac * scale)).max()))
    return out
