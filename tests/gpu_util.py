"""Helpers shared by the GPU parity tests: build problems from the seeded
synthetic inputs and pull device results back for comparison with the oracle."""
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
    return field.Problem(x, y, z, S, P, m, spacing, cap=cap or m, **kw)


def host_params(pb):
    return pb.p[:, :pb.m()].detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)
