"""The allocation-free normalisation entry point.

Some callers cannot allocate device memory when they need the Eq. 3-10 target
map: an application that only hands out buffers from its own pool, or a loop
that must not allocate once it runs.  serbf_normalize_sdf_noalloc serves them
with a fixed scratch array inside the library.  This test calls it through the
C ABI twice in a row and checks each result against serbf_normalize_sdf, which
uses a caller-allocated workspace.  The file is named so that pytest runs it
last.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _workspace_normalize(N, torch, S):
    sizes = N.WsSizes(max(S.numel(), 1), 16, 8, 0, 16, 2, 0)
    nbytes = N.serbf_workspace_bytes(sizes)
    buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    off = (-buf.data_ptr()) % 256
    ws = N.workspace_struct()
    N.serbf_workspace_init(ws, buf[off:off + nbytes], sizes)
    t = torch.zeros_like(S)
    mh = torch.zeros(2, dtype=torch.float64, device="cuda")
    N.serbf_normalize_sdf(S, t, mh, ws)
    return t, mh


def test_noalloc_normalize_matches_workspace_version_twice():
    torch = torch_cuda()
    from paper_2505_02350_gb300 import build
    build.build()
    from paper_2505_02350_gb300 import _native as N
    x, y, z = synth.grid(64)
    inputs = [synth.sdf_torus(x, y, z), synth.sdf_sphere(*synth.grid(33))[:30001]]
    for S_host in inputs:  # two calls in a row, different sizes: stale scratch must not leak in
        S = torch.as_tensor(S_host, device="cuda")
        t = torch.full_like(S, -1.0)
        mh = torch.zeros(2, dtype=torch.float64, device="cuda")
        N.serbf_normalize_sdf_noalloc(S, t, mh)
        t_ref, mh_ref = _workspace_normalize(N, torch, S)
        torch.cuda.synchronize()
        assert torch.equal(mh, mh_ref)
        assert torch.equal(t, t_ref)  # same arithmetic in the same order: identical targets
        assert float(mh[0]) == float(S_host.min())


def test_noalloc_normalize_rejects_sizes_beyond_its_scratch():
    torch_cuda()
    from paper_2505_02350_gb300 import _native as N
    rc = N.lib.serbf_normalize_sdf_noalloc(C.c_void_p(16), C.c_void_p(16), 67108865, C.c_void_p(16), None)
    assert rc == N.SERBF_ECAPACITY
