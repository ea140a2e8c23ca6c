"""Batched solve through the C ABI (serbf_batch_init / serbf_epoch_batched):
fields of uneven sizes advanced by one persistent forward + adjoint launch per
epoch give the same bits as the same fields advanced one at a time with the
same warps per item -- parameters, kernel counts, Adam moments, optimiser
states and loss terms, over epochs in which the L1 phase, deletions and
additions all happen."""
import numpy as np
import pytest

import synth
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def _fields(torch, count, seed, fwd_warps):
    from paper_2505_02350_gb300 import field
    out = []
    for sh in synth.batch_workload(count, seed=seed):
        if sh["n"] > 64:
            continue
        pb = field.Problem(sh["x"], sh["y"], sh["z"], sh["S"], sh["P"], sh["m"], sh["spacing"], cap=2 * sh["m"])
        # short windows so that the Algorithm 3 gates fire within a few
        # epochs: L1 on at epoch 5, a deletion due at 10, an addition at 12
        pb.cfg.k_l2, pb.cfg.tau_l2 = 5, 1e30
        pb.cfg.k_l1, pb.cfg.tau_l1 = 12, 1e30
        pb.cfg.fwd_warps = fwd_warps
        from paper_2505_02350_gb300 import _native as N
        N.serbf_state_init(pb.state, pb.cfg)
        out.append(pb)
    return out


@pytest.mark.parametrize("warps", [1, 2])
def test_batched_epochs_equal_single_field_epochs(warps):
    torch = torch_cuda()
    from paper_2505_02350_gb300 import batch, build
    build.build()
    singles = _fields(torch, 10, 700, warps)
    batched = _fields(torch, 10, 700, warps)
    assert len(singles) >= 4
    bt = batch.Batch(batched, fwd_warps=warps)
    assert bt.fwd_warps == warps
    added = pruned = 0
    for e in range(16):
        for pb in singles:
            pb.epoch()
        bt.epoch()
        torch.cuda.synchronize()
        for a, b in zip(singles, batched):
            sa = a.state_host()
            added = max(added, sa.m_added)
            pruned = max(pruned, sa.m_pruned)
            assert a.m() == b.m(), e
            m = a.m()
            assert torch.equal(a.p[:, :m], b.p[:, :m]), e
            assert torch.equal(a.adam_m[:, :m], b.adam_m[:, :m]) and torch.equal(a.adam_v[:, :m], b.adam_v[:, :m])
            assert torch.equal(a.stats[:10], b.stats[:10]), e
            assert torch.equal(a.state, b.state), e
    assert added > 0 and pruned > 0  # both the deletion and the addition happened along the way
    for pb in batched:
        assert pb.status()[0] == 0


def test_batched_epoch_replays_as_one_graph():
    torch = torch_cuda()
    from paper_2505_02350_gb300 import batch, build
    build.build()
    a = _fields(torch, 6, 800, 2)
    b = _fields(torch, 6, 800, 2)
    ba, bb = batch.Batch(a, fwd_warps=2), batch.Batch(b, fwd_warps=2)
    for _ in range(3):
        ba.epoch()
    bb.capture()  # one eager epoch, then the capture
    for _ in range(2):
        bb.epoch_graph()
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        m = x.m()
        assert m == y.m() and torch.equal(x.p[:, :m], y.p[:, :m]) and torch.equal(x.stats[:6], y.stats[:6])
