"""The comparison helpers of the GPU parity tests, checked on the CPU: a
planted mistake in one kernel's gradient must fail the kernel-by-kernel bar,
and gradients within the fixed-point rounding floor must pass it."""
import numpy as np

from gpu_util import per_kernel_errors, rel_l2


def _grads(seed=0, m=512):
    g = np.random.default_rng(seed)
    # magnitudes spread over ten decades, as at the fringe of a band
    return g.normal(size=(10, m)) * 10.0 ** g.uniform(-10, 0, size=m)


def test_rounding_floor_passes():
    g_o = _grads()
    scale = np.abs(g_o).max()
    noisy = g_o * (1 + 1e-6 * np.random.default_rng(1).normal(size=g_o.shape))
    noisy += 1e-9 * scale * np.random.default_rng(2).normal(size=g_o.shape)
    assert max(per_kernel_errors(noisy, g_o)) <= 1.0


def test_one_wrong_small_kernel_fails_though_the_group_norm_passes():
    g_o = _grads()
    norms = np.linalg.norm(g_o[6:9], axis=0)
    j = int(np.argsort(norms)[-40])  # a kernel well below the largest
    assert norms[j] < 0.5 * norms.max()
    bad = g_o.copy()
    bad[6:9, j] *= -1.0  # sign of one kernel's rotation gradient flipped
    assert rel_l2(bad[6:9], g_o[6:9]) > 0  # the group norm sees little ...
    assert per_kernel_errors(bad, g_o)[2] > 1.0  # ... the per-kernel bar fails


def test_degenerate_group_uses_the_floor():
    g_o = _grads()
    g_o[6:9] = 1e-17  # an all-rounding group (isotropic kernels)
    g = g_o.copy()
    g[6:9] = 0.0
    assert per_kernel_errors(g, g_o, floor=1e-6)[2] <= 1.0
    assert per_kernel_errors(g, g_o)[2] > 1.0
