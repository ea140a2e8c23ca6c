"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
finite differences, invariants, brute force on tiny inputs, or a library
routine that computes a special case.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import synth
from fp32 import fmaf, support_d2

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


def _params(m, g, rotate=True, iso=False, centre=0.4, lo=0.2, hi=0.6):
    P = np.zeros((10, m), np.float64)
    P[0:3] = g.uniform(-centre, centre, (3, m))
    if iso:
        P[3:6] = 1.0 / g.uniform(lo, hi, m)[None, :]
    else:
        P[3:6] = 1.0 / g.uniform(lo, hi, (3, m))
    if rotate:
        P[6:9] = g.uniform(-math.pi, math.pi, (3, m))
    P[9] = g.normal(0.0, 0.5, m)
    return P.astype(np.float32).astype(np.float64)


# ---------------------------------------------------------------- Eq. 3-10
def test_normalize_fixed_points(orc):
    m = -0.3
    rows = _golden("eq3_10_fixed_points.txt")
    S = np.array([float(r[0]) * abs(m) for r in rows] + [0.2, -0.1], np.float32)
    t, mm, h = orc.normalize(S)
    assert mm == float(np.float32(m))
    assert h == pytest.approx(math.log(2) / mm ** 2, rel=1e-15)
    for k, r in enumerate(rows):
        assert t[k] == pytest.approx(float(r[1]), rel=1e-6)
    # interior maps into (1, 2], exterior into (0, 1)
    assert 1.0 < t[-1] <= 2.0 and 0.0 < t[-2] < 1.0


def test_normalize_exact_surface_value(orc):
    S = np.array([-0.25, 0.0, 0.25, 1.0], np.float32)
    t, _, _ = orc.normalize(S)
    assert t[1] == pytest.approx(1.0, abs=1e-15)
    assert t[0] == pytest.approx(2.0, abs=1e-15)
    assert t[2] == pytest.approx(0.125, abs=1e-15)


def test_hyperparameter_defaults(orc):
    g = {r[0]: float(r[1]) for r in _golden("alg3_hyperparameters.txt")}
    c = orc.default_cfg()
    assert c.lr0 == g["lr"] and c.tau_m == g["tau_m"] and c.tau_d == g["tau_d"]
    assert c.tau_l1 == g["tau_l1"] and c.tau_l2 == g["tau_l2"]
    assert c.k_l1 == g["k_l1"] and c.k_l2 == g["k_l2"] and c.T_e == g["T_e"] and c.M_e == g["M_e"]


# ---------------------------------------------------------------- rotation
def _Rx(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _Ry(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, -s], [0, 1, 0], [s, 0, c]])


def _Rz(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def test_rotation_is_product_of_eq3_6_matrices(orc):
    g = np.random.default_rng(0)
    for _ in range(20):
        a, b, c = g.uniform(-math.pi, math.pi, 3)
        R = orc.rotation(a, b, c)
        # App. A entries = R_z(theta_x) R_y(theta_y) R_x(theta_z) of Eq. 3-6's factors
        np.testing.assert_allclose(R, _Rz(a) @ _Ry(b) @ _Rx(c), atol=1e-14)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
    np.testing.assert_allclose(orc.rotation(0, 0, 0), np.eye(3), atol=0)


# ---------------------------------------------------------------- Eq. 3-7 / 3-26
def test_single_erbf_closed_forms(orc):
    g = np.random.default_rng(1)
    P = _params(1, g)
    c = P[0:3, 0]
    R = orc.rotation(*P[6:9, 0])
    assert orc.erbf(c, P, 0) == pytest.approx(1.0, abs=1e-15)
    for k in range(3):
        for s in (0.05, 0.1, 0.3):
            v = c + s * R.T[:, k]  # offset along the k-th principal axis
            assert orc.erbf(v, P, 0) == pytest.approx(math.exp(-(P[3 + k, 0] * s) ** 2), rel=1e-12)


def test_forward_single_kernel_and_superposition(orc):
    g = np.random.default_rng(2)
    P = _params(3, g)
    P[9, 1] = -abs(P[9, 1])  # a negative signed-square weight
    x, y, z = (g.uniform(-0.5, 0.5, 50).astype(np.float32) for _ in range(3))
    t = np.zeros(50, np.float32)
    psi_all = orc.forward(x, y, z, t, P, 3, use_cutoff=False)[0]
    total = np.zeros(50)
    for j in range(3):
        Pj = P[:, j:j + 1].copy()
        psi_j = orc.forward(x, y, z, t, Pj, 1, use_cutoff=False)[0]
        phi = np.array([orc.erbf((x[i], y[i], z[i]), Pj, 0) for i in range(50)])
        np.testing.assert_allclose(psi_j, P[9, j] * abs(P[9, j]) * phi, rtol=1e-13)
        total += psi_j
    np.testing.assert_allclose(psi_all, total, rtol=1e-12, atol=1e-15)


def test_forward_permutation_invariance(orc):
    g = np.random.default_rng(3)
    m = 12
    P = _params(m, g)
    x, y, z = (g.uniform(-0.7, 0.7, 300).astype(np.float32) for _ in range(3))
    t = g.uniform(0.5, 1.5, 300).astype(np.float32)
    perm = g.permutation(m)
    a = orc.forward(x, y, z, t, P, m)
    b = orc.forward(x, y, z, t, P[:, perm].copy(), m)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-12, atol=1e-15)
    ga, _ = orc.backward(x, y, z, a[1], P, m)
    gb, _ = orc.backward(x, y, z, a[1], P[:, perm].copy(), m)
    np.testing.assert_allclose(ga[:, perm], gb, rtol=1e-12, atol=1e-15)


def test_cutoff_excludes_outside_exactly(orc):
    # one isotropic kernel at the origin, d = 10 -> radius sqrt(16.118)/10 = 0.4015
    P = np.zeros((10, 1))
    P[3:6, 0] = 10.0
    P[9, 0] = 1.0
    x = np.array([0.0, 0.39, 0.41, 0.6], np.float32)
    zero = np.zeros(4, np.float32)
    psi_c = orc.forward(x, zero, zero, zero, P, 1, use_cutoff=True)[0]
    psi_n = orc.forward(x, zero, zero, zero, P, 1, use_cutoff=False)[0]
    assert psi_c[2] == 0.0 and psi_c[3] == 0.0
    assert psi_c[0] == psi_n[0] == 1.0 and psi_c[1] == psi_n[1]
    assert psi_n[2] == pytest.approx(math.exp(-(10 * 0.41) ** 2), rel=1e-6)
    # the value dropped at the radius is at most eps
    assert psi_n[2] < 1e-7


def test_mask_cases_eq3_18(orc):
    # one very wide kernel gives Psi ~= a at points near the centre
    P = np.zeros((10, 1))
    P[3:6, 0] = 1e-3
    for a, t, inside in [(0.95, 0.95, True), (0.95, 0.5, True), (0.5, 0.5, False),
                         (1.05, 1.5, True), (1.5, 1.5, False), (0.5, 1.05, True),
                         (0.95, 0.9, True), (0.85, 0.9, False), (1.05, 1.1, True), (1.15, 1.1, False)]:
        P[9, 0] = math.sqrt(a)
        x = np.zeros(1, np.float32)
        psi, err, mask, st = orc.forward(x, x, x, np.array([t], np.float32), P, 1)
        assert psi[0] == pytest.approx(a, rel=1e-12)
        assert bool(mask[0]) == inside, (a, t)
        assert err[0] == (pytest.approx(a - float(np.float32(t)), abs=1e-12) if inside else 0.0)
        assert st[0] == pytest.approx(err[0] ** 2) and st[3] == float(inside)


def test_loss_stats_sum_over_id_all(orc):
    g = np.random.default_rng(4)
    P = _params(6, g)
    x, y, z = (g.uniform(-0.7, 0.7, 400).astype(np.float32) for _ in range(3))
    t = g.uniform(0.0, 2.0, 400).astype(np.float32)
    psi, err, mask, st = orc.forward(x, y, z, t, P, 6)
    sel = mask.astype(bool)
    assert st[0] == pytest.approx(np.sum((psi[sel] - t[sel].astype(np.float64)) ** 2), rel=1e-12)
    assert st[1] == pytest.approx(np.abs(P[9, :6]).sum(), rel=1e-12)
    assert st[3] == sel.sum() and np.all(err[~sel] == 0.0)


# ---------------------------------------------------------------- Eq. 3-15 predicate
def test_support_predicate_fp64_margin(orc):
    g = np.random.default_rng(5)
    P = _params(30, g, centre=0.5, lo=0.1, hi=0.4)
    x, y, z = (g.uniform(-1, 1, 3000).astype(np.float32) for _ in range(3))
    krow, kcol, _, _ = orc.neighbors(x, y, z, P, 30)
    nle = -math.log(1e-7)
    for j in range(30):
        members = np.zeros(3000, bool)
        members[kcol[krow[j]:krow[j + 1]]] = True
        r = math.sqrt(nle / np.min(P[3:6, j] ** 2))
        dist = np.sqrt((x - P[0, j]) ** 2 + (y - P[1, j]) ** 2 + (z - P[2, j]) ** 2)
        assert members[dist < r * (1 - 1e-5)].all()
        assert not members[dist > r * (1 + 1e-5)].any()


def test_support_predicate_is_strict(orc):
    assert not orc.in_support((2.0, 0.0, 0.0), (0.0, 0.0, 0.0), 4.0)
    assert orc.in_support((np.nextafter(np.float32(2.0), np.float32(0)), 0.0, 0.0), (0, 0, 0), 4.0)
    assert orc.support_r2(4.0, 2.0, 8.0) == np.float32(np.float32(-math.log(1e-7)) / np.float32(4.0))


def _np_member(px, py, pz, cx, cy, cz, r2):
    f = np.float32
    dx, dy, dz = f(px) - f(cx), f(py) - f(cy), f(pz) - f(cz)
    return support_d2(dx, dy, dz) < f(r2)


def test_fmaf_helper_rounds_once():
    """The float32 fma of the pins against exact rational arithmetic."""
    from fractions import Fraction
    g = np.random.default_rng(30)
    a, b, c = (g.normal(0, 1, 400).astype(np.float32) for _ in range(3))
    # a case whose float64 sum lies exactly halfway between two float32 values
    a = np.append(a, np.float32(1.0)); b = np.append(b, np.float32(1.0))
    c = np.append(c, np.float32(2.0 ** -24) + np.float32(2.0 ** -60))
    got = fmaf(a, b, c)
    for k in range(a.size):
        exact = Fraction(float(a[k])) * Fraction(float(b[k])) + Fraction(float(c[k]))
        lo = np.float32(float(exact))
        cands = [np.nextafter(lo, np.float32(-np.inf)), lo, np.nextafter(lo, np.float32(np.inf))]
        dist = [abs(Fraction(float(v)) - exact) for v in cands]
        best = min(dist)
        assert abs(Fraction(float(got[k])) - exact) == best, k


def test_support_predicate_uses_the_fma_form(orc):
    """Where the canonical form fma(dz, dz, fma(dy, dy, fl(dx dx))) and the
    unfused sum of rounded squares give different floats, the oracle's test
    follows the canonical form (r2 set between the two values)."""
    g = np.random.default_rng(31)
    d = g.uniform(-0.3, 0.3, (3, 400000)).astype(np.float32)
    canon = support_d2(d[0], d[1], d[2])
    plain = ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]).astype(np.float32)
    diff = np.flatnonzero(canon != plain)
    assert diff.size >= 20
    for k in diff[:40]:
        r2 = max(canon[k], plain[k])  # strictly above the smaller one only
        p = (float(d[0, k]), float(d[1, k]), float(d[2, k]))
        assert orc.in_support(p, (0.0, 0.0, 0.0), float(r2)) == bool(canon[k] < r2)


def test_neighbors_match_numpy_bruteforce(orc):
    g = np.random.default_rng(6)
    m, n = 25, 700
    P = _params(m, g, centre=0.6, lo=0.1, hi=0.5)
    x, y, z = (g.uniform(-1, 1, n).astype(np.float32) for _ in range(3))
    krow, kcol, prow, pcol = orc.neighbors(x, y, z, P, m)
    f = np.float32
    nle = f(-math.log(1e-7))
    member = np.zeros((n, m), bool)
    for j in range(m):
        d2 = (P[3:6, j].astype(np.float32)) ** 2
        r2 = nle / d2.min()
        member[:, j] = _np_member(x, y, z, P[0, j], P[1, j], P[2, j], r2)
    for j in range(m):
        np.testing.assert_array_equal(kcol[krow[j]:krow[j + 1]], np.nonzero(member[:, j])[0])
    for i in range(n):
        np.testing.assert_array_equal(pcol[prow[i]:prow[i + 1]], np.nonzero(member[i])[0])
    assert krow[-1] == prow[-1] == member.sum()


# ---------------------------------------------------------------- binning
@pytest.mark.parametrize("sf", [1, 3, 4])
def test_binning_matches_lexsort(orc, sf):
    g = np.random.default_rng(7)
    x, y, z = (g.uniform(-1, 1, 5000).astype(np.float32) for _ in range(3))
    x[:10] = x[10:20]  # ties in the key
    y[:10] = y[10:20]
    z[:10] = z[10:20]
    o = np.float32(-1.05)
    h = np.float32(0.13)
    nc = 17
    perm = orc.bin_points(x, y, z, (o, o, o), h, (nc, nc, nc), sf)

    def ax(v):
        k = np.floor((v - o) / h)
        return np.clip(k, 0, nc - 1).astype(np.int64)

    kx, ky, kz = ax(x), ax(y), ax(z)
    ns = -(-nc // sf)
    sup = ((kz // sf) * ns + ky // sf) * ns + kx // sf
    loc = ((kz % sf) * sf + ky % sf) * sf + kx % sf
    ref = np.lexsort((np.arange(5000), loc, sup))
    np.testing.assert_array_equal(perm, ref)


# ---------------------------------------------------------------- App. A gradients
def _loss(orc, x, y, z, t, P, m):
    psi = orc.forward(x, y, z, t, P, m, use_cutoff=False, tau1=-1e30, tau2=1e30)[0]
    return float(np.sum((psi - t.astype(np.float64)) ** 2))


@pytest.mark.parametrize("iso", [False, True])
def test_gradients_match_central_differences(orc, iso):
    g = np.random.default_rng(8 + iso)
    m, n = 4, 120
    P = _params(m, g, iso=iso, lo=0.3, hi=0.8)
    x, y, z = (g.uniform(-0.7, 0.7, n).astype(np.float32) for _ in range(3))
    t = g.uniform(0.0, 1.5, n).astype(np.float32)
    psi = orc.forward(x, y, z, t, P, m, use_cutoff=False, tau1=-1e30, tau2=1e30)[0]
    E = psi - t.astype(np.float64)
    grad, _ = orc.backward(x, y, z, E, P, m, use_cutoff=False)
    h = 1e-6
    for r in range(10):
        for j in range(m):
            Pp, Pm = P.copy(), P.copy()
            Pp[r, j] += h
            Pm[r, j] -= h
            fd = (_loss(orc, x, y, z, t, Pp, m) - _loss(orc, x, y, z, t, Pm, m)) / (2 * h)
            assert grad[r, j] == pytest.approx(fd, rel=2e-6, abs=2e-7), (r, j)


def test_isotropic_kernels_have_zero_angle_gradient(orc):
    g = np.random.default_rng(10)
    m, n = 6, 300
    P = _params(m, g, iso=True)
    x, y, z = (g.uniform(-0.7, 0.7, n).astype(np.float32) for _ in range(3))
    E = g.normal(0, 1, n)
    grad, _ = orc.backward(x, y, z, E, P, m)
    scale = np.abs(grad).max()
    assert np.abs(grad[6:9]).max() <= 1e-12 * scale


def test_single_pair_axis_closed_form(orc):
    # identity rotation, point on the k-th axis at distance s: phi = exp(-(d_k s)^2)
    P = np.zeros((10, 1))
    P[3:6, 0] = [3.0, 5.0, 7.0]
    P[9, 0] = -0.7
    a = P[9, 0] * abs(P[9, 0])
    for k in range(3):
        v = np.zeros(3, np.float32)
        v[k] = 0.125
        s = 0.125
        phi = math.exp(-(P[3 + k, 0] * s) ** 2)
        E = np.array([0.3])
        gr, npair = orc.backward(v[0:1], v[1:2], v[2:3], E, P, 1)
        assert npair == 1
        assert gr[9, 0] == pytest.approx(4 * abs(P[9, 0]) * phi * 0.3, rel=1e-12)
        assert gr[3 + k, 0] == pytest.approx(-4 * a * P[3 + k, 0] * s * s * phi * 0.3, rel=1e-12)
        # dPsi/dc_k = 2 a d_k^2 s phi along the axis
        assert gr[k, 0] == pytest.approx(4 * a * P[3 + k, 0] ** 2 * s * phi * 0.3, rel=1e-12)


# ---------------------------------------------------------------- Eq. 3-21
def test_alpha_is_min_norm_point(orc):
    g = np.random.default_rng(11)
    grid = np.linspace(0, 1, 200001)
    for trial in range(6):
        m = 40
        w = g.normal(0, 1, m)
        w[:3] = 0.0
        g2 = g.normal(0, 0.3 if trial % 2 else 3.0, m)
        g1 = np.sign(w)
        a = orc.alpha(g2, w)
        vals = np.array([np.sum((al * g2 + (1 - al) * g1) ** 2) for al in grid[::100]])
        best = grid[::100][vals.argmin()]
        assert abs(a - best) <= 1e-3 + 1e-12
        assert 0.0 <= a <= 1.0
    w = np.array([1.0, -2.0, 0.5])
    assert orc.alpha(np.sign(w), w) == 1.0


# ---------------------------------------------------------------- Adam
def test_adam_matches_torch(orc):
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(12)
    p0 = g.normal(0, 1, 37)
    p = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    q, mo, v = p0.copy(), np.zeros(37), np.zeros(37)
    for t in range(1, 8):
        gr = g.normal(0, 1, 37)
        p.grad = torch.tensor(gr)
        opt.step()
        q, mo, v = orc.adam(q, gr, mo, v, t, 0.01)
        np.testing.assert_allclose(q, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def _line_search_alpha(g2, g1):
    """argmin over [0, 1] of ||a g2 + (1 - a) g1||^2 by ternary search on the
    convex objective (no use of the Eq. 3-21 closed form)."""
    f = lambda a: float(np.sum((a * g2 + (1.0 - a) * g1) ** 2))
    lo, hi = 0.0, 1.0
    for _ in range(200):
        a, b = lo + (hi - lo) / 3.0, hi - (hi - lo) / 3.0
        if f(a) <= f(b):
            hi = b
        else:
            lo = a
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("gscale", [0.3, 3.0])
def test_step_with_l1_term_is_adam_on_the_combined_gradient(orc, gscale):
    """Eq. 3-21 inside the Algorithm 3 step: with l1_optim set and max|E| <
    tau_m, the update is Adam on alpha g for the centre, axis and angle rows
    and on alpha g_w + beta sign(w) for the weight row (App. A, Eq. grad),
    with alpha the minimiser of ||a g2 + (1 - a) g1||^2 over [0, 1] found by
    a line search here.  Reference: torch.optim.Adam in float64 on those
    gradients; two steps in a row, so the moments carry over."""
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(21)
    m, cap = 23, 29
    cfg = orc.default_cfg()
    st = orc.state_init(cfg)
    st.l1_optim = 1
    P = np.zeros((10, cap))
    P[:, :m] = g.normal(0, 1, (10, m))
    P[9, :3] = 0.0  # sign(0) = 0: no L1 pull on these weights
    P[9, 3:6] = -np.abs(P[9, 3:6])
    mo, v = np.zeros((10, cap)), np.zeros((10, cap))
    tp = torch.tensor(P[:, :m].copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=cfg.lr0, betas=(cfg.beta1, cfg.beta2), eps=cfg.adam_eps)
    alphas = []
    for it in range(2):
        grad = g.normal(0, gscale, (10, m))
        w = tp.detach().numpy()[9].copy()
        g1 = np.sign(w)
        a_ls = _line_search_alpha(grad[9], g1)
        assert 0.0 < a_ls < 1.0  # the branch under test mixes both terms
        orc.step(P, m, grad, mo, v, 1.0, 0.5 * cfg.tau_m, cfg, st)
        # the flat minimum limits the search to about sqrt(machine eps)
        assert st.alpha == pytest.approx(a_ls, abs=1e-7)
        assert st.beta == 1.0 - st.alpha
        a = st.alpha
        comb = a * grad
        comb[9] += (1.0 - a) * g1
        tp.grad = torch.tensor(comb)
        opt.step()
        alphas.append(a)
        assert st.adam_t == it + 1
        np.testing.assert_allclose(P[:, :m], tp.detach().numpy(), rtol=1e-9, atol=1e-11)
        s = opt.state[tp]
        np.testing.assert_allclose(mo[:, :m], s["exp_avg"].numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(v[:, :m], s["exp_avg_sq"].numpy(), rtol=1e-9, atol=1e-14)
        assert not P[:, m:].any() and not mo[:, m:].any()  # columns past m untouched
    assert alphas[0] != alphas[1]


def test_step_without_the_gate_is_plain_adam(orc):
    """l1_optim set but max|E| >= tau_m (Eq. l1_activate2 false), and l1_optim
    off with a small max|E|: alpha = 1, beta = 0, Adam on the raw gradient."""
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(22)
    m = 17
    cfg = orc.default_cfg()
    for l1, maxe in ((1, 2.0 * cfg.tau_m), (0, 0.1 * cfg.tau_m)):
        st = orc.state_init(cfg)
        st.l1_optim = l1
        P = g.normal(0, 1, (10, m))
        mo, v = np.zeros((10, m)), np.zeros((10, m))
        tp = torch.tensor(P.copy(), dtype=torch.float64, requires_grad=True)
        opt = torch.optim.Adam([tp], lr=cfg.lr0, betas=(cfg.beta1, cfg.beta2), eps=cfg.adam_eps)
        grad = g.normal(0, 1, (10, m))
        tp.grad = torch.tensor(grad)
        opt.step()
        orc.step(P, m, grad, mo, v, 1.0, maxe, cfg, st)
        assert st.alpha == 1.0 and st.beta == 0.0
        np.testing.assert_allclose(P, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- Algorithm 3 gates
def _run_gates(orc, l2_seq, w_seq, cfg, maxE=1.0):
    m = len(w_seq[0])
    st = orc.state_init(cfg)
    hist = []
    for e, (l2, w) in enumerate(zip(l2_seq, w_seq)):
        P = np.zeros((10, m))
        P[9] = w
        mo = np.zeros((10, m))
        v = np.zeros((10, m))
        grad = np.zeros((10, m))
        orc.step(P, m, grad, mo, v, l2, maxE, cfg, st)
        hist.append((st.epoch, st.l1_optim, st.do_prune, st.do_add, st.phase2, st.lr))
    return hist


def test_gate_l1_activation_after_k_l2_stable_epochs(orc):
    cfg = orc.default_cfg(T_e=1600, M_e=2000)
    l2 = [100.0 - 20 * k for k in range(5)] + [3.0] * 20
    w = [np.full(8, 0.5)] * len(l2)
    h = _run_gates(orc, l2, w, cfg)
    on = [e for (e, l1, *_r) in h if l1]
    # the first window of 10 epochs with std < 0.5 ends at epoch 15 (epochs 6..15 all 3.0)
    assert on[0] == 15
    assert all(e >= 15 for e in on)


def test_gate_prune_every_k_l2_epochs_while_l1(orc):
    cfg = orc.default_cfg()
    cfg.tau_l1 = -1.0  # never add
    l2 = [5.0] * 40
    w = [np.full(8, 0.5)] * 40
    h = _run_gates(orc, l2, w, cfg)
    prune_epochs = [e for (e, l1, pr, *_r) in h if pr]
    # L1 switches on at epoch 10 (end of that epoch); prunes are due at 20, 30, 40
    assert prune_epochs == [20, 30, 40]


def test_gate_add_after_k_l1_stable_basis_counts(orc):
    cfg = orc.default_cfg()
    n = 60
    l2 = [5.0] * n
    w = [np.full(8, 0.5)] * n
    h = _run_gates(orc, l2, w, cfg)
    adds = [e for (e, l1, pr, ad, *_r) in h if ad]
    # L1 on at epoch 10; b_f history is full (50 values) at epoch 50 -> add, L1 off.
    # With L2 and b_f held constant both gates hold again at once, so the literal
    # Algorithm 3 re-activates L1 and adds again every epoch.
    assert adds == list(range(50, 61))
    assert all(l1 == 0 for (e, l1, pr, ad, *_r) in h if ad)


def test_gate_add_blocked_by_basis_count_swing(orc):
    cfg = orc.default_cfg()
    n = 100
    l2 = [5.0] * n
    w = []
    for e in range(n):
        v = np.full(20, 0.5)
        if 30 <= e < 40:
            v[:6] = 0.0  # b_f drops by 6 >= tau^l1 = 5 for ten epochs
        w.append(v)
    h = _run_gates(orc, l2, w, cfg)
    adds = [e for (e, l1, pr, ad, *_r) in h if ad]
    # the window of the last 50 b_f values holds the swing until epoch 40 + 50 - 1
    assert adds[0] == 90


def test_gate_phase2_cosine_lr(orc):
    cfg = orc.default_cfg(T_e=20, M_e=30)
    h = _run_gates(orc, [1e6 * (k % 2) for k in range(30)], [np.full(4, 0.5)] * 30, cfg)
    lr = {e: r for (e, *_x, r) in h}
    assert lr[19] == 0.01
    assert lr[20] == pytest.approx(1e-3)
    assert lr[25] == pytest.approx(1e-5 + (1e-3 - 1e-5) * 0.5 * (1 + math.cos(math.pi * 0.5)))
    assert lr[30] == pytest.approx(1e-5)
    assert all(ph for (e, l1, pr, ad, ph, r) in h if e >= 20)


def test_minibatch_epoch_gates_follow_the_epoch_sum(orc):
    """Algorithm 3 with mini-batches: Adam runs per batch, the gates once per
    epoch on the sum of the batch L2 values -- the same gate sequence as a
    full-batch run fed those sums."""
    m, cap, nb = 4, 4, 3
    P = np.zeros((10, cap))
    P[3:6] = 5.0
    P[9] = 0.5
    zero = np.zeros((10, m))
    cfg_b = orc.default_cfg(T_e=40, M_e=50, epoch_steps=nb)
    cfg_f = orc.default_cfg(T_e=40, M_e=50)
    sb, sf = orc.state_init(cfg_b), orc.state_init(cfg_f)
    Pb, Pf = P.copy(), P.copy()
    mb, vb, mf, vf = (np.zeros((10, cap)) for _ in range(4))
    for e in range(45):
        parts = [30.0 - e + 0.25 * k if e < 8 else 1.0 + 0.1 * k for k in range(nb)]
        for k in range(nb):
            orc.step(Pb, m, zero, mb, vb, parts[k], 0.5, cfg_b, sb)
            if k < nb - 1:
                assert sb.epoch == e and sb.step == k + 1
        orc.step(Pf, m, zero, mf, vf, (parts[0] + parts[1]) + parts[2], 0.5, cfg_f, sf)
        assert (sb.epoch, sb.l1_optim, sb.phase2, sb.do_prune, sb.do_add, sb.step) == \
            (sf.epoch, sf.l1_optim, sf.phase2, sf.do_prune, sf.do_add, 0), e
        assert list(sb.l2_hist[:10]) == list(sf.l2_hist[:10])
        assert sb.adam_t == nb * sf.adam_t
        assert sb.lr == sf.lr


# ---------------------------------------------------------------- Eq. 3-27
def test_prune_keeps_order_and_threshold(orc):
    g = np.random.default_rng(13)
    m = 50
    P = g.normal(0, 1, (10, m + 5))
    P[9, :m] = g.normal(0, 0.02, m)
    keep = np.abs(P[9, :m]) >= 0.01
    ref = P[:, :m][:, keep]
    m2 = orc.prune(P, m, 0.01)
    assert m2 == keep.sum()
    np.testing.assert_array_equal(P[:, :m2], ref)


# ---------------------------------------------------------------- Algorithm 2 / Eq. 3-24
def test_topk_matches_sorted(orc):
    g = np.random.default_rng(14)
    n = 2000
    E = g.normal(0, 0.05, n).astype(np.float32)
    E[100:110] = E[5]  # ties
    E[200:205] = -E[5]
    mask = (g.uniform(size=n) < 0.6).astype(np.uint8)
    mask[[5, 100, 200]] = 1
    th = 0.01
    for k in (1, 7, 50, 10 ** 6):
        got = orc.select_topk(E, mask, th, k)
        cand = [i for i in range(n) if mask[i] and abs(float(E[i])) > th]
        ref = sorted(cand, key=lambda i: (-abs(float(E[i])), i))[:k]
        np.testing.assert_array_equal(got, ref)


def test_local_max_bruteforce(orc):
    g = np.random.default_rng(15)
    n = 600
    x, y, z = (g.uniform(-1, 1, n).astype(np.float32) for _ in range(3))
    E = g.normal(0, 1, n).astype(np.float32)
    mask = (g.uniform(size=n) < 0.7).astype(np.uint8)
    cand = np.nonzero(mask)[0].astype(np.int32)
    r2 = np.float32(0.04)
    got = orc.local_max(x, y, z, E, mask, cand, r2)
    ref = []
    for i in cand:
        d2 = support_d2(x - x[i], y - y[i], z - z[i])
        nb = (d2 <= r2) & mask.astype(bool)
        if np.all(np.abs(E[nb]) <= abs(E[i])):
            ref.append(i)
    np.testing.assert_array_equal(got, ref)


def test_new_kernel_eq3_24(orc):
    for e, dbar in [(0.05, 0.1), (-0.3, 0.02), (0.011, 0.5)]:
        k = orc.new_kernel((0.1, -0.2, 0.3), e, dbar)
        np.testing.assert_allclose(k[0:3], np.float32([0.1, -0.2, 0.3]))
        assert k[9] == pytest.approx(-np.float32(e))
        assert np.all(k[6:9] == 0.0) and k[3] == k[4] == k[5]
        # the new basis function has decayed to eps/|E| at distance dbar from its centre
        P = k.reshape(10, 1)
        v = np.array(k[0:3]) + np.array([dbar, 0, 0])
        assert orc.erbf(v, P, 0) == pytest.approx(1e-7 / abs(float(np.float32(e))), rel=1e-9)


def test_synthetic_grid_and_sphere_targets(orc):
    x, y, z = synth.grid(16)
    S = synth.sdf_sphere(x, y, z)
    t, m, h = orc.normalize(S)
    assert m == S.min()
    assert np.all((t > 1.0) == (S < 0)) and t.max() == pytest.approx(2.0)


# ---------------------------------------------------------------- Algorithm 1, Eq. 3-12
def test_inscribed_hand_example(orc):
    # five interior points on a line (t in (1, 2)); |S| = 0.30 at x=0 covers
    # x = 0.25 (d^2 = 0.0625 <= 0.09); the next largest uncovered is x = 0.8
    # (|S| 0.1) which covers x = 0.72 but not x = 1.1 (d^2 = 0.09 > 0.01)
    x = np.array([0.0, 0.25, 0.72, 0.8, 1.1], np.float32)
    z0 = np.zeros(5, np.float32)
    S = np.array([-0.30, -0.20, -0.05, -0.10, -0.02], np.float32)
    t = np.full(5, 1.5, np.float32)
    idx, n = orc.inscribed(x, z0, z0, t, S)
    assert n == 3 and list(idx) == [0, 3, 4]


def test_inscribed_skips_exterior_and_takes_first_of_ties(orc):
    x = np.array([0.0, 5.0, 10.0, 15.0], np.float32)
    z0 = np.zeros(4, np.float32)
    S = np.array([-1.0, -2.0, -2.0, 0.5], np.float32)
    t = np.array([1.5, 1.5, 1.5, 0.5], np.float32)  # the last point is outside (t < 1)
    idx, n = orc.inscribed(x, z0, z0, t, S)
    assert list(idx) == [1, 2, 0]


def test_inscribed_properties_on_sphere(orc):
    x, y, z = synth.grid(24)
    S = synth.sdf_sphere(x, y, z)
    t = orc.normalize(S)[0].astype(np.float32)
    idx, n = orc.inscribed(x, y, z, t, S)
    interior = np.flatnonzero((t > 1) & (t < 2))
    r = np.abs(S[idx]).astype(np.float32)
    # the first centre is the deepest interior point; radii never grow
    assert idx[0] == interior[np.argmax(np.abs(S[interior]))]
    assert np.all(np.diff(r) <= 0)
    d2 = lambda i, j: support_d2(np.float32(x[i] - x[j]), np.float32(y[i] - y[j]), np.float32(z[i] - z[j]))
    # every interior point lies in some selected sphere; no centre lies in an earlier one
    cover = np.zeros(interior.size, bool)
    for c, rc in zip(idx, r):
        cover |= d2(interior, c) <= rc * rc
    assert cover.all()
    for a in range(1, len(idx)):
        assert np.all(d2(idx[a], idx[:a]) > r[:a] * r[:a])


def test_init_shape_satisfies_eq3_11(orc):
    g = np.random.default_rng(21)
    c = g.uniform(-1, 1, (7, 3))
    w = g.uniform(1.05, 2.0, 7)
    r = g.uniform(0.1, 0.3, 7)
    gamma = 1e-3
    d = orc.init_shape(c, w, r, gamma)
    for j in range(7):
        dhat = min(np.linalg.norm(c[j] - c[i]) for i in range(7) if i != j)
        assert w[j] ** 2 * np.exp(-d[j] ** 2 * (dhat / 2) ** 2) == pytest.approx(gamma, rel=1e-12)
    d1 = orc.init_shape(c[:1], w[:1], r[:1], gamma)
    assert w[0] ** 2 * np.exp(-d1[0] ** 2 * r[0] ** 2) == pytest.approx(gamma, rel=1e-12)  # dhat = 2 r


# ---------------------------------------------------------------- Sec. 3.4.2 octree layers (input generator)
def test_octree_layers_structure():
    sphere = lambda x, y, z: np.sqrt(x * x + y * y + z * z) - 0.5
    L = synth.octree_layers(sphere, 3, 6)
    assert L[0][0].size == 9 ** 3  # every cell of the first level is kept
    keys = set()
    for l, (x, y, z, S, edge) in enumerate(L, start=3):
        assert edge == 2.0 / 2 ** l
        ijk = np.stack([x, y, z], 1).astype(np.float64)
        lat = (ijk + 1.0) / edge
        assert np.allclose(lat, np.round(lat), atol=1e-4)  # on the level-l lattice
        k = set(map(tuple, np.round((ijk + 1.0) * 2 ** 6 / 2).astype(int).tolist()))
        assert not (k & keys) and len(k) == x.size  # no point repeats a coarser one
        keys |= k
        np.testing.assert_allclose(S, sphere(x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)),
                                   atol=1e-6)
        if l > 3:
            # corners of children of cells the surface may cross
            assert np.abs(S).max() <= 1.5 * np.sqrt(3) * 2 * edge + 1e-6
    # every finest-lattice point close to the surface is present
    x, y, z = synth.grid(2 ** 6 + 1)
    close = np.abs(sphere(x.astype(np.float64), y.astype(np.float64), z.astype(np.float64))) < 0.5 * 2.0 / 2 ** 6
    want = set(map(tuple, np.round((np.stack([x, y, z], 1)[close] + 1.0) * 2 ** 6 / 2).astype(int).tolist()))
    assert want <= keys


# ---------------------------------------------------------------- surface extraction and Sec. 4 metrics
def _vertex_grid_field(n, fn):
    x, y, z = synth.grid(n)
    return fn(x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)).astype(np.float32)


def _areas(tri):
    t = tri.astype(np.float64).reshape(-1, 3, 3)
    return 0.5 * np.linalg.norm(np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]), axis=1)


def test_marching_tets_plane_is_exact(orc):
    n = 9
    f = _vertex_grid_field(n, lambda x, y, z: z - 0.3)
    tri = orc.marching_tets(f, (n, n, n), (-1, -1, -1), 2.0 / (n - 1))
    assert np.allclose(tri.reshape(-1, 3)[:, 2], 0.3, atol=1e-6)
    assert _areas(tri).sum() == pytest.approx(4.0, rel=1e-6)  # the [-1, 1]^2 cross-section


def test_marching_tets_sphere_area_converges(orc):
    errs = []
    for n in (17, 33, 65):
        f = _vertex_grid_field(n, lambda x, y, z: np.sqrt(x * x + y * y + z * z) - 0.5)
        tri = orc.marching_tets(f, (n, n, n), (-1, -1, -1), 2.0 / (n - 1))
        v = tri.reshape(-1, 3).astype(np.float64)
        assert np.abs(np.linalg.norm(v, axis=1) - 0.5).max() < 2.0 / (n - 1)  # vertices near the sphere
        errs.append(abs(_areas(tri).sum() / (4 * np.pi * 0.25) - 1))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 0.01


def test_surface_samples_and_metrics_closed_forms(orc):
    n = 9
    tri = orc.marching_tets(_vertex_grid_field(n, lambda x, y, z: z - 0.3), (n, n, n), (-1, -1, -1), 2.0 / (n - 1))
    u = np.random.default_rng(4).uniform(size=(4000, 3))
    A, nA = orc.sample_surface(tri, u)
    assert np.allclose(A[:, 2], 0.3, atol=1e-6) and np.allclose(np.abs(nA[:, 2]), 1.0)
    assert abs(A[:, 0].mean()) < 0.05 and A[:, 0].var() == pytest.approx(1 / 3, rel=0.05)  # uniform on the square
    hd, cd, cs = orc.surface_metrics(A, nA, A, nA)
    assert (hd, cd, cs) == (0.0, 0.0, 1.0)
    B = A.copy()
    B[:, 2] += np.float32(0.125)  # translated along the normal: every nearest point is the copy
    hd, cd, cs = orc.surface_metrics(A, nA, B, nA)
    assert hd == pytest.approx(0.125, rel=1e-6) and cd == pytest.approx(0.125, rel=1e-6) and cs == 1.0
