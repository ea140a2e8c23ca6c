"""ctypes binding of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the cpu_baseline / reference legs
of ``bench.py`` may import this package.  It never touches the CUDA library.
All arrays are numpy; parameter arrays are 10 x cap (row order cx, cy, cz,
d1, d2, d3, theta_x, theta_y, theta_z, w).
"""
import ctypes as C
import math

import numpy as np

from . import build as _build

_lib = None

f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


class State(C.Structure):
    _fields_ = [("epoch", C.c_int32), ("l1_optim", C.c_int32), ("phase2", C.c_int32),
                ("adam_t", C.c_int32), ("do_prune", C.c_int32), ("do_add", C.c_int32),
                ("n_l2", C.c_int32), ("n_bf", C.c_int32), ("step", C.c_int32), ("pad", C.c_int32),
                ("lr", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("l2_epoch", C.c_double),
                ("l2_hist", C.c_double * 64), ("bf_hist", C.c_int32 * 256)]


class Cfg(C.Structure):
    _fields_ = [("lr0", C.c_double), ("lr_p2", C.c_double), ("lr_min", C.c_double),
                ("beta1", C.c_double), ("beta2", C.c_double), ("adam_eps", C.c_double),
                ("tau_m", C.c_double), ("tau_d", C.c_double), ("tau_l1", C.c_double),
                ("tau_l2", C.c_double), ("k_l1", C.c_int32), ("k_l2", C.c_int32), ("T_e", C.c_int32),
                ("M_e", C.c_int32), ("epoch_steps", C.c_int32), ("pad", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_version.restype = C.c_int
        L.oracle_set_threads.argtypes = [C.c_int]
        L.oracle_support_r2.restype = C.c_float
        L.oracle_support_r2.argtypes = [C.c_float] * 4
        L.oracle_in_support.restype = C.c_int
        L.oracle_in_support.argtypes = [C.c_float] * 7
        L.oracle_rotation.argtypes = [C.c_double, C.c_double, C.c_double, f64p]
        L.oracle_erbf.restype = C.c_double
        L.oracle_erbf.argtypes = [C.c_double, C.c_double, C.c_double, f64p, C.c_int32, C.c_int32]
        L.oracle_normalize.argtypes = [f32p, C.c_int64, f64p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.oracle_cell_keys.argtypes = [f32p, f32p, f32p, C.c_int64, C.c_float, C.c_float, C.c_float,
                                       C.c_float, C.c_int32, C.c_int32, C.c_int32, C.c_int32, u32p]
        L.oracle_bin.argtypes = [f32p, f32p, f32p, C.c_int64, C.c_float, C.c_float, C.c_float,
                                 C.c_float, C.c_int32, C.c_int32, C.c_int32, C.c_int32, u32p]
        L.oracle_neighbors.restype = C.c_int64
        L.oracle_neighbors.argtypes = [f32p, f32p, f32p, C.c_int64, f64p, C.c_int32, C.c_int32,
                                       C.c_float, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.oracle_forward.argtypes = [f32p, f32p, f32p, f32p, C.c_int64, f64p, C.c_int32, C.c_int32,
                                     C.c_float, C.c_double, C.c_double, C.c_int, f64p, f64p, u8p, f64p]
        L.oracle_backward.argtypes = [f32p, f32p, f32p, C.c_int64, f64p, f64p, C.c_int32, C.c_int32,
                                      C.c_float, C.c_int, f64p, C.POINTER(C.c_int64)]
        L.oracle_alpha.restype = C.c_double
        L.oracle_alpha.argtypes = [f64p, f64p, C.c_int32]
        L.oracle_adam.argtypes = [f64p, f64p, f64p, f64p, C.c_int64, C.c_int32, C.c_double,
                                  C.c_double, C.c_double, C.c_double]
        L.oracle_state_init.argtypes = [C.POINTER(State), C.POINTER(Cfg)]
        L.oracle_step.argtypes = [f64p, C.c_int32, C.c_int32, f64p, f64p, f64p, C.c_double,
                                  C.c_double, C.POINTER(Cfg), C.POINTER(State)]
        L.oracle_prune.restype = C.c_int32
        L.oracle_prune.argtypes = [f64p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_double]
        L.oracle_select_topk.restype = C.c_int32
        L.oracle_select_topk.argtypes = [f32p, u8p, C.c_int64, C.c_double, C.c_int64, i32p]
        L.oracle_local_max.restype = C.c_int32
        L.oracle_local_max.argtypes = [f32p, f32p, f32p, f32p, u8p, C.c_int64, i32p, C.c_int32,
                                       C.c_float, i32p]
        L.oracle_new_kernel.argtypes = [C.c_float, C.c_float, C.c_float, C.c_float, C.c_double,
                                        C.c_double, f64p]
        L.oracle_marching_tets.restype = C.c_int64
        L.oracle_marching_tets.argtypes = [f32p, C.c_int, C.c_int, C.c_int, f32p, C.c_float, C.c_float, f32p,
                                           C.c_int64]
        L.oracle_sample_surface.restype = C.c_int
        L.oracle_sample_surface.argtypes = [f32p, C.c_int64, f64p, C.c_int64, f32p, f32p]
        L.oracle_surface_metrics.argtypes = [f32p, f32p, C.c_int64, f32p, f32p, C.c_int64, f64p]
        L.oracle_inscribed.restype = C.c_int32
        L.oracle_inscribed.argtypes = [f32p, f32p, f32p, f32p, f32p, C.c_int64, i32p, C.c_int32]
        L.oracle_init_shape.argtypes = [f64p, f64p, f64p, f64p, f64p, C.c_int32, C.c_double, f64p]
        _lib = L
    return _lib


def set_threads(n):
    lib().oracle_set_threads(int(n))


def neg_ln_eps(eps=1e-7):
    """-ln(eps) rounded once to float: the numerator of the support radius (Eq. 3-15)."""
    return float(np.float32(-math.log(eps)))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _p64(P):
    """Parameters widened to float64 (float32 inputs widen exactly)."""
    return np.ascontiguousarray(P, dtype=np.float64)


def support_r2(d1, d2, d3, eps=1e-7):
    return lib().oracle_support_r2(d1, d2, d3, neg_ln_eps(eps))


def in_support(p, c, r2):
    return bool(lib().oracle_in_support(p[0], p[1], p[2], c[0], c[1], c[2], r2))


def rotation(tx, ty, tz):
    R = np.zeros(9, np.float64)
    lib().oracle_rotation(tx, ty, tz, R)
    return R.reshape(3, 3)


def erbf(v, P, j):
    P = _p64(P)
    return lib().oracle_erbf(float(v[0]), float(v[1]), float(v[2]), P, P.shape[1], j)


def normalize(S):
    S = _f32(S)
    t = np.zeros(S.shape[0], np.float64)
    m = C.c_double()
    h = C.c_double()
    lib().oracle_normalize(S, S.shape[0], t, C.byref(m), C.byref(h))
    return t, m.value, h.value


def cell_keys(x, y, z, origin, h, ncell, sf):
    x, y, z = _f32(x), _f32(y), _f32(z)
    k = np.zeros(x.shape[0], np.uint32)
    lib().oracle_cell_keys(x, y, z, x.shape[0], origin[0], origin[1], origin[2], h,
                           ncell[0], ncell[1], ncell[2], sf, k)
    return k


def bin_points(x, y, z, origin, h, ncell, sf):
    x, y, z = _f32(x), _f32(y), _f32(z)
    perm = np.zeros(x.shape[0], np.uint32)
    lib().oracle_bin(x, y, z, x.shape[0], origin[0], origin[1], origin[2], h,
                     ncell[0], ncell[1], ncell[2], sf, perm)
    return perm


def neighbors(x, y, z, P, m, eps=1e-7, cols=True):
    """Eq. 3-15-1 lists: returns (krow, kcol, prow, pcol)."""
    x, y, z, P = _f32(x), _f32(y), _f32(z), _p64(P)
    n = x.shape[0]
    krow = np.zeros(m + 1, np.int64)
    prow = np.zeros(n + 1, np.int64)
    tot = lib().oracle_neighbors(x, y, z, n, P, P.shape[1], m, neg_ln_eps(eps),
                                 krow.ctypes.data, None, prow.ctypes.data, None)
    if not cols:
        return krow, None, prow, None
    kcol = np.zeros(max(tot, 1), np.uint32)
    pcol = np.zeros(max(tot, 1), np.uint32)
    lib().oracle_neighbors(x, y, z, n, P, P.shape[1], m, neg_ln_eps(eps),
                           krow.ctypes.data, kcol.ctypes.data, prow.ctypes.data, pcol.ctypes.data)
    return krow, kcol[:tot], prow, pcol[:tot]


def forward(x, y, z, t, P, m, eps=1e-7, tau1=0.9, tau2=1.1, use_cutoff=True):
    """Returns psi, err, mask, stats(L2, L1, max|E|, |id_all|, pairs)."""
    x, y, z, t, P = _f32(x), _f32(y), _f32(z), _f32(t), _p64(P)
    n = x.shape[0]
    psi = np.zeros(n, np.float64)
    err = np.zeros(n, np.float64)
    mask = np.zeros(n, np.uint8)
    st = np.zeros(5, np.float64)
    lib().oracle_forward(x, y, z, t, n, P, P.shape[1], m, neg_ln_eps(eps), tau1, tau2,
                         int(use_cutoff), psi, err, mask, st)
    return psi, err, mask, st


def backward(x, y, z, err, P, m, eps=1e-7, use_cutoff=True):
    """App. A gradients (10 x m) of sum_i err_i^2, and the number of pairs used."""
    x, y, z, P = _f32(x), _f32(y), _f32(z), _p64(P)
    err = np.ascontiguousarray(err, dtype=np.float64)
    g = np.zeros((10, m), np.float64)
    npairs = C.c_int64()
    lib().oracle_backward(x, y, z, x.shape[0], err, P, P.shape[1], m, neg_ln_eps(eps),
                          int(use_cutoff), g.reshape(-1), C.byref(npairs))
    return g, npairs.value


def alpha(g2w, w):
    g2w = np.ascontiguousarray(g2w, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    return lib().oracle_alpha(g2w, w, g2w.shape[0])


def adam(p, g, mo, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    p = np.array(p, np.float64)
    mo = np.array(mo, np.float64)
    v = np.array(v, np.float64)
    g = np.ascontiguousarray(g, np.float64)
    lib().oracle_adam(p, g, mo, v, p.size, t, lr, b1, b2, eps)
    return p, mo, v


def default_cfg(T_e=1600, M_e=2000, lr0=0.01, epoch_steps=1):
    """Algorithm 3 input line and Sec. 4.1 settings; Adam moments at the usual defaults."""
    return Cfg(lr0=lr0, lr_p2=1e-3, lr_min=1e-5, beta1=0.9, beta2=0.999, adam_eps=1e-8,
               tau_m=0.02, tau_d=0.01, tau_l1=5.0, tau_l2=0.5, k_l1=50, k_l2=10, T_e=T_e, M_e=M_e,
               epoch_steps=epoch_steps)


def state_init(cfg):
    st = State()
    lib().oracle_state_init(C.byref(st), C.byref(cfg))
    return st


def step(P, m, grad, mo, v, l2, max_abs_e, cfg, st):
    """One Algorithm 3 update in place on float64 arrays P, mo, v (10 x cap); the
    epoch tail runs after every cfg.epoch_steps-th call."""
    cap = P.shape[1]
    lib().oracle_step(P.reshape(-1), cap, m, np.ascontiguousarray(grad, np.float64).reshape(-1),
                      mo.reshape(-1), v.reshape(-1), l2, max_abs_e, C.byref(cfg), C.byref(st))


def prune(P, m, tau_d=0.01, mo=None, v=None):
    cap = P.shape[1]
    return lib().oracle_prune(P.reshape(-1), None if mo is None else mo.ctypes.data,
                              None if v is None else v.ctypes.data, cap, m, tau_d)


def select_topk(E, mask, thresh, k):
    E = _f32(E)
    mask = np.ascontiguousarray(mask, np.uint8)
    out = np.zeros(max(E.shape[0], 1), np.int32)
    n = lib().oracle_select_topk(E, mask, E.shape[0], thresh, k, out)
    return out[:n].copy()


def local_max(x, y, z, E, mask, cand, r2):
    x, y, z, E = _f32(x), _f32(y), _f32(z), _f32(E)
    mask = np.ascontiguousarray(mask, np.uint8)
    cand = np.ascontiguousarray(cand, np.int32)
    out = np.zeros(max(cand.shape[0], 1), np.int32)
    n = lib().oracle_local_max(x, y, z, E, mask, x.shape[0], cand, cand.shape[0],
                               np.float32(r2), out)
    return out[:n].copy()


def new_kernel(p, e, dbar, eps=1e-7):
    out = np.zeros(10, np.float64)
    lib().oracle_new_kernel(float(p[0]), float(p[1]), float(p[2]), float(e), dbar, eps, out)
    return out


def inscribed(x, y, z, t, S, max_out=1 << 20):
    """Algorithm 1: indices of the selected centres, in order."""
    x, y, z, t, S = _f32(x), _f32(y), _f32(z), _f32(t), _f32(S)
    out = np.zeros(max(max_out, 1), np.int32)
    n = lib().oracle_inscribed(x, y, z, t, S, x.shape[0], out, max_out)
    return out[:min(n, max_out)].copy(), n


def init_shape(c, w, r, gamma=1e-3):
    """Eq. 3-12 for centres c (M x 3), weights w, radii r: the axis parameter d."""
    c = np.ascontiguousarray(c, np.float64)
    w, r = np.ascontiguousarray(w, np.float64), np.ascontiguousarray(r, np.float64)
    d = np.zeros(max(len(w), 1))
    lib().oracle_init_shape(np.ascontiguousarray(c[:, 0]), np.ascontiguousarray(c[:, 1]),
                            np.ascontiguousarray(c[:, 2]), w, r, len(w), gamma, d)
    return d[:len(w)]


def marching_tets(f, shape, origin, h, iso=0.0):
    """Zero level set (value < iso inside) of a grid field f (x fastest), shape
    (nx, ny, nz): triangles as an (ntri, 9) float32 array."""
    f = _f32(f)
    nx, ny, nz = shape
    o = np.asarray(origin, np.float32)
    n = lib().oracle_marching_tets(f, nx, ny, nz, o, h, iso, np.zeros(9, np.float32), 0)
    tri = np.zeros((max(n, 1), 9), np.float32)
    lib().oracle_marching_tets(f, nx, ny, nz, o, h, iso, tri, n)
    return tri[:n]


def sample_surface(tri, u):
    """Area-weighted samples; u: (ns, 3) uniform numbers in [0, 1)."""
    tri = _f32(tri)
    u = np.ascontiguousarray(u, np.float64)
    ns = u.shape[0]
    pts = np.zeros((ns, 3), np.float32)
    nrm = np.zeros((ns, 3), np.float32)
    rc = lib().oracle_sample_surface(tri, tri.shape[0], u, ns, pts, nrm)
    if rc:
        raise ValueError("surface has no area")
    return pts, nrm


def surface_metrics(A, nA, B, nB):
    """(HD, CD, CS) of two sampled surfaces (Sec. 4)."""
    out = np.zeros(3)
    lib().oracle_surface_metrics(_f32(A), _f32(nA), A.shape[0], _f32(B), _f32(nB), B.shape[0], out)
    return tuple(out)
