"""ctypes binding of libserbf.so (include/serbf.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Array
arguments are torch tensors (device memory owned by the caller) or None for a
NULL pointer; the stream defaults to torch's current CUDA stream.  A missing or
unloadable library raises at import time: there is no fallback.
"""
import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libserbf.so")

SERBF_OK = 0
SERBF_EINVAL = -1
SERBF_ENOMEM = -2
SERBF_ECAPACITY = -3
SERBF_ECUDA = -4
SERBF_ETIMEOUT = -5

FLAG_SUPER_LIST, FLAG_ADD_CAPACITY, FLAG_FIX_RANGE = 1, 4, 8

STAT_L2, STAT_L1, STAT_MAXE, STAT_COUNT, STAT_PAIRS_FWD, STAT_PAIRS_BWD = 0, 1, 2, 3, 4, 5
STAT_ALPHA, STAT_BETA, STAT_BF, STAT_LOSS, NSTATS = 6, 7, 8, 9, 16


class SerbfError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__("%s failed: %s (%d)" % (fn, _lib.serbf_status_string(code).decode(), code))
        self.code = code


class Config(C.Structure):
    _fields_ = [("eps", C.c_double), ("tau1", C.c_double), ("tau2", C.c_double), ("tau_m", C.c_double),
                ("tau_d", C.c_double), ("tau_l1", C.c_double), ("tau_l2", C.c_double), ("lr", C.c_double),
                ("lr_p2", C.c_double), ("lr_min", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("adam_eps", C.c_double), ("topk_frac", C.c_double), ("add_radius", C.c_double),
                ("dbar_min", C.c_double), ("k_l1", C.c_int32), ("k_l2", C.c_int32), ("T_e", C.c_int32),
                ("M_e", C.c_int32), ("kahan", C.c_int32), ("fwd_warps", C.c_int32),
                ("epoch_steps", C.c_int32), ("rebuild_levels", C.c_int32)]


class State(C.Structure):
    _fields_ = [("epoch", C.c_int32), ("l1_optim", C.c_int32), ("phase2", C.c_int32), ("adam_t", C.c_int32),
                ("do_prune", C.c_int32), ("do_add", C.c_int32), ("n_l2", C.c_int32), ("n_bf", C.c_int32),
                ("m_added", C.c_int32), ("m_pruned", C.c_int32), ("step", C.c_int32), ("reserved", C.c_int32),
                ("lr", C.c_double), ("alpha", C.c_double), ("beta", C.c_double), ("l2_epoch", C.c_double),
                ("l2_hist", C.c_double * 64), ("bf_hist", C.c_int32 * 256)]


class Points(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("t", C.c_void_p), ("n", C.c_int64)]


class Params(C.Structure):
    _fields_ = [("p", C.c_void_p), ("m", C.c_void_p), ("cap", C.c_int32)]


class Csr(C.Structure):
    _fields_ = [("rowptr", C.c_void_p), ("col", C.c_void_p), ("cap", C.c_int64)]


class Grid(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("h", C.c_float), ("n", C.c_int32 * 3)]


class WsSizes(C.Structure):
    _fields_ = [("max_points", C.c_int64), ("max_kernels", C.c_int32), ("max_cells", C.c_int32),
                ("reserved0", C.c_int32), ("super_cap", C.c_int32), ("super_factor", C.c_int32),
                ("reserved", C.c_int32)]


class Field(C.Structure):
    _fields_ = [("pts", Points), ("S_raw", C.c_void_p), ("psi", C.c_void_p), ("err", C.c_void_p),
                ("mask", C.c_void_p), ("prm", Params), ("grad", C.c_void_p), ("adam_m", C.c_void_p),
                ("adam_v", C.c_void_p), ("st", C.c_void_p), ("stats", C.c_void_p), ("cfg", C.POINTER(Config)),
                ("ws", C.c_void_p)]


VP = C.c_void_p
_SIGS = {
    "serbf_version": (C.c_char_p, []),
    "serbf_status_string": (C.c_char_p, [C.c_int]),
    "serbf_config_default": (C.c_int, [C.POINTER(Config)]),
    "serbf_workspace_struct_size": (C.c_size_t, []),
    "serbf_workspace_bytes": (C.c_int, [C.POINTER(WsSizes), C.POINTER(C.c_size_t)]),
    "serbf_workspace_init": (C.c_int, [VP, VP, C.c_size_t, C.POINTER(WsSizes)]),
    "serbf_workspace_release": (C.c_int, [VP]),
    "serbf_status": (C.c_int, [VP, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.c_int, VP]),
    "serbf_state_init": (C.c_int, [VP, C.POINTER(Config), VP]),
    "serbf_normalize_sdf": (C.c_int, [VP, VP, C.c_int64, VP, VP, VP]),
    "serbf_normalize_sdf_noalloc": (C.c_int, [VP, VP, C.c_int64, VP, VP]),
    "serbf_bin_points": (C.c_int, [VP, VP, VP, C.c_int64, C.POINTER(Grid), VP, VP, VP, VP, VP, VP]),
    "serbf_gather": (C.c_int, [VP, VP, VP, C.c_int64, VP]),
    "serbf_build_neighbors": (C.c_int, [C.POINTER(Points), C.POINTER(Params), C.POINTER(Config),
                                        C.POINTER(Csr), C.POINTER(Csr), C.POINTER(C.c_int64), VP, VP]),
    "serbf_init_kernels": (C.c_int, [C.POINTER(Points), VP, C.c_double, C.POINTER(Params), C.POINTER(C.c_int32), VP,
                                     VP]),
    "serbf_marching_tets": (C.c_int, [VP, C.POINTER(C.c_int32 * 3), C.POINTER(C.c_float * 3), C.c_float, C.c_float,
                                      VP, C.c_int64, C.POINTER(C.c_int64), VP, VP]),
    "serbf_sample_surface": (C.c_int, [VP, C.c_int64, VP, C.c_int64, VP, VP, VP, VP]),
    "serbf_surface_metrics": (C.c_int, [VP, VP, C.c_int64, VP, VP, C.c_int64, C.POINTER(C.c_double * 3), VP, VP]),
    "serbf_denormalize_sdf": (C.c_int, [VP, VP, C.c_int64, VP, VP]),
    "serbf_scatter": (C.c_int, [VP, VP, VP, C.c_int64, VP]),
    "serbf_forward": (C.c_int, [C.POINTER(Points), C.POINTER(Params), C.POINTER(Config), VP, VP, VP, VP,
                                VP, VP]),
    "serbf_forward_backward": (C.c_int, [C.POINTER(Points), C.POINTER(Params), C.POINTER(Config), VP, VP, VP, VP,
                                         VP, VP, VP]),
    "serbf_backward": (C.c_int, [C.POINTER(Points), C.POINTER(Params), C.POINTER(Config), VP, VP, VP, VP,
                                 VP]),
    "serbf_step": (C.c_int, [C.POINTER(Params), VP, VP, VP, VP, VP, C.POINTER(Config), VP, VP]),
    "serbf_prune": (C.c_int, [C.POINTER(Params), VP, VP, VP, C.POINTER(Config), VP]),
    "serbf_add_kernels": (C.c_int, [C.POINTER(Points), VP, VP, VP, C.POINTER(Params), VP, VP, VP, VP,
                                    C.POINTER(Config), C.c_int, VP, VP]),
    "serbf_refine": (C.c_int, [VP, VP, VP, VP, VP, C.c_int64, VP, VP, VP, VP, VP, C.c_int64, C.POINTER(Grid),
                               VP, VP, VP, VP, VP, VP, VP, VP]),
    "serbf_batch_struct_size": (C.c_size_t, []),
    "serbf_batch_bytes": (C.c_int, [C.c_int32, C.POINTER(C.c_size_t)]),
    "serbf_batch_init": (C.c_int, [VP, C.POINTER(Field), C.c_int32, C.c_int32, VP, C.c_size_t, VP]),
    "serbf_batch_warps": (C.c_int, [VP]),
    "serbf_epoch_batched": (C.c_int, [VP, VP]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libserbf.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
lib = _lib


def symbols():
    return sorted(_SIGS)


def _p(t):
    """Device pointer of a tensor (None -> NULL)."""
    return None if t is None else t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(name, rc, ok=(SERBF_OK,)):
    if rc not in ok:
        raise SerbfError(name, rc)
    return rc


def version():
    """serbf_version(): the library's version string."""
    return _lib.serbf_version().decode()


def config_default(**over):
    c = Config()
    _check("serbf_config_default", _lib.serbf_config_default(C.byref(c)))
    for k, v in over.items():
        setattr(c, k, v)
    return c


def serbf_workspace_bytes(sizes):
    b = C.c_size_t()
    _check("serbf_workspace_bytes", _lib.serbf_workspace_bytes(C.byref(sizes), C.byref(b)))
    return b.value


def serbf_workspace_init(ws_host, dev, sizes):
    return _check("serbf_workspace_init",
                  _lib.serbf_workspace_init(C.addressof(ws_host), _p(dev), dev.numel() * dev.element_size(),
                                            C.byref(sizes)))


def serbf_workspace_release(ws_host):
    return _check("serbf_workspace_release", _lib.serbf_workspace_release(C.addressof(ws_host)))


def serbf_status(ws_host, clear=False, stream=None):
    f = C.c_int32()
    nd = (C.c_int64 * 4)()
    rc = _lib.serbf_status(C.addressof(ws_host), C.byref(f), nd, int(clear), _stream(stream))
    _check("serbf_status", rc, ok=(SERBF_OK, SERBF_ECAPACITY))
    return f.value, list(nd)


def serbf_state_init(st, cfg, stream=None):
    return _check("serbf_state_init", _lib.serbf_state_init(_p(st), C.byref(cfg), _stream(stream)))


def serbf_normalize_sdf(S, t, mh, ws_host, stream=None):
    return _check("serbf_normalize_sdf", _lib.serbf_normalize_sdf(_p(S), _p(t), S.numel(), _p(mh),
                                                                  C.addressof(ws_host), _stream(stream)))


def serbf_normalize_sdf_noalloc(S, t, mh, stream=None, n=None):
    """Eq. 3-10 without a workspace (for callers that cannot allocate device memory)."""
    n = S.numel() if n is None else n
    rc = _lib.serbf_normalize_sdf_noalloc(_p(S), _p(t), n, _p(mh), _stream(stream))
    if rc == SERBF_ECAPACITY:
        raise SerbfError("serbf_normalize_sdf_noalloc (n > 67,108,864 points)", rc)
    return _check("serbf_normalize_sdf_noalloc", rc)


def serbf_bin_points(x, y, z, grid, perm, xb, yb, zb, ws_host, stream=None):
    return _check("serbf_bin_points", _lib.serbf_bin_points(_p(x), _p(y), _p(z), x.numel(), C.byref(grid), _p(perm),
                                                            _p(xb), _p(yb), _p(zb), C.addressof(ws_host),
                                                            _stream(stream)))


def serbf_gather(src, perm, dst, n=None, stream=None):
    n = perm.numel() if n is None else n
    return _check("serbf_gather", _lib.serbf_gather(_p(src), _p(perm), _p(dst), n, _stream(stream)))


def points(x, y, z, t, n=None):
    return Points(_p(x), _p(y), _p(z), _p(t), x.numel() if n is None else n)


def params(p, m_dev):
    return Params(_p(p), _p(m_dev), p.shape[1])


def csr(rowptr, col):
    return Csr(_p(rowptr), _p(col), 0 if col is None else col.numel())


def serbf_build_neighbors(pts, prm, cfg, ws_host, kmajor=None, pmajor=None, stream=None):
    npairs = C.c_int64(-1)
    rc = _lib.serbf_build_neighbors(C.byref(pts), C.byref(prm), C.byref(cfg),
                                    None if kmajor is None else C.byref(kmajor),
                                    None if pmajor is None else C.byref(pmajor), C.byref(npairs),
                                    C.addressof(ws_host), _stream(stream))
    _check("serbf_build_neighbors", rc, ok=(SERBF_OK, SERBF_ECAPACITY))
    return rc, npairs.value


def serbf_init_kernels(pts, S_raw, gamma, prm, ws_host, stream=None):
    """Algorithm 1 + Eq. 3-12; returns (status, number of centres found)."""
    mo = C.c_int32(0)
    rc = _lib.serbf_init_kernels(C.byref(pts), _p(S_raw), float(gamma), C.byref(prm), C.byref(mo),
                                 C.addressof(ws_host), _stream(stream))
    _check("serbf_init_kernels", rc, ok=(SERBF_OK, SERBF_ECAPACITY))
    return rc, mo.value


def serbf_marching_tets(f, dims, origin, h, iso, tri, ntri_cap, scratch, stream=None):
    """Returns (status, triangle count); tri may be None with ntri_cap 0 to count."""
    n = C.c_int64(0)
    rc = _lib.serbf_marching_tets(_p(f), C.byref((C.c_int32 * 3)(*dims)), C.byref((C.c_float * 3)(*origin)), h, iso,
                                  _p(tri), ntri_cap, C.byref(n), _p(scratch), _stream(stream))
    _check("serbf_marching_tets", rc, ok=(SERBF_OK, SERBF_ECAPACITY))
    return rc, n.value


def serbf_sample_surface(tri, ntri, u, ns, pts, nrm, scratch, stream=None):
    return _check("serbf_sample_surface", _lib.serbf_sample_surface(_p(tri), ntri, _p(u), ns, _p(pts), _p(nrm),
                                                                    _p(scratch), _stream(stream)))


def serbf_surface_metrics(A, nA, na, B, nB, nb, scratch, stream=None):
    out = (C.c_double * 3)()
    _check("serbf_surface_metrics", _lib.serbf_surface_metrics(_p(A), _p(nA), na, _p(B), _p(nB), nb, C.byref(out),
                                                               _p(scratch), _stream(stream)))
    return tuple(out)


def serbf_denormalize_sdf(t, S, n, mh, stream=None):
    return _check("serbf_denormalize_sdf", _lib.serbf_denormalize_sdf(_p(t), _p(S), n, _p(mh), _stream(stream)))


def serbf_scatter(src, idx, dst, n, stream=None):
    return _check("serbf_scatter", _lib.serbf_scatter(_p(src), _p(idx), _p(dst), n, _stream(stream)))


def serbf_forward(pts, prm, cfg, psi, err, mask, stats, ws_host, stream=None):
    return _check("serbf_forward", _lib.serbf_forward(C.byref(pts), C.byref(prm), C.byref(cfg), _p(psi), _p(err),
                                                      _p(mask), _p(stats), C.addressof(ws_host), _stream(stream)))


def serbf_forward_backward(pts, prm, cfg, psi, err, mask, grad, stats, ws_host, stream=None):
    return _check("serbf_forward_backward",
                  _lib.serbf_forward_backward(C.byref(pts), C.byref(prm), C.byref(cfg), _p(psi), _p(err), _p(mask),
                                              _p(grad), _p(stats), C.addressof(ws_host), _stream(stream)))


def serbf_backward(pts, prm, cfg, err, grad, stats, ws_host, stream=None):
    return _check("serbf_backward", _lib.serbf_backward(C.byref(pts), C.byref(prm), C.byref(cfg), _p(err),
                                                        _p(grad), _p(stats), C.addressof(ws_host),
                                                        _stream(stream)))


def serbf_step(prm, grad, adam_m, adam_v, st, stats, cfg, ws_host, stream=None):
    return _check("serbf_step", _lib.serbf_step(C.byref(prm), _p(grad), _p(adam_m), _p(adam_v), _p(st), _p(stats),
                                                C.byref(cfg), C.addressof(ws_host), _stream(stream)))


def serbf_prune(prm, adam_m, adam_v, st, cfg, stream=None):
    return _check("serbf_prune", _lib.serbf_prune(C.byref(prm), _p(adam_m), _p(adam_v), _p(st), C.byref(cfg),
                                                  _stream(stream)))


def serbf_add_kernels(pts, S_raw, err, mask, prm, adam_m, adam_v, st, stats, cfg, ws_host, force=False,
                      stream=None):
    return _check("serbf_add_kernels",
                  _lib.serbf_add_kernels(C.byref(pts), _p(S_raw), _p(err), _p(mask), C.byref(prm), _p(adam_m),
                                         _p(adam_v), _p(st), _p(stats), C.byref(cfg), int(force),
                                         C.addressof(ws_host), _stream(stream)))


def serbf_refine(x_all, y_all, z_all, t_all, s_all, n_old, x_new, y_new, z_new, t_new, s_new, grid, perm, xb, yb,
                 zb, tb, sb, ws_host, stream=None):
    n_new = x_new.numel()
    return _check("serbf_refine",
                  _lib.serbf_refine(_p(x_all), _p(y_all), _p(z_all), _p(t_all), _p(s_all), n_old, _p(x_new),
                                    _p(y_new), _p(z_new), _p(t_new), _p(s_new), n_new, C.byref(grid), _p(perm),
                                    _p(xb), _p(yb), _p(zb), _p(tb), _p(sb), C.addressof(ws_host),
                                    _stream(stream)))


def workspace_struct():
    """Host storage for one serbf_workspace (opaque)."""
    return C.create_string_buffer(_lib.serbf_workspace_struct_size())


def batch_struct():
    """Host storage for one serbf_batch (opaque)."""
    return C.create_string_buffer(_lib.serbf_batch_struct_size())


def serbf_batch_bytes(nfields):
    b = C.c_size_t()
    _check("serbf_batch_bytes", _lib.serbf_batch_bytes(int(nfields), C.byref(b)))
    return b.value


def serbf_batch_init(b_host, fields, fwd_warps, dev, stream=None):
    arr = (Field * len(fields))(*fields)
    return _check("serbf_batch_init", _lib.serbf_batch_init(C.addressof(b_host), arr, len(fields), int(fwd_warps),
                                                            _p(dev), dev.numel() * dev.element_size(),
                                                            _stream(stream)))


def serbf_batch_warps(b_host):
    return _lib.serbf_batch_warps(C.addressof(b_host))


def serbf_epoch_batched(b_host, stream=None):
    return _check("serbf_epoch_batched", _lib.serbf_epoch_batched(C.addressof(b_host), _stream(stream)))


STATE_BYTES = C.sizeof(State)
