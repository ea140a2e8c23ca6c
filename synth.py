"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no arithmetic of the fitting method: it only makes signed
distance samples of analytic shapes on vertex grids, point subsets, and the
random initial kernel parameters the workloads start from.  The paper's own
inputs (octree grids of meshes from public datasets, SDFs computed by a mesh
library) are not available here; these analytic shapes stand in for them.

Grids are vertex grids over [-1, 1]^3 with x_i = -1 + 2 i / (n - 1), linear
index (iz * n + iy) * n + ix.  Parameter arrays are float32, 10 rows of `cap`
columns in the order cx, cy, cz, d1, d2, d3, theta_x, theta_y, theta_z, w,
with d = 1 / (axis length).
"""
import math

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def grid(n):
    """Vertex grid n^3 over [-1,1]^3 as float32 x, y, z (x fastest)."""
    a = -1.0 + 2.0 * np.arange(n, dtype=np.float64) / (n - 1)
    z, y, x = np.meshgrid(a, a, a, indexing="ij")
    return (x.reshape(-1).astype(np.float32), y.reshape(-1).astype(np.float32),
            z.reshape(-1).astype(np.float32))


def spacing(n):
    return 2.0 / (n - 1)


def sdf_sphere(x, y, z, r=0.5):
    x, y, z = (np.asarray(v, np.float64) for v in (x, y, z))
    return (np.sqrt(x * x + y * y + z * z) - r).astype(np.float32)


def sdf_torus(x, y, z, R=0.5, r=0.2):
    x, y, z = (np.asarray(v, np.float64) for v in (x, y, z))
    q = np.sqrt(x * x + y * y) - R
    return (np.sqrt(q * q + z * z) - r).astype(np.float32)


def _random_rotation(g):
    """Uniform random rotation matrix from a unit quaternion."""
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def random_primitives(seed, count, centre=0.7, size=(0.05, 0.3)):
    """Union of `count` random ellipsoids, boxes and capsules (list of dicts)."""
    g = rng(seed)
    prims = []
    for k in range(count):
        kind = ("ellipsoid", "box", "capsule")[k % 3]
        prims.append(dict(kind=kind, c=g.uniform(-centre, centre, 3), R=_random_rotation(g),
                          s=g.uniform(size[0], size[1], 3)))
    return prims


def sdf_primitives(prims, x, y, z):
    p = np.stack([np.asarray(v, np.float64) for v in (x, y, z)], axis=1)
    out = np.full(p.shape[0], np.inf)
    for pr in prims:
        lp = (p - pr["c"]) @ pr["R"]  # coordinates in the primitive frame
        s = pr["s"]
        if pr["kind"] == "ellipsoid":
            d = (np.linalg.norm(lp / s, axis=1) - 1.0) * s.min()
        elif pr["kind"] == "box":
            q = np.abs(lp) - s
            d = np.linalg.norm(np.maximum(q, 0.0), axis=1) + np.minimum(q.max(axis=1), 0.0)
        else:  # capsule along local z, half length s[2], radius s[0]
            zc = np.clip(lp[:, 2], -s[2], s[2])
            d = np.sqrt(lp[:, 0] ** 2 + lp[:, 1] ** 2 + (lp[:, 2] - zc) ** 2) - s[0]
        out = np.minimum(out, d)
    return out.astype(np.float32)


def band_far_mask(S, band=0.1, stride=8):
    """Narrow band |S| < band plus every `stride`-th point of the rest (by linear index)."""
    idx = np.arange(S.shape[0])
    return (np.abs(S) < band) | (idx % stride == 0)


def haar_angles(g, m):
    """Angles with the Haar distribution for R = Rz(a) Ry(b) Rx(c): a, c uniform, sin b uniform."""
    a = g.uniform(-math.pi, math.pi, m)
    b = np.arcsin(g.uniform(-1.0, 1.0, m))
    c = g.uniform(-math.pi, math.pi, m)
    return a, b, c


def init_kernels(seed, m, cap=None, centre=0.6, length=0.15, length_range=None, rotate=False,
                 w_std=0.1):
    """Random initial parameters (10 x cap float32)."""
    cap = m if cap is None else cap
    g = rng(seed)
    P = np.zeros((10, cap), np.float32)
    P[0:3, :m] = g.uniform(-centre, centre, (3, m))
    if length_range is None:
        P[3:6, :m] = 1.0 / length
    else:
        P[3:6, :m] = 1.0 / g.uniform(length_range[0], length_range[1], (3, m))
    if rotate:
        a, b, c = haar_angles(g, m)
        P[6, :m], P[7, :m], P[8, :m] = a, b, c
    P[9, :m] = g.normal(0.0, w_std, m)
    return P


CONFIGS = {
    # sphere |x|-0.5 on 32^3, 64 isotropic kernels of length 0.15, identity rotation
    "c1": dict(shape="sphere", grids=[32], m=64, seed=1, length=0.15, length_range=None,
               rotate=False, steps=200),
    # torus (R=0.5, r=0.2) on 64^3 with a 32^3 coarse layer first, 512 anisotropic rotated kernels
    "c2": dict(shape="torus", grids=[32, 64], m=512, seed=2, length=None, length_range=(0.05, 0.2),
               rotate=True, steps=200),
    # union of 20 random primitives on 128^3, 4096 kernels
    "c3": dict(shape="prims20", grids=[128], m=4096, seed=3, length=None,
               length_range=(0.05 * 0.5, 0.2 * 0.5), rotate=True, steps=200),
    # union of 60 random primitives on 256^3, band |S|<0.1 plus 1/8 far field, 16384 kernels
    "c4": dict(shape="prims60", grids=[256], m=16384, seed=4, length=None,
               length_range=(0.05 * (512 / 16384) ** (1 / 3), 0.2 * (512 / 16384) ** (1 / 3)),
               rotate=True, steps=50, band=0.1),
}


def shape_sdf(name, seed, x, y, z):
    if name == "sphere":
        return sdf_sphere(x, y, z)
    if name == "torus":
        return sdf_torus(x, y, z)
    if name.startswith("prims"):
        return sdf_primitives(random_primitives(seed + 1000, int(name[5:])), x, y, z)
    raise ValueError(name)


def layer(cfg, n):
    """One grid layer of a config: x, y, z, S (float32), optionally band-restricted."""
    x, y, z = grid(n)
    S = shape_sdf(cfg["shape"], cfg["seed"], x, y, z)
    if cfg.get("band"):
        keep = band_far_mask(S, cfg["band"])
        x, y, z, S = x[keep], y[keep], z[keep], S[keep]
    return x, y, z, S


def workload(name, cap=None, layers=None):
    """Training layers (coarse to fine) and initial parameters of a named config."""
    cfg = dict(CONFIGS[name])
    grids = cfg["grids"] if layers is None else layers
    lay = [layer(cfg, n) for n in grids]
    P = init_kernels(cfg["seed"], cfg["m"], cap=cap, length=cfg["length"] or 0.15,
                     length_range=cfg["length_range"], rotate=cfg["rotate"])
    return cfg, lay, P


def sdf_primitives_torch(prims, x, y, z, device):
    """sdf_primitives evaluated with torch (float64) on `device`; same formulas."""
    import torch
    p = torch.stack([torch.as_tensor(np.asarray(v, np.float64), device=device) for v in (x, y, z)], dim=1)
    out = torch.full((p.shape[0],), float("inf"), dtype=torch.float64, device=device)
    for pr in prims:
        c = torch.as_tensor(pr["c"], device=device)
        R = torch.as_tensor(pr["R"], device=device)
        s = torch.as_tensor(pr["s"], device=device)
        lp = (p - c) @ R
        if pr["kind"] == "ellipsoid":
            d = (torch.linalg.norm(lp / s, dim=1) - 1.0) * s.min()
        elif pr["kind"] == "box":
            q = lp.abs() - s
            d = torch.linalg.norm(q.clamp(min=0.0), dim=1) + q.max(dim=1).values.clamp(max=0.0)
        else:
            zc = lp[:, 2].clamp(-s[2], s[2])
            d = torch.sqrt(lp[:, 0] ** 2 + lp[:, 1] ** 2 + (lp[:, 2] - zc) ** 2) - s[0]
        out = torch.minimum(out, d)
    return out.to(torch.float32).cpu().numpy()


def batch_workload(count=64, seed=500, device=None):
    """Independent random-primitive shapes with uneven grids and kernel counts:
    per shape 5..40 primitives, a vertex grid of 32, 48, 64, 96 or 128 points
    per axis, 64..2048 kernels (log-uniform) with lengths
    U(0.05, 0.2) (512 / M)^(1/3) and random rotations.  Returns a list of
    dicts (x, y, z, S, P, m, spacing, n, prims).  With a torch device the
    distances are evaluated there (same formulas)."""
    out = []
    for k in range(count):
        g = rng(seed + k)
        nprim = int(g.integers(5, 41))
        n = int(g.choice([32, 48, 64, 96, 128]))
        m = int(round(math.exp(g.uniform(math.log(64), math.log(2048)))))
        x, y, z = grid(n)
        prims = random_primitives(seed + 1000 + k, nprim)
        S = sdf_primitives(prims, x, y, z) if device is None else sdf_primitives_torch(prims, x, y, z, device)
        scale = (512.0 / m) ** (1.0 / 3.0)
        P = init_kernels(seed + 2000 + k, m, length_range=(0.05 * scale, 0.2 * scale), rotate=True)
        out.append(dict(x=x, y=y, z=z, S=S, P=P, m=m, spacing=spacing(n), n=n, prims=nprim))
    return out


def octree_layers(sdf, l_min, l_max, lo=-1.0, hi=1.0):
    """Grid points of an adaptive octree over [lo, hi]^3 (Sec. 3.4.2's
    hierarchical grids), layer by layer.

    Level l has cells of edge (hi - lo) / 2^l.  Every cell of level l_min is
    kept; a kept cell of level l is split into its 8 children when the
    surface may cross it: |sdf(centre)| <= half its diagonal (exact for a
    true distance function).  Layer l holds the corners of the kept cells of
    level l that are not corners of a coarser layer.  `sdf` maps float64
    arrays (x, y, z) to distances.  Returns a list of (x, y, z, S, spacing)
    with float32 coordinates and S, from l_min to l_max."""
    layers = []
    seen = set()
    res = 2 ** l_max  # integer coordinates on the finest lattice
    cells = np.stack(np.meshgrid(*[np.arange(2 ** l_min)] * 3, indexing="ij"), -1).reshape(-1, 3)
    for l in range(l_min, l_max + 1):
        step = res // (2 ** l)
        edge = (hi - lo) / 2 ** l
        corners = (cells[:, None, :] + np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)])[None])
        corners = np.unique(corners.reshape(-1, 3) * step, axis=0)
        key = (corners[:, 0] * (res + 1) + corners[:, 1]) * (res + 1) + corners[:, 2]
        new = np.array([k not in seen for k in key.tolist()], bool)
        seen.update(key[new].tolist())
        pts = corners[new]
        # z slowest, x fastest, as the vertex grids
        order = np.lexsort((pts[:, 0], pts[:, 1], pts[:, 2]))
        pts = pts[order]
        xyz = lo + (hi - lo) * pts.astype(np.float64) / res
        S = np.asarray(sdf(xyz[:, 0], xyz[:, 1], xyz[:, 2]), np.float64)
        layers.append((xyz[:, 0].astype(np.float32), xyz[:, 1].astype(np.float32), xyz[:, 2].astype(np.float32),
                       S.astype(np.float32), edge))
        if l == l_max:
            break
        centre = lo + edge * (cells.astype(np.float64) + 0.5)
        near = np.abs(np.asarray(sdf(centre[:, 0], centre[:, 1], centre[:, 2]), np.float64)) <= 0.5 * math.sqrt(3) * edge
        kids = cells[near]
        cells = (2 * kids[:, None, :] + np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)])[None]
                 ).reshape(-1, 3)
    return layers
