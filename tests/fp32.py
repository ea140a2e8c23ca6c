"""Exact float32 arithmetic helpers for the CPU pins: a correctly rounded
float32 fused multiply-add, and the canonical float32 squared distance of
the support test (the differences, fl(dx dx), then two fused multiply-adds)."""
import numpy as np


def fmaf(a, b, c):
    """float32 fma(a, b, c), rounded once.  The product of two float32 values
    is exact in float64; TwoSum gives the float64 sum s and its exact
    residual, and the residual breaks the tie when s lies exactly halfway
    between two float32 neighbours."""
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    p = a * b
    s = p + c
    bb = s - p
    err = (p - (s - bb)) + (c - bb)
    r = s.astype(np.float32)
    r64 = r.astype(np.float64)
    other = np.nextafter(r, np.where(s > r64, np.float32(np.inf), np.float32(-np.inf)).astype(np.float32))
    mid = (r64 + other.astype(np.float64)) * 0.5
    tie = (s == mid) & (err != 0)
    up = other.astype(np.float64) > r64
    pick_other = tie & (((err > 0) & up) | ((err < 0) & ~up))
    return np.where(pick_other, other, r).astype(np.float32)


def support_d2(dx, dy, dz):
    dx, dy, dz = (np.asarray(v, np.float32) for v in (dx, dy, dz))
    return fmaf(dz, dz, fmaf(dy, dy, (dx * dx).astype(np.float32)))
