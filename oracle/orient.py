"""Parity-based normal orientation (Sec. 2.2): point-cloud ray casting with a
finite detection radius and the three-iteration refinement.  Test
infrastructure only: the CUDA path never imports it.

Steps, in the paper's order and notation:
  r_{d,0} = 1/2 max_i min_{j != i} |x_i - x_j|          (Eq. baseline_detection_radius)
  r_d     = gamma_r r_{d,0}                             (Eq. expanded_detection_radius)
  y_{i,m} = x_i + m ds u_i,  m = 0, 1, ..., M           (probe points, u_i = n_i / |n_i|)
  d_{i,m} = 1 if some x_j lies within r_d of y_{i,m}    (detection array)
  N_all   = #{m >= 1 : d_{i,m} = 0 and d_{i,m-1} = 1}   (1 -> 0 transitions)
  N_i     = N_all - 1                                   (Eq. N_i_define)
  N_one   = the number of leading ones of d_{i,.}
  iteration 0: flip if N_i is odd                       (Eq. basic_parity_flip)
  iteration 1: flip if N_i != 0 or N_one > N_tol
  iteration 2: flip if N_i > N_i^- (N_i^- along -n_i)

Readings where the paper is silent:
  * ds = r_d (consecutive probe balls overlap; a surface band of a sampled
    surface holds at least one probe when gamma_r r_{d,0} >= ds / 2 + r_{d,0});
  * M is the first probe outside the cloud's bounding box widened by r_d on
    every side (that probe detects nothing, so the array ends with a 0);
  * every iteration looks at every point, along its current normal.  Only
    signs change, so the patterns along +n_i and -n_i (as given) settle all
    three iterations;
  * the ray direction is the normal scaled to unit length in float32,
    u = n / sqrt((n_x^2 + n_y^2) + n_z^2), each operation rounded (D-PCA
    normals are unit already; the scaling bounds the probe count);
  * the integer decisions (nearest-neighbour distances, detections, the box
    exit) are taken in float32, the precision of the paper's kernels:
    d2 = ((dx*dx + dy*dy) + dz*dz) with every operation rounded, probes
    y = x + (m ds) u rounded per operation, r_{d,0} = 0.5 sqrt(max d2) and
    r_d = gamma_r r_{d,0} rounded to float32;
  * a zero or non-finite normal, a non-finite point, or r_d = 0 (fewer than
    two distinct points) leaves the normal as it is, with zero statistics.
    Non-finite points are not part of the cloud.  A flip negates the normal
    as given.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree


def _d2_f32(A, b):
    """Squared float32 distances of the rows of A to b, ((dx^2 + dy^2) + dz^2)
    with every operation rounded to float32."""
    d = np.asarray(A, dtype=np.float32) - np.asarray(b, dtype=np.float32)
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def detection_radius(points, gamma: float = 2.5):
    """(r_d, r_{d,0}) as float32 for the finite points of the cloud."""
    P = np.asarray(points, dtype=np.float64)
    P = P[np.isfinite(P).all(axis=1)]
    if len(P) < 2:
        return np.float32(0), np.float32(0)
    P32 = P.astype(np.float32)
    tree = cKDTree(P)
    k = min(9, len(P))
    dist, idx = tree.query(P, k=k)
    best = np.full(len(P), np.inf, dtype=np.float32)
    for c in range(k):
        other = idx[:, c] != np.arange(len(P))
        d2 = _d2_f32(P32[idx[:, c]], P32)
        best = np.where(other & (d2 < best), d2, best)
    # nearest distance in FP64 (column 1 unless duplicates sit at distance 0)
    nn64 = np.where(idx[:, 0] == np.arange(len(P)), dist[:, 1], dist[:, 0]) if k > 1 else dist[:, 0]
    # where the k-th neighbour is not clearly farther than the nearest, the
    # float32 minimum could lie beyond the k found: test the whole ball
    unsure = dist[:, -1] <= nn64 * (1 + 1e-5) + 1e-30
    for i in np.nonzero(unsure)[0]:
        cand = np.asarray(tree.query_ball_point(P[i], nn64[i] * (1 + 1e-5) + 1e-30), dtype=np.int64)
        cand = cand[cand != i]
        if len(cand):
            best[i] = min(best[i], _d2_f32(P32[cand], P32[i]).min())
    r0 = np.float32(0.5) * np.sqrt(np.float32(best.max()))
    return np.float32(np.float32(gamma) * r0), np.float32(r0)


class _Detector:
    """d(y) = 1 iff some cloud point lies within r_d of y (float32 test)."""

    def __init__(self, P, rd):
        self.P32 = np.asarray(P, dtype=np.float32)
        self.tree = cKDTree(self.P32.astype(np.float64))
        self.rd = np.float32(rd)
        self.rd2 = np.float32(self.rd * self.rd)

    def __call__(self, Y32):
        Y32 = np.asarray(Y32, dtype=np.float32).reshape(-1, 3)
        if len(Y32) == 0:
            return np.zeros(0, dtype=bool)
        dist, j = self.tree.query(Y32.astype(np.float64), k=1)
        rd = float(self.rd)
        out = dist < rd * (1 - 1e-5)
        band = np.nonzero(np.abs(dist - rd) <= rd * 1e-5)[0]
        for b in band:
            cand = np.asarray(self.tree.query_ball_point(Y32[b].astype(np.float64), rd * (1 + 1e-5)),
                              dtype=np.int64)
            out[b] = bool(len(cand)) and bool((_d2_f32(self.P32[cand], Y32[b]) <= self.rd2).any())
        return out


def unit_direction(n):
    """n / |n| in float32, or None for a zero or non-finite normal."""
    n32 = np.asarray(n, dtype=np.float32)
    ss = (n32[0] * n32[0] + n32[1] * n32[1]) + n32[2] * n32[2]
    if not (ss > 0 and np.isfinite(ss)):
        return None
    return n32 / np.sqrt(ss)


def detection_array(x, n, rd, det: _Detector, lo, hi):
    """d_{i,0..M} along y_m = x + m ds n, ds = r_d, ending at the first probe
    outside [lo - r_d, hi + r_d] (float32 throughout)."""
    x32 = np.asarray(x, dtype=np.float32)
    n32 = np.asarray(n, dtype=np.float32)
    rd = np.float32(rd)
    lo_e = np.asarray(lo, dtype=np.float32) - rd
    hi_e = np.asarray(hi, dtype=np.float32) + rd
    out = []
    m0 = 0
    chunk = 64
    while True:
        m = np.arange(m0, m0 + chunk, dtype=np.float32)
        t = m * rd
        Y = x32[None, :] + t[:, None] * n32[None, :]
        outside = ((Y < lo_e) | (Y > hi_e)).any(axis=1)
        stop = np.nonzero(outside)[0]
        last = stop[0] if len(stop) else chunk
        d = det(Y[:last])
        out.extend(d.tolist())
        if len(stop):
            out.append(False)
            return np.array(out, dtype=bool)
        m0 += chunk


def crossings(d):
    """(N_i, N_one) of a detection array: N_i = #(1 -> 0 transitions) - 1 and
    the number of leading ones."""
    d = np.asarray(d, dtype=bool)
    n_all = int(np.count_nonzero(~d[1:] & d[:-1]))
    zeros = np.nonzero(~d)[0]
    n_one = int(zeros[0]) if len(zeros) else len(d)
    return n_all - 1, n_one


def orient(points, normals, gamma: float = 2.5, n_tol: int = 2, only=None):
    """Oriented normals and per-point statistics int64 [n, 5]:
    (N along +n, N_one along +n, N along -n, N_one along -n, flags) with flag
    bits 1, 2, 4 = flipped by iteration 0, 1, 2 and 8 = final normal is -n.
    Also returns r_d.  `only` (indices) restricts the rays to those points;
    r_d and the detections still use the whole cloud."""
    P = np.asarray(points, dtype=np.float64)
    Nrm = np.asarray(normals, dtype=np.float32).copy()
    n = len(P)
    stats = np.zeros((n, 5), dtype=np.int64)
    ok = np.isfinite(P).all(axis=1) if n else np.zeros(0, dtype=bool)
    rd, _ = detection_radius(P, gamma)
    if n == 0 or rd == 0:
        return Nrm, stats, rd
    C = P[ok]
    det = _Detector(C, rd)
    lo = C.astype(np.float32).min(axis=0)
    hi = C.astype(np.float32).max(axis=0)
    P32 = P.astype(np.float32)
    todo = np.nonzero(ok)[0] if only is None else [i for i in np.asarray(only) if ok[i]]
    for i in todo:
        nv = Nrm[i]
        u = unit_direction(nv)
        if u is None:
            continue
        Np, op = crossings(detection_array(P32[i], u, rd, det, lo, hi))
        Nm, om = crossings(detection_array(P32[i], -u, rd, det, lo, hi))
        s, flags = 1, 0
        # iteration 0: standard parity along the estimated normal
        if Np % 2 == 1:
            s, flags = -s, flags | 1
        # iteration 1: along the current normal
        Nc, oc = (Np, op) if s > 0 else (Nm, om)
        if Nc != 0 or oc > n_tol:
            s, flags = -s, flags | 2
        # iteration 2: the current direction against the opposite one
        Nc, No = (Np, Nm) if s > 0 else (Nm, Np)
        if Nc > No:
            s, flags = -s, flags | 4
        if s < 0:
            flags |= 8
            Nrm[i] = -nv
        stats[i] = (Np, op, Nm, om, flags)
    return Nrm, stats, rd
