"""CPU oracle (FP64) for the periodic neighbor query, RDF and Steinhardt q_l.

TEST INFRASTRUCTURE: only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg
of `bench.py` may import this package.  It shares no code with the CUDA library
(`paper_1906_06317_gb300`) and never imports it.

The arithmetic lives in `oracle.c` (plain loops, one query at a time); this module only
marshals numpy arrays through ctypes and splits query ranges over host threads (ctypes
releases the GIL during the call, so the threads run the C loops in parallel).
"""
from __future__ import annotations

import ctypes
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import build as _build

OK, ERR_ARG, ERR_BOX_TOO_SMALL, ERR_OOM = 0, -1, -2, -3

_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int
_D = ctypes.c_double


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_box_widths.argtypes = [_P, _P]
        L.orc_min_image.argtypes = [_P, _P, _P, _P, _P]
        L.orc_cells_dims.argtypes = [_P, _D, _P]
        L.orc_cells_build.argtypes = [_P, _P, _I64, _P, _P, _P]
        L.orc_ball_query.argtypes = [_P, _P, _I64, _P, _P, _P, _P, _I64, _I64, _D, _I32, _P, _P, _P, _P]
        L.orc_knn.argtypes = [_P, _P, _I64, _P, _P, _P, _P, _I64, _I64, _I32, _I32, _P, _P, _P]
        L.orc_rdf_edges.argtypes = [_I32, _D, _D, _P]
        L.orc_rdf.argtypes = [_P, _P, _I64, _P, _P, _P, _P, _I64, _I64, _I32, _D, _D, _I32, _P]
        L.orc_ylm.argtypes = [_I32, _I32, _D, _D, _D, _P, _P]
        L.orc_steinhardt_ylm.argtypes = [_P, _P, _I64, _P, _P, _I32, _P, _I64, _P, _P]
        L.orc_descriptors.argtypes = [_P, _P, _P, _I64, _P, _P, _I32, _I32, _P]
        L.orc_steinhardt_legendre.argtypes = [_P, _P, _I64, _P, _P, _I32, _P, _I64, _P]
        L.orc_q_grad.argtypes = [_P, _P, _I64, _P, _P, _I32, _P]
        L.orc_pmftxy.argtypes = [_P, _P, _P, _P, _I64, _P, _P, _D, _D, _I32, _I32, _P, _P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(code, what):
    if code != OK:
        raise OracleError(code, what)


def _box(box) -> np.ndarray:
    b = np.asarray(box.params() if hasattr(box, "params") else box, dtype=np.float64)
    assert b.shape == (6,)
    return np.ascontiguousarray(b)


def _pts(x) -> np.ndarray:
    x = np.asarray(x)
    assert x.ndim == 2 and x.shape[1] == 3
    return np.ascontiguousarray(x.astype(np.float64))


def default_threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _ranges(n, threads, min_chunk=256):
    chunks = max(1, min(threads * 4, (n + min_chunk - 1) // min_chunk))
    edges = np.linspace(0, n, chunks + 1).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


def box_widths(box) -> np.ndarray:
    w = np.zeros(3)
    lib().orc_box_widths(_ptr(_box(box)), _ptr(w))
    return w


def min_image(box, xi, xj):
    """Minimum-image displacement x_j - x_i (exact FP64 sequence) and its length."""
    d = np.zeros(3)
    r = np.zeros(1)
    lib().orc_min_image(_ptr(_box(box)), _ptr(np.asarray(xi, np.float64)), _ptr(np.asarray(xj, np.float64)),
                        _ptr(d), _ptr(r))
    return d, float(r[0])


class Cells:
    """Cell list used by the oracle only to prune candidates."""

    def __init__(self, box, points, r_cell: float):
        self.b = _box(box)
        self.pts = _pts(points)
        self.nc = np.zeros(3, dtype=np.int32)
        _check(lib().orc_cells_dims(_ptr(self.b), float(r_cell), _ptr(self.nc)), "cells_dims")
        ncell = int(np.prod(self.nc.astype(np.int64)))
        self.cell_start = np.zeros(ncell + 1, dtype=np.int64)
        self.order = np.zeros(max(1, len(self.pts)), dtype=np.int64)
        _check(lib().orc_cells_build(_ptr(self.b), _ptr(self.pts), len(self.pts), _ptr(self.nc),
                                     _ptr(self.cell_start), _ptr(self.order)), "cells_build")


def _setup(box, points, r_cell, brute, query_points):
    b = _box(box)
    pts = _pts(points)
    qpts = pts if query_points is None else _pts(query_points)
    cells = None if brute else Cells(b, pts, r_cell)
    return b, pts, qpts, cells


def _cargs(cells):
    if cells is None:
        return None, None, None
    return _ptr(cells.nc), _ptr(cells.cell_start), _ptr(cells.order)


def ball_query(box, points, r_max, exclude_ii=True, query_points=None, brute=False, queries=None,
               threads=None):
    """Neighbor list of a ball query.

    Returns (counts, offsets, point_indices, distances) for the queries in
    `queries` = (q0, q1) (default all): segment t = offsets[t]..offsets[t+1] holds the
    neighbors of query q0+t sorted by point index.
    """
    b, pts, qpts, cells = _setup(box, points, r_max, brute, query_points)
    q0, q1 = (0, len(qpts)) if queries is None else queries
    nq = q1 - q0
    threads = threads or default_threads()
    counts = np.zeros(nq, dtype=np.int64)
    L = lib()
    nc, cs, od = _cargs(cells)

    def count(rg):
        a, z = rg
        return L.orc_ball_query(_ptr(b), _ptr(pts), len(pts), nc, cs, od, _ptr(qpts), q0 + a, q0 + z,
                                float(r_max), int(exclude_ii), _ptr(counts[a:z]), None, None, None)

    rgs = _ranges(nq, threads)
    with ThreadPoolExecutor(threads) as ex:
        for st in ex.map(count, rgs):
            _check(st, "ball_query(count)")
    offsets = np.zeros(nq + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    pj = np.zeros(max(1, offsets[-1]), dtype=np.int64)
    dist = np.zeros(max(1, offsets[-1]), dtype=np.float64)

    def fill(rg):
        a, z = rg
        rel = np.ascontiguousarray(offsets[a:z])
        return L.orc_ball_query(_ptr(b), _ptr(pts), len(pts), nc, cs, od, _ptr(qpts), q0 + a, q0 + z,
                                float(r_max), int(exclude_ii), None, _ptr(rel), _ptr(pj), _ptr(dist))

    with ThreadPoolExecutor(threads) as ex:
        for st in ex.map(fill, rgs):
            _check(st, "ball_query(fill)")
    m = int(offsets[-1])
    return counts, offsets, pj[:m], dist[:m]


def knn(box, points, k, exclude_ii=True, query_points=None, brute=False, queries=None, threads=None,
        r_cell=None):
    """k nearest neighbors ordered by (r2, index).  Returns (n_found, idx (nq,k), dist (nq,k))."""
    b = _box(box)
    pts = _pts(points)
    qpts = pts if query_points is None else _pts(query_points)
    cells = None
    if not brute:
        if r_cell is None:
            if b[2] == 0.0:  # 2D box: disc holding about k+1 points
                r_cell = 1.2 * ((k + 1) * b[0] * b[1] / (math.pi * max(1, len(pts)))) ** 0.5
            else:
                vol = abs(np.prod(b[:3]))
                r_cell = 1.2 * (3.0 * (k + 1) * vol / (4.0 * math.pi * max(1, len(pts)))) ** (1.0 / 3.0)
        cells = Cells(b, pts, r_cell)
    q0, q1 = (0, len(qpts)) if queries is None else queries
    nq = q1 - q0
    threads = threads or default_threads()
    out_j = np.full((nq, k), -1, dtype=np.int64)
    out_r = np.zeros((nq, k), dtype=np.float64)
    out_n = np.zeros(nq, dtype=np.int64)
    L = lib()
    nc, cs, od = _cargs(cells)

    def run(rg):
        a, z = rg
        oj = np.zeros((z - a, k), dtype=np.int64)
        orr = np.zeros((z - a, k), dtype=np.float64)
        on = np.zeros(z - a, dtype=np.int64)
        st = L.orc_knn(_ptr(b), _ptr(pts), len(pts), nc, cs, od, _ptr(qpts), q0 + a, q0 + z, int(k),
                       int(exclude_ii), _ptr(oj), _ptr(orr), _ptr(on))
        out_j[a:z], out_r[a:z], out_n[a:z] = oj, orr, on
        return st

    with ThreadPoolExecutor(threads) as ex:
        for st in ex.map(run, _ranges(nq, threads, 64)):
            _check(st, "knn")
    for t in range(nq):
        out_j[t, out_n[t]:] = -1
    return out_n, out_j, out_r


def rdf_edges(bins, r_min, r_max) -> np.ndarray:
    e = np.zeros(bins + 1)
    _check(lib().orc_rdf_edges(int(bins), float(r_min), float(r_max), _ptr(e)), "rdf_edges")
    return e


def rdf_counts(box, points, bins, r_max, r_min=0.0, exclude_ii=True, query_points=None, brute=False,
               queries=None, threads=None) -> np.ndarray:
    """Ordered-pair histogram counts (uint64) over bins of [r_min, r_max)."""
    b, pts, qpts, cells = _setup(box, points, r_max, brute, query_points)
    q0, q1 = (0, len(qpts)) if queries is None else queries
    threads = threads or default_threads()
    L = lib()
    nc, cs, od = _cargs(cells)

    def run(rg):
        a, z = rg
        c = np.zeros(bins, dtype=np.uint64)
        st = L.orc_rdf(_ptr(b), _ptr(pts), len(pts), nc, cs, od, _ptr(qpts), q0 + a, q0 + z, int(bins),
                       float(r_min), float(r_max), int(exclude_ii), _ptr(c))
        _check(st, "rdf")
        return c

    total = np.zeros(bins, dtype=np.uint64)
    with ThreadPoolExecutor(threads) as ex:
        for c in ex.map(run, _ranges(q1 - q0, threads)):
            total += c
    return total


def rdf_normalize(counts, n_query, n_points, volume, bins, r_min, r_max, dim=3):
    """g_b = counts_b / (N_q (N_p / V) (4 pi / 3)(R_{b+1}^3 - R_b^3)) and the bin centres
    r_min + (b + 1/2) (r_max - r_min)/bins.  With several frames accumulated, pass
    n_query * n_points / volume summed over frames as `n_query` and n_points = volume = 1.
    dim=2: V is the box area and the shell the annulus pi (R_{b+1}^2 - R_b^2)."""
    e = rdf_edges(bins, r_min, r_max)
    if dim == 2:
        shell = math.pi * (e[1:] ** 2 - e[:-1] ** 2)
    else:
        shell = 4.0 / 3.0 * math.pi * (e[1:] ** 3 - e[:-1] ** 3)
    g = np.asarray(counts, dtype=np.float64) / (n_query * (n_points / volume) * shell)
    delta = (r_max - r_min) / bins
    centers = r_min + (np.arange(bins) + 0.5) * delta
    return g, centers


def ylm(l, m, v):
    re = np.zeros(1)
    im = np.zeros(1)
    _check(lib().orc_ylm(int(l), int(m), float(v[0]), float(v[1]), float(v[2]), _ptr(re), _ptr(im)), "ylm")
    return complex(re[0], im[0])


def _nl(offsets, pj):
    return np.ascontiguousarray(np.asarray(offsets, np.int64)), np.ascontiguousarray(np.asarray(pj, np.int64))


def steinhardt(box, points, offsets, pj, l, which=None, with_qlm=False, threads=None):
    """q_l per particle from the spherical-harmonic definition (optionally Q_lm, m = 0..l)."""
    b = _box(box)
    pts = _pts(points)
    off, j = _nl(offsets, pj)
    idx = np.arange(len(pts), dtype=np.int64) if which is None else np.ascontiguousarray(np.asarray(which, np.int64))
    q = np.zeros(len(idx))
    Q = np.zeros((len(idx), l + 1, 2)) if with_qlm else None
    threads = threads or default_threads()
    L = lib()

    def run(rg):
        a, z = rg
        sub = np.ascontiguousarray(idx[a:z])
        qq = np.zeros(z - a)
        QQ = np.zeros((z - a, l + 1, 2)) if with_qlm else None
        st = L.orc_steinhardt_ylm(_ptr(b), _ptr(pts), len(pts), _ptr(off), _ptr(j), int(l), _ptr(sub), z - a,
                                  _ptr(qq), _ptr(QQ))
        _check(st, "steinhardt")
        q[a:z] = qq
        if with_qlm:
            Q[a:z] = QQ
        return st

    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(run, _ranges(len(idx), threads, 64)))
    if with_qlm:
        return q, Q[..., 0] + 1j * Q[..., 1]
    return q


def steinhardt_legendre(box, points, offsets, pj, l, which=None):
    """q_l per particle through the Legendre addition theorem (independent second form)."""
    b = _box(box)
    pts = _pts(points)
    off, j = _nl(offsets, pj)
    idx = np.arange(len(pts), dtype=np.int64) if which is None else np.ascontiguousarray(np.asarray(which, np.int64))
    q = np.zeros(len(idx))
    _check(lib().orc_steinhardt_legendre(_ptr(b), _ptr(pts), len(pts), _ptr(off), _ptr(j), int(l), _ptr(idx),
                                         len(idx), _ptr(q)), "steinhardt_legendre")
    return q


def q_grad(box, points, offsets, pj, l):
    """dQ/dx for Q = mean_i q_l(i), neighbor list fixed; (N, 3) float64."""
    b = _box(box)
    pts = _pts(points)
    off, j = _nl(offsets, pj)
    g = np.zeros((len(pts), 3))
    _check(lib().orc_q_grad(_ptr(b), _ptr(pts), len(pts), _ptr(off), _ptr(j), int(l), _ptr(g)), "q_grad")
    return g


# ------------------------------------------------------------- Steinhardt variants


def wigner3j(j1, j2, j3, m1, m2, m3) -> float:
    """Wigner 3j symbol from Racah's formula, summed exactly in rational arithmetic.

    (j1 j2 j3; m1 m2 m3) = (-1)^(j1-j2-m3) sqrt(D (j1+m1)!(j1-m1)!(j2+m2)!(j2-m2)!(j3+m3)!(j3-m3)!)
                           * sum_k (-1)^k / [k! (j3-j2+k+m1)! (j3-j1+k-m2)! (j1+j2-j3-k)! (j1-k-m1)! (j2-k+m2)!],
    D = (j1+j2-j3)!(j1-j2+j3)!(-j1+j2+j3)!/(j1+j2+j3+1)!; zero unless m1+m2+m3 = 0 and the
    triangle and |m| <= j conditions hold.
    """
    from fractions import Fraction
    f = math.factorial
    if m1 + m2 + m3 != 0 or j3 < abs(j1 - j2) or j3 > j1 + j2:
        return 0.0
    if abs(m1) > j1 or abs(m2) > j2 or abs(m3) > j3:
        return 0.0
    d = Fraction(f(j1 + j2 - j3) * f(j1 - j2 + j3) * f(-j1 + j2 + j3), f(j1 + j2 + j3 + 1))
    pre2 = d * f(j1 + m1) * f(j1 - m1) * f(j2 + m2) * f(j2 - m2) * f(j3 + m3) * f(j3 - m3)
    s = Fraction(0)
    for k in range(0, j1 + j2 - j3 + 1):
        args = (k, j3 - j2 + k + m1, j3 - j1 + k - m2, j1 + j2 - j3 - k, j1 - k - m1, j2 - k + m2)
        if min(args) < 0:
            continue
        den = 1
        for a in args:
            den *= f(a)
        s += Fraction((-1) ** k, den)
    val2 = pre2 * s * s
    sign = (-1) ** ((j1 - j2 - m3) % 2) * (1 if s >= 0 else -1)
    return sign * math.sqrt(float(val2))


def _full_qlm(Q, l):
    """(n, l+1) complex Q_lm, m >= 0 -> (n, 2l+1) for m = -l..l."""
    n = Q.shape[0]
    F = np.zeros((n, 2 * l + 1), dtype=complex)
    for m in range(l + 1):
        F[:, l + m] = Q[:, m]
        F[:, l - m] = (-1) ** m * np.conj(Q[:, m])
    return F


def wl_from_qlm(Q, l, normalize=True):
    """W_l per particle from Q_lm (Steinhardt, Nelson and Ronchetti 1983), FP64."""
    F = _full_qlm(np.asarray(Q), l)
    w = np.zeros(F.shape[0])
    for m1 in range(-l, l + 1):
        for m2 in range(-l, l + 1):
            m3 = -m1 - m2
            if abs(m3) > l:
                continue
            c = wigner3j(l, l, l, m1, m2, m3)
            w += c * np.real(F[:, l + m1] * F[:, l + m2] * F[:, l + m3])
    if normalize:
        s = np.sum(np.abs(F) ** 2, axis=1)
        w = np.where(s > 0, w / np.where(s > 0, s, 1.0) ** 1.5, 0.0)
    return w


def wl(box, points, offsets, pj, l, normalize=True):
    _, Q = steinhardt(box, points, offsets, pj, l, with_qlm=True)
    return wl_from_qlm(Q, l, normalize)


def steinhardt_average(box, points, offsets, pj, l, with_qlm=False):
    """Neighbor-averaged q_l (Lechner and Dellago 2008): Qbar_lm(i) = (Q_lm(i) + sum over
    the neighbors k of Q_lm(k)) / (n_i + 1), qbar = sqrt(4 pi/(2l+1) sum_m |Qbar_lm|^2)."""
    _, Q = steinhardt(box, points, offsets, pj, l, with_qlm=True)
    off, j = _nl(offsets, pj)
    n = len(off) - 1
    S = Q.copy()
    for i in range(n):
        a, z = off[i], off[i + 1]
        if z > a:
            S[i] += Q[j[a:z]].sum(axis=0)
    S /= (np.diff(off) + 1)[:, None]
    w = np.ones(l + 1)
    w[1:] = 2.0
    q = np.sqrt(4.0 * math.pi / (2 * l + 1) * np.sum(w * np.abs(S) ** 2, axis=1))
    return (q, S) if with_qlm else q


def local_descriptors(box, points, qi, pj, l_max, negative_m=True, query_points=None):
    """(n_pairs, n_sph) complex Y_lm of every bond, l <= l_max (m = -l..l or 0..l)."""
    b = _box(box)
    pts = _pts(points)
    qpts = pts if query_points is None else _pts(query_points)
    qi = np.ascontiguousarray(np.asarray(qi, np.int64))
    pj = np.ascontiguousarray(np.asarray(pj, np.int64))
    nsph = (l_max + 1) ** 2 if negative_m else (l_max + 1) * (l_max + 2) // 2
    out = np.zeros((len(qi), nsph, 2))
    _check(lib().orc_descriptors(_ptr(b), _ptr(pts), _ptr(qpts), len(qi), _ptr(qi), _ptr(pj), int(l_max),
                                 int(bool(negative_m)), _ptr(out)), "descriptors")
    return out[..., 0] + 1j * out[..., 1]


# ------------------------------------------------------------------------ clusters


def clusters(n, qi, pj, mask=None):
    """Connected components of the points joined by bonds (qi[e], pj[e]) with mask[e]
    (all when None); numbered by decreasing size, ties by smallest member.  Returns
    (cluster index per point, sizes)."""
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    qi = np.asarray(qi, np.int64)
    pj = np.asarray(pj, np.int64)
    for e in range(len(qi)):
        if mask is not None and not mask[e]:
            continue
        a, b = find(int(qi[e])), find(int(pj[e]))
        if a != b:
            parent[max(a, b)] = min(a, b)
    root = np.array([find(i) for i in range(n)], np.int64)
    members = {}
    for i in range(n):
        members.setdefault(root[i], []).append(i)
    order = sorted(members, key=lambda r: (-len(members[r]), min(members[r])))
    idx = np.empty(n, np.int64)
    for c, r in enumerate(order):
        idx[members[r]] = c
    return idx, np.array([len(members[r]) for r in order], np.int64)


def cluster_properties(box, points, cluster_idx):
    """Centers and gyration tensors: members unwrapped to the image nearest the
    cluster's smallest member (the defining minimum image), centre = that member + mean
    offset wrapped into the box, gyration = mean outer product of offsets from the centre."""
    b = _box(box)
    pts = _pts(points)
    idx = np.asarray(cluster_idx, np.int64)
    nc = int(idx.max()) + 1 if len(idx) else 0
    L = lib()
    centers = np.zeros((nc, 3))
    gyr = np.zeros((nc, 3, 3))
    M = np.asarray(box.matrix(), np.float64)
    Minv = np.linalg.inv(M)
    for c in range(nc):
        mem = np.nonzero(idx == c)[0]
        r = mem[0]
        d = np.zeros((len(mem), 3))
        for k, j in enumerate(mem):
            out = np.zeros(3)
            rr = np.zeros(1)
            _check(L.orc_min_image(_ptr(b), _ptr(np.ascontiguousarray(pts[r])), _ptr(np.ascontiguousarray(pts[j])),
                                   _ptr(out), _ptr(rr)), "min_image")
            d[k] = out
        mean = d.mean(axis=0)
        p = pts[r] + mean
        s = Minv @ p + 0.5
        centers[c] = p - M @ np.floor(s)
        e = d - mean
        gyr[c] = e.T @ e / len(mem)
    return centers, gyr


def solid_liquid(box, points, offsets, pj, l, q_threshold, solid_threshold, normalize_q=True):
    """Solid-liquid order parameter (ten Wolde, Ruiz-Montero and Frenkel 1996) in FP64:
    bond scores s_ij = Re sum_m Q_lm(i) conj(Q_lm(j)) (normalised by |Q_l(i)| |Q_l(j)|),
    solid-like bonds s_ij > q_threshold, solid particles with >= solid_threshold of them,
    clusters of solid particles joined by solid-like bonds.  Returns (s_ij, connections,
    cluster index, cluster sizes)."""
    _, Q = steinhardt(box, points, offsets, pj, l, with_qlm=True)
    F = _full_qlm(Q, l)
    off, j = _nl(offsets, pj)
    qi = np.repeat(np.arange(len(off) - 1), np.diff(off))
    dot = np.real(np.sum(F[qi] * np.conj(F[j]), axis=1))
    if normalize_q:
        na = np.sqrt(np.sum(np.abs(F) ** 2, axis=1))
        den = na[qi] * na[j]
        s = np.where(den > 0, dot / np.where(den > 0, den, 1.0), 0.0)
    else:
        s = dot
    solid_bond = s > q_threshold
    conn = np.zeros(len(off) - 1, np.int64)
    np.add.at(conn, qi, solid_bond.astype(np.int64))
    join = solid_bond & (conn[qi] >= solid_threshold) & (conn[j] >= solid_threshold)
    idx, sizes = clusters(len(off) - 1, qi, j, join)
    return s, conn, idx, sizes


def pmftxy(box, points, theta, x_max, y_max, bins_x, bins_y, query_points=None, qi=None, pj=None,
           with_xy=False):
    """PMFT(x, y) bin counts (int64, (bins_x, bins_y), x major): every bond (i, j) of the
    list in the frame of query particle i (orientation angle theta[i] about z), counted in
    [-x_max, x_max) x [-y_max, y_max).  Without a list the bonds are every pair (i != j
    when query_points is None); only those within sqrt(x_max^2 + y_max^2) can land in a
    bin, so the ball query at (1 + 1e-6) times that radius supplies them (the factor
    keeps a bond at the corner whatever the rounding of its rotation).  with_xy also returns the rotated bond
    (x', y') per bond and the bonds (qi, pj)."""
    b = _box(box)
    pts = _pts(points)
    qpts = pts if query_points is None else _pts(query_points)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    assert th.shape == (len(qpts),)
    if qi is None:
        r = math.sqrt(x_max * x_max + y_max * y_max) * (1.0 + 1e-6)
        _, off, pj, _ = ball_query(b, pts, r, exclude_ii=query_points is None, query_points=query_points)
        qi = np.repeat(np.arange(len(qpts), dtype=np.int64), np.diff(off))
    qi = np.ascontiguousarray(np.asarray(qi, dtype=np.int64))
    pj = np.ascontiguousarray(np.asarray(pj, dtype=np.int64))
    counts = np.zeros((bins_x, bins_y), dtype=np.int64)
    xy = np.zeros((len(qi), 2)) if with_xy else None
    _check(lib().orc_pmftxy(_ptr(b), _ptr(pts), _ptr(qpts), _ptr(th), len(qi), _ptr(qi), _ptr(pj), float(x_max),
                            float(y_max), int(bins_x), int(bins_y), _ptr(counts), _ptr(xy)), "pmftxy")
    return (counts, xy, qi, pj) if with_xy else counts


def pmft_normalize(counts, norm, x_max, y_max):
    """pcf = counts / (norm * bin area), norm = sum over frames of N_query N_points / A
    (A the box area), and PMFT = -log(pcf) in units of k_B T (Section "Potentials of Mean
    Force and Torque": the negative logarithm of the accumulated histogram; +inf where a
    bin is empty)."""
    c = np.asarray(counts, dtype=np.float64)
    bx, by = c.shape
    area = (2.0 * x_max / bx) * (2.0 * y_max / by)
    pcf = c / (norm * area) if norm > 0 else np.zeros_like(c)
    with np.errstate(divide="ignore"):
        pmft = np.where(pcf > 0, -np.log(np.where(pcf > 0, pcf, 1.0)), np.inf)
    return pcf, pmft
