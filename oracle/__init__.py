"""FP64 CPU oracle for STKDE -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct evaluations of the paper's density (Section 2.1)
by Algorithm 1 (VB) and Algorithm 2 (PB), in ``stkde_oracle.c``.  Only the test
suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The GPU library never does, and the two share no code:
the only thing both sides take from elsewhere is the seeded input generator.

Kernel constants: ``CS_PRINTED = pi/2`` and ``CT_PRINTED = 3/4`` are the
constants printed with k_s and k_t; ``CS_UNIT_MASS = 24/(13 pi)`` makes the
spatial kernel c_s (1-u^2)(1-v^2) integrate to 1 over the unit disk, so that
the density integrates to 1 when every cylinder lies inside the grid.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stkde_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CS_PRINTED = math.pi / 2.0
CT_PRINTED = 0.75
CS_UNIT_MASS = 24.0 / (13.0 * math.pi)


class Params(ctypes.Structure):
    _fields_ = [
        ("x0", ctypes.c_double), ("y0", ctypes.c_double), ("t0", ctypes.c_double),
        ("sres", ctypes.c_double), ("tres", ctypes.c_double),
        ("gx", ctypes.c_int64), ("gy", ctypes.c_int64), ("gt", ctypes.c_int64),
        ("hs", ctypes.c_double), ("ht", ctypes.c_double),
        ("cs", ctypes.c_double), ("ct", ctypes.c_double),
        ("sample_off", ctypes.c_double),
        ("round_fp32", ctypes.c_int32), ("nthreads", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        l = ctypes.CDLL(build())
        P = ctypes.POINTER(Params)
        dp = ctypes.c_void_p
        i64 = ctypes.c_int64
        l.oracle_vb.argtypes = [P, dp, i64, dp]
        l.oracle_vb_voxels.argtypes = [P, dp, i64, dp, i64, dp]
        l.oracle_pb.argtypes = [P, dp, i64, dp, dp]
        l.oracle_pb_box.argtypes = [P, dp, i64, i64, i64, i64, i64, i64, i64, dp, dp]
        l.oracle_pb_boxes.argtypes = [P, dp, i64, dp, i64, dp, dp, dp]
        l.oracle_count_updates.argtypes = [P, dp, i64, dp]
        l.oracle_max_threads.argtypes = []
        l.oracle_vb_adaptive.argtypes = [P, dp, dp, dp, i64, dp]
        l.oracle_pb_adaptive.argtypes = [P, dp, dp, dp, i64, dp, dp]
        l.oracle_pb_adaptive_boxes.argtypes = [P, dp, dp, dp, i64, dp, i64, dp, dp, dp]
        l.oracle_abramson.argtypes = [P, dp, i64, dp, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, dp, dp, dp]
        for f in ("oracle_vb", "oracle_vb_voxels", "oracle_pb", "oracle_pb_box",
                  "oracle_pb_boxes", "oracle_count_updates", "oracle_max_threads",
                  "oracle_vb_adaptive", "oracle_pb_adaptive", "oracle_pb_adaptive_boxes",
                  "oracle_abramson"):
            getattr(l, f).restype = ctypes.c_int
        _lib = l
    return _lib


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def params(gx, gy, gt, hs, ht, *, x0=0.0, y0=0.0, t0=0.0, sres=1.0, tres=1.0,
           cs=CS_PRINTED, ct=CT_PRINTED, sample_off=0.5, round_fp32=True, nthreads=0) -> Params:
    return Params(float(x0), float(y0), float(t0), float(sres), float(tres),
                  int(gx), int(gy), int(gt), float(hs), float(ht), float(cs), float(ct),
                  float(sample_off), int(bool(round_fp32)), int(nthreads))


def _pts(points) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    return a


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def vb(points, p: Params) -> np.ndarray:
    """Algorithm 1 on the whole grid, shape (gx, gy, gt)."""
    a = _pts(points)
    out = np.empty((p.gx, p.gy, p.gt), dtype=np.float64)
    rc = lib().oracle_vb(ctypes.byref(p), _ptr(a), a.shape[0], out.ctypes.data)
    assert rc == 0
    return out


def vb_voxels(points, p: Params, vox) -> np.ndarray:
    """Algorithm 1 at the listed voxels (m, 3) of (X, Y, T)."""
    a = _pts(points)
    v = np.ascontiguousarray(np.asarray(vox, dtype=np.int64).reshape(-1, 3))
    vals = np.empty(v.shape[0], dtype=np.float64)
    rc = lib().oracle_vb_voxels(ctypes.byref(p), _ptr(a), a.shape[0], _ptr(v), v.shape[0],
                                _ptr(vals))
    assert rc == 0
    return vals


def pb(points, p: Params, with_slack: bool = False):
    """Algorithm 2 on the whole grid, shape (gx, gy, gt); optionally the tie slack."""
    a = _pts(points)
    out = np.empty((p.gx, p.gy, p.gt), dtype=np.float64)
    slack = np.empty_like(out) if with_slack else None
    rc = lib().oracle_pb(ctypes.byref(p), _ptr(a), a.shape[0], out.ctypes.data,
                         slack.ctypes.data if with_slack else None)
    assert rc == 0
    return (out, slack) if with_slack else out


def pb_boxes(points, p: Params, boxes, with_slack: bool = True, pair_counts: bool = False):
    """Algorithm 2 restricted to boxes (bx0, bx1, by0, by1, bt0, bt1); returns a
    list of (values, slack) arrays shaped like each box, plus the per-box count
    of in-cylinder (event, voxel) pairs when ``pair_counts``."""
    a = _pts(points)
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int64).reshape(-1, 6))
    sizes = (b[:, 1] - b[:, 0]) * (b[:, 3] - b[:, 2]) * (b[:, 5] - b[:, 4])
    tot = int(sizes.sum())
    out = np.empty(tot, dtype=np.float64)
    slack = np.empty(tot, dtype=np.float64) if with_slack else None
    npairs = np.zeros(b.shape[0], dtype=np.uint64)
    rc = lib().oracle_pb_boxes(ctypes.byref(p), _ptr(a), a.shape[0], _ptr(b), b.shape[0],
                               _ptr(out), _ptr(slack) if with_slack else None, _ptr(npairs))
    if rc != 0:
        raise ValueError("box outside the grid or empty")
    res, off = [], 0
    for j in range(b.shape[0]):
        shp = (int(b[j, 1] - b[j, 0]), int(b[j, 3] - b[j, 2]), int(b[j, 5] - b[j, 4]))
        sz = int(sizes[j])
        res.append((out[off:off + sz].reshape(shp),
                    slack[off:off + sz].reshape(shp) if with_slack else None))
        off += sz
    return (res, npairs) if pair_counts else res


def count_updates(points, p: Params) -> int:
    """Number of (event, in-grid voxel) pairs inside the bandwidth cylinder."""
    a = _pts(points)
    c = np.zeros(1, dtype=np.uint64)
    rc = lib().oracle_count_updates(ctypes.byref(p), _ptr(a), a.shape[0], c.ctypes.data)
    assert rc == 0
    return int(c[0])


def _bw(a, n: int) -> np.ndarray:
    b = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    assert b.shape[0] == n, "one bandwidth per event"
    return b


def vb_adaptive(points, hs, ht, p: Params) -> np.ndarray:
    """Algorithm 1 with per-event bandwidths hs[i], ht[i] (domain units) and
    per-event normalisation 1/(n hs_i^2 ht_i); p.hs, p.ht unused."""
    a = _pts(points)
    h, t = _bw(hs, a.shape[0]), _bw(ht, a.shape[0])
    out = np.empty((p.gx, p.gy, p.gt), dtype=np.float64)
    rc = lib().oracle_vb_adaptive(ctypes.byref(p), _ptr(a), _ptr(h), _ptr(t), a.shape[0],
                                  out.ctypes.data)
    assert rc == 0
    return out


def pb_adaptive(points, hs, ht, p: Params, with_slack: bool = False):
    """Algorithm 2 with per-event bandwidths (box per event); returns the grid, and
    the binary32 tie slack when ``with_slack``."""
    a = _pts(points)
    h, t = _bw(hs, a.shape[0]), _bw(ht, a.shape[0])
    out = np.empty((p.gx, p.gy, p.gt), dtype=np.float64)
    slack = np.empty_like(out) if with_slack else None
    rc = lib().oracle_pb_adaptive(ctypes.byref(p), _ptr(a), _ptr(h), _ptr(t), a.shape[0],
                                  out.ctypes.data, slack.ctypes.data if with_slack else None)
    assert rc == 0
    return (out, slack) if with_slack else out


def pb_adaptive_boxes(points, hs, ht, p: Params, boxes, with_slack: bool = True,
                      pair_counts: bool = False):
    """Adaptive Algorithm 2 restricted to boxes; list of (values, slack), plus the
    per-box count of in-cylinder pairs when ``pair_counts``."""
    a = _pts(points)
    h, t = _bw(hs, a.shape[0]), _bw(ht, a.shape[0])
    b = np.ascontiguousarray(np.asarray(boxes, dtype=np.int64).reshape(-1, 6))
    sizes = (b[:, 1] - b[:, 0]) * (b[:, 3] - b[:, 2]) * (b[:, 5] - b[:, 4])
    tot = int(sizes.sum())
    out = np.empty(tot, dtype=np.float64)
    slack = np.empty(tot, dtype=np.float64) if with_slack else None
    npairs = np.zeros(b.shape[0], dtype=np.uint64)
    rc = lib().oracle_pb_adaptive_boxes(ctypes.byref(p), _ptr(a), _ptr(h), _ptr(t), a.shape[0],
                                        _ptr(b), b.shape[0], _ptr(out),
                                        _ptr(slack) if with_slack else None, _ptr(npairs))
    assert rc == 0
    res, off = [], 0
    for j in range(b.shape[0]):
        sz = int(sizes[j])
        shape = (int(b[j, 1] - b[j, 0]), int(b[j, 3] - b[j, 2]), int(b[j, 5] - b[j, 4]))
        v = out[off:off + sz].reshape(shape)
        s_ = slack[off:off + sz].reshape(shape) if with_slack else None
        res.append((v, s_))
        off += sz
    return (res, npairs) if pair_counts else res


def abramson(points, p: Params, alpha: float = 0.5, lam_min: float = 0.125, lam_max: float = 8.0,
             pilot=None):
    """Per-event bandwidths by Abramson's law from a pilot density with the fixed
    pair (p.hs, p.ht) (computed here by PB unless given); returns (hs_i, ht_i, lambda_i)."""
    a = _pts(points)
    if pilot is None:
        pilot = pb(a, p)
    pil = np.ascontiguousarray(np.asarray(pilot, dtype=np.float64))
    assert pil.shape == (p.gx, p.gy, p.gt)
    n = a.shape[0]
    hs, ht, lam = np.empty(n), np.empty(n), np.empty(n)
    rc = lib().oracle_abramson(ctypes.byref(p), _ptr(a), n, _ptr(pil), float(alpha), float(lam_min),
                               float(lam_max), _ptr(hs), _ptr(ht), _ptr(lam))
    assert rc == 0
    return hs, ht, lam
