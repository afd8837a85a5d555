"""CPU oracle for the adaptive equi-join path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The product library never does, and this
package imports nothing from it: the two share no code.

Every function here is a thin numpy marshalling layer over ``oracle.cpp``,
which holds the definitions (see the comments there for the paper passages).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

_lib = None

I32, I64 = 0, 1
HLL_P = 14
HLL_M = 1 << HLL_P


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    c = ctypes
    lib.oracle_h64.restype = c.c_uint64
    lib.oracle_h64.argtypes = [c.c_uint64]
    lib.oracle_join.restype = c.c_int64
    lib.oracle_join.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_void_p, c.c_int64,
                                c.c_void_p, c.c_void_p, c.c_int64]
    lib.oracle_join_mt.restype = c.c_int64
    lib.oracle_join_mt.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_void_p, c.c_int64,
                                   c.c_void_p, c.c_void_p, c.c_int64, c.c_int]
    lib.oracle_join_fingerprint.restype = c.c_int64
    lib.oracle_join_fingerprint.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_void_p, c.c_int64, c.c_int,
                                            c.POINTER(c.c_uint64), c.POINTER(c.c_uint64)]
    lib.oracle_join_count.restype = c.c_int64
    lib.oracle_join_count.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_void_p, c.c_int64]
    lib.oracle_join_sum.restype = c.c_int64
    lib.oracle_join_sum.argtypes = [c.c_int, c.c_void_p, c.c_void_p, c.c_int64, c.c_void_p,
                                    c.c_void_p, c.c_int64, c.c_int, c.POINTER(c.c_int64)]
    lib.oracle_stats.restype = None
    lib.oracle_stats.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.POINTER(c.c_int64),
                                 c.POINTER(c.c_int64), c.c_void_p]
    lib.oracle_hll_estimate.restype = c.c_double
    lib.oracle_hll_estimate.argtypes = [c.c_void_p]
    lib.oracle_groupby.restype = c.c_int64
    lib.oracle_groupby.argtypes = [c.c_int, c.c_void_p, c.c_int64, c.c_int, c.c_void_p, c.c_void_p,
                                   c.c_void_p, c.c_void_p, c.c_void_p, c.c_int64]
    lib.oracle_exact_ndv.restype = c.c_int64
    lib.oracle_exact_ndv.argtypes = [c.c_int, c.c_void_p, c.c_int64]
    _lib = lib
    return lib


def _keys(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.int32:
        return a, I32
    if a.dtype == np.int64:
        return a, I64
    raise TypeError(f"keys must be int32 or int64, got {a.dtype}")


def _ptr(a):
    return a.ctypes.data if a.size else None


def h64(x: int) -> int:
    return int(_load().oracle_h64(ctypes.c_uint64(x & 0xFFFFFFFFFFFFFFFF)))


def join(build_keys, probe_keys, cap=None):
    """Canonically sorted join pairs ``(build_idx, probe_idx)`` as uint32 arrays.

    ``cap`` bounds how many pairs are materialised; the returned count is |J|
    regardless. With the default cap every pair is returned.
    """
    bk, dt = _keys(build_keys)
    pk, dt2 = _keys(probe_keys)
    if dt != dt2:
        raise TypeError("build and probe keys must share a dtype")
    lib = _load()
    if cap is None:
        cap = lib.oracle_join_count(dt, _ptr(bk), bk.size, _ptr(pk), pk.size)
    out_b = np.empty(max(cap, 1), np.uint32)
    out_p = np.empty(max(cap, 1), np.uint32)
    n = lib.oracle_join(dt, _ptr(bk), bk.size, _ptr(pk), pk.size, _ptr(out_b), _ptr(out_p), cap)
    k = min(n, cap)
    return out_b[:k].copy(), out_p[:k].copy(), int(n)


def join_mt(build_keys, probe_keys, threads: int):
    """``join`` with the probe loop split over ``threads`` host threads (the
    oracle's -t N mode); the output is identical to ``join``'s."""
    bk, dt = _keys(build_keys)
    pk, dt2 = _keys(probe_keys)
    if dt != dt2:
        raise TypeError("build and probe keys must share a dtype")
    lib = _load()
    cap = lib.oracle_join_count(dt, _ptr(bk), bk.size, _ptr(pk), pk.size)
    out_b = np.empty(max(cap, 1), np.uint32)
    out_p = np.empty(max(cap, 1), np.uint32)
    n = lib.oracle_join_mt(dt, _ptr(bk), bk.size, _ptr(pk), pk.size, _ptr(out_b), _ptr(out_p), cap,
                           int(threads))
    return out_b[:n].copy(), out_p[:n].copy(), int(n)


def join_fingerprint(build_keys, probe_keys, threads: int = 1):
    """(|J|, fp_sum, fp_xor) of the join's pair multiset without storing it:
    with w = build_idx * 2^32 + probe_idx per pair, fp_sum = sum of h64(w)
    mod 2^64 and fp_xor = xor of h64(w + 0x9E3779B97F4A7C15), both as Python
    ints in [0, 2^64). For results too large to sort on the host."""
    bk, dt = _keys(build_keys)
    pk, dt2 = _keys(probe_keys)
    if dt != dt2:
        raise TypeError("build and probe keys must share a dtype")
    s = ctypes.c_uint64(0)
    x = ctypes.c_uint64(0)
    n = _load().oracle_join_fingerprint(dt, _ptr(bk), bk.size, _ptr(pk), pk.size, int(threads),
                                        ctypes.byref(s), ctypes.byref(x))
    return int(n), int(s.value), int(x.value)


def join_wide(build_keys, probe_keys, build_cols=(), probe_cols=()):
    """The wide join in canonical order: (build_idx, probe_idx, build column
    values, probe column values), where match (i, j) carries row i of every
    build column and row j of every probe column (Sec. 3.2 materialisation;
    both strategies compute this same result)."""
    b, p, _ = join(build_keys, probe_keys)
    return (b, p, [np.asarray(c)[b.astype(np.int64)] for c in build_cols],
            [np.asarray(c)[p.astype(np.int64)] for c in probe_cols])


def join_count(build_keys, probe_keys) -> int:
    bk, dt = _keys(build_keys)
    pk, _ = _keys(probe_keys)
    return int(_load().oracle_join_count(dt, _ptr(bk), bk.size, _ptr(pk), pk.size))


def join_sum(build_keys, build_pay, probe_keys, probe_pay):
    """(sum over matches of build_pay + probe_pay mod 2^64 as int64, |J|)."""
    bk, dt = _keys(build_keys)
    pk, _ = _keys(probe_keys)
    bp = np.ascontiguousarray(build_pay)
    pp = np.ascontiguousarray(probe_pay)
    if bp.dtype != pp.dtype or bp.dtype not in (np.int32, np.int64):
        raise TypeError("payloads must both be int32 or both int64")
    cnt = ctypes.c_int64(0)
    s = _load().oracle_join_sum(dt, _ptr(bk), _ptr(bp), bk.size, _ptr(pk), _ptr(pp), pk.size,
                                bp.dtype.itemsize, ctypes.byref(cnt))
    return int(s), int(cnt.value)


def stats(keys):
    """(min, max, registers uint8[2^14]) by one sequential pass."""
    k, dt = _keys(keys)
    mn = ctypes.c_int64(0)
    mx = ctypes.c_int64(0)
    regs = np.zeros(HLL_M, np.uint8)
    _load().oracle_stats(dt, _ptr(k), k.size, ctypes.byref(mn), ctypes.byref(mx), _ptr(regs))
    return int(mn.value), int(mx.value), regs


def hll_estimate(regs) -> float:
    r = np.ascontiguousarray(regs, dtype=np.uint8)
    if r.size != HLL_M:
        raise ValueError("expected 2^14 registers")
    return float(_load().oracle_hll_estimate(_ptr(r)))


def exact_ndv(keys) -> int:
    k, dt = _keys(keys)
    return int(_load().oracle_exact_ndv(dt, _ptr(k), k.size))


AGG_OPS = {"sum": 0, "count": 1, "min": 2, "max": 3}


def groupby(keys, aggs):
    """Group-by in ascending key order: (keys int64[g], [int64[g] per aggregate]).
    ``aggs`` is a list of (op, values) with op in sum/count/min/max and values
    an int32/int64 array (None for count)."""
    k, dt = _keys(keys)
    n = k.size
    ops = np.array([AGG_OPS[o] for o, _ in aggs], np.int32)
    cols = [np.ascontiguousarray(v) if v is not None else np.zeros(1, np.int64) for _, v in aggs]
    vb = np.array([c.dtype.itemsize for c in cols], np.int32)
    ptrs = (ctypes.c_void_p * max(len(cols), 1))(*[c.ctypes.data for c in cols])
    lib = _load()
    g = lib.oracle_groupby(dt, _ptr(k), n, len(aggs), ops.ctypes.data, vb.ctypes.data, ptrs, None, None, 0)
    out_k = np.empty(max(g, 1), np.int64)
    out_a = np.empty(max(g, 1) * max(len(aggs), 1), np.int64)
    lib.oracle_groupby(dt, _ptr(k), n, len(aggs), ops.ctypes.data, vb.ctypes.data, ptrs, out_k.ctypes.data,
                       out_a.ctypes.data, g)
    return out_k[:g].copy(), [out_a[a * g:(a + 1) * g].copy() for a in range(len(aggs))]
