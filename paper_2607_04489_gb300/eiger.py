"""Python binding of libeiger's C ABI (``include/eiger.h``).

Argument marshalling only: tensors become device pointers, the current torch
stream becomes the ``stream`` argument, statuses become exceptions. Every step
of the join runs in the library's CUDA kernels; if ``libeiger.so`` is missing
or cannot be loaded, every call raises instead of computing anything here.

PyTorch supplies device memory (inputs, outputs, workspace) and streams.
"""

from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libeiger.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_WORKSPACE, ERR_TABLE_FULL, ERR_CUDA, ERR_INTERNAL = range(7)
I32, I64 = 0, 1
BATCH_SMALL_MAX_I32, BATCH_SMALL_MAX_I64 = 2048, 1024  # build rows of a shared-memory batch table
AUTO, NPHJ, PHJ1, PHJ2, STATIC, SMJ = range(6)
VARIANTS = {"auto": AUTO, "nphj": NPHJ, "phj1": PHJ1, "phj2": PHJ2, "static": STATIC, "smj": SMJ}
GFUR, GFTR, MAT_AUTO = range(3)
MATERIALIZE = {"gfur": GFUR, "gftr": GFTR, "auto": MAT_AUTO}
MATERIALIZE_NAMES = {GFUR: "gfur", GFTR: "gftr"}
MAX_COLS = 4
VARIANT_NAMES = {v: k for k, v in VARIANTS.items()}
HLL_M = 16384

_STATUS = {
    ERR_INVALID_ARG: "EIGER_ERR_INVALID_ARG",
    ERR_CAPACITY: "EIGER_ERR_CAPACITY",
    ERR_WORKSPACE: "EIGER_ERR_WORKSPACE",
    ERR_TABLE_FULL: "EIGER_ERR_TABLE_FULL",
    ERR_CUDA: "EIGER_ERR_CUDA",
    ERR_INTERNAL: "EIGER_ERR_INTERNAL",
}


class EigerError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class StatsT(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("min", ctypes.c_int64), ("max", ctypes.c_int64),
                ("estimate", ctypes.c_double), ("hll", ctypes.c_uint8 * HLL_M)]


class StageT(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("ms", ctypes.c_float), ("launches", ctypes.c_int32),
                ("bytes", ctypes.c_double)]


class JoinDescT(ctypes.Structure):
    _fields_ = [("build_keys", ctypes.c_void_p), ("probe_keys", ctypes.c_void_p), ("nb", ctypes.c_int64),
                ("np", ctypes.c_int64), ("out_bidx", ctypes.c_void_p), ("out_pidx", ctypes.c_void_p),
                ("capacity", ctypes.c_int64)]


class BatchKnobsT(ctypes.Structure):
    _fields_ = [("block_threads", ctypes.c_int32), ("chunk_rows", ctypes.c_int32),
                ("load_factor", ctypes.c_float), ("small_rows", ctypes.c_int32)]


class PlanT(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("bits1", ctypes.c_int32), ("bits2", ctypes.c_int32),
                ("narrow", ctypes.c_int32), ("load_factor", ctypes.c_float),
                ("selector", ctypes.c_int32), ("key_min", ctypes.c_int64),
                ("key_max", ctypes.c_int64), ("materialize", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


MAX_AGGS = 4
GB_AUTO, GB_HASH, GB_PARTITION = range(3)
GB_VARIANTS = {"auto": GB_AUTO, "hash": GB_HASH, "partition": GB_PARTITION}
GB_VARIANT_NAMES = {v: k for k, v in GB_VARIANTS.items()}
AGG_SUM, AGG_COUNT, AGG_MIN, AGG_MAX = range(4)
AGG_OPS = {"sum": AGG_SUM, "count": AGG_COUNT, "min": AGG_MIN, "max": AGG_MAX}


class AggsT(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("op", ctypes.c_int32 * MAX_AGGS), ("bytes", ctypes.c_int32 * MAX_AGGS),
                ("vals", ctypes.c_void_p * MAX_AGGS), ("out", ctypes.c_void_p * MAX_AGGS)]


class GbPlanT(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("bits1", ctypes.c_int32), ("bits2", ctypes.c_int32),
                ("narrow", ctypes.c_int32), ("table_slots", ctypes.c_int64), ("estimate", ctypes.c_double),
                ("selector", ctypes.c_int32), ("attempts", ctypes.c_int32)]


@dataclass
class GbPlan:
    variant: str
    bits1: int = 0
    bits2: int = 0
    narrow: int = 0
    table_slots: int = 0
    estimate: float = 0.0
    selector: int = 0
    attempts: int = 0

    @classmethod
    def from_c(cls, p: "GbPlanT") -> "GbPlan":
        return cls(GB_VARIANT_NAMES.get(p.variant, str(p.variant)), p.bits1, p.bits2, p.narrow, p.table_slots,
                   p.estimate, p.selector, p.attempts)

    def to_c(self) -> "GbPlanT":
        p = GbPlanT()
        p.variant = GB_VARIANTS[self.variant]
        p.bits1, p.bits2, p.narrow, p.table_slots = self.bits1, self.bits2, self.narrow, self.table_slots
        return p


class ColumnsT(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("bytes", ctypes.c_int32 * MAX_COLS),
                ("cols", ctypes.c_void_p * MAX_COLS), ("out", ctypes.c_void_p * MAX_COLS)]


@dataclass
class Stats:
    n: int
    min: int
    max: int
    estimate: float
    hll: np.ndarray

    @classmethod
    def from_c(cls, s: StatsT) -> "Stats":
        return cls(s.n, s.min, s.max, s.estimate, np.frombuffer(bytes(s.hll), np.uint8).copy())

    def to_c(self) -> StatsT:
        s = StatsT()
        s.n, s.min, s.max, s.estimate = self.n, self.min, self.max, self.estimate
        ctypes.memmove(s.hll, np.ascontiguousarray(self.hll, np.uint8).ctypes.data, HLL_M)
        return s


@dataclass
class Plan:
    variant: str
    bits1: int = 0
    bits2: int = 0
    narrow: int = 0
    load_factor: float = 0.5
    selector: int = 0
    key_min: int = 0
    key_max: int = 0
    materialize: str = "gfur"

    @classmethod
    def from_c(cls, p: PlanT) -> "Plan":
        return cls(VARIANT_NAMES.get(p.variant, str(p.variant)), p.bits1, p.bits2, p.narrow,
                   p.load_factor, p.selector, p.key_min, p.key_max,
                   MATERIALIZE_NAMES.get(p.materialize, str(p.materialize)))

    def to_c(self) -> PlanT:
        p = PlanT()
        p.variant = VARIANTS[self.variant]
        p.bits1, p.bits2, p.narrow = self.bits1, self.bits2, self.narrow
        p.load_factor, p.selector = self.load_factor, self.selector
        return p


_lib = None

# Every symbol include/eiger.h declares (checked against the header by the tests).
SYMBOLS = ("eiger_stats_workspace", "eiger_stats", "eiger_plan", "eiger_join_workspace", "eiger_join",
           "eiger_join_sum", "eiger_join_batched_workspace", "eiger_join_batched",
           "eiger_mlp_param_count", "eiger_mlp_forward", "eiger_mlp_grad_workspace", "eiger_mlp_grad",
           "eiger_mlp_adam", "eiger_features", "eiger_class_plan", "eiger_selector_set",
           "eiger_join_static_noalloc", "eiger_profile", "eiger_profile_read", "eiger_last_error",
           "eiger_version", "eiger_join_wide_workspace", "eiger_join_wide", "eiger_groupby_workspace",
           "eiger_groupby", "eiger_join_sum_workspace")
MLP_IN, MLP_HIDDEN, MLP_OUT = 12, 64, 15


def load():
    """Load libeiger.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    c = ctypes
    vp, i64, i32, sz = c.c_void_p, c.c_int64, c.c_int32, c.c_size_t
    lib.eiger_last_error.restype = c.c_char_p
    lib.eiger_last_error.argtypes = []
    lib.eiger_version.restype = c.c_char_p
    lib.eiger_version.argtypes = []
    lib.eiger_stats_workspace.restype = c.c_int
    lib.eiger_stats_workspace.argtypes = [i64, c.c_int, c.POINTER(sz)]
    lib.eiger_stats.restype = c.c_int
    lib.eiger_stats.argtypes = [vp, i64, c.c_int, c.POINTER(StatsT), vp, sz, vp]
    lib.eiger_plan.restype = c.c_int
    lib.eiger_plan.argtypes = [c.POINTER(StatsT), c.POINTER(StatsT), i64, i64, c.c_int,
                               c.POINTER(PlanT)]
    lib.eiger_join_workspace.restype = c.c_int
    lib.eiger_join_workspace.argtypes = [i64, i64, c.c_int, c.c_int, c.POINTER(PlanT), c.POINTER(sz)]
    lib.eiger_join.restype = c.c_int
    lib.eiger_join.argtypes = [c.c_int, vp, vp, i64, vp, vp, i64, i32, c.c_int, c.POINTER(PlanT),
                               vp, vp, vp, vp, i64, c.POINTER(i64), vp, sz, c.POINTER(PlanT), vp]
    lib.eiger_join_sum.restype = c.c_int
    lib.eiger_join_sum.argtypes = [c.c_int, vp, vp, i64, vp, vp, i64, i32, c.c_int, c.c_int,
                                   c.POINTER(PlanT), c.POINTER(i64), c.POINTER(i64), vp, sz,
                                   c.POINTER(PlanT), vp]
    lib.eiger_join_sum_workspace.restype = c.c_int
    lib.eiger_join_sum_workspace.argtypes = [i64, i64, c.c_int, i32, c.c_int, c.c_int, c.POINTER(PlanT),
                                             c.POINTER(sz)]
    lib.eiger_join_wide_workspace.restype = c.c_int
    lib.eiger_join_wide_workspace.argtypes = [i64, i64, c.c_int, c.POINTER(ColumnsT), c.POINTER(ColumnsT),
                                              c.c_int, c.c_int, c.POINTER(PlanT), c.POINTER(sz)]
    lib.eiger_join_wide.restype = c.c_int
    lib.eiger_join_wide.argtypes = [c.c_int, vp, i64, c.POINTER(ColumnsT), vp, i64, c.POINTER(ColumnsT),
                                    c.c_int, c.c_int, c.POINTER(PlanT), vp, vp, i64, c.POINTER(i64), vp, sz,
                                    c.POINTER(PlanT), vp]
    lib.eiger_groupby_workspace.restype = c.c_int
    lib.eiger_groupby_workspace.argtypes = [i64, c.c_int, c.POINTER(AggsT), c.c_int32, c.POINTER(sz)]
    lib.eiger_groupby.restype = c.c_int
    lib.eiger_groupby.argtypes = [c.c_int, vp, i64, c.POINTER(AggsT), c.c_int32, c.POINTER(GbPlanT), vp, i64,
                                  c.POINTER(i64), vp, sz, c.POINTER(GbPlanT), vp]
    lib.eiger_join_batched_workspace.restype = c.c_int
    lib.eiger_join_batched_workspace.argtypes = [c.POINTER(JoinDescT), c.c_int32, c.c_int,
                                                 c.POINTER(BatchKnobsT), c.POINTER(sz)]
    lib.eiger_join_batched.restype = c.c_int
    lib.eiger_join_batched.argtypes = [c.c_int, vp, c.c_int32, vp, vp, c.POINTER(BatchKnobsT), vp, sz, vp]
    fp = c.POINTER(c.c_float)
    lib.eiger_mlp_param_count.restype = c.c_int32
    lib.eiger_mlp_param_count.argtypes = []
    lib.eiger_mlp_forward.restype = c.c_int
    lib.eiger_mlp_forward.argtypes = [vp, vp, c.c_int32, vp, vp]
    lib.eiger_mlp_grad_workspace.restype = c.c_int
    lib.eiger_mlp_grad_workspace.argtypes = [c.c_int32, c.POINTER(sz)]
    lib.eiger_mlp_grad.restype = c.c_int
    lib.eiger_mlp_grad.argtypes = [vp, vp, vp, c.c_int32, c.c_float, vp, vp, vp, sz, vp]
    lib.eiger_mlp_adam.restype = c.c_int
    lib.eiger_mlp_adam.argtypes = [vp, vp, vp, vp, c.c_int32, c.c_float, vp]
    lib.eiger_features.restype = c.c_int
    lib.eiger_features.argtypes = [c.POINTER(StatsT), c.POINTER(StatsT), i64, i64, c.c_int, sz, fp]
    lib.eiger_class_plan.restype = c.c_int
    lib.eiger_class_plan.argtypes = [c.c_int32, c.POINTER(PlanT)]
    lib.eiger_selector_set.restype = c.c_int
    lib.eiger_selector_set.argtypes = [vp, fp, fp]
    lib.eiger_join_static_noalloc.restype = c.c_int
    lib.eiger_join_static_noalloc.argtypes = [c.c_int, vp, i64, vp, i64, vp, vp, i64, c.POINTER(i64),
                                              vp]
    lib.eiger_profile.restype = c.c_int
    lib.eiger_profile.argtypes = [c.c_int]
    lib.eiger_profile_read.restype = c.c_int
    lib.eiger_profile_read.argtypes = [c.POINTER(StageT), c.c_int]
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise EigerError(status, load().eiger_last_error().decode())


def last_error() -> str:
    return load().eiger_last_error().decode()


def version() -> str:
    return load().eiger_version().decode()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return I32
    if t.dtype == torch.int64:
        return I64
    raise TypeError(f"join keys must be int32 or int64, got {t.dtype}")


def _ptr(t):
    return None if t is None or t.numel() == 0 else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _variant(v) -> int:
    return VARIANTS[v] if isinstance(v, str) else int(v)


def _dev(t: torch.Tensor | None, device) -> torch.Tensor | None:
    """Host tensors are copied to the device (the end-to-end path)."""
    if t is None:
        return None
    t = t.contiguous()
    return t if t.is_cuda else t.to(device, non_blocking=True)


# ------------------------------------------------------------------ API

def profile(enable: bool = True) -> None:
    """eiger_profile: time every kernel launch of later calls on this thread."""
    _check(load().eiger_profile(1 if enable else 0))


def profile_read() -> list[tuple[str, float, int, float]]:
    """(name, device ms, kernel launches, algorithmic bytes) of each stage of
    the last call on this thread."""
    lib = load()
    n = lib.eiger_profile_read(None, 0)
    buf = (StageT * max(n, 1))()
    n = lib.eiger_profile_read(buf, n)
    return [(buf[i].name.decode(), float(buf[i].ms), int(buf[i].launches), float(buf[i].bytes))
            for i in range(n)]


def stats_workspace(n: int, dtype: int) -> int:
    out = ctypes.c_size_t(0)
    _check(load().eiger_stats_workspace(n, dtype, ctypes.byref(out)))
    return out.value


def stats(keys: torch.Tensor, workspace: torch.Tensor | None = None, stream=None) -> Stats:
    """eiger_stats: min, max, HyperLogLog++ registers and estimate of a key column."""
    lib = load()
    keys = _dev(keys, torch.device("cuda"))
    dt = _dtype_code(keys)
    n = keys.numel()
    if workspace is None:
        workspace = torch.empty(stats_workspace(n, dt), dtype=torch.uint8, device=keys.device)
    out = StatsT()
    _check(lib.eiger_stats(_ptr(keys), n, dt, ctypes.byref(out), _ptr(workspace), workspace.numel(),
                           _stream(stream)))
    return Stats.from_c(out)


def plan(build: Stats, probe: Stats | None, nb: int, np_: int, dtype: int) -> Plan:
    """eiger_plan: the rule-based selector (host only)."""
    out = PlanT()
    b = build.to_c()
    p = probe.to_c() if probe is not None else None
    _check(load().eiger_plan(ctypes.byref(b), ctypes.byref(p) if p is not None else None, nb, np_,
                             dtype, ctypes.byref(out)))
    return Plan.from_c(out)


def join_workspace(nb: int, np_: int, dtype: int, variant="auto", knobs: Plan | None = None) -> int:
    out = ctypes.c_size_t(0)
    k = knobs.to_c() if knobs is not None else None
    _check(load().eiger_join_workspace(nb, np_, dtype, _variant(variant),
                                       ctypes.byref(k) if k is not None else None, ctypes.byref(out)))
    return out.value


@dataclass
class JoinResult:
    count: int
    build_idx: torch.Tensor | None
    probe_idx: torch.Tensor | None
    build_pay: torch.Tensor | None
    probe_pay: torch.Tensor | None
    plan: Plan


def join_into(build_keys, probe_keys, *, build_pay=None, probe_pay=None, variant="auto",
              knobs: Plan | None = None, out_bidx=None, out_pidx=None, out_bpay=None, out_ppay=None,
              capacity: int = 0, workspace: torch.Tensor, stream=None):
    """eiger_join into caller-allocated device outputs. Returns (status, count, plan)."""
    lib = load()
    dt = _dtype_code(build_keys)
    pay_bytes = build_pay.element_size() if build_pay is not None else (
        probe_pay.element_size() if probe_pay is not None else 0)
    cnt = ctypes.c_int64(0)
    used = PlanT()
    k = knobs.to_c() if knobs is not None else None
    st = lib.eiger_join(dt, _ptr(build_keys), _ptr(build_pay), build_keys.numel(), _ptr(probe_keys),
                        _ptr(probe_pay), probe_keys.numel(), pay_bytes, _variant(variant),
                        ctypes.byref(k) if k is not None else None, _ptr(out_bidx), _ptr(out_pidx),
                        _ptr(out_bpay), _ptr(out_ppay), capacity, ctypes.byref(cnt),
                        _ptr(workspace), workspace.numel() if workspace is not None else 0,
                        ctypes.byref(used), _stream(stream))
    return st, cnt.value, Plan.from_c(used)


def join(build_keys: torch.Tensor, probe_keys: torch.Tensor, *, build_pay=None, probe_pay=None,
         variant="auto", knobs: Plan | None = None, indices: bool = True, payloads: bool = False,
         capacity: int | None = None, workspace: torch.Tensor | None = None, stream=None,
         to_host: bool = False) -> JoinResult:
    """eiger_join: all matching (build_idx, probe_idx) pairs, and optionally the
    matched payloads. Host (CPU) inputs are copied to the GPU first; with
    ``to_host`` the results are copied back. Retries once with the exact
    capacity when the first guess (``capacity`` or |S|) is too small."""
    dev = torch.device("cuda")
    bk, pk = _dev(build_keys, dev), _dev(probe_keys, dev)
    bp, pp = _dev(build_pay, dev), _dev(probe_pay, dev)
    if _dtype_code(bk) != _dtype_code(pk):
        raise TypeError("build and probe keys must share a dtype")
    if workspace is None:
        workspace = torch.empty(join_workspace(bk.numel(), pk.numel(), _dtype_code(bk), variant,
                                               knobs), dtype=torch.uint8, device=dev)
    cap = pk.numel() if capacity is None else capacity
    for attempt in range(2):
        c = max(cap, 1)
        ob = torch.empty(c, dtype=torch.int32, device=dev) if indices else None
        op = torch.empty(c, dtype=torch.int32, device=dev) if indices else None
        obp = torch.empty(c, dtype=bp.dtype, device=dev) if payloads and bp is not None else None
        opp = torch.empty(c, dtype=pp.dtype, device=dev) if payloads and pp is not None else None
        st, n, used = join_into(bk, pk, build_pay=bp, probe_pay=pp, variant=variant, knobs=knobs,
                                out_bidx=ob, out_pidx=op, out_bpay=obp, out_ppay=opp, capacity=cap,
                                workspace=workspace, stream=stream)
        if st == ERR_CAPACITY and attempt == 0:
            cap = n
            continue
        _check(st)
        break
    cut = lambda t: None if t is None else (t[:n].cpu() if to_host else t[:n])
    return JoinResult(n, cut(ob), cut(op), cut(obp), cut(opp), used)


def join_sum_workspace(nb: int, np_: int, dtype: int, payload_bytes: int, variant="auto",
                       materialize="auto", knobs: Plan | None = None) -> int:
    out = ctypes.c_size_t(0)
    k = knobs.to_c() if knobs is not None else None
    _check(load().eiger_join_sum_workspace(nb, np_, dtype, payload_bytes, _variant(variant), _mat(materialize),
                                           ctypes.byref(k) if k is not None else None, ctypes.byref(out)))
    return out.value


def join_sum(build_keys, build_pay, probe_keys, probe_pay, *, variant="auto", materialize="auto",
             knobs: Plan | None = None, workspace: torch.Tensor | None = None, stream=None):
    """eiger_join_sum: (sum over matches of build_pay + probe_pay mod 2^64, |J|, plan)."""
    lib = load()
    dev = torch.device("cuda")
    bk, pk = _dev(build_keys, dev), _dev(probe_keys, dev)
    bp, pp = _dev(build_pay, dev), _dev(probe_pay, dev)
    dt = _dtype_code(bk)
    if bp.dtype != pp.dtype:
        raise TypeError("payload columns must share a dtype")
    if workspace is None:
        workspace = torch.empty(join_sum_workspace(bk.numel(), pk.numel(), dt, bp.element_size(), variant,
                                                   materialize, knobs),
                                dtype=torch.uint8, device=dev)
    s = ctypes.c_int64(0)
    cnt = ctypes.c_int64(0)
    used = PlanT()
    k = knobs.to_c() if knobs is not None else None
    _check(lib.eiger_join_sum(dt, _ptr(bk), _ptr(bp), bk.numel(), _ptr(pk), _ptr(pp), pk.numel(),
                              bp.element_size(), _variant(variant), _mat(materialize),
                              ctypes.byref(k) if k is not None else None, ctypes.byref(s),
                              ctypes.byref(cnt), _ptr(workspace), workspace.numel(),
                              ctypes.byref(used), _stream(stream)))
    return s.value, cnt.value, Plan.from_c(used)


def _columns(cols, outs=None) -> ColumnsT | None:
    """eiger_columns of one side from a list of 4- or 8-byte device tensors
    (and the matching output tensors)."""
    if not cols:
        return None
    if len(cols) > MAX_COLS:
        raise ValueError(f"at most {MAX_COLS} payload columns per side")
    c = ColumnsT()
    c.n = len(cols)
    for q, t in enumerate(cols):
        c.bytes[q] = t.element_size()
        c.cols[q] = t.data_ptr() if t.numel() else None
        if outs is not None:
            c.out[q] = outs[q].data_ptr() if outs[q].numel() else None
    return c


def _mat(m) -> int:
    return MATERIALIZE[m] if isinstance(m, str) else int(m)


def join_wide_workspace(nb: int, np_: int, dtype: int, build_cols=(), probe_cols=(), variant="auto",
                        materialize="auto", knobs: Plan | None = None) -> int:
    out = ctypes.c_size_t(0)
    b, p = _columns(list(build_cols)), _columns(list(probe_cols))
    k = knobs.to_c() if knobs is not None else None
    _check(load().eiger_join_wide_workspace(nb, np_, dtype, ctypes.byref(b) if b is not None else None,
                                            ctypes.byref(p) if p is not None else None, _variant(variant),
                                            _mat(materialize), ctypes.byref(k) if k is not None else None,
                                            ctypes.byref(out)))
    return out.value


def join_wide_into(build_keys, probe_keys, build_cols, probe_cols, build_out, probe_out, *, variant="auto",
                   materialize="auto", knobs: Plan | None = None, out_bidx=None, out_pidx=None,
                   capacity: int = 0, workspace: torch.Tensor, stream=None):
    """eiger_join_wide into caller-allocated device outputs (one output tensor
    per payload column). Returns (status, count, plan)."""
    lib = load()
    dt = _dtype_code(build_keys)
    b, p = _columns(list(build_cols), build_out), _columns(list(probe_cols), probe_out)
    cnt = ctypes.c_int64(0)
    used = PlanT()
    k = knobs.to_c() if knobs is not None else None
    st = lib.eiger_join_wide(dt, _ptr(build_keys), build_keys.numel(), ctypes.byref(b) if b is not None else None,
                             _ptr(probe_keys), probe_keys.numel(), ctypes.byref(p) if p is not None else None,
                             _variant(variant), _mat(materialize), ctypes.byref(k) if k is not None else None,
                             _ptr(out_bidx), _ptr(out_pidx), capacity, ctypes.byref(cnt), _ptr(workspace),
                             workspace.numel() if workspace is not None else 0, ctypes.byref(used),
                             _stream(stream))
    return st, cnt.value, Plan.from_c(used)


@dataclass
class WideResult:
    count: int
    build_idx: torch.Tensor | None
    probe_idx: torch.Tensor | None
    build_cols: list
    probe_cols: list
    plan: Plan


def join_wide(build_keys, probe_keys, build_cols=(), probe_cols=(), *, variant="auto", materialize="auto",
              knobs: Plan | None = None, indices: bool = True, capacity: int | None = None,
              workspace: torch.Tensor | None = None, stream=None) -> WideResult:
    """eiger_join_wide: every match with its build and probe payload columns
    (and the tuple IDs when ``indices``). Host inputs are copied to the GPU.
    Retries once with the exact capacity when the first guess is too small."""
    dev = torch.device("cuda")
    bk, pk = _dev(build_keys, dev), _dev(probe_keys, dev)
    bc = [_dev(t, dev) for t in build_cols]
    pc = [_dev(t, dev) for t in probe_cols]
    dt = _dtype_code(bk)
    if workspace is None:
        workspace = torch.empty(join_wide_workspace(bk.numel(), pk.numel(), dt, bc, pc, variant, materialize,
                                                    knobs), dtype=torch.uint8, device=dev)
    cap = pk.numel() if capacity is None else capacity
    for attempt in range(2):
        c = max(cap, 1)
        ob = torch.empty(c, dtype=torch.int32, device=dev) if indices else None
        op = torch.empty(c, dtype=torch.int32, device=dev) if indices else None
        bo = [torch.empty(c, dtype=t.dtype, device=dev) for t in bc]
        po = [torch.empty(c, dtype=t.dtype, device=dev) for t in pc]
        st, n, used = join_wide_into(bk, pk, bc, pc, bo, po, variant=variant, materialize=materialize,
                                     knobs=knobs, out_bidx=ob, out_pidx=op, capacity=cap, workspace=workspace,
                                     stream=stream)
        if st == ERR_CAPACITY and attempt == 0:
            cap = n
            continue
        _check(st)
        break
    cut = lambda t: None if t is None else t[:n]
    return WideResult(n, cut(ob), cut(op), [t[:n] for t in bo], [t[:n] for t in po], used)


def _aggs(aggs, outs=None) -> AggsT:
    """eiger_aggs from a list of (op, values tensor or None for count)."""
    if len(aggs) > MAX_AGGS:
        raise ValueError(f"at most {MAX_AGGS} aggregates")
    a = AggsT()
    a.n = len(aggs)
    for q, (op, vals) in enumerate(aggs):
        a.op[q] = AGG_OPS[op] if isinstance(op, str) else int(op)
        a.bytes[q] = vals.element_size() if vals is not None else 8
        a.vals[q] = vals.data_ptr() if vals is not None and vals.numel() else None
        if outs is not None:
            a.out[q] = outs[q].data_ptr() if outs[q].numel() else None
    return a


def _gb_variant(v) -> int:
    return GB_VARIANTS[v] if isinstance(v, str) else int(v)


def groupby_workspace(n: int, dtype: int, aggs, variant="auto") -> int:
    out = ctypes.c_size_t(0)
    a = _aggs(list(aggs))
    _check(load().eiger_groupby_workspace(n, dtype, ctypes.byref(a), _gb_variant(variant), ctypes.byref(out)))
    return out.value


def groupby_into(keys, aggs, out_keys, outs, *, variant="auto", knobs: GbPlan | None = None, capacity: int = 0,
                 workspace: torch.Tensor, stream=None):
    """eiger_groupby into caller-allocated outputs. Returns (status, groups, plan)."""
    lib = load()
    a = _aggs(list(aggs), outs)
    cnt = ctypes.c_int64(0)
    used = GbPlanT()
    k = knobs.to_c() if knobs is not None else None
    st = lib.eiger_groupby(_dtype_code(keys), _ptr(keys), keys.numel(), ctypes.byref(a), _gb_variant(variant),
                           ctypes.byref(k) if k is not None else None, _ptr(out_keys), capacity, ctypes.byref(cnt),
                           _ptr(workspace), workspace.numel() if workspace is not None else 0, ctypes.byref(used),
                           _stream(stream))
    return st, cnt.value, GbPlan.from_c(used)


@dataclass
class GroupByResult:
    groups: int
    keys: torch.Tensor
    aggs: list
    plan: GbPlan


def groupby(keys, aggs=(), *, variant="auto", knobs: GbPlan | None = None, capacity: int | None = None,
            workspace: torch.Tensor | None = None, stream=None) -> GroupByResult:
    """eiger_groupby: every distinct key with its aggregates (int64 each).
    ``aggs``: list of (op, values) with op in sum/count/min/max (values None
    for count). Host inputs are copied to the GPU. Retries once with the exact
    capacity when the first guess is too small."""
    dev = torch.device("cuda")
    k = _dev(keys, dev)
    ag = [(op, _dev(v, dev)) for op, v in aggs]
    dt = _dtype_code(k)
    if workspace is None:
        workspace = torch.empty(groupby_workspace(k.numel(), dt, ag, variant), dtype=torch.uint8, device=dev)
    cap = min(k.numel(), 1 << 20) if capacity is None else capacity
    for attempt in range(2):
        c = max(cap, 1)
        ok = torch.empty(c, dtype=k.dtype, device=dev)
        outs = [torch.empty(c, dtype=torch.int64, device=dev) for _ in ag]
        st, n, used = groupby_into(k, ag, ok, outs, variant=variant, knobs=knobs, capacity=cap, workspace=workspace,
                                   stream=stream)
        if st == ERR_CAPACITY and attempt == 0:
            cap = n
            continue
        _check(st)
        break
    return GroupByResult(n, ok[:n], [o[:n] for o in outs], used)


def join_static_noalloc_into(build_keys, probe_keys, out_bidx, out_pidx, capacity: int,
                             stream=None):
    """eiger_join_static_noalloc into caller-owned outputs: the static join
    with its scratch in the library's fixed device array (for callers that
    cannot allocate). Returns (status, count).

    The kernels read and write through raw pointers, so every argument is
    checked here first, as join() does: both key columns contiguous CUDA
    tensors of one dtype (int32 or int64); each output None or a contiguous
    int32 CUDA tensor of at least `capacity` entries."""
    if capacity < 0:
        raise ValueError("capacity must be >= 0")
    for name, t in (("build_keys", build_keys), ("probe_keys", probe_keys)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA tensor")
    if build_keys.dtype != probe_keys.dtype:
        raise TypeError("build and probe keys must share a dtype")
    dt = _dtype_code(build_keys)
    if capacity > 0 and out_bidx is None and out_pidx is None:
        raise ValueError("capacity > 0 needs at least one output tensor")
    for name, t in (("out_bidx", out_bidx), ("out_pidx", out_pidx)):
        if t is None:
            continue
        if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous() or t.dtype != torch.int32:
            raise TypeError(f"{name} must be a contiguous int32 CUDA tensor")
        if t.numel() < capacity:
            raise ValueError(f"{name} holds {t.numel()} entries < capacity {capacity}")
    lib = load()
    cnt = ctypes.c_int64(0)
    st = lib.eiger_join_static_noalloc(dt, _ptr(build_keys), build_keys.numel(), _ptr(probe_keys),
                                       probe_keys.numel(), _ptr(out_bidx), _ptr(out_pidx), capacity,
                                       ctypes.byref(cnt), _stream(stream))
    return st, cnt.value


@dataclass
class BatchKnobs:
    block_threads: int = 256
    chunk_rows: int = 16384
    load_factor: float = 0.5
    small_rows: int = 1024  # joins with at most this many build rows use a shared-memory table

    def to_c(self) -> BatchKnobsT:
        return BatchKnobsT(self.block_threads, self.chunk_rows, self.load_factor, self.small_rows)


class BatchedJoin:
    """k independent joins run by one eiger_join_batched call.

    Build and probe key columns are given as lists of device tensors (one
    dtype). Outputs live in two concatenated uint32 buffers; join j's pairs are
    out_bidx[off[j] : off[j] + counts[j]] (capped at its capacity). ``run``
    enqueues the call on the current stream; ``capture`` records it into a CUDA
    graph whose replays redo the whole batch.
    """

    def __init__(self, builds, probes, capacities=None, knobs: "BatchKnobs | None" = None):
        if len(builds) != len(probes):
            raise ValueError("builds and probes differ in length")
        lib = load()
        self.k = len(builds)
        self.builds = [b.contiguous() for b in builds]
        self.probes = [p.contiguous() for p in probes]
        dts = {_dtype_code(t) for t in self.builds + self.probes} or {I32}
        if len(dts) != 1:
            raise TypeError("all key columns of a batch must share one dtype")
        self.dtype = dts.pop()
        dev = torch.device("cuda")
        caps = [p.numel() for p in self.probes] if capacities is None else list(capacities)
        self.capacities = caps
        self.off = np.zeros(self.k + 1, np.int64)
        self.off[1:] = np.cumsum(caps)
        total = int(self.off[-1])
        self.out_bidx = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        self.out_pidx = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
        descs = (JoinDescT * max(self.k, 1))()
        for j in range(self.k):
            d = descs[j]
            d.build_keys = self.builds[j].data_ptr() if self.builds[j].numel() else None
            d.probe_keys = self.probes[j].data_ptr() if self.probes[j].numel() else None
            d.nb, d.np = self.builds[j].numel(), self.probes[j].numel()
            d.out_bidx = self.out_bidx.data_ptr() + 4 * int(self.off[j])
            d.out_pidx = self.out_pidx.data_ptr() + 4 * int(self.off[j])
            d.capacity = int(caps[j])
        self.knobs = knobs if knobs is not None else (load_tuned_batch_knobs() or BatchKnobs())
        kc = self.knobs.to_c()
        ws = ctypes.c_size_t(0)
        _check(lib.eiger_join_batched_workspace(descs, self.k, self.dtype, ctypes.byref(kc),
                                                ctypes.byref(ws)))
        self.workspace = torch.empty(max(ws.value, 1), dtype=torch.uint8, device=dev)
        raw = bytes(descs)[: ctypes.sizeof(JoinDescT) * self.k]
        self.d_descs = torch.frombuffer(bytearray(raw or b"\0"), dtype=torch.uint8).to(dev)
        self.counts = torch.zeros(max(self.k, 1), dtype=torch.int64, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        self._kc = kc

    def run(self, stream=None):
        _check(load().eiger_join_batched(self.dtype, _ptr(self.d_descs), self.k, _ptr(self.counts),
                                         _ptr(self.status), ctypes.byref(self._kc), _ptr(self.workspace),
                                         self.workspace.numel(), _stream(stream)))

    def capture(self):
        """Record one batch into a CUDA graph (runs it once eagerly first)."""
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def result(self, j):
        """(count, build_idx, probe_idx) of join j (device tensors, capped at capacity)."""
        n = int(self.counts[j])
        m = min(n, int(self.capacities[j]))
        a, b = int(self.off[j]), int(self.off[j]) + m
        return n, self.out_bidx[a:b], self.out_pidx[a:b]


_TUNED = os.path.join(_HERE, "tuned_batch.json")


def load_tuned_batch_knobs() -> "BatchKnobs | None":
    """Knobs the autotuner stored for this GPU model, if any."""
    import json

    try:
        with open(_TUNED) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    try:
        name = torch.cuda.get_device_name() if torch.cuda.is_available() else None
    except Exception:
        name = None
    if name is not None and d.get("device") not in (None, name):
        return None
    k = d.get("knobs", {})
    return BatchKnobs(int(k.get("block_threads", 256)), int(k.get("chunk_rows", 16384)),
                      float(k.get("load_factor", 0.5)), int(k.get("small_rows", 1024)))


# ------------------------------------------------------------------ selector network

def mlp_param_count() -> int:
    return int(load().eiger_mlp_param_count())


def mlp_forward(params: torch.Tensor, x: torch.Tensor, stream=None) -> torch.Tensor:
    """Logits [n, 15] of the selector network (device float32 tensors)."""
    n = x.shape[0]
    z = torch.empty((n, MLP_OUT), dtype=torch.float32, device=x.device)
    _check(load().eiger_mlp_forward(_ptr(params), _ptr(x), n, _ptr(z), _stream(stream)))
    return z


def mlp_grad(params, x, cost, tau: float = 0.0, workspace=None, stream=None):
    """(mean loss, gradient) from the library's gradient kernels: the expected
    regret for tau = 0, the soft-target cross-entropy for tau > 0."""
    lib = load()
    n = x.shape[0]
    if workspace is None:
        b = ctypes.c_size_t(0)
        _check(lib.eiger_mlp_grad_workspace(n, ctypes.byref(b)))
        workspace = torch.empty(max(b.value, 1), dtype=torch.uint8, device=x.device)
    g = torch.empty_like(params)
    L = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib.eiger_mlp_grad(_ptr(params), _ptr(x), _ptr(cost), n, tau, _ptr(g), _ptr(L), _ptr(workspace),
                              workspace.numel(), _stream(stream)))
    return L, g


def mlp_adam(params, grad, m, v, step: int, lr: float, stream=None):
    _check(load().eiger_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, _stream(stream)))


def features(build: Stats, probe_sample: "Stats | None", nb: int, np_: int, dtype: int,
             l2_bytes: int = 0) -> np.ndarray:
    out = (ctypes.c_float * MLP_IN)()
    b = build.to_c()
    p = probe_sample.to_c() if probe_sample is not None else None
    _check(load().eiger_features(ctypes.byref(b), ctypes.byref(p) if p is not None else None, nb, np_, dtype,
                                 l2_bytes, out))
    return np.array(out[:], dtype=np.float32)


def class_plan(cls: int) -> Plan:
    p = PlanT()
    _check(load().eiger_class_plan(cls, ctypes.byref(p)))
    return Plan.from_c(p)


_SELECTOR_KEEP = []


def selector_set(params: "torch.Tensor | None", mean=None, scale=None) -> None:
    """Let EIGER_AUTO use the network (device params kept alive here); None
    restores the rule-based selector."""
    lib = load()
    if params is None:
        _check(lib.eiger_selector_set(None, None, None))
        _SELECTOR_KEEP.clear()
        return
    m = (ctypes.c_float * MLP_IN)(*[float(v) for v in mean])
    s = (ctypes.c_float * MLP_IN)(*[float(v) for v in scale])
    _check(lib.eiger_selector_set(_ptr(params), m, s))
    _SELECTOR_KEEP[:] = [params]
