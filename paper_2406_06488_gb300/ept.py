"""Thin ctypes binding of libept (include/ept.h): argument marshalling only.

Every step of a test runs in libept's CUDA kernels; there is no CPU fallback.  If
``_build/libept.so`` is missing the import of the library fails with an error
telling how to build it.

Arrays may be numpy arrays (host memory: the library copies them to the GPU) or
CUDA torch tensors (device memory: the library works in place and returns the
permuted statistics as a CUDA tensor).  One call may not mix the two.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libept.so")

STAT = {"ed": 0, "mmd": 1, "mmd_gauss": 1, "mmd_laplace": 2}
SIGMA_MEDIAN = -1.0   # EPT_SIGMA_MEDIAN: bandwidth from the median heuristic
ABI_VERSION = 6       # EPT_ABI_VERSION this binding's structures follow
PREC = {"plain_fp32": 0, "split_bf16": 1, "pooled_fp32": 2}   # pooled_fp32: Algorithm 5 baseline
STATUS = {0: "EPT_OK", 1: "EPT_EINVAL", 2: "EPT_ENOMEM", 3: "EPT_EBUSY", 4: "EPT_ECUDA", 5: "EPT_ETIMEOUT",
          6: "EPT_ECANCELLED", 7: "EPT_ENOTFOUND", 8: "EPT_EUNSUPPORTED", 9: "EPT_EINTERNAL"}

# every entry point declared in include/ept.h
EXPORTS = ["ept_abi_version", "ept_build_info", "ept_last_error", "ept_create", "ept_destroy", "ept_estimate_bytes", "ept_test",
           "ept_test_masks", "ept_perm_masks", "ept_build_blocks", "ept_test_static", "ept_test_batch",
           "ept_set_option", "ept_submit", "ept_poll", "ept_wait", "ept_cancel", "ept_test_range",
           "ept_serving_stats", "ept_create_ex", "ept_plan_check", "ept_serving_lanes"]


class EptError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, str(status)), message))
        self.status = status


class _TestDesc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("Y", ctypes.c_void_p), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("p", ctypes.c_int64), ("stat", ctypes.c_int), ("sigma", ctypes.c_double), ("B", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("perm_stats", ctypes.c_void_p)]


class _Result(ctypes.Structure):
    _fields_ = [("observed", ctypes.c_double), ("p_value", ctypes.c_double), ("n_ge", ctypes.c_int64),
                ("n_near_tie", ctypes.c_int64), ("n_fixup", ctypes.c_int64), ("ms_build", ctypes.c_double),
                ("ms_perm", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_masks", ctypes.c_double),
                ("ms_contract", ctypes.c_double), ("sigma", ctypes.c_double), ("n_windows", ctypes.c_int64),
                ("n_refined", ctypes.c_int64), ("tuning", ctypes.c_int64), ("tune_candidates", ctypes.c_int64),
                ("refine_launches", ctypes.c_int64)]


class _PlanInfo(ctypes.Structure):
    _fields_ = [("units", ctypes.c_int64), ("chunks", ctypes.c_int64), ("stored_blocks", ctypes.c_int64),
                ("partials", ctypes.c_int64), ("cta_kblocks_max", ctypes.c_int64), ("cta_kblocks_min", ctypes.c_int64),
                ("windows", ctypes.c_int64), ("scratch_bytes", ctypes.c_size_t)]


# ept_allocator: device memory from the caller (ept_create_ex)
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _Allocator(ctypes.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", ctypes.c_void_p)]


@dataclass
class Result:
    observed: float
    p_value: float
    n_ge: int
    n_near_tie: int
    n_fixup: int
    ms_build: float
    ms_perm: float
    ms_total: float
    ms_masks: float
    ms_contract: float
    sigma: float
    n_windows: int = 0
    n_refined: int = 0
    tuning: int = 0
    tune_candidates: int = 0
    refine_launches: int = 0
    stats: Optional[object] = field(default=None, repr=False)


def _result(r, buf) -> "Result":
    return Result(r.observed, r.p_value, r.n_ge, r.n_near_tie, r.n_fixup, r.ms_build, r.ms_perm, r.ms_total,
                  r.ms_masks, r.ms_contract, r.sigma, r.n_windows, r.n_refined, r.tuning, r.tune_candidates,
                  r.refine_launches, buf)


_lib = None


def load():
    """Load libept.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libept.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`"
                           % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, u64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    lib.ept_abi_version.argtypes = []
    lib.ept_abi_version.restype = i32
    if lib.ept_abi_version() != ABI_VERSION:
        raise RuntimeError("libept ABI version %d, binding expects %d: rebuild the library"
                           % (lib.ept_abi_version(), ABI_VERSION))
    lib.ept_last_error.argtypes = []
    lib.ept_last_error.restype = ctypes.c_char_p
    lib.ept_build_info.argtypes = []
    lib.ept_build_info.restype = ctypes.c_char_p
    lib.ept_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_size_t]
    lib.ept_create.restype = i32
    lib.ept_create_ex.argtypes = [ctypes.POINTER(vp), i32, ctypes.c_size_t, ctypes.POINTER(_Allocator)]
    lib.ept_create_ex.restype = i32
    lib.ept_destroy.argtypes = [vp]
    lib.ept_destroy.restype = i32
    lib.ept_estimate_bytes.argtypes = [i64, i64, i64, i64, i32]
    lib.ept_estimate_bytes.restype = ctypes.c_size_t
    lib.ept_plan_check.argtypes = [vp, vp, vp, vp, i32, i32, i32, i64, ctypes.POINTER(_PlanInfo)]
    lib.ept_plan_check.restype = i32
    lib.ept_test.argtypes = [vp, vp, i64, vp, i64, i64, i32, i32, f64, i64, u64, i32, vp, ctypes.POINTER(_Result), vp]
    lib.ept_test.restype = i32
    lib.ept_test_range.argtypes = [vp, vp, i64, vp, i64, i64, i32, i32, f64, i64, i64, u64, i32, vp,
                                   ctypes.POINTER(_Result), vp]
    lib.ept_test_range.restype = i32
    lib.ept_test_masks.argtypes = [vp, vp, i64, vp, i64, i64, i32, i32, f64, vp, i64, i32, vp,
                                   ctypes.POINTER(_Result), vp]
    lib.ept_test_masks.restype = i32
    lib.ept_perm_masks.argtypes = [vp, u64, i64, i64, i64, i64, vp, i32, vp]
    lib.ept_perm_masks.restype = i32
    lib.ept_build_blocks.argtypes = [vp, vp, i64, vp, i64, i64, i32, i32, f64, i32, vp, vp]
    lib.ept_build_blocks.restype = i32
    lib.ept_test_static.argtypes = [vp, i64, vp, i64, i64, i32, f64, i64, u64, vp, ctypes.POINTER(_Result), vp]
    lib.ept_test_static.restype = i32
    lib.ept_test_batch.argtypes = [vp, ctypes.POINTER(_TestDesc), i64, i32, i32, ctypes.POINTER(_Result), vp]
    lib.ept_test_batch.restype = i32
    lib.ept_set_option.argtypes = [vp, i32, i64]
    lib.ept_set_option.restype = i32
    lib.ept_submit.argtypes = [vp, ctypes.POINTER(_TestDesc), i32, ctypes.POINTER(u64)]
    lib.ept_submit.restype = i32
    lib.ept_poll.argtypes = [vp, u64, ctypes.POINTER(i32)]
    lib.ept_poll.restype = i32
    lib.ept_wait.argtypes = [vp, u64, vp, ctypes.POINTER(_Result), i64]
    lib.ept_wait.restype = i32
    lib.ept_serving_stats.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(i64),
                                      ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.ept_serving_stats.restype = i32
    lib.ept_serving_lanes.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.ept_serving_lanes.restype = i32
    lib.ept_cancel.argtypes = [vp, u64]
    lib.ept_cancel.restype = i32
    _lib = lib
    return lib


def _check(status: int):
    if status != 0:
        raise EptError(status, load().ept_last_error().decode(errors="replace"))


def _is_torch_cuda(a) -> bool:
    return type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _stat(stat) -> int:
    if isinstance(stat, str):
        return STAT[stat.lower()]
    return int(stat)


def _sigma(sigma) -> float:
    """Kernel bandwidth: a number, or "median" for the median heuristic."""
    if isinstance(sigma, str):
        if sigma.lower() != "median":
            raise ValueError("sigma must be a number or 'median'")
        return SIGMA_MEDIAN
    return float(sigma)


def _prec(prec) -> int:
    if isinstance(prec, str):
        return PREC[prec.lower()]
    return int(prec)


def build_info() -> str:
    """How the loaded library was built (ABI, host and GPU architecture, nvcc, date)."""
    return load().ept_build_info().decode()


def estimate_bytes(nx: int, ny: int, p: int, B: int, prec="split_bf16") -> int:
    return int(load().ept_estimate_bytes(nx, ny, p, B, _prec(prec)))


def plan_check(shapes, unit_kb: int = 8, num_sms: int = 152, stream_blocks: int = 0) -> dict:
    """The run planner on the host alone (ept_plan_check): shapes = [(nx, ny, p, B), ...].
    Returns the plan's totals; raises EptError if an argument is bad or an invariant breaks."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(shapes, dtype=np.int64).reshape(-1, 4).T)
    info = _PlanInfo()
    _check(load().ept_plan_check(a[0].ctypes.data, a[1].ctypes.data, a[2].ctypes.data, a[3].ctypes.data,
                                 a.shape[1], unit_kb, num_sms, stream_blocks, ctypes.byref(info)))
    return {name: int(getattr(info, name)) for name, _ in _PlanInfo._fields_}


OPTION = {"graphs": 1, "autotune": 2, "serve_lanes": 3, "serve_slots": 4, "draw_mode": 5,
          "fault_inject_alloc": 6, "fault_inject_stall": 7, "debug_checks": 8, "stream_blocks": 9,
          "wait_limit_ms": 10, "max_chunk": 11, "refine": 12, "contraction": 13, "unit_kb": 14}


class Context:
    """One libept context on one CUDA device (owns its scratch memory and stream)."""

    def __init__(self, device: int = 0, budget_bytes: int = 0, allocator=None):
        """allocator: optional (alloc, free) pair of callables for the context's device
        scratch -- alloc(nbytes, stream) -> device address (int, 256-byte aligned; 0 on
        failure), free(address, stream); `stream` is the cudaStream_t (int) whose work
        uses the memory (ept_allocator in ept.h)."""
        lib = load()
        h = ctypes.c_void_p()
        self._alloc_keep = None
        if allocator is None:
            _check(lib.ept_create(ctypes.byref(h), int(device), int(budget_bytes)))
        else:
            a_fn, f_fn = allocator

            def _a(nbytes, stream, user):
                return int(a_fn(int(nbytes), int(stream or 0))) or None

            def _f(ptr, stream, user):
                f_fn(int(ptr or 0), int(stream or 0))

            st = _Allocator(_ALLOC_FN(_a), _FREE_FN(_f), None)
            self._alloc_keep = st   # the callbacks must outlive the context
            _check(lib.ept_create_ex(ctypes.byref(h), int(device), int(budget_bytes), ctypes.byref(st)))
        self._h = h
        self.device = int(device)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().ept_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ helpers
    def _arrays(self, X, Y):
        dev = _is_torch_cuda(X)
        if dev != _is_torch_cuda(Y):
            raise TypeError("X and Y must both be numpy arrays or both CUDA tensors")
        if dev:
            import torch
            if X.dtype != torch.float32 or Y.dtype != torch.float32:
                raise TypeError("X and Y must be float32")
            X = X.contiguous()
            Y = Y.contiguous()
            if X.dim() != 2 or Y.dim() != 2 or X.shape[1] != Y.shape[1]:
                raise ValueError("X and Y must be 2-D with the same number of columns")
            stream = torch.cuda.current_stream(X.device).cuda_stream
            return X, Y, X.data_ptr(), Y.data_ptr(), 1, stream
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        if X.ndim != 2 or Y.ndim != 2 or X.shape[1] != Y.shape[1]:
            raise ValueError("X and Y must be 2-D with the same number of columns")
        return X, Y, X.ctypes.data, Y.ctypes.data, 0, None

    def _stats_buffer(self, X, count: int, on_dev: int):
        if count <= 0:
            return None, None
        if on_dev:
            import torch
            buf = torch.empty(count, dtype=torch.float64, device=X.device)
            return buf, buf.data_ptr()
        buf = np.empty(count, dtype=np.float64)
        return buf, buf.ctypes.data

    # ------------------------------------------------------------------ API
    def test(self, X, Y, B: int, seed: int = 0, stat="ed", sigma: float = 1.0, prec="split_bf16",
             want_stats: bool = True) -> Result:
        """Permutation test (Algorithm 1): observed statistic, B permuted statistics
        (draws 1..B of the stream of `seed`) and the p-value."""
        X, Y, px, py, on_dev, stream = self._arrays(X, Y)
        buf, pbuf = self._stats_buffer(X, B if want_stats else 0, on_dev)
        r = _Result()
        _check(load().ept_test(self._h, px, X.shape[0], py, Y.shape[0], X.shape[1], on_dev, _stat(stat),
                               _sigma(sigma), int(B), ctypes.c_uint64(seed), _prec(prec), pbuf, ctypes.byref(r),
                               stream))
        return _result(r, buf)

    def test_range(self, X, Y, b_first: int, count: int, seed: int = 0, stat="ed", sigma: float = 1.0,
                   prec="split_bf16", want_stats: bool = True) -> Result:
        """The observed statistic and draws b_first .. b_first + count - 1 of the stream
        of `seed` (a range of ept_test's relabelings; p_value is the range's own)."""
        X, Y, px, py, on_dev, stream = self._arrays(X, Y)
        buf, pbuf = self._stats_buffer(X, count if want_stats else 0, on_dev)
        r = _Result()
        _check(load().ept_test_range(self._h, px, X.shape[0], py, Y.shape[0], X.shape[1], on_dev, _stat(stat),
                                     _sigma(sigma), int(b_first), int(count), ctypes.c_uint64(seed), _prec(prec),
                                     pbuf, ctypes.byref(r), stream))
        return _result(r, buf)

    def test_masks(self, X, Y, masks, stat="ed", sigma: float = 1.0, prec="split_bf16") -> Result:
        """The test on caller-given relabelings: masks [count, ceil(n/32)] uint32
        (pooled row t = bit t%32 of word t//32; set = row goes to x*)."""
        X, Y, px, py, on_dev, stream = self._arrays(X, Y)
        if on_dev:
            import torch
            if not _is_torch_cuda(masks):
                raise TypeError("masks must be a CUDA tensor when X and Y are")
            masks = masks.contiguous()
            count = masks.shape[0]
            pm = masks.data_ptr()
        else:
            masks = np.ascontiguousarray(masks, dtype=np.uint32)
            if masks.ndim != 2:
                raise ValueError("masks must be 2-D")
            count = masks.shape[0]
            pm = masks.ctypes.data if count > 0 else None
        n = X.shape[0] + Y.shape[0]
        if count > 0 and masks.shape[1] != (n + 31) // 32:
            raise ValueError("masks need ceil(n/32) = %d words per relabeling" % ((n + 31) // 32))
        buf, pbuf = self._stats_buffer(X, count, on_dev)
        r = _Result()
        _check(load().ept_test_masks(self._h, px, X.shape[0], py, Y.shape[0], X.shape[1], on_dev, _stat(stat),
                                     _sigma(sigma), pm, int(count), _prec(prec), pbuf, ctypes.byref(r), stream))
        return _result(r, buf)

    def test_batch(self, tests, prec="split_bf16", want_stats: bool = True):
        """Many tests in one batched run.  tests: sequence of dicts with keys X, Y, B and
        optionally seed, stat, sigma (all X/Y numpy, or all CUDA tensors).  Returns a
        list of Result (stats: B permuted statistics each when want_stats)."""
        return self.prepare_batch(tests, prec, want_stats).run()

    def prepare_batch(self, tests, prec="split_bf16", want_stats: bool = True) -> "PreparedBatch":
        """The descriptors and output buffers of a batch, built once; `run()` runs it
        (again) on whatever the arrays hold at that time."""
        return PreparedBatch(self, tests, prec, want_stats)

    def set_option(self, option: str, value: int) -> None:
        _check(load().ept_set_option(self._h, OPTION[option], int(value)))

    # ------------------------------------------------------------------ serving
    def submit(self, X, Y, B: int, seed: int = 0, stat="ed", sigma: float = 1.0, prec="split_bf16") -> int:
        """Queue one test (host arrays, copied before returning); returns a ticket."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        d = _TestDesc(X.ctypes.data, Y.ctypes.data, X.shape[0], Y.shape[0], X.shape[1], _stat(stat), _sigma(sigma),
                      int(B), int(seed), None)
        t = ctypes.c_uint64(0)
        _check(load().ept_submit(self._h, ctypes.byref(d), _prec(prec), ctypes.byref(t)))
        self._pending_B = getattr(self, "_pending_B", {})
        self._pending_B[t.value] = int(B)
        return t.value

    def poll(self, ticket: int) -> bool:
        done = ctypes.c_int(0)
        _check(load().ept_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(done)))
        return bool(done.value)

    def wait(self, ticket: int, timeout_ms: int = -1) -> Result:
        B = getattr(self, "_pending_B", {}).get(ticket, 0)
        buf = np.empty(B, dtype=np.float64) if B > 0 else None
        r = _Result()
        st = load().ept_wait(self._h, ctypes.c_uint64(ticket), buf.ctypes.data if buf is not None else None,
                             ctypes.byref(r), int(timeout_ms))
        if st != 5:   # a timeout keeps the ticket
            self._pending_B.pop(ticket, None)
        _check(st)
        return _result(r, buf)

    def serving_stats(self) -> dict:
        b = ctypes.c_size_t(0)
        run, q, fin = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(load().ept_serving_stats(self._h, ctypes.byref(b), ctypes.byref(run), ctypes.byref(q),
                                        ctypes.byref(fin)))
        return {"bytes_in_use": b.value, "running": run.value, "queued": q.value, "finished": fin.value}

    def serving_lanes(self) -> dict:
        """Lanes busy now, the most busy at once so far, and requests submitted while a
        batch was running (ept_serving_lanes)."""
        b, pk, sb = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        _check(load().ept_serving_lanes(self._h, ctypes.byref(b), ctypes.byref(pk), ctypes.byref(sb)))
        return {"busy": b.value, "peak_busy": pk.value, "submits_while_busy": sb.value}

    def cancel(self, ticket: int) -> None:
        _check(load().ept_cancel(self._h, ctypes.c_uint64(ticket)))

    def perm_masks(self, seed: int, nx: int, ny: int, b0: int, count: int) -> np.ndarray:
        """Draws b0 .. b0+count-1 of the permutation stream, generated on the GPU:
        uint32 [count, ceil((nx+ny)/32)]."""
        nwu = (nx + ny + 31) // 32
        out = np.zeros((count, nwu), dtype=np.uint32)
        _check(load().ept_perm_masks(self._h, ctypes.c_uint64(seed), nx, ny, b0, count,
                                     out.ctypes.data if count else None, 0, None))
        return out

    def build_blocks(self, X, Y, stat="ed", sigma: float = 1.0, prec="split_bf16") -> np.ndarray:
        """Phase 1 alone: the pooled [[D_XX, D_XY], [D_XY', D_YY]] as built (FP32 numpy)."""
        X, Y, px, py, on_dev, stream = self._arrays(X, Y)
        n = X.shape[0] + Y.shape[0]
        if on_dev:
            import torch
            out = torch.empty((n, n), dtype=torch.float32, device=X.device)
            pout = out.data_ptr()
        else:
            out = np.empty((n, n), dtype=np.float32)
            pout = out.ctypes.data
        _check(load().ept_build_blocks(self._h, px, X.shape[0], py, Y.shape[0], X.shape[1], on_dev, _stat(stat),
                                       _sigma(sigma), _prec(prec), pout, stream))
        return out


class PreparedBatch:
    """A batch of tests with its descriptors and output buffers built once."""

    def __init__(self, ctx: Context, tests, prec, want_stats: bool):
        self.ctx = ctx
        self.n = n = len(tests)
        self.prec = _prec(prec)
        self.descs = (_TestDesc * max(n, 1))()
        self.res = (_Result * max(n, 1))()
        self.keep, self.bufs = [], []
        self.on_dev, self.stream = 0, None
        for k, t in enumerate(tests):
            X, Y, px, py, dev, st = ctx._arrays(t["X"], t["Y"])
            if k == 0:
                self.on_dev, self.stream = dev, st
            elif self.on_dev != dev:
                raise TypeError("all tests of a batch must use the same memory space")
            B = int(t["B"])
            buf, pbuf = ctx._stats_buffer(X, B if want_stats else 0, dev)
            self.keep.append((X, Y))
            self.bufs.append(buf)
            self.descs[k] = _TestDesc(px, py, X.shape[0], Y.shape[0], X.shape[1], _stat(t.get("stat", "ed")),
                                      _sigma(t.get("sigma", 1.0)), B, int(t.get("seed", 0)), pbuf)

    def run(self):
        if self.n == 0:
            return []
        _check(load().ept_test_batch(self.ctx._h, self.descs, self.n, self.on_dev, self.prec, self.res, self.stream))
        return [_result(self.res[k], self.bufs[k]) for k in range(self.n)]
