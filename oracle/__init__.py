"""FP64 CPU oracle for the efficient permutation two-sample test (arXiv 2406.06488).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package.

The arithmetic lives in ``ept_oracle.c`` (plain C, IEEE double); this module only
compiles it with gcc and marshals numpy arrays.  Every function names the passage
of the paper it follows:

* Eq. 1 (energy distance V-statistic) and Eq. 2 (biased MMD^2), pairwise distances
  as in Algorithm 3 (Appendix A.1), Gaussian kernel exp(-||x-y||^2 / (2 sigma^2))
  or Laplacian kernel exp(-||x-y|| / sigma);
* the median-heuristic bandwidth (lower median of the pooled pairwise distances)
  -- ``median_pairs``;
* Algorithm 4 (standard permutation test: statistics recomputed from permuted
  raw rows) -- ``test_direct``;
* Algorithm 5 (pre-computed pooled matrix) -- ``test_pooled``;
* Algorithm 1 with Algorithm 2 (three blocks, twelve block assignments) --
  ``test_blocks``; Algorithm 2 alone -- ``alg2_indices``;
* the p-value of Section 3.1 -- ``pvalue``;
* the permutation stream (Philox4x32-10 + Knuth's Algorithm S, the library's
  reading of SampleWithoutReplacement) -- ``perm_select``;
* exhaustive enumeration of all relabelings -- ``exhaustive``;
* the statistic of one relabeling recomputed from permuted raw rows with threads
  over rows (Algorithm 4, for sampled checks at full size) -- ``stat_select``;
* the sum and trace of the pooled matrix and the closed-form mean of the
  permutation distribution (Section 3.1's null) -- ``pooled_moments``,
  ``permutation_mean``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ept_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libept_oracle.so")

STAT_ED = 0
STAT_MMD = 1
STAT_MMD_LAPLACE = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile ept_oracle.c with gcc (-O2, OpenMP, no fast-math).  Returns the path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_mutant(k: int) -> str:
    """Compile a copy with the test-only switch EO_MUTANT = k (one planted mistake)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    out = os.path.join(_OUT_DIR, "libept_oracle_mutant%d.so" % k)
    if os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
                    "-ffp-contract=off", "-DEO_MUTANT=%d" % k, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, out)
    return out


def use_library(path=None):
    """Point the wrappers at another build of ept_oracle.c (None = the oracle itself).
    Returns the previously loaded library handle."""
    global _lib
    prev = _lib
    _lib = None
    _load(path)
    return prev


def _load(path=None):
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        build()
        path = _LIB_PATH
    lib = ctypes.CDLL(path)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    f32p = ctypes.POINTER(ctypes.c_float)
    f64p = ctypes.POINTER(ctypes.c_double)
    i64 = ctypes.c_int64
    lib.eo_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.eo_philox4x32_10.restype = None
    lib.eo_perm_select.argtypes = [ctypes.c_uint64, i64, i64, i64, u8p]
    lib.eo_perm_select.restype = None
    lib.eo_perm_select_many.argtypes = [ctypes.c_uint64, i64, i64, i64, i64, u8p]
    lib.eo_perm_select_many.restype = None
    lib.eo_alg2_indices.argtypes = [i64, i64, i64p, i64p, i64p]
    lib.eo_alg2_indices.restype = ctypes.c_int
    lib.eo_block_matrix.argtypes = [f64p, i64, f64p, i64, i64, ctypes.c_int, ctypes.c_double, f64p]
    lib.eo_block_matrix.restype = None
    lib.eo_stat_direct.argtypes = [f64p, i64, f64p, i64, i64, ctypes.c_int, ctypes.c_double]
    lib.eo_stat_direct.restype = ctypes.c_double
    for name in ("eo_test_direct", "eo_test_pooled", "eo_test_blocks"):
        fn = getattr(lib, name)
        fn.argtypes = [f32p, i64, f32p, i64, i64, ctypes.c_int, ctypes.c_double, u8p, i64, f64p]
        fn.restype = ctypes.c_int
    lib.eo_pvalue.argtypes = [f64p, i64, ctypes.c_double, i64p]
    lib.eo_pvalue.restype = ctypes.c_double
    lib.eo_exhaustive.argtypes = [f32p, i64, f32p, i64, i64, ctypes.c_int, ctypes.c_double, i64,
                                  u8p, f64p]
    lib.eo_exhaustive.restype = i64
    lib.eo_stat_select_mt.argtypes = [f32p, i64, f32p, i64, i64, ctypes.c_int, ctypes.c_double, u8p]
    lib.eo_stat_select_mt.restype = ctypes.c_double
    lib.eo_pooled_moments.argtypes = [f32p, i64, f32p, i64, i64, ctypes.c_int, ctypes.c_double, f64p, f64p]
    lib.eo_pooled_moments.restype = None
    lib.eo_median_pairs.argtypes = [f32p, i64, f32p, i64, i64]
    lib.eo_median_pairs.restype = ctypes.c_double
    lib.eo_permutation_mean.argtypes = [ctypes.c_double, ctypes.c_double, i64, i64, ctypes.c_int]
    lib.eo_permutation_mean.restype = ctypes.c_double
    lib.eo_num_threads.argtypes = []
    lib.eo_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _stat_code(stat) -> int:
    if stat in (STAT_ED, "ed", "ED"):
        return STAT_ED
    if stat in (STAT_MMD, "mmd", "MMD"):
        return STAT_MMD
    if stat in (STAT_MMD_LAPLACE, "mmd_laplace"):
        return STAT_MMD_LAPLACE
    raise ValueError("stat must be 'ed', 'mmd' or 'mmd_laplace'")


def num_threads() -> int:
    return int(_load().eo_num_threads())


def philox4x32_10(counter, key) -> np.ndarray:
    """Philox4x32-10 block function (Salmon et al., SC'11): 4 counter words, 2 key words."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.eo_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def perm_select(seed: int, nx: int, ny: int, b0: int, count: int) -> np.ndarray:
    """Draws b0 .. b0+count-1 of the permutation stream as a bool array [count, n]
    (True = the pooled row goes to x*).  Draw 0 is the identity relabeling."""
    lib = _load()
    n = nx + ny
    out = np.zeros((count, n), dtype=np.uint8)
    lib.eo_perm_select_many(ctypes.c_uint64(seed), nx, ny, b0, count, _ptr(out, ctypes.c_uint8))
    return out.astype(bool)


def pack_masks(sel: np.ndarray) -> np.ndarray:
    """Pack a bool array [count, n] into uint32 words [count, ceil(n/32)]:
    pooled row t is bit (t % 32) of word t // 32.  (Layout conversion only.)"""
    sel = np.asarray(sel, dtype=bool)
    count, n = sel.shape
    nw = (n + 31) // 32
    padded = np.zeros((count, nw * 32), dtype=np.uint8)
    padded[:, :n] = sel
    by = np.packbits(padded, axis=1, bitorder="little")
    return np.ascontiguousarray(by).view("<u4").reshape(count, nw).astype(np.uint32)


def unpack_masks(words: np.ndarray, n: int) -> np.ndarray:
    words = np.ascontiguousarray(words, dtype="<u4")
    count = words.shape[0]
    by = words.view(np.uint8).reshape(count, -1)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :n].astype(bool)


def alg2_indices(nx: int, ny: int, idx_p1) -> dict:
    """Algorithm 2 from a given draw idx_p1 (1-based pooled indexes, length nx)."""
    lib = _load()
    p1 = np.ascontiguousarray(idx_p1, dtype=np.int64)
    if p1.shape != (nx,):
        raise ValueError("idx_p1 must have nx entries")
    out = np.zeros(2 * (nx + ny), dtype=np.int64)
    lens = np.zeros(8, dtype=np.int64)
    rc = lib.eo_alg2_indices(nx, ny, _ptr(p1, ctypes.c_int64), _ptr(out, ctypes.c_int64),
                             _ptr(lens, ctypes.c_int64))
    if rc != 0:
        raise ValueError("idx_p1 is not a set of nx distinct indexes in 1..n")
    names = ["i1", "i2", "i1s", "i2s", "j1", "j2", "j1s", "j2s"]
    res, off = {}, 0
    for name, ln in zip(names, lens):
        res[name] = out[off:off + ln].tolist()
        off += int(ln)
    return res


def block_matrix(a, b, stat="ed", sigma: float = 1.0) -> np.ndarray:
    """Algorithm 3: matrix of Euclidean distances (or Gaussian kernel values) between
    the rows of a and b, in FP64."""
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros((a.shape[0], b.shape[0]), dtype=np.float64)
    lib.eo_block_matrix(_ptr(a, ctypes.c_double), a.shape[0], _ptr(b, ctypes.c_double), b.shape[0],
                        a.shape[1], _stat_code(stat), float(sigma), _ptr(out, ctypes.c_double))
    return out


def stat_direct(x, y, stat="ed", sigma: float = 1.0) -> float:
    """Eq. 1 (ED) or Eq. 2 (biased MMD^2) recomputed from raw rows, in FP64."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib.eo_stat_direct(_ptr(x, ctypes.c_double), x.shape[0], _ptr(y, ctypes.c_double),
                                    y.shape[0], x.shape[1], _stat_code(stat), float(sigma)))


def _run_test(fn_name, X, Y, sel, stat, sigma):
    lib = _load()
    X = _f32(X)
    Y = _f32(Y)
    sel = np.ascontiguousarray(sel, dtype=np.uint8)
    nperm = sel.shape[0]
    if sel.shape[1] != X.shape[0] + Y.shape[0]:
        raise ValueError("relabelings must have nx + ny entries")
    stats = np.zeros(nperm, dtype=np.float64)
    rc = getattr(lib, fn_name)(_ptr(X, ctypes.c_float), X.shape[0], _ptr(Y, ctypes.c_float),
                               Y.shape[0], X.shape[1], _stat_code(stat), float(sigma),
                               _ptr(sel, ctypes.c_uint8), nperm, _ptr(stats, ctypes.c_double))
    if rc != 0:
        raise ValueError("%s: malformed relabeling or allocation failure" % fn_name)
    return stats


def test_direct(X, Y, sel, stat="ed", sigma: float = 1.0) -> np.ndarray:
    """Algorithm 4: statistic of each relabeling recomputed from permuted raw rows."""
    return _run_test("eo_test_direct", X, Y, sel, stat, sigma)


def test_pooled(X, Y, sel, stat="ed", sigma: float = 1.0) -> np.ndarray:
    """Algorithm 5: statistic of each relabeling sliced from the pooled matrix."""
    return _run_test("eo_test_pooled", X, Y, sel, stat, sigma)


def test_blocks(X, Y, sel, stat="ed", sigma: float = 1.0) -> np.ndarray:
    """Algorithm 1 + Algorithm 2: statistic of each relabeling by block swapping."""
    return _run_test("eo_test_blocks", X, Y, sel, stat, sigma)


def pvalue(stats, observed: float):
    """Section 3.1: (1 + #{stats >= observed}) / (1 + B); returns (p, n_ge)."""
    lib = _load()
    s = np.ascontiguousarray(stats, dtype=np.float64)
    nge = ctypes.c_int64(0)
    p = lib.eo_pvalue(_ptr(s, ctypes.c_double), s.shape[0], float(observed), ctypes.byref(nge))
    return float(p), int(nge.value)


def permutation_test(X, Y, B: int, seed: int, stat="ed", sigma: float = 1.0,
                     method: str = "direct"):
    """Whole test: observed statistic (draw 0), B permuted statistics (draws 1..B of
    the stream) and the p-value.  method: 'direct' (Algorithm 4), 'pooled'
    (Algorithm 5) or 'blocks' (Algorithm 1)."""
    nx, ny = X.shape[0], Y.shape[0]
    sel = perm_select(seed, nx, ny, 0, B + 1)
    fn = {"direct": test_direct, "pooled": test_pooled, "blocks": test_blocks}[method]
    all_stats = fn(X, Y, sel, stat, sigma)
    observed = float(all_stats[0])
    stats = all_stats[1:]
    p, nge = pvalue(stats, observed)
    return {"observed": observed, "stats": stats, "p_value": p, "n_ge": nge}


def stat_select(X, Y, sel, stat="ed", sigma: float = 1.0) -> float:
    """Eq. 1 / Eq. 2 of ONE relabeling (bool [n]) recomputed from the permuted raw
    rows (Algorithm 4), threads splitting the rows.  For sampled checks at full size."""
    lib = _load()
    X = _f32(X)
    Y = _f32(Y)
    s = np.ascontiguousarray(sel, dtype=np.uint8)
    if s.shape != (X.shape[0] + Y.shape[0],):
        raise ValueError("relabeling must have nx + ny entries")
    return float(lib.eo_stat_select_mt(_ptr(X, ctypes.c_float), X.shape[0], _ptr(Y, ctypes.c_float), Y.shape[0],
                                       X.shape[1], _stat_code(stat), float(sigma), _ptr(s, ctypes.c_uint8)))


def pooled_moments(X, Y, stat="ed", sigma: float = 1.0):
    """(S, trace) of the pooled matrix W of Algorithm 3 entries over all pooled pairs."""
    lib = _load()
    X = _f32(X)
    Y = _f32(Y)
    S = ctypes.c_double(0.0)
    tr = ctypes.c_double(0.0)
    lib.eo_pooled_moments(_ptr(X, ctypes.c_float), X.shape[0], _ptr(Y, ctypes.c_float), Y.shape[0], X.shape[1],
                          _stat_code(stat), float(sigma), ctypes.byref(S), ctypes.byref(tr))
    return float(S.value), float(tr.value)


def permutation_mean(S: float, trace: float, nx: int, ny: int, stat="ed") -> float:
    """Closed-form mean of the permutation distribution of Eq. 1 / Eq. 2 under a uniform
    random nx-subset of the pooled rows, from S = 1'W1 and tr W of the pooled matrix
    (E[s_i] = nx/n, E[s_i s_j] = nx(nx-1)/(n(n-1)); the statistic is linear in
    T = s'Ws and L = s'W1)."""
    return float(_load().eo_permutation_mean(float(S), float(trace), int(nx), int(ny), _stat_code(stat)))


def exhaustive(X, Y, stat="ed", sigma: float = 1.0, max_count: int = 1_000_000):
    """All C(n, nx) relabelings in lexicographic order: (sel [count, n], stats [count])."""
    lib = _load()
    X = _f32(X)
    Y = _f32(Y)
    nx, ny = X.shape[0], Y.shape[0]
    count = comb(nx + ny, nx)
    if count > max_count:
        raise ValueError("too many relabelings")
    sel = np.zeros((count, nx + ny), dtype=np.uint8)
    stats = np.zeros(count, dtype=np.float64)
    got = lib.eo_exhaustive(_ptr(X, ctypes.c_float), nx, _ptr(Y, ctypes.c_float), ny, X.shape[1],
                            _stat_code(stat), float(sigma), max_count, _ptr(sel, ctypes.c_uint8),
                            _ptr(stats, ctypes.c_double))
    if got != count:
        raise RuntimeError("exhaustive enumeration failed")
    return sel.astype(bool), stats


def median_pairs(X, Y) -> float:
    """Median-heuristic bandwidth: the lower median of the distances between distinct
    pooled rows (C, FP64)."""
    lib = _load()
    X, Y = _f32(X), _f32(Y)
    v = lib.eo_median_pairs(_ptr(X, ctypes.c_float), X.shape[0], _ptr(Y, ctypes.c_float), Y.shape[0], X.shape[1])
    if v < 0:
        raise ValueError("median of pairwise distances needs at least two rows")
    return float(v)
