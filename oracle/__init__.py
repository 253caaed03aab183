"""CPU oracle for grayscale lambda-thinning (TEST INFRASTRUCTURE ONLY).

Plain, slow, single-threaded restatement of the paper's definitions
(Sec. 2.1) and lowering loop (Sec. 2.2) in a fixed 2x2-parity subfield
schedule, compiled from ``thin_oracle.c`` with gcc and called through ctypes.
Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package; the CUDA library shares no code with it.

Every function here takes and returns numpy arrays of shape (H, W)
(row = y, column = x).  Images of any integer dtype are widened to int32.

Parity pins: the point test is pinned by exhaustive brute force (global
component counts on tiny images) and by the (8,4) identity T+ = T-- away from
interior and isolated points; the schedule by invariants (lowering only,
fixed point, per-level topology at lambda = 0) and by hand-worked cases.
Rule R2 (F^-(c) = min over c) is "parity unpinned": the paper never defines
F^-, and only constant-valued basins, where R1 and R2 agree, pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "thin_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

RULE_MAX = 0  # F^-(c) = max of F over c  (reading R1, default)
RULE_MIN = 1  # F^-(c) = min of F over c  (reading R2)
ADJ_8_4 = 0      # (n, nbar) = (8, 4): 8-adjacency for sections of F, 4 for their complements
ADJ_4_8 = 1      # (n, nbar) = (4, 8)
OP_THIN = 0      # lambda-thinning: lower lambda-destructible points
OP_SKELETON = 1  # lambda-skeleton (Sec. 2.2): lower lambda-deletable points that are not lambda-end


class OracleStats(ctypes.Structure):
    _fields_ = [
        ("phases", ctypes.c_int64),
        ("rounds", ctypes.c_int64),
        ("lowered", ctypes.c_int64),
        ("last_change_phase", ctypes.c_int64),
        ("end_phase", ctypes.c_int64),
        ("converged", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile thin_oracle.c into liboracle.so (gcc, -O2).  Returns the path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".%d.tmp" % os.getpid()
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_mask_numbers.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.oracle_tplusplus.argtypes = [ctypes.c_uint]
    lib.oracle_lambda_destructible.argtypes = [i32p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int, i32p]
    lib.oracle_lambda_skeleton_point.argtypes = lib.oracle_lambda_destructible.argtypes
    lib.oracle_mask_numbers_adj.argtypes = [ctypes.c_int] + lib.oracle_mask_numbers.argtypes
    lib.oracle_lowerable.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int,
                                     i32p]
    lib.oracle_thin.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32,
                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                ctypes.POINTER(OracleStats)]
    lib.oracle_thin_queue.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_thin_queue.restype = ctypes.c_int64
    lib.oracle_thin_minvalue.argtypes = lib.oracle_thin_queue.argtypes
    lib.oracle_thin_minvalue.restype = ctypes.c_int64
    lib.oracle_count_lambda_destructible.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                                     ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_count_lambda_destructible.restype = ctypes.c_int64
    lib.oracle_count_section_components.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                                     ctypes.c_int32, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_int]
    lib.oracle_count_section_components.restype = ctypes.c_int64
    lib.oracle_global_destructible.argtypes = [i32p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                               ctypes.c_int, ctypes.c_int]
    lib.oracle_global_destructible_adj.argtypes = [ctypes.c_int] + lib.oracle_global_destructible.argtypes
    _lib = lib
    return lib


def _i32(img) -> np.ndarray:
    """A fresh C-contiguous int32 copy: the C routines work in place and must
    never touch the caller's array."""
    a = np.array(np.asarray(img), dtype=np.int32, order="C", copy=True)
    if a.ndim != 2:
        raise ValueError("image must be 2-D (H, W)")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def mask_numbers(lower_mask: int, adj: int = ADJ_8_4):
    """(T+, T--, labels) for a point whose strictly lower neighbours form
    ``lower_mask`` (ring order E, NE, N, NW, W, SW, S, SE = bits 0..7)."""
    lib = _load()
    tp, tm = ctypes.c_int(), ctypes.c_int()
    lab = (ctypes.c_int * 8)()
    lib.oracle_mask_numbers_adj(int(adj), lower_mask, ctypes.byref(tp), ctypes.byref(tm), lab)
    return tp.value, tm.value, list(lab)


def tplusplus(greater_mask: int) -> int:
    return _load().oracle_tplusplus(greater_mask)


def lambda_destructible(nb, fx: int, lam: int, rule: int = RULE_MAX):
    """(is_lambda_destructible, alpha^-) for value fx with ring-ordered neighbours nb."""
    lib = _load()
    arr = (ctypes.c_int32 * 8)(*[int(v) for v in nb])
    alpha = ctypes.c_int32(int(fx))
    r = lib.oracle_lambda_destructible(arr, int(fx), int(lam), int(rule), ctypes.byref(alpha))
    return bool(r), int(alpha.value)


def lambda_skeleton_point(nb, fx: int, lam: int, rule: int = RULE_MAX):
    """(lowerable by the lambda-skeleton, alpha^-) for value fx with ring-ordered neighbours nb."""
    lib = _load()
    arr = (ctypes.c_int32 * 8)(*[int(v) for v in nb])
    alpha = ctypes.c_int32(int(fx))
    r = lib.oracle_lambda_skeleton_point(arr, int(fx), int(lam), int(rule), ctypes.byref(alpha))
    return bool(r), int(alpha.value)


def lowerable(nb, fx: int, lam: int, rule: int = RULE_MAX, op: int = OP_THIN, adj: int = ADJ_8_4):
    """(the test of op under adj accepts the point, alpha^-) for value fx with ring-ordered neighbours nb."""
    lib = _load()
    arr = (ctypes.c_int32 * 8)(*[int(v) for v in nb])
    alpha = ctypes.c_int32(int(fx))
    r = lib.oracle_lowerable(int(op), int(adj), arr, int(fx), int(lam), int(rule), ctypes.byref(alpha))
    return bool(r), int(alpha.value)


def thin(img, lam: int, rule: int = RULE_MAX, start_phase: int = 0, max_phases: int = -1, op: int = OP_THIN,
         adj: int = ADJ_8_4):
    """Subfield-schedule lambda-thinning (op = OP_THIN) or lambda-skeleton
    (op = OP_SKELETON) under the adjacency pair ``adj``.  Returns (result,
    stats dict); the result keeps the input's dtype."""
    a = _i32(img)
    h, w = a.shape
    st = OracleStats()
    rc = _load().oracle_thin(_ptr(a), w, h, w, int(lam), int(rule), int(op), int(adj), int(start_phase),
                             int(max_phases), ctypes.byref(st))
    d = st.as_dict()
    d["capped"] = bool(rc)
    return a.astype(np.asarray(img).dtype), d


def thin_queue(img, lam: int, rule: int = RULE_MAX, op: int = OP_THIN, adj: int = ADJ_8_4):
    """FIFO-order sequential thinning (invariants-only cross-check).  Returns (result, lowered)."""
    a = _i32(img)
    h, w = a.shape
    n = _load().oracle_thin_queue(_ptr(a), w, h, w, int(lam), int(rule), int(op), int(adj))
    if n < 0:
        raise MemoryError("oracle_thin_queue")
    return a.astype(np.asarray(img).dtype), int(n)


def thin_minvalue(img, lam: int, rule: int = RULE_MAX, op: int = OP_THIN, adj: int = ADJ_8_4):
    """Minimal-value-first sequential thinning (Sec. 2.2 selection).  Returns (result, lowered)."""
    a = _i32(img)
    h, w = a.shape
    n = _load().oracle_thin_minvalue(_ptr(a), w, h, w, int(lam), int(rule), int(op), int(adj))
    if n < 0:
        raise MemoryError("oracle_thin_minvalue")
    return a.astype(np.asarray(img).dtype), int(n)


def count_lambda_destructible(img, lam: int, rule: int = RULE_MAX, op: int = OP_THIN, adj: int = ADJ_8_4) -> int:
    """Interior points the test of ``op`` accepts (0 at a fixed point)."""
    a = _i32(img)
    h, w = a.shape
    return int(_load().oracle_count_lambda_destructible(_ptr(a), w, h, w, int(lam), int(rule), int(op), int(adj)))


def count_section_components(img, k: int, n: int, complement: bool = False, flip=None) -> int:
    """Components of {F >= k} (n-adjacency) or of {F < k}; ``flip`` = (x, y) toggles one point."""
    a = _i32(img)
    h, w = a.shape
    fx, fy = flip if flip is not None else (-1, -1)
    r = _load().oracle_count_section_components(_ptr(a), w, h, w, int(k), int(n), int(bool(complement)),
                                                int(fx), int(fy))
    if r < 0:
        raise MemoryError("oracle_count_section_components")
    return int(r)


def global_destructible(img, x: int, y: int, adj: int = ADJ_8_4) -> bool:
    a = _i32(img)
    h, w = a.shape
    r = _load().oracle_global_destructible_adj(int(adj), _ptr(a), w, h, w, int(x), int(y))
    if r < 0:
        raise MemoryError("oracle_global_destructible")
    return bool(r)


def level_topology(img, levels=None, adj: int = ADJ_8_4):
    """Per-level topology signature: for each k, (#n-components of F_k,
    #nbar-components of its complement), (n, nbar) the pair ``adj``.
    ``levels`` defaults to every value present in the image plus one above
    the maximum."""
    a = _i32(img)
    n, nbar = (4, 8) if adj == ADJ_4_8 else (8, 4)
    if levels is None:
        vals = np.unique(a)
        levels = list(vals) + [int(vals.max()) + 1]
    return {int(k): (count_section_components(a, k, n, False), count_section_components(a, k, nbar, True))
            for k in levels}
