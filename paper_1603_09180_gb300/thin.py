"""Python binding of libthin.so (ctypes).  Argument marshalling only.

Every step of lambda-thinning runs in the library's CUDA kernels; PyTorch
supplies device memory and the current stream.  There is no CPU fallback: if
the library is missing or fails to load, these functions raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthin.so")

THIN_OK = 0
THIN_ERR_ARG = -1
THIN_ERR_UNSUPPORTED = -2
THIN_ERR_OOM = -3
THIN_ERR_NOT_CONVERGED = -4
THIN_ERR_TIMEOUT = -5
THIN_ERR_CUDA = -6
THIN_EAGAIN = -7
THIN_ERR_TOO_LARGE = -8
ERRORS = {THIN_ERR_ARG: "bad argument", THIN_ERR_UNSUPPORTED: "unsupported", THIN_ERR_OOM: "out of memory",
          THIN_ERR_NOT_CONVERGED: "not converged", THIN_ERR_TIMEOUT: "device wait timed out",
          THIN_ERR_CUDA: "CUDA error", THIN_EAGAIN: "over budget, try again",
          THIN_ERR_TOO_LARGE: "image too large for the fixed scratch"}

U8, U16 = 0, 1
ADJ_8_4, ADJ_4_8 = 0, 1
RULE_MAX, RULE_MIN = 0, 1
OP_THINNING, OP_SKELETON = 0, 1
KERNEL_AUTO, KERNEL_NAIVE, KERNEL_TILED, KERNEL_RESIDENT = 0, 1, 2, 3


class ThinError(RuntimeError):
    def __init__(self, code, what=""):
        super().__init__("%s: %s (%d)" % (what, ERRORS.get(code, "error"), code))
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_int32), ("kernel", ctypes.c_int32), ("tile_w", ctypes.c_int32),
                ("tile_h", ctypes.c_int32), ("halo", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("start_phase", ctypes.c_int64), ("max_phases", ctypes.c_int64), ("op", ctypes.c_int32),
                ("reserved2", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("converged", ctypes.c_int32), ("phases", ctypes.c_int64),
                ("lowered", ctypes.c_int64), ("last_change_phase", ctypes.c_int64), ("end_phase", ctypes.c_int64),
                ("tiles_visited", ctypes.c_int64), ("steps", ctypes.c_int64), ("tested", ctypes.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Job(ctypes.Structure):
    _fields_ = [("img_dev", ctypes.c_void_p), ("w", ctypes.c_int32), ("h", ctypes.c_int32),
                ("pitch", ctypes.c_size_t), ("dtype", ctypes.c_int32), ("lam", ctypes.c_uint32)]


EXPORTS = ["thin_default_options", "thin_run", "thin_batch", "thin_point_table", "thin_version",
           "thin_serve_create", "thin_serve_submit", "thin_serve_poll", "thin_serve_wait_any",
           "thin_serve_destroy", "thin_run_noalloc", "thin_plan_create", "thin_plan_launch", "thin_plan_stats",
           "thin_plan_destroy", "thin_autotune", "thin_point_table_adj", "thin_plan_tiling"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libthin.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libthin.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, u32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t
    lib.thin_default_options.argtypes = [ctypes.POINTER(Options)]
    lib.thin_default_options.restype = None
    lib.thin_run.argtypes = [vp, i32, i32, sz, i32, u32, i32, vp, ctypes.POINTER(Options), ctypes.POINTER(Stats)]
    lib.thin_run.restype = i32
    lib.thin_batch.argtypes = [ctypes.POINTER(Job), i32, i32, vp, ctypes.POINTER(Options), ctypes.POINTER(Stats)]
    lib.thin_batch.restype = i32
    lib.thin_point_table.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
    lib.thin_point_table.restype = None
    lib.thin_point_table_adj.argtypes = [i32, ctypes.POINTER(ctypes.c_uint32)]
    lib.thin_point_table_adj.restype = None
    lib.thin_version.restype = ctypes.c_char_p
    lib.thin_serve_create.argtypes = [sz, i32, i32, ctypes.POINTER(vp)]
    lib.thin_serve_create.restype = i32
    lib.thin_serve_submit.argtypes = [vp, vp, i32, i32, sz, i32, u32, ctypes.POINTER(ctypes.c_uint64)]
    lib.thin_serve_submit.restype = i32
    lib.thin_serve_poll.argtypes = [vp, ctypes.c_uint64, vp, sz, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(Stats)]
    lib.thin_serve_poll.restype = i32
    lib.thin_serve_wait_any.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.thin_serve_wait_any.restype = i32
    lib.thin_serve_destroy.argtypes = [vp]
    lib.thin_serve_destroy.restype = i32
    lib.thin_plan_create.argtypes = [ctypes.POINTER(Job), i32, i32, ctypes.POINTER(Options), ctypes.POINTER(vp)]
    lib.thin_plan_create.restype = i32
    lib.thin_plan_launch.argtypes = [vp, vp]
    lib.thin_plan_launch.restype = i32
    lib.thin_plan_stats.argtypes = [vp, vp, ctypes.POINTER(Stats)]
    lib.thin_plan_stats.restype = i32
    lib.thin_plan_tiling.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]
    lib.thin_plan_tiling.restype = i32
    lib.thin_plan_destroy.argtypes = [vp]
    lib.thin_plan_destroy.restype = i32
    lib.thin_autotune.argtypes = [vp, i32, i32, sz, i32, u32, vp, ctypes.c_int64, ctypes.POINTER(Options),
                                  ctypes.POINTER(ctypes.c_float)]
    lib.thin_autotune.restype = i32
    lib.thin_run_noalloc.argtypes = lib.thin_run.argtypes
    lib.thin_run_noalloc.restype = i32
    _lib = lib
    return lib


def options(rule=RULE_MAX, kernel=KERNEL_AUTO, tile=None, halo=0, start_phase=0, max_phases=-1, debug=0,
            op=OP_THINNING):
    o = Options()
    load().thin_default_options(ctypes.byref(o))
    o.rule = {"max": RULE_MAX, "min": RULE_MIN}.get(rule, rule)
    o.kernel = {"auto": KERNEL_AUTO, "naive": KERNEL_NAIVE, "tiled": KERNEL_TILED,
                "resident": KERNEL_RESIDENT}.get(kernel, kernel)
    if tile is not None:
        o.tile_w, o.tile_h = (tile, tile) if isinstance(tile, int) else tile
    o.halo = halo or 0
    o.start_phase = start_phase
    o.max_phases = max_phases
    o.reserved = debug
    o.op = {"thinning": OP_THINNING, "skeleton": OP_SKELETON}.get(op, op)
    return o


def _adj_code(adj):
    return {"8,4": ADJ_8_4, "4,8": ADJ_4_8, (8, 4): ADJ_8_4, (4, 8): ADJ_4_8}.get(adj, adj)


def point_table(adj=ADJ_8_4):
    out = (ctypes.c_uint32 * 256)()
    load().thin_point_table_adj(_adj_code(adj), out)
    return list(out)


def version() -> str:
    return load().thin_version().decode()


def _dtype_code(t):
    import torch
    if t.dtype == torch.uint8:
        return U8
    if t.dtype == torch.uint16:
        return U16
    raise TypeError("image must be torch.uint8 or torch.uint16")


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_image(img):
    if not img.is_cuda:
        raise ValueError("image must be a CUDA tensor")
    if img.dim() != 2 or (img.numel() and img.stride(1) != 1):
        raise ValueError("image must be 2-D with unit column stride")


def run(img, lam: int, *, rule="max", kernel="auto", tile=None, halo=0, start_phase=0, max_phases=-1,
        stream=None, stats=True, check=True, debug=0, op="thinning", adj=ADJ_8_4):
    """Lambda-thin a CUDA tensor (H x W, uint8/uint16, unit column stride) in place.

    Returns the stats dict (stats=True waits for the stream), else None."""
    _check_image(img)
    h, w = img.shape
    es = img.element_size()
    pitch = img.stride(0) * es if h > 1 else w * es
    st = Stats()
    o = options(rule, kernel, tile, halo, start_phase, max_phases, debug, op)
    rc = load().thin_run(ctypes.c_void_p(img.data_ptr() if img.numel() else 0), w, h, pitch, _dtype_code(img),
                         int(lam), _adj_code(adj), _stream_ptr(stream), ctypes.byref(o),
                         ctypes.byref(st) if stats else None)
    if check and rc not in (THIN_OK, THIN_ERR_NOT_CONVERGED):
        raise ThinError(rc, "thin_run")
    if stats:
        d = st.as_dict()
        d["rc"] = rc
        return d
    return rc


def autotune(img, lam: int, *, trial_phases: int = -1, rule="max", op="thinning", stream=None):
    """Best (tile, halo) of the tiled engine for this image (timed on a scratch copy).

    Returns ({"tile": (tw, th), "halo": h}, best_ms)."""
    _check_image(img)
    h, w = img.shape
    es = img.element_size()
    pitch = img.stride(0) * es if h > 1 else w * es
    o = options(rule, KERNEL_TILED, op=op)
    ms = ctypes.c_float()
    rc = load().thin_autotune(ctypes.c_void_p(img.data_ptr() if img.numel() else 0), w, h, pitch, _dtype_code(img),
                              int(lam), _stream_ptr(stream), int(trial_phases), ctypes.byref(o), ctypes.byref(ms))
    if rc != THIN_OK:
        raise ThinError(rc, "thin_autotune")
    return {"tile": (o.tile_w, o.tile_h), "halo": o.halo}, ms.value


def run_raw(ptr: int, w: int, h: int, pitch: int, dtype: int, lam: int, adj: int = ADJ_8_4, stream_ptr: int = 0,
            opts: Options | None = None, want_stats: bool = True):
    """Direct C-ABI call with plain integers (device pointer as int).  Returns (rc, stats dict)."""
    st = Stats()
    rc = load().thin_run(ctypes.c_void_p(ptr), w, h, pitch, dtype, lam, adj, ctypes.c_void_p(stream_ptr),
                         ctypes.byref(opts) if opts is not None else None, ctypes.byref(st) if want_stats else None)
    return rc, st.as_dict()


def batch(imgs, lams, *, rule="max", kernel="auto", tile=None, halo=0, start_phase=0, max_phases=-1, stream=None,
          stats=True, check=True, debug=0, op="thinning", adj=ADJ_8_4):
    """Lambda-thin a list of CUDA tensors (each H x W, uint8/uint16) in place, in one device-driven run."""
    n = len(imgs)
    if len(lams) != n:
        raise ValueError("one lambda per image")
    jobs = (Job * max(n, 1))()
    for k, (t, lam) in enumerate(zip(imgs, lams)):
        if not t.is_cuda or t.dim() != 2 or (t.numel() and t.stride(1) != 1):
            raise ValueError("image %d must be a 2-D CUDA tensor with unit column stride" % k)
        h, w = t.shape
        es = t.element_size()
        jobs[k].img_dev = t.data_ptr() if t.numel() else None
        jobs[k].w, jobs[k].h = w, h
        jobs[k].pitch = t.stride(0) * es if h > 1 else w * es
        jobs[k].dtype = _dtype_code(t)
        jobs[k].lam = int(lam)
    sts = (Stats * max(n, 1))()
    o = options(rule, kernel, tile, halo, start_phase, max_phases, debug, op)
    rc = load().thin_batch(jobs, n, _adj_code(adj), _stream_ptr(stream), ctypes.byref(o), sts if stats else None)
    if check and rc not in (THIN_OK, THIN_ERR_NOT_CONVERGED):
        raise ThinError(rc, "thin_batch")
    if stats:
        return [sts[k].as_dict() for k in range(n)], rc
    return None, rc


class BatchPlan:
    """A batch whose job records are marshalled once; ``run`` calls thin_batch.

    The tensors must stay alive (and at the same addresses) while the plan is used."""

    def __init__(self, imgs, lams, *, rule="max", kernel="auto", tile=None, halo=0, start_phase=0, max_phases=-1,
                 debug=0, op="thinning", adj=ADJ_8_4):
        self._fill(imgs, lams, rule, kernel, tile, halo, start_phase, max_phases, debug, op)
        self.adj = _adj_code(adj)

    def _fill(self, imgs, lams, rule, kernel, tile, halo, start_phase, max_phases, debug, op):
        self.n = len(imgs)
        if len(lams) != self.n:
            raise ValueError("one lambda per image")
        self.jobs = (Job * max(self.n, 1))()
        for k, (t, lam) in enumerate(zip(imgs, lams)):
            if not t.is_cuda or t.dim() != 2 or (t.numel() and t.stride(1) != 1):
                raise ValueError("image %d must be a 2-D CUDA tensor with unit column stride" % k)
            h, w = t.shape
            es = t.element_size()
            self.jobs[k].img_dev = t.data_ptr() if t.numel() else None
            self.jobs[k].w, self.jobs[k].h = w, h
            self.jobs[k].pitch = t.stride(0) * es if h > 1 else w * es
            self.jobs[k].dtype = _dtype_code(t)
            self.jobs[k].lam = int(lam)
        self.opts = options(rule, kernel, tile, halo, start_phase, max_phases, debug, op)
        self.stats = (Stats * max(self.n, 1))()

    def run(self, stream=None, stats=False, check=True):
        rc = load().thin_batch(self.jobs, self.n, self.adj, _stream_ptr(stream), ctypes.byref(self.opts),
                               self.stats if stats else None)
        if check and rc not in (THIN_OK, THIN_ERR_NOT_CONVERGED):
            raise ThinError(rc, "thin_batch")
        if stats:
            return [self.stats[k].as_dict() for k in range(self.n)], rc
        return None, rc


class Server:
    """A serving instance (thin_serve_*): host numpy images in, host images out.

    submit returns a ticket, or raises ThinError (THIN_EAGAIN when the
    admission queue is full); poll and wait_any collect finished requests."""

    def __init__(self, budget_bytes: int, max_slots: int = 256, queue_cap: int = 1024):
        self._lib = load()
        self._h = ctypes.c_void_p()
        rc = self._lib.thin_serve_create(int(budget_bytes), int(max_slots), int(queue_cap), ctypes.byref(self._h))
        if rc != THIN_OK:
            raise ThinError(rc, "thin_serve_create")
        self.shapes = {}

    def submit(self, img: np.ndarray, lam: int) -> int:
        if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16) or (img.size and img.strides[1] != img.itemsize):
            raise ValueError("image must be a 2-D uint8/uint16 array with unit column stride")
        h, w = img.shape
        t = ctypes.c_uint64()
        rc = self._lib.thin_serve_submit(self._h, ctypes.c_void_p(img.ctypes.data if img.size else 0), w, h,
                                         img.strides[0] if h > 1 else w * img.itemsize,
                                         U16 if img.dtype == np.uint16 else U8, int(lam), ctypes.byref(t))
        if rc != THIN_OK:
            raise ThinError(rc, "thin_serve_submit")
        self.shapes[t.value] = (h, w, img.dtype)
        return t.value

    def poll(self, ticket: int):
        """(done, result array or None, stats dict or None, rc)."""
        h, w, dt = self.shapes[ticket]
        out = np.empty((h, w), dt)
        done = ctypes.c_int()
        st = Stats()
        rc = self._lib.thin_serve_poll(self._h, ctypes.c_uint64(ticket), ctypes.c_void_p(out.ctypes.data if out.size else 0),
                                       w * out.itemsize, ctypes.byref(done), ctypes.byref(st))
        if not done.value:
            if rc != THIN_OK:
                raise ThinError(rc, "thin_serve_poll")
            return False, None, None, rc
        del self.shapes[ticket]
        return True, out, st.as_dict(), rc

    def wait_any(self, timeout_ms: int = 1000):
        """Ticket of a finished, unpolled request, or None on timeout."""
        t = ctypes.c_uint64()
        rc = self._lib.thin_serve_wait_any(self._h, int(timeout_ms), ctypes.byref(t))
        if rc == THIN_EAGAIN:
            return None
        if rc != THIN_OK:
            raise ThinError(rc, "thin_serve_wait_any")
        return t.value

    def close(self):
        if self._h:
            self._lib.thin_serve_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class GraphPlan(BatchPlan):
    """thin_plan_*: the batch prepared once and replayed as one CUDA graph per ``run``."""

    def __init__(self, imgs, lams, *, rule="max", kernel="auto", tile=None, halo=0, start_phase=0, max_phases=-1,
                 debug=0, op="thinning", adj=ADJ_8_4):
        self._fill(imgs, lams, rule, kernel, tile, halo, start_phase, max_phases, debug, op)
        self.adj = _adj_code(adj)
        self._h = ctypes.c_void_p()
        rc = load().thin_plan_create(self.jobs, self.n, self.adj, ctypes.byref(self.opts), ctypes.byref(self._h))
        if rc != THIN_OK:
            raise ThinError(rc, "thin_plan_create")

    def run(self, stream=None, stats=False, check=True):
        lib = load()
        rc = lib.thin_plan_launch(self._h, _stream_ptr(stream))
        if rc == THIN_OK and stats:
            rc = lib.thin_plan_stats(self._h, _stream_ptr(stream), self.stats)
        if check and rc not in (THIN_OK, THIN_ERR_NOT_CONVERGED):
            raise ThinError(rc, "thin_plan")
        if stats:
            return [self.stats[k].as_dict() for k in range(self.n)], rc
        return None, rc

    def tiling(self):
        """(tile_w, tile_h, halo) the plan autotuned for its tiled images, zeros if none."""
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        rc = load().thin_plan_tiling(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        if rc != THIN_OK:
            raise ThinError(rc, "thin_plan_tiling")
        return a.value, b.value, c.value

    def close(self):
        if self._h:
            load().thin_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
