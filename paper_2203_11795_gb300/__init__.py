"""Python binding of libfftu, the GB300 cyclic multidimensional FFT.

Argument marshalling only: every step of the transform runs in the CUDA
kernels of ``libfftu.so`` (built in-tree by ``_build.py``).  The functions
below carry the C ABI's names (``include/fftu.h``) and take raw device
pointers; ``Plan`` is a small convenience wrapper over torch tensors.  PyTorch
supplies device memory and streams only.

There is no CPU fallback: the first call into the library raises ImportError
if ``libfftu.so`` has not been built, and every call raises ``FFTUError`` on a
non-OK status.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfftu.so")

FFTU_MAX_DIMS = 8
FFTU_C64, FFTU_C128 = 1, 2
FFTU_FORWARD, FFTU_INVERSE = -1, 1
FFTU_PHASE_A, FFTU_PHASE_B, FFTU_PHASE_ALL = 1, 2, 3
FFTU_SCHED_AUTO, FFTU_SCHED_GENERIC, FFTU_SCHED_FUSED, FFTU_SCHED_GENERIC_A = 0, 1, 2, 3
FFTU_PREC_NATIVE, FFTU_PREC_SPLIT_BF16, FFTU_PREC_SPLIT_FP16 = 0, 1, 2
FFTU_LAYOUT_NATURAL, FFTU_LAYOUT_CYCLIC = 0, 1
FFTU_WORKSPACE_PLAN, FFTU_WORKSPACE_CALLER = 0, 1
STATUS_NAMES = {0: "FFTU_OK", 1: "FFTU_ERR_ARG", 2: "FFTU_ERR_DIVISIBILITY", 3: "FFTU_ERR_UNSUPPORTED",
                4: "FFTU_ERR_NOMEM", 5: "FFTU_ERR_CUDA", 6: "FFTU_ERR_TIMEOUT", 7: "FFTU_ERR_INTERNAL"}

# Every entry point the header declares (checked by the test suite).
EXPORTS = ("fftu_plan", "fftu_plan_ex", "fftu_exec", "fftu_exec_phase", "fftu_exec_pointwise", "fftu_destroy",
           "fftu_plan_info",
           "fftu_check_device_status", "fftu_exec_noalloc", "fftu_noalloc_check_status",
           "fftu_noalloc_selftest_timeout", "fftu_batch_create", "fftu_batch_exec",
           "fftu_batch_check_status", "fftu_batch_destroy", "fftu_wisdom_export", "fftu_wisdom_import",
           "fftu_wisdom_forget", "fftu_workspace_size", "fftu_set_workspace", "fftu_selftest_bounded_wait",
           "fftu_measure_fp64_rate",
           "fftu_status_string",
           "fftu_last_error", "fftu_version",
           # include/fftu_serve.h
           "fftu_server_create", "fftu_server_submit", "fftu_server_warm", "fftu_server_poll", "fftu_server_drain",
           "fftu_server_stats_get", "fftu_server_destroy")


class FFTUError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        name = STATUS_NAMES.get(status, f"status {status}")
        super().__init__(f"{where}: {name}" + (f" ({detail})" if detail else ""))


class fftu_options(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("tune", ctypes.c_int), ("precision", ctypes.c_int),
                ("layout", ctypes.c_int), ("workspace_mode", ctypes.c_int), ("tile", ctypes.c_int),
                ("radix", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


class fftu_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64 * FFTU_MAX_DIMS), ("p", ctypes.c_int64 * FFTU_MAX_DIMS),
                ("dtype", ctypes.c_int), ("dir", ctypes.c_int), ("schedule", ctypes.c_int),
                ("launches_phase_a", ctypes.c_int), ("launches_phase_b", ctypes.c_int),
                ("N", ctypes.c_int64), ("alg_bytes", ctypes.c_int64), ("table_bytes", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("tuned", ctypes.c_int), ("precision", ctypes.c_int),
                ("workspace_need", ctypes.c_int64), ("layout", ctypes.c_int), ("workspace_mode", ctypes.c_int),
                ("tile", ctypes.c_int), ("radix", ctypes.c_int)]


class fftu_server_config(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("max_batch", ctypes.c_int), ("streams", ctypes.c_int),
                ("large_elems", ctypes.c_int64), ("use_graphs", ctypes.c_int), ("max_inflight", ctypes.c_int),
                ("copy_piece_mib", ctypes.c_int), ("max_inflight_solo", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


class fftu_request(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64 * FFTU_MAX_DIMS), ("dtype", ctypes.c_int),
                ("dir", ctypes.c_int), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("tag", ctypes.c_uint64)]


class fftu_completion(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("status", ctypes.c_int), ("batch_size", ctypes.c_int),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double), ("done_s", ctypes.c_double)]


class fftu_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "submitted", "completed", "rejected", "batches", "graph_replays", "graph_builds", "direct_launches",
        "kernel_launches", "instances", "plans", "bytes_in_use", "peak_bytes", "budget_bytes", "evictions",
        "bytes_h2d", "bytes_d2h", "instance_creations")] + [
        ("creation_s", ctypes.c_double), ("max_launch_s", ctypes.c_double), ("max_loop_gap_s", ctypes.c_double),
        ("last_cuda_error", ctypes.c_int), ("last_error_site", ctypes.c_int)]


def _load_library() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfftu.so is not built ({LIB_PATH}); run __graft_entry__.build() or "
                          "python -m paper_2203_11795_gb300._build")
    lib = ctypes.CDLL(LIB_PATH)
    i64p = ctypes.POINTER(ctypes.c_int64)
    vp = ctypes.c_void_p
    h = ctypes.c_void_p
    lib.fftu_plan.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(h)]
    lib.fftu_plan_ex.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(fftu_options), ctypes.POINTER(h)]
    lib.fftu_exec.argtypes = [h, vp, vp, vp]
    lib.fftu_exec_phase.argtypes = [h, ctypes.c_int, vp, vp, vp]
    lib.fftu_exec_pointwise.argtypes = [h, h, vp, vp, vp, vp, vp]
    lib.fftu_destroy.argtypes = [h]
    lib.fftu_plan_info.argtypes = [h, ctypes.POINTER(fftu_info)]
    lib.fftu_check_device_status.argtypes = [h]
    lib.fftu_exec_noalloc.argtypes = [ctypes.c_int, i64p, i64p, ctypes.c_int, ctypes.c_int, vp, vp, vp]
    lib.fftu_noalloc_check_status.argtypes = [vp]
    lib.fftu_noalloc_selftest_timeout.argtypes = [ctypes.c_double, vp]
    lib.fftu_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(h), ctypes.POINTER(h)]
    lib.fftu_batch_exec.argtypes = [h, ctypes.POINTER(vp), ctypes.POINTER(vp), vp]
    lib.fftu_batch_check_status.argtypes = [h]
    lib.fftu_batch_destroy.argtypes = [h]
    lib.fftu_wisdom_export.argtypes = [ctypes.c_char_p]
    lib.fftu_wisdom_import.argtypes = [ctypes.c_char_p]
    lib.fftu_wisdom_forget.argtypes = []
    lib.fftu_workspace_size.argtypes = [h, ctypes.POINTER(ctypes.c_size_t)]
    lib.fftu_set_workspace.argtypes = [h, vp, ctypes.c_size_t]
    lib.fftu_selftest_bounded_wait.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    lib.fftu_measure_fp64_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.fftu_server_create.argtypes = [ctypes.POINTER(fftu_server_config), ctypes.POINTER(h)]
    lib.fftu_server_submit.argtypes = [h, ctypes.POINTER(fftu_request)]
    lib.fftu_server_poll.argtypes = [h, ctypes.POINTER(fftu_completion), ctypes.c_int]
    lib.fftu_server_drain.argtypes = [h, ctypes.c_double]
    lib.fftu_server_warm.argtypes = [h, ctypes.POINTER(fftu_request), ctypes.c_int, ctypes.c_double]
    lib.fftu_server_stats_get.argtypes = [h, ctypes.POINTER(fftu_server_stats)]
    lib.fftu_server_destroy.argtypes = [h]
    lib.fftu_status_string.argtypes = [ctypes.c_int]
    lib.fftu_status_string.restype = ctypes.c_char_p
    lib.fftu_last_error.restype = ctypes.c_char_p
    lib.fftu_version.restype = ctypes.c_char_p
    for name in ("fftu_plan", "fftu_plan_ex", "fftu_exec", "fftu_exec_phase", "fftu_exec_pointwise", "fftu_destroy",
                 "fftu_plan_info", "fftu_check_device_status", "fftu_exec_noalloc", "fftu_noalloc_check_status",
                 "fftu_noalloc_selftest_timeout", "fftu_batch_create",
                 "fftu_batch_exec", "fftu_batch_check_status", "fftu_batch_destroy", "fftu_wisdom_export",
                 "fftu_wisdom_import", "fftu_wisdom_forget", "fftu_workspace_size", "fftu_set_workspace",
                 "fftu_selftest_bounded_wait", "fftu_measure_fp64_rate",
                 "fftu_server_create", "fftu_server_submit", "fftu_server_warm",
                 "fftu_server_poll", "fftu_server_drain", "fftu_server_stats_get", "fftu_server_destroy"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


class _LazyLib:
    """Loads libfftu.so on first attribute access (so the build module can be
    imported before the library exists); raises ImportError if it is missing."""

    def __init__(self):
        self._cdll = None

    def __getattr__(self, name):
        if self._cdll is None:
            self._cdll = _load_library()
        return getattr(self._cdll, name)


_lib = _LazyLib()


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise FFTUError(rc, where, fftu_last_error())


def _i64(vals):
    if vals is None:
        return None
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


# ---- C ABI, same names -----------------------------------------------------------------

def fftu_plan(d: int, n, p, dtype: int, direction: int) -> int:
    h = ctypes.c_void_p()
    _check(_lib.fftu_plan(int(d), _i64(n), _i64(p), int(dtype), int(direction), ctypes.byref(h)), "fftu_plan")
    return h.value


def fftu_plan_ex(d: int, n, p, dtype: int, direction: int, schedule: int = FFTU_SCHED_AUTO,
                 tune: bool = False, precision: int = FFTU_PREC_NATIVE, layout: int = FFTU_LAYOUT_NATURAL,
                 workspace_mode: int = FFTU_WORKSPACE_PLAN, tile: int = 0, radix: int = 0) -> int:
    h = ctypes.c_void_p()
    opts = fftu_options(schedule=int(schedule), tune=int(bool(tune)), precision=int(precision), layout=int(layout),
                        workspace_mode=int(workspace_mode), tile=int(tile), radix=int(radix))
    _check(_lib.fftu_plan_ex(int(d), _i64(n), _i64(p), int(dtype), int(direction), ctypes.byref(opts),
                             ctypes.byref(h)), "fftu_plan_ex")
    return h.value


def fftu_exec(plan: int, in_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check(_lib.fftu_exec(plan, in_ptr, out_ptr, stream or None), "fftu_exec")


def fftu_exec_phase(plan: int, phase: int, in_ptr, out_ptr: int, stream: int = 0) -> None:
    _check(_lib.fftu_exec_phase(plan, int(phase), in_ptr, out_ptr, stream or None), "fftu_exec_phase")


def fftu_exec_pointwise(fwd: int, inv: int, in_ptr: int, mul_ptr: int, tmp_ptr: int, out_ptr: int,
                        stream: int = 0) -> None:
    _check(_lib.fftu_exec_pointwise(fwd, inv, in_ptr, mul_ptr, tmp_ptr, out_ptr, stream or None),
           "fftu_exec_pointwise")


def fftu_destroy(plan: int) -> None:
    _check(_lib.fftu_destroy(plan), "fftu_destroy")


def fftu_plan_info(plan: int) -> dict:
    info = fftu_info()
    _check(_lib.fftu_plan_info(plan, ctypes.byref(info)), "fftu_plan_info")
    d = info.d
    return {"d": d, "n": list(info.n[:d]), "p": list(info.p[:d]), "dtype": info.dtype, "dir": info.dir,
            "schedule": info.schedule, "launches_phase_a": info.launches_phase_a,
            "launches_phase_b": info.launches_phase_b, "N": info.N, "alg_bytes": info.alg_bytes,
            "table_bytes": info.table_bytes, "workspace_bytes": info.workspace_bytes, "tuned": info.tuned,
            "precision": info.precision, "workspace_need": info.workspace_need, "layout": info.layout,
            "workspace_mode": info.workspace_mode, "tile": info.tile, "radix": info.radix}


def fftu_check_device_status(plan: int) -> None:
    _check(_lib.fftu_check_device_status(plan), "fftu_check_device_status")


def fftu_exec_noalloc(d: int, n, p, dtype: int, direction: int, in_ptr: int, out_ptr: int,
                      stream: int = 0) -> None:
    """Whole transform with no device allocation (static device scratch); see include/fftu.h."""
    _check(_lib.fftu_exec_noalloc(int(d), _i64(n), _i64(p), int(dtype), int(direction), in_ptr, out_ptr,
                                  stream or None), "fftu_exec_noalloc")


def fftu_noalloc_check_status(stream: int = 0) -> None:
    """Read and clear fftu_exec_noalloc's shared device status word (raises FFTUError on a recorded error)."""
    _check(_lib.fftu_noalloc_check_status(stream or None), "fftu_noalloc_check_status")


def fftu_noalloc_selftest_timeout(limit_s: float, stream: int = 0) -> None:
    """Let a bounded device wait expire into fftu_exec_noalloc's status word (failure-detection self-test)."""
    _check(_lib.fftu_noalloc_selftest_timeout(float(limit_s), stream or None), "fftu_noalloc_selftest_timeout")


def fftu_batch_create(plans) -> int:
    hs = (ctypes.c_void_p * len(plans))(*plans)
    b = ctypes.c_void_p()
    _check(_lib.fftu_batch_create(len(plans), hs, ctypes.byref(b)), "fftu_batch_create")
    return b.value


def fftu_batch_exec(batch: int, in_ptrs, out_ptrs, stream: int = 0) -> None:
    ins = (ctypes.c_void_p * len(in_ptrs))(*in_ptrs)
    outs = (ctypes.c_void_p * len(out_ptrs))(*out_ptrs)
    _check(_lib.fftu_batch_exec(batch, ins, outs, stream or None), "fftu_batch_exec")


def fftu_batch_check_status(batch: int) -> None:
    _check(_lib.fftu_batch_check_status(batch), "fftu_batch_check_status")


def fftu_batch_destroy(batch: int) -> None:
    _check(_lib.fftu_batch_destroy(batch), "fftu_batch_destroy")


def fftu_wisdom_export(path: str) -> None:
    _check(_lib.fftu_wisdom_export(path.encode()), "fftu_wisdom_export")


def fftu_wisdom_import(path: str) -> None:
    _check(_lib.fftu_wisdom_import(path.encode()), "fftu_wisdom_import")


def fftu_wisdom_forget() -> None:
    _check(_lib.fftu_wisdom_forget(), "fftu_wisdom_forget")


def fftu_server_create(device_bytes: int = 0, max_batch: int = 0, streams: int = 0, large_elems: int = 0,
                       use_graphs: bool = True, max_inflight: int = 0, copy_piece_mib: int = 0,
                       max_inflight_solo: int = 0) -> int:
    cfg = fftu_server_config(device_bytes=int(device_bytes), max_batch=int(max_batch), streams=int(streams),
                             large_elems=int(large_elems), use_graphs=int(bool(use_graphs)),
                             max_inflight=int(max_inflight), copy_piece_mib=int(copy_piece_mib),
                             max_inflight_solo=int(max_inflight_solo))
    h = ctypes.c_void_p()
    _check(_lib.fftu_server_create(ctypes.byref(cfg), ctypes.byref(h)), "fftu_server_create")
    return h.value


def fftu_server_submit(server: int, n, dtype: int, direction: int, in_ptr: int, out_ptr: int, tag: int) -> None:
    n = [int(v) for v in n]
    r = fftu_request(d=len(n), dtype=int(dtype), dir=int(direction), in_=in_ptr, out=out_ptr, tag=int(tag))
    for i, v in enumerate(n):
        r.n[i] = v
    _check(_lib.fftu_server_submit(server, ctypes.byref(r)), "fftu_server_submit")


def fftu_server_warm(server: int, n, dtype: int, direction: int, in_ptr: int, out_ptr: int, max_k: int,
                     timeout_s: float = 120.0) -> None:
    """Pre-build the key's resident instances and graphs for batch sizes up to max_k (fftu_serve.h)."""
    n = [int(v) for v in n]
    r = fftu_request(d=len(n), dtype=int(dtype), dir=int(direction), in_=in_ptr, out=out_ptr, tag=0)
    for i, v in enumerate(n):
        r.n[i] = v
    _check(_lib.fftu_server_warm(server, ctypes.byref(r), int(max_k), float(timeout_s)), "fftu_server_warm")


def fftu_server_poll(server: int, max_items: int = 1024) -> list:
    buf = (fftu_completion * max_items)()
    k = _lib.fftu_server_poll(server, buf, max_items)
    if k < 0:
        raise FFTUError(1, "fftu_server_poll")
    return [{"tag": c.tag, "status": c.status, "batch_size": c.batch_size, "submit_s": c.submit_s,
             "start_s": c.start_s, "done_s": c.done_s} for c in buf[:k]]


def fftu_server_drain(server: int, timeout_s: float = 60.0) -> None:
    _check(_lib.fftu_server_drain(server, float(timeout_s)), "fftu_server_drain")


def fftu_server_stats_get(server: int) -> dict:
    st = fftu_server_stats()
    _check(_lib.fftu_server_stats_get(server, ctypes.byref(st)), "fftu_server_stats_get")
    return {name: getattr(st, name) for name, _ in fftu_server_stats._fields_}


def fftu_server_destroy(server: int) -> None:
    _check(_lib.fftu_server_destroy(server), "fftu_server_destroy")


def fftu_workspace_size(plan: int) -> int:
    b = ctypes.c_size_t()
    _check(_lib.fftu_workspace_size(plan, ctypes.byref(b)), "fftu_workspace_size")
    return int(b.value)


def fftu_set_workspace(plan: int, ptr, nbytes: int) -> None:
    _check(_lib.fftu_set_workspace(plan, ptr, int(nbytes)), "fftu_set_workspace")


def fftu_measure_fp64_rate(reps: int = 3) -> float:
    """Sustained FP64 FMA rate of the current device, GFLOP/s (best of reps timed launches)."""
    g = ctypes.c_double(0.0)
    _check(_lib.fftu_measure_fp64_rate(int(reps), ctypes.byref(g)), "fftu_measure_fp64_rate")
    return float(g.value)


def fftu_selftest_bounded_wait(limit_s: float) -> float:
    """Seconds the device waited before its bounded wait gave up with FFTU_ERR_TIMEOUT."""
    w = ctypes.c_double()
    _check(_lib.fftu_selftest_bounded_wait(float(limit_s), ctypes.byref(w)), "fftu_selftest_bounded_wait")
    return w.value


def fftu_status_string(status: int) -> str:
    return _lib.fftu_status_string(int(status)).decode()


def fftu_last_error() -> str:
    return _lib.fftu_last_error().decode()


def fftu_version() -> str:
    return _lib.fftu_version().decode()


# ---- torch convenience -----------------------------------------------------------------

def _dtype_code(torch_dtype) -> int:
    import torch
    if torch_dtype == torch.complex64:
        return FFTU_C64
    if torch_dtype == torch.complex128:
        return FFTU_C128
    raise TypeError(f"unsupported dtype {torch_dtype}; use torch.complex64 or torch.complex128")


class Plan:
    """A plan for one shape, cyclic grid p, dtype and direction (fftu_plan)."""

    def __init__(self, n, p=None, dtype=None, inverse: bool = False, schedule: int = FFTU_SCHED_AUTO,
                 tune: bool = False, precision: int = FFTU_PREC_NATIVE, layout: int = FFTU_LAYOUT_NATURAL,
                 workspace_mode: int = FFTU_WORKSPACE_PLAN, tile: int = 0, radix: int = 0):
        import torch
        self.n = tuple(int(v) for v in n)
        self.dtype = dtype if dtype is not None else torch.complex64
        code = _dtype_code(self.dtype)
        self.inverse = bool(inverse)
        self.handle = fftu_plan_ex(len(self.n), self.n, None if p is None else list(p), code,
                                   FFTU_INVERSE if inverse else FFTU_FORWARD, schedule, tune, precision, layout,
                                   workspace_mode, tile, radix)
        self.p = tuple(self.info["p"])

    def _validate(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype or tuple(t.shape) != self.n or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor of shape {self.n}")

    def exec(self, x, out=None, stream=None):
        """Whole transform; out defaults to a new tensor; out may be x (in place)."""
        import torch
        self._validate(x, "x")
        if out is None:
            out = torch.empty_like(x)
        self._validate(out, "out")
        s = stream if stream is not None else torch.cuda.current_stream(x.device)
        fftu_exec(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    def exec_phase(self, phase: int, x, out, stream=None):
        import torch
        self._validate(out, "out")
        if x is not None:
            self._validate(x, "x")
        s = stream if stream is not None else torch.cuda.current_stream(out.device)
        fftu_exec_phase(self.handle, phase, None if x is None else x.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    @property
    def info(self) -> dict:
        """fftu_plan_info, read now (workspace fields change with fftu_set_workspace)."""
        return fftu_plan_info(self.handle)

    def check_device_status(self):
        fftu_check_device_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            fftu_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
