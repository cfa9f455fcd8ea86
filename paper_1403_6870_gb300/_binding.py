"""Thin Python binding of libzig.so (include/zig.h), same names as the C ABI.

Argument marshalling only: every step of generation runs in the library's
CUDA kernels.  Device buffers are PyTorch CUDA tensors (or raw device
addresses as ints); streams are torch.cuda.Stream objects, raw cudaStream_t
ints, or None for the tensor's current stream.  A non-OK status raises
ZigError.  The module fails to import when libzig.so has not been built:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libzig.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with paper_1403_6870_gb300.build.build() "
        "(or __graft_entry__.build()); there is no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

ZIG_OK, ZIG_E_INVAL, ZIG_E_NOTINIT, ZIG_E_CUDA, ZIG_E_NOMEM = 0, 1, 2, 3, 4
ZIG_E_ALIGN, ZIG_E_RANGE, ZIG_E_LOOP_LIMIT, ZIG_E_TABLE, ZIG_E_TIMEOUT = 5, 6, 7, 8, 9
ZIG_F32, ZIG_F64 = 0, 1
ZIG_EXP, ZIG_NORMAL = 0, 1

_u64 = ctypes.c_uint64
_vp = ctypes.c_void_p
_int = ctypes.c_int


class ZigError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        super().__init__(f"{where}: {zig_strerror(status)} (status {status})")


class zig_tables_export(ctypes.Structure):
    _fields_ = [
        ("dist", ctypes.c_int32), ("L", ctypes.c_int32), ("imax", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("X", ctypes.c_double * 257), ("f", ctypes.c_double * 257),
        ("dX", ctypes.c_double * 257), ("df", ctypes.c_double * 257),
        ("A", ctypes.c_double * 257),
        ("eps", ctypes.c_double), ("tau", ctypes.c_double), ("rinv", ctypes.c_double),
        ("X32", ctypes.c_float * 257), ("f32", ctypes.c_float * 257),
        ("dX32", ctypes.c_float * 257), ("df32", ctypes.c_float * 257),
        ("rinv32", ctypes.c_float), ("reserved2", ctypes.c_float),
        ("T", ctypes.c_uint64 * 256), ("alias", ctypes.c_uint8 * 256),
    ]


def _sig(name, restype, argtypes):
    fn = getattr(_lib, name)
    fn.restype = restype
    fn.argtypes = argtypes
    return fn


_strerror = _sig("zig_strerror", ctypes.c_char_p, [_int])
_build_tables = _sig("zig_build_tables", _int, [])
_export_tables = _sig("zig_export_tables", _int, [_int, ctypes.POINTER(zig_tables_export)])
_exponential = _sig("zig_exponential", _int, [_vp, _u64, _u64, _u64, _int, _vp])
_normal = _sig("zig_normal", _int, [_vp, _u64, _u64, _u64, _int, _vp])
_status_poll = _sig("zig_status_poll", _int, [_vp])
_generate = _sig("zig_generate", _int, [_int, _int, _int, _vp, _u64, _u64, _u64, _int, _vp])
ZIG_KEY_INDEX, ZIG_KEY_PACKED = 0, 1
_moments_ws = _sig("zig_moments_workspace_bytes", ctypes.c_size_t, [_int, _int])
_moments = _sig("zig_moments", _int, [_int, _int, _u64, _u64, _u64, _vp, _vp, _vp,
                                      ctypes.c_size_t, _vp])
_batch_ws = _sig("zig_batch_workspace_bytes", ctypes.c_size_t, [ctypes.c_uint32])
_batch_validate = _sig("zig_batch_validate", _int, [_vp, ctypes.c_uint32])
_batch = _sig("zig_batch", _int, [_vp, ctypes.c_uint32, _vp, _vp, ctypes.c_size_t, _vp])
_moments_keyed = _sig("zig_moments_keyed", _int, [_int, _int, _int, _u64, _u64, _u64, _vp, _vp,
                                                  _vp, ctypes.c_size_t, _vp])
_moments_noalloc = _sig("zig_moments_noalloc", _int, [_int, _int, _u64, _u64, _u64, _vp, _vp,
                                                      _vp])
_set_limits = _sig("zig_set_fringe_limits", _int, [_int, _int])


class zig_tables_ex(ctypes.Structure):
    _fields_ = [
        ("dist", ctypes.c_int32), ("L", ctypes.c_int32), ("imax", ctypes.c_int32),
        ("index_bits", ctypes.c_int32),
        ("X", ctypes.c_double * 1025), ("f", ctypes.c_double * 1025),
        ("dX", ctypes.c_double * 1025), ("df", ctypes.c_double * 1025),
        ("A", ctypes.c_double * 1025),
        ("eps", ctypes.c_double), ("tau", ctypes.c_double), ("rinv", ctypes.c_double),
        ("X32", ctypes.c_float * 1025), ("f32", ctypes.c_float * 1025),
        ("dX32", ctypes.c_float * 1025), ("df32", ctypes.c_float * 1025),
        ("rinv32", ctypes.c_float), ("reserved", ctypes.c_float),
        ("T", ctypes.c_uint64 * 1024), ("alias", ctypes.c_uint16 * 1024),
        ("acc52", ctypes.c_uint64 * 1025), ("rej52", ctypes.c_uint64 * 1025),
        ("acc23", ctypes.c_uint64 * 1025), ("rej23", ctypes.c_uint64 * 1025),
    ]


_export_tables_ex = _sig("zig_export_tables_ex", _int, [_int, _int, ctypes.POINTER(zig_tables_ex)])


def zig_export_tables_ex(dist: int, index_bits: int) -> zig_tables_ex:
    t = zig_tables_ex()
    _check(_export_tables_ex(int(dist), int(index_bits), ctypes.byref(t)), "zig_export_tables_ex")
    return t


class zig_tune_entry(ctypes.Structure):
    _fields_ = [("V", ctypes.c_int32), ("R", ctypes.c_int32), ("min_blocks", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("gsamples_s", ctypes.c_double)]


_TuneP = ctypes.POINTER(zig_tune_entry)
_tune_candidates = _sig("zig_tune_candidates", _int, [_int, _TuneP, _int])
_autotune = _sig("zig_autotune", _int, [_int, _int, _vp, ctypes.c_size_t, _int, _vp, _TuneP, _int,
                                        ctypes.POINTER(_int), _TuneP])
_tune_get = _sig("zig_tune_get", _int, [_int, _int, _TuneP])
_tune_set = _sig("zig_tune_set", _int, [_int, _int, _TuneP])
_tune_save = _sig("zig_tune_save", _int, [ctypes.c_char_p])
_tune_load = _sig("zig_tune_load", _int, [ctypes.c_char_p])


def zig_strerror(status: int) -> str:
    return _strerror(int(status)).decode()


def _check(st: int, where: str) -> None:
    if st != ZIG_OK:
        raise ZigError(st, where)


def _stream_handle(stream, tensor=None):
    if stream is None:
        if tensor is not None and hasattr(tensor, "device") and tensor.is_cuda:
            import torch

            return torch.cuda.current_stream(tensor.device).cuda_stream
        if tensor is not None and hasattr(tensor, "device"):
            import torch

            return torch.cuda.current_stream().cuda_stream
        return 0
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _out_args(out, n, dtype):
    """(device address, n, dtype code) from a tensor or a raw address."""
    if hasattr(out, "data_ptr"):
        import torch

        if not (out.is_cuda or out.is_pinned()):
            raise ValueError("out must be a CUDA tensor or a pinned host tensor")
        if not out.is_contiguous():
            raise ValueError("out must be contiguous")
        code = {torch.float32: ZIG_F32, torch.float64: ZIG_F64}.get(out.dtype)
        if code is None:
            raise ValueError("out must be float32 or float64")
        if dtype is not None and dtype != code:
            raise ValueError("dtype does not match the tensor")
        if n is None:
            n = out.numel()
        elif n > out.numel():
            raise ValueError("n exceeds the tensor size")
        return out.data_ptr(), int(n), code
    if dtype is None or n is None:
        raise ValueError("raw addresses need explicit n and dtype")
    return int(out), int(n), int(dtype)


def zig_build_tables() -> None:
    _check(_build_tables(), "zig_build_tables")


def zig_export_tables(dist: int) -> zig_tables_export:
    t = zig_tables_export()
    _check(_export_tables(int(dist), ctypes.byref(t)), "zig_export_tables")
    return t


def zig_exponential(out, n=None, seed: int = 0, offset: int = 0, dtype=None, stream=None) -> None:
    ptr, n, code = _out_args(out, n, dtype)
    _check(_exponential(ptr, n, seed & (2**64 - 1), offset & (2**64 - 1), code,
                        _stream_handle(stream, out)), "zig_exponential")


def zig_normal(out, n=None, seed: int = 0, offset: int = 0, dtype=None, stream=None) -> None:
    ptr, n, code = _out_args(out, n, dtype)
    _check(_normal(ptr, n, seed & (2**64 - 1), offset & (2**64 - 1), code,
                   _stream_handle(stream, out)), "zig_normal")


def zig_generate(dist: int, keying: int, out, n=None, seed: int = 0, offset: int = 0, dtype=None,
                 stream=None, index_bits: int = 8) -> None:
    """zig_exponential / zig_normal with a keying (ZIG_KEY_INDEX or
    ZIG_KEY_PACKED) and a table width (index_bits 8 or 10)."""
    ptr, n, code = _out_args(out, n, dtype)
    _check(_generate(int(dist), int(keying), int(index_bits), ptr, n, seed & (2**64 - 1),
                     offset & (2**64 - 1), code, _stream_handle(stream, out)), "zig_generate")


def zig_moments_workspace_bytes(dist: int, dtype: int) -> int:
    return int(_moments_ws(int(dist), int(dtype)))


def zig_moments(dist: int, dtype: int, n: int, seed: int, offset: int, sums, hist, workspace,
                stream=None) -> None:
    """Fused generate-and-reduce into sums (4 float64) and hist (4098 int64
    or uint64) device tensors; workspace is a device tensor of at least
    zig_moments_workspace_bytes(dist, dtype) bytes."""
    import torch

    if sums.dtype != torch.float64 or sums.numel() < 4 or not sums.is_cuda:
        raise ValueError("sums must be a CUDA float64 tensor of 4 elements")
    if hist.element_size() != 8 or hist.numel() < 4098 or not hist.is_cuda:
        raise ValueError("hist must be a CUDA 64-bit integer tensor of 4098 elements")
    wbytes = workspace.numel() * workspace.element_size()
    _check(_moments(int(dist), int(dtype), n, seed & (2**64 - 1), offset & (2**64 - 1),
                    sums.data_ptr(), hist.data_ptr(), workspace.data_ptr(), wbytes,
                    _stream_handle(stream, sums)), "zig_moments")


def zig_moments_keyed(dist: int, dtype: int, keying: int, n: int, seed: int, offset: int, sums,
                      hist, workspace, stream=None) -> None:
    """zig_moments over the variates of a keying (ZIG_KEY_INDEX or
    ZIG_KEY_PACKED)."""
    import torch

    if sums.dtype != torch.float64 or sums.numel() < 4 or not sums.is_cuda:
        raise ValueError("sums must be a CUDA float64 tensor of 4 elements")
    if hist.element_size() != 8 or hist.numel() < 4098 or not hist.is_cuda:
        raise ValueError("hist must be a CUDA 64-bit integer tensor of 4098 elements")
    wbytes = workspace.numel() * workspace.element_size()
    _check(_moments_keyed(int(dist), int(dtype), int(keying), n, seed & (2**64 - 1),
                          offset & (2**64 - 1), sums.data_ptr(), hist.data_ptr(),
                          workspace.data_ptr(), wbytes, _stream_handle(stream, sums)),
           "zig_moments_keyed")


def zig_moments_noalloc(dist: int, dtype: int, n: int, seed: int, offset: int, sums, hist,
                        stream=None) -> None:
    """zig_moments with the library's static scratch instead of a workspace,
    for callers that cannot allocate device memory (see include/zig.h)."""
    import torch

    if sums.dtype != torch.float64 or sums.numel() < 4 or not sums.is_cuda:
        raise ValueError("sums must be a CUDA float64 tensor of 4 elements")
    if hist.element_size() != 8 or hist.numel() < 4098 or not hist.is_cuda:
        raise ValueError("hist must be a CUDA 64-bit integer tensor of 4098 elements")
    _check(_moments_noalloc(int(dist), int(dtype), n, seed & (2**64 - 1), offset & (2**64 - 1),
                            sums.data_ptr(), hist.data_ptr(), _stream_handle(stream, sums)),
           "zig_moments_noalloc")


REQUEST_DTYPE = None


def request_dtype():
    """numpy structured dtype laid out like zig_request (56 bytes)."""
    global REQUEST_DTYPE
    if REQUEST_DTYPE is None:
        import numpy as np

        REQUEST_DTYPE = np.dtype([("out", "<u8"), ("n", "<u8"), ("seed", "<u8"), ("offset", "<u8"),
                                  ("dist", "<u4"), ("dtype", "<u4"), ("p0", "<f8"), ("p1", "<f8")])
        assert REQUEST_DTYPE.itemsize == 56
    return REQUEST_DTYPE


def pack_requests(reqs) -> "numpy.ndarray":
    """Pack dicts with keys out (device address), n, seed, offset, dist,
    dtype, p0, p1 into a zig_request array (host memory)."""
    import numpy as np

    a = np.zeros(len(reqs), dtype=request_dtype())
    for k, q in enumerate(reqs):
        a[k] = (int(q["out"]), int(q["n"]), int(q["seed"]) & (2**64 - 1),
                int(q["offset"]) & (2**64 - 1), int(q["dist"]), int(q["dtype"]),
                float(q["p0"]), float(q["p1"]))
    return a


def zig_batch_workspace_bytes(count: int) -> int:
    return int(_batch_ws(int(count)))


def zig_batch_validate(h_reqs) -> int:
    """Host-side check of a packed request array; returns the status code."""
    return int(_batch_validate(h_reqs.ctypes.data, len(h_reqs)))


def zig_batch(d_reqs, count: int, workspace, done_ns=None, stream=None) -> None:
    """Serve `count` packed requests held in the device tensor d_reqs."""
    wbytes = workspace.numel() * workspace.element_size()
    _check(_batch(d_reqs.data_ptr(), int(count), None if done_ns is None else done_ns.data_ptr(),
                  workspace.data_ptr(), wbytes, _stream_handle(stream, workspace)), "zig_batch")


class zig_batch_tune_entry(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_uint32), ("ms", ctypes.c_double)]


_batch_autotune = _sig("zig_batch_autotune", _int,
                       [_vp, ctypes.c_uint32, _vp, ctypes.c_size_t, _int, _vp,
                        ctypes.POINTER(zig_batch_tune_entry), _int, ctypes.POINTER(_int),
                        ctypes.POINTER(ctypes.c_uint32)])
_batch_set_chunk = _sig("zig_batch_set_chunk", _int, [ctypes.c_uint32])
_batch_get_chunk = _sig("zig_batch_get_chunk", ctypes.c_uint32, [])


def zig_batch_autotune(d_reqs, count: int, workspace, reps: int = 3, stream=None):
    """Time zig_batch with each candidate chunk size on this batch and keep
    the fastest; returns (chosen chunk, [{"chunk", "ms"}, ...])."""
    wbytes = workspace.numel() * workspace.element_size()
    buf = (zig_batch_tune_entry * 16)()
    n = _int(0)
    chosen = ctypes.c_uint32(0)
    _check(_batch_autotune(d_reqs.data_ptr(), int(count), workspace.data_ptr(), wbytes, int(reps),
                           _stream_handle(stream, workspace), buf, 16, ctypes.byref(n),
                           ctypes.byref(chosen)), "zig_batch_autotune")
    return int(chosen.value), [{"chunk": int(buf[k].chunk), "ms": float(buf[k].ms)}
                               for k in range(min(n.value, 16))]


def zig_batch_set_chunk(chunk: int) -> None:
    _check(_batch_set_chunk(int(chunk)), "zig_batch_set_chunk")


def zig_batch_get_chunk() -> int:
    return int(_batch_get_chunk())


def zig_status_poll(stream=None) -> int:
    """Returns the device status (ZIG_OK or ZIG_E_LOOP_LIMIT) and clears it."""
    st = _status_poll(_stream_handle(stream))
    if st not in (ZIG_OK, ZIG_E_LOOP_LIMIT, ZIG_E_TIMEOUT, ZIG_E_INVAL):
        raise ZigError(st, "zig_status_poll")
    return st


def zig_set_fringe_limits(max_attempts: int = 64, max_tail: int = 16) -> None:
    _check(_set_limits(int(max_attempts), int(max_tail)), "zig_set_fringe_limits")


def _entry_dict(e: zig_tune_entry) -> dict:
    return {"V": e.V, "R": e.R, "min_blocks": e.min_blocks, "blocks_per_sm": e.blocks_per_sm,
            "gsamples_s": e.gsamples_s}


def zig_tune_candidates(dtype: int) -> list:
    """Compiled candidate shapes for dtype (the first is the default)."""
    buf = (zig_tune_entry * 64)()
    k = int(_tune_candidates(int(dtype), buf, 64))
    return [_entry_dict(buf[i]) for i in range(min(k, 64))]


def zig_autotune(dist: int, dtype: int, scratch, reps: int = 3, stream=None):
    """Time every candidate shape on the device tensor `scratch` and select
    the fastest for (dist, dtype); returns (chosen, all measured) dicts."""
    buf = (zig_tune_entry * 64)()
    n = _int(0)
    chosen = zig_tune_entry()
    nbytes = scratch.numel() * scratch.element_size()
    _check(_autotune(int(dist), int(dtype), scratch.data_ptr(), nbytes, int(reps),
                     _stream_handle(stream, scratch), buf, 64, ctypes.byref(n),
                     ctypes.byref(chosen)), "zig_autotune")
    return _entry_dict(chosen), [_entry_dict(buf[i]) for i in range(min(n.value, 64))]


def zig_tune_get(dist: int, dtype: int) -> dict:
    e = zig_tune_entry()
    _check(_tune_get(int(dist), int(dtype), ctypes.byref(e)), "zig_tune_get")
    return _entry_dict(e)


def zig_tune_set(dist: int, dtype: int, entry: dict) -> None:
    e = zig_tune_entry(int(entry["V"]), int(entry["R"]), int(entry["min_blocks"]),
                       int(entry.get("blocks_per_sm", 0)), float(entry.get("gsamples_s", 0.0)))
    _check(_tune_set(int(dist), int(dtype), ctypes.byref(e)), "zig_tune_set")


def zig_tune_save(path: str) -> None:
    _check(_tune_save(os.fsencode(path)), "zig_tune_save")


def zig_tune_load(path: str) -> None:
    _check(_tune_load(os.fsencode(path)), "zig_tune_load")


def raw_call(name: str, *args) -> int:  # noqa: C901
    """Call an exported function with raw C arguments and return its status
    (used to exercise argument checks without raising)."""
    table = {"zig_exponential": _exponential, "zig_normal": _normal, "zig_moments": _moments,
             "zig_generate": _generate,
             "zig_set_fringe_limits": _set_limits, "zig_status_poll": _status_poll,
             "zig_batch_autotune": _batch_autotune}
    return int(table[name](*args))
