"""ctypes wrapper for the CPU oracle (zig_oracle.c).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
CPU-baseline / reference legs may import this module; the product library in
paper_1403_6870_gb300/ never does.  The oracle follows Table 1 (modified
column) of McFarland, arXiv:1403.6870, with the tables of Sec. 2 built in
binary128; see zig_oracle.h for the passages and readings each function
follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "zig_oracle.c")
LIB = os.path.join(HERE, "liborc.so")
# Mutation tests point this at a deliberately broken copy of the oracle.
LIB_OVERRIDE = os.environ.get("ZIG_ORACLE_LIB")

EXP, NORMAL = 0, 1
F32, F64 = 0, 1
MAXCOLS = 1024

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liborc.so with gcc (contraction off, as the readings require)."""
    if LIB_OVERRIDE:
        return LIB_OVERRIDE
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "zig_oracle.h"))
    ):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=gnu11", SRC, "-o", tmp, "-lm", "-lpthread",
        ]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


class Tables(ctypes.Structure):
    _fields_ = [
        ("dist", ctypes.c_int32), ("imax", ctypes.c_int32), ("ibits", ctypes.c_int32),
        ("L", ctypes.c_int32), ("ubits", ctypes.c_int32), ("abits", ctypes.c_int32),
        ("pad0", ctypes.c_int32), ("pad1", ctypes.c_int32),
        ("X", ctypes.c_double * (MAXCOLS + 1)),
        ("f", ctypes.c_double * (MAXCOLS + 1)),
        ("dX", ctypes.c_double * (MAXCOLS + 1)),
        ("df", ctypes.c_double * (MAXCOLS + 1)),
        ("A", ctypes.c_double * (MAXCOLS + 1)),
        ("eps_j", ctypes.c_double * (MAXCOLS + 1)),
        ("eps", ctypes.c_double), ("tau", ctypes.c_double), ("rinv", ctypes.c_double),
        ("X32", ctypes.c_float * (MAXCOLS + 1)),
        ("f32", ctypes.c_float * (MAXCOLS + 1)),
        ("dX32", ctypes.c_float * (MAXCOLS + 1)),
        ("df32", ctypes.c_float * (MAXCOLS + 1)),
        ("rinv32", ctypes.c_float), ("padf", ctypes.c_float),
        ("q", ctypes.c_uint64 * MAXCOLS),
        ("T", ctypes.c_uint64 * MAXCOLS),
        ("alias", ctypes.c_uint16 * MAXCOLS),
    ]

    def arr(self, name: str) -> np.ndarray:
        return np.ctypeslib.as_array(getattr(self, name)).copy()


class Words(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("dtype", ctypes.c_int), ("dom", ctypes.c_uint32),
        ("seed", ctypes.c_uint64), ("g", ctypes.c_uint64),
        ("block", ctypes.c_uint32), ("half", ctypes.c_int), ("r", ctypes.c_uint32 * 4),
        ("script", ctypes.POINTER(ctypes.c_uint64)), ("nscript", ctypes.c_int),
        ("pos", ctypes.c_int), ("overrun", ctypes.c_int), ("used", ctypes.c_int),
    ]


class Diag(ctypes.Structure):
    _fields_ = [("words", ctypes.c_int), ("err", ctypes.c_int), ("margin", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            L = _lib
            P = ctypes.POINTER
            L.orc_tables_size.restype = ctypes.c_size_t
            assert L.orc_tables_size() == ctypes.sizeof(Tables), "orc_tables layout mismatch"
            L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
            L.orc_build_tables.argtypes = [ctypes.c_int] * 4 + [P(Tables)]
            L.orc_words_philox.argtypes = [P(Words), ctypes.c_uint64, ctypes.c_uint64]
            L.orc_words_script.argtypes = [P(Words), P(ctypes.c_uint64), ctypes.c_int]
            L.orc_words_packed.argtypes = [P(Words), ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            L.orc_next.argtypes = [P(Words)]
            L.orc_next.restype = ctypes.c_uint64
            L.orc_set_limits.argtypes = [ctypes.c_int, ctypes.c_int]
            L.orc_overhang_attempt64.argtypes = [P(Tables), ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, P(ctypes.c_double),
                                                 P(ctypes.c_double)]
            L.orc_alias_pick.argtypes = [P(Tables), ctypes.c_uint64]
            for name, rt in (("orc_exp64", ctypes.c_double), ("orc_exp32", ctypes.c_float)):
                getattr(L, name).argtypes = [P(Tables), P(Words), P(Diag)]
                getattr(L, name).restype = rt
            for name, rt in (("orc_normal64", ctypes.c_double), ("orc_normal32", ctypes.c_float)):
                getattr(L, name).argtypes = [P(Tables), P(Tables), P(Words), P(Diag)]
                getattr(L, name).restype = rt
            L.orc_fill.argtypes = [P(Tables), P(Tables), ctypes.c_int, ctypes.c_int,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_int]
            L.orc_fill.restype = ctypes.c_int64
            L.orc_fill_keyed.argtypes = [P(Tables), P(Tables), ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            L.orc_fill_keyed.restype = ctypes.c_int64
            L.orc_moments.argtypes = [P(Tables), P(Tables), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int]
            L.orc_moments.restype = ctypes.c_int64
            L.orc_moments_keyed.argtypes = [P(Tables), P(Tables), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int]
            L.orc_moments_keyed.restype = ctypes.c_int64
            L.orc_enum_overhang.argtypes = [P(Tables), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
            L.orc_enum_overhang.restype = ctypes.c_int64
            L.orc_transform64.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double]
            L.orc_transform64.restype = ctypes.c_double
            L.orc_transform32.argtypes = [ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                          ctypes.c_double]
            L.orc_transform32.restype = ctypes.c_float
            L.orc_request_values.argtypes = [P(Tables), P(Tables), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64,
                                             ctypes.c_void_p, ctypes.c_int]
            L.orc_request_values.restype = ctypes.c_int64
            L.orc_first_words.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                          ctypes.c_uint64, ctypes.c_void_p]
            L.orc_first_words.restype = None
        return _lib


def philox(ctr, key) -> tuple:
    """One Philox4x32-10 block for counter ctr[4] and key key[2]."""
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(o)


_tables_cache: dict = {}


def tables(dist: int, ibits: int = 8, ubits: int = 52, abits: int = 56) -> Tables:
    key = (dist, ibits, ubits, abits)
    if key not in _tables_cache:
        t = Tables()
        rc = lib().orc_build_tables(dist, ibits, ubits, abits, ctypes.byref(t))
        if rc != 0:
            raise ValueError(f"orc_build_tables failed for {key}")
        _tables_cache[key] = t
    return _tables_cache[key]


def set_limits(max_attempts: int = 64, max_tail: int = 16) -> None:
    lib().orc_set_limits(max_attempts, max_tail)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def fill(dist: int, dtype: int, seed: int, offset: int, n: int, idx=None,
         want_words: bool = False, want_margin: bool = False, nthreads: int | None = None,
         te: Tables | None = None, tn: Tables | None = None, keying: int = 0):
    """Samples at counters offset + pos (pos = idx[k] or k); keying 0 =
    per-index words, 1 = packed keying (orc_words_packed).

    Returns (values, errors, words_or_None, margin_or_None)."""
    te = te or tables(EXP)
    tn = tn or tables(NORMAL)
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.uint64)
        n = int(idx.size)
    out = np.empty(n, dtype=np.float64 if dtype == F64 else np.float32)
    words = np.empty(n, dtype=np.uint8) if want_words else None
    margin = np.empty(n, dtype=np.float64) if want_margin else None
    errs = lib().orc_fill_keyed(
        ctypes.byref(te), ctypes.byref(tn), dist, dtype, int(keying), seed & (2**64 - 1),
        offset & (2**64 - 1),
        n, None if idx is None else idx.ctypes.data, out.ctypes.data,
        None if words is None else words.ctypes.data,
        None if margin is None else margin.ctypes.data,
        nthreads or default_threads())
    return out, int(errs), words, margin


def moments(dist: int, dtype: int, seed: int, offset: int, n: int, nthreads: int | None = None,
            keying: int = 0):
    """Exact-order (binary128) power sums, absolute power sums and histogram
    (keying 0 per index, 1 packed)."""
    te, tn = tables(EXP), tables(NORMAL)
    sums = np.zeros(4, dtype=np.float64)
    abss = np.zeros(4, dtype=np.float64)
    hist = np.zeros(4098, dtype=np.uint64)
    errs = lib().orc_moments_keyed(ctypes.byref(te), ctypes.byref(tn), dist, dtype, int(keying),
                                   seed, offset, n, sums.ctypes.data, abss.ctypes.data,
                                   hist.ctypes.data, nthreads or default_threads())
    return sums, abss, hist, int(errs)


def sample_script(dist: int, words, dtype: int = F64, te: Tables | None = None,
                  tn: Tables | None = None):
    """Run one sampler call on a scripted word list.

    Returns (value, words_used, overrun, err)."""
    te = te or tables(EXP)
    tn = tn or tables(NORMAL)
    arr = (ctypes.c_uint64 * max(1, len(words)))(*[int(w) & (2**64 - 1) for w in words])
    w = Words()
    lib().orc_words_script(ctypes.byref(w), arr, len(words))
    d = Diag()
    L = lib()
    if dist == EXP:
        fn = L.orc_exp64 if dtype == F64 else L.orc_exp32
        x = fn(ctypes.byref(te), ctypes.byref(w), ctypes.byref(d))
    else:
        fn = L.orc_normal64 if dtype == F64 else L.orc_normal32
        x = fn(ctypes.byref(te), ctypes.byref(tn), ctypes.byref(w), ctypes.byref(d))
    return float(x), int(w.used), bool(w.overrun), bool(d.err)


def philox_words(seed: int, g: int, count: int) -> list:
    """The first `count` words of the word stream of counter g."""
    w = Words()
    lib().orc_words_philox(ctypes.byref(w), seed, g)
    return [int(lib().orc_next(ctypes.byref(w))) for _ in range(count)]


def packed_words(seed: int, g: int, dtype: int, count: int) -> list:
    """The first `count` words of counter g under packed keying."""
    w = Words()
    lib().orc_words_packed(ctypes.byref(w), seed, g, dtype)
    return [int(lib().orc_next(ctypes.byref(w))) for _ in range(count)]


def alias_pick(t: Tables, w: int) -> int:
    return int(lib().orc_alias_pick(ctypes.byref(t), w & (2**64 - 1)))


def overhang_attempt(t: Tables, j: int, ux: float, uy: float):
    x = ctypes.c_double()
    m = ctypes.c_double(float("inf"))
    ok = lib().orc_overhang_attempt64(ctypes.byref(t), j, ux, uy, ctypes.byref(x), ctypes.byref(m))
    return bool(ok), float(x.value)


def enum_overhang(t: Tables, j: int, bits: int) -> np.ndarray:
    buf = np.empty(1 << (2 * bits), dtype=np.float64)
    cnt = lib().orc_enum_overhang(ctypes.byref(t), j, bits, buf.ctypes.data)
    return buf[:cnt].copy()


def request_values(req: dict, idx) -> np.ndarray:
    """Variates of one batched request at positions idx: the standard variate
    of each counter mapped by transform() (float64; FP32 results widened
    exactly)."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.float64)
    te, tn = tables(EXP), tables(NORMAL)
    rc = lib().orc_request_values(ctypes.byref(te), ctypes.byref(tn), req["dist"],
                                  req["dtype"], req["seed"] & (2**64 - 1),
                                  req["offset"] & (2**64 - 1), float(req["p0"]),
                                  float(req["p1"]), idx.ctypes.data, idx.size, out.ctypes.data,
                                  default_threads())
    if rc < 0:
        raise MemoryError("orc_request_values could not allocate its scratch")
    return out


def first_words(seed: int, offset: int, idx) -> np.ndarray:
    """First word (block 0, r0 | r1 << 32) of counters offset + idx."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.uint64)
    lib().orc_first_words(seed & (2**64 - 1), offset & (2**64 - 1), idx.ctypes.data, idx.size,
                          out.ctypes.data)
    return out


def transform(dist: int, dtype: int, x: float, p0: float, p1: float) -> float:
    if dtype == F64:
        return float(lib().orc_transform64(dist, x, p0, p1))
    return float(lib().orc_transform32(dist, x, p0, p1))
