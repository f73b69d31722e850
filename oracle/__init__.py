"""CPU oracle for DF Louvain -- test infrastructure only.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  The GPU library never calls it, and it
never calls the GPU library: the two share nothing but the seeded inputs of
`synth`.

The arithmetic lives in `dfl_oracle.cpp` (single-threaded C++, exact integer
delta-modularity); this module compiles it with g++ and wraps its C ABI with
ctypes.  See the header of `dfl_oracle.cpp` for the schedule it fixes and for
which parts are pinned by the CPU tests.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dfl_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

ND, DS, DF = 0, 1, 2

ERRORS = {0: "ok", -1: "invalid", -2: "not_found", -3: "overflow", -4: "nomem", -7: "state"}


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"oracle error {code} ({ERRORS.get(code, '?')}) {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, no GPU code)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_libs = {}


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file (this one, or a deliberately mutated copy
    used by the tests that check the pins catch mistakes) to a shared library."""
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out, src])
    return out


def _load(path: str | None = None):
    path = path or build()
    if path not in _libs:
        lib = ct.CDLL(path)
        P = ct.c_void_p
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
        lib.orc_create.restype = P
        lib.orc_create.argtypes = [ct.c_uint32, u64p, u32p, u32p, ct.POINTER(ct.c_int)]
        lib.orc_create_ex.restype = P
        lib.orc_create_ex.argtypes = [ct.c_uint32, u64p, u32p, u32p, ct.c_uint32,
                                      ct.POINTER(ct.c_int)]
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_options.argtypes = [P, ct.c_uint32, ct.c_uint32, ct.c_uint64, ct.c_uint64,
                                        ct.c_uint64, ct.c_double, ct.c_uint32]
        lib.orc_static.argtypes = [P]
        lib.orc_apply_batch.argtypes = [P, u32p, ct.c_uint64, u32p, ct.c_uint64]
        lib.orc_update.argtypes = [P, ct.c_int]
        lib.orc_mark.argtypes = [P, ct.c_int, u8p, u8p]
        lib.orc_set_membership.argtypes = [P, u32p]
        lib.orc_louvain_from.argtypes = [P, u8p, u8p]
        lib.orc_move_iteration.argtypes = [P, u8p, u8p, u8p, i64p]
        lib.orc_delta_q_num.argtypes = [P, ct.c_uint32, ct.c_uint32, i64p]
        lib.orc_aggregate.argtypes = [P, ct.POINTER(ct.c_uint32), ct.POINTER(ct.c_uint64),
                                      P, P, P]
        lib.orc_num_arcs.restype = ct.c_uint64
        lib.orc_num_arcs.argtypes = [P]
        lib.orc_graph.argtypes = [P, u64p, u32p, u32p]
        lib.orc_membership.argtypes = [P, u32p]
        lib.orc_weights.argtypes = [P, i64p, i64p, ct.POINTER(ct.c_int64)]
        lib.orc_modularity.argtypes = [P, ct.POINTER(ct.c_double), i64p]
        lib.orc_stats.argtypes = [P, u64p, ct.c_uint32]
        lib.orc_trace.argtypes = [P, u64p, ct.c_uint32]
        lib.orc_last_error.restype = ct.c_char_p
        lib.orc_last_error.argtypes = [P]
        _libs[path] = lib
    return _libs[path]


def _i128(hi: int, lo: int) -> int:
    v = ((hi & 0xFFFFFFFFFFFFFFFF) << 64) | (lo & 0xFFFFFFFFFFFFFFFF)
    return v - (1 << 128) if v >> 127 else v


def _edges(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32).reshape(-1, 3))
    return a


class Oracle:
    """Single-threaded DF Louvain state (graph, K, Sigma, 2m, membership)."""

    def __init__(self, n: int, offsets, indices, weights, allow_self_loops: bool = False,
                 library: str | None = None):
        lib = _load(library)
        st = ct.c_int(0)
        self.n = int(n)
        self._h = lib.orc_create_ex(self.n, np.ascontiguousarray(offsets, np.uint64),
                                    np.ascontiguousarray(indices, np.uint32),
                                    np.ascontiguousarray(weights, np.uint32),
                                    1 if allow_self_loops else 0, ct.byref(st))
        if not self._h:
            raise OracleError(st.value, "create")
        self._lib = lib

    def close(self):
        if getattr(self, "_h", None):
            self._lib.orc_destroy(self._h)
            self._h = None

    __del__ = close

    def _check(self, rc: int):
        if rc != 0:
            raise OracleError(rc, self._lib.orc_last_error(self._h).decode())

    def set_options(self, max_iterations=20, max_passes=10, tau_num=1, tau_den=100,
                    tolerance_drop=10, tau_agg=0.8, substeps=4):
        self._check(self._lib.orc_set_options(self._h, max_iterations, max_passes, tau_num,
                                              tau_den, tolerance_drop, float(tau_agg), substeps))

    def static(self):
        self._check(self._lib.orc_static(self._h))

    def apply_batch(self, dels, ins) -> int:
        d, i = _edges(dels), _edges(ins)
        return self._lib.orc_apply_batch(self._h, d.reshape(-1), d.shape[0], i.reshape(-1),
                                         i.shape[0])

    def update(self, mode: int):
        self._check(self._lib.orc_update(self._h, mode))

    def mark(self, mode: int):
        F = np.zeros(self.n, np.uint8)
        R = np.zeros(self.n, np.uint8)
        self._check(self._lib.orc_mark(self._h, mode, F, R))
        return F, R

    def set_membership(self, C):
        self._check(self._lib.orc_set_membership(self._h, np.ascontiguousarray(C, np.uint32)))

    def louvain_from(self, F0, R0):
        self._check(self._lib.orc_louvain_from(self._h, np.ascontiguousarray(F0, np.uint8),
                                               np.ascontiguousarray(R0, np.uint8)))

    def move_iteration(self, F, R):
        F = np.array(F, np.uint8)
        moved = np.zeros(self.n, np.uint8)
        dq = np.zeros(2, np.int64)
        self._check(self._lib.orc_move_iteration(self._h, F, np.ascontiguousarray(R, np.uint8),
                                                 moved, dq))
        return F, moved, _i128(int(dq[0]), int(dq[1]))

    def delta_q_num(self, i: int, c: int) -> int:
        out = np.zeros(2, np.int64)
        self._check(self._lib.orc_delta_q_num(self._h, i, c, out))
        return _i128(int(out[0]), int(out[1]))

    def aggregate(self):
        nv = ct.c_uint32(0)
        na = ct.c_uint64(0)
        self._check(self._lib.orc_aggregate(self._h, ct.byref(nv), ct.byref(na), None, None,
                                            None))
        off = np.zeros(nv.value + 1, np.uint64)
        idx = np.zeros(max(na.value, 1), np.uint32)
        w = np.zeros(max(na.value, 1), np.uint64)
        self._check(self._lib.orc_aggregate(self._h, ct.byref(nv), ct.byref(na),
                                            off.ctypes.data, idx.ctypes.data, w.ctypes.data))
        return off, idx[: na.value], w[: na.value]

    def graph(self):
        na = self._lib.orc_num_arcs(self._h)
        off = np.zeros(self.n + 1, np.uint64)
        idx = np.zeros(max(na, 1), np.uint32)
        w = np.zeros(max(na, 1), np.uint32)
        self._check(self._lib.orc_graph(self._h, off, idx, w))
        return off, idx[:na], w[:na]

    def membership(self) -> np.ndarray:
        out = np.zeros(self.n, np.uint32)
        self._check(self._lib.orc_membership(self._h, out))
        return out

    def weights(self):
        K = np.zeros(self.n, np.int64)
        S = np.zeros(self.n, np.int64)
        m2 = ct.c_int64(0)
        self._check(self._lib.orc_weights(self._h, K, S, ct.byref(m2)))
        return K, S, int(m2.value)

    def modularity(self):
        q = ct.c_double(0)
        parts = np.zeros(4, np.int64)
        self._check(self._lib.orc_modularity(self._h, ct.byref(q), parts))
        return q.value, _i128(int(parts[0]), int(parts[1])), _i128(int(parts[2]), int(parts[3]))

    def stats(self) -> dict:
        out = np.zeros(4 + 64, np.uint64)
        self._check(self._lib.orc_stats(self._h, out, out.shape[0]))
        passes = int(out[0])
        return {"passes": passes, "affected_initial": int(out[1]),
                "affected_ever": int(out[2]), "trace_len": int(out[3]),
                "iterations": [int(x) for x in out[4:4 + passes]]}

    def trace(self):
        t = self.stats()["trace_len"]
        out = np.zeros(4 * max(t, 1), np.uint64)
        self._check(self._lib.orc_trace(self._h, out, t))
        return [(int(out[4 * k]), int(out[4 * k + 1]), (int(out[4 * k + 2]) << 64) | int(out[4 * k + 3]))
                for k in range(t)]
