"""GB300 (sm_103a) Dynamic Frontier Louvain: Python binding of libdfl.so.

Thin ctypes marshalling over the C ABI declared in include/dfl.h: the module
functions carry the C names (dfl_create, dfl_static, dfl_apply_batch,
dfl_update, dfl_membership, dfl_modularity, ...) and the `Dfl` class wraps a
handle.  Every step of the computation runs in the CUDA kernels of
`csrc/`; this module only converts arguments.  Host inputs are numpy arrays;
device inputs are CUDA tensors (PyTorch supplies device memory and streams).
There is no CPU fallback: if the library is not built, importing the
functions raises.
"""
from __future__ import annotations

import ctypes as ct
import glob
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libdfl.so")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")

ND, DS, DF = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
FLAG_PROFILE = 1
FLAG_NO_GRAPH = 4
FLAG_SERIAL_BINS = 8
FLAG_PERSISTENT = 16
FLAG_GRAPH = 32
FLAG_PROFILE_MOVE = 64
FLAG_RECOMPUTE_AUX = 128
FLAG_TEST_UNREACHABLE_BARRIER = 256
PROF_NAMES = ["apply", "mark", "move", "commit", "aggregate", "other", "bin0", "bin1", "bin2",
              "bin3"]
PROF_APPLY, PROF_MARK, PROF_MOVE, PROF_COMMIT, PROF_AGG, PROF_OTHER = range(6)

ERRORS = {0: "ok", -1: "invalid", -2: "not_found", -3: "overflow", -4: "nomem", -5: "cuda",
          -6: "timeout", -7: "state"}

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
              "-Xcompiler", "-fPIC"]


class DflError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"dfl error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a (one nvcc per file, in parallel) and link
    _build/libdfl.so.  Rebuilds only what is older than its sources."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(_CSRC, "*.cu")))
    headers = glob.glob(os.path.join(_CSRC, "*.cuh")) + glob.glob(os.path.join(_INCLUDE, "*.h"))
    newest_hdr = max(os.path.getmtime(p) for p in headers)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(_BUILD, os.path.basename(src)[:-3] + ".o")
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(os.path.getmtime(src), newest_hdr)):
            return obj
        cmd = [nvcc] + NVCC_FLAGS + ["-c", src, "-o", obj + ".tmp"]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        os.replace(obj + ".tmp", obj)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(map(os.path.getmtime, objs)):
        tmp = _LIB + ".tmp"
        subprocess.check_call([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a"] + objs
                              + ["-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class Options(ct.Structure):
    _fields_ = [("max_iterations", ct.c_uint32), ("max_passes", ct.c_uint32),
                ("tau_num", ct.c_uint64), ("tau_den", ct.c_uint64),
                ("tolerance_drop", ct.c_uint64), ("tau_agg", ct.c_double),
                ("substeps", ct.c_uint32), ("flags", ct.c_uint32)]


class Stats(ct.Structure):
    _fields_ = [("passes", ct.c_uint32), ("iterations", ct.c_uint32 * 16),
                ("affected_initial", ct.c_uint64), ("affected_ever", ct.c_uint64),
                ("kernel_launches", ct.c_uint64), ("num_arcs", ct.c_uint64),
                ("arc_pool", ct.c_uint64), ("max_degree", ct.c_uint32),
                ("num_communities", ct.c_uint32), ("graph_captures", ct.c_uint64),
                ("graph_capture_ms", ct.c_double)]


class Profile(ct.Structure):
    _fields_ = [("launches", ct.c_uint64 * 10), ("ms", ct.c_double * 10), ("bytes", ct.c_uint64 * 10)]


class Tuning(ct.Structure):
    _fields_ = [("bin_warp", ct.c_uint32), ("bin_warp_hash", ct.c_uint32),
                ("bin_block", ct.c_uint32), ("block_threads", ct.c_uint32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# Every function the header declares, with its argument types.
_P = ct.c_void_p
_SIGS = {
    "dfl_default_options": (None, [ct.POINTER(Options)]),
    "dfl_create": (ct.c_int, [ct.POINTER(_P), ct.c_uint32, _P, _P, _P, ct.c_uint64, ct.c_int,
                              ct.POINTER(Options), _P]),
    "dfl_destroy": (None, [_P]),
    "dfl_set_options": (ct.c_int, [_P, ct.POINTER(Options)]),
    "dfl_set_stream": (ct.c_int, [_P, _P]),
    "dfl_static": (ct.c_int, [_P]),
    "dfl_apply_batch": (ct.c_int, [_P, _P, ct.c_uint64, _P, ct.c_uint64, ct.c_int]),
    "dfl_update": (ct.c_int, [_P, ct.c_int]),
    "dfl_step": (ct.c_int, [_P, _P, ct.c_uint64, _P, ct.c_uint64, ct.c_int, ct.c_int]),
    "dfl_membership": (ct.c_int, [_P, _P, ct.c_int]),
    "dfl_modularity": (ct.c_int, [_P, ct.POINTER(ct.c_double), _P]),
    "dfl_weights": (ct.c_int, [_P, _P, _P, ct.POINTER(ct.c_int64), ct.c_int]),
    "dfl_num_arcs": (ct.c_int, [_P, ct.POINTER(ct.c_uint64)]),
    "dfl_compact": (ct.c_int, [_P, ct.POINTER(ct.c_uint64), ct.POINTER(ct.c_uint64)]),
    "dfl_graph": (ct.c_int, [_P, _P, _P, _P, ct.c_int]),
    "dfl_stats": (ct.c_int, [_P, ct.POINTER(Stats)]),
    "dfl_profile": (ct.c_int, [_P, ct.POINTER(Profile), ct.c_int]),
    "dfl_trace": (ct.c_int, [_P, _P, ct.c_uint32, ct.POINTER(ct.c_uint32)]),
    "dfl_last_error": (ct.c_char_p, [_P]),
    "dfl_set_membership": (ct.c_int, [_P, _P, ct.c_int]),
    "dfl_mark": (ct.c_int, [_P, ct.c_int, _P, _P, ct.c_int]),
    "dfl_louvain_from": (ct.c_int, [_P, _P, _P, ct.c_int]),
    "dfl_move_iteration": (ct.c_int, [_P, _P, _P, _P, _P, ct.c_int]),
    "dfl_aggregate": (ct.c_int, [_P, ct.POINTER(ct.c_uint32), ct.POINTER(ct.c_uint64), _P, _P, _P]),
    "dfl_get_tuning": (ct.c_int, [_P, ct.POINTER(Tuning)]),
    "dfl_set_tuning": (ct.c_int, [_P, ct.POINTER(Tuning)]),
    "dfl_autotune": (ct.c_int, [_P, ct.c_int, ct.c_uint32, ct.POINTER(Tuning),
                                ct.POINTER(ct.c_double)]),
    "dfl_group_create": (ct.c_int, [ct.POINTER(_P), ct.c_uint32, _P, _P, _P, _P,
                                    ct.POINTER(Options), _P]),
    "dfl_group_static": (ct.c_int, [_P]),
    "dfl_group_apply_batch": (ct.c_int, [_P, _P, _P, _P, _P, ct.c_int]),
    "dfl_group_update": (ct.c_int, [_P, ct.c_int]),
    "dfl_group_membership": (ct.c_int, [_P, ct.c_uint32, _P, ct.c_int]),
    "dfl_group_modularity": (ct.c_int, [_P, ct.c_uint32, ct.POINTER(ct.c_double), _P]),
    "dfl_group_stats": (ct.c_int, [_P, ct.c_uint32, ct.POINTER(Stats)]),
    "dfl_test_fail_allocations": (ct.c_int, [ct.c_int64]),
    "dfl_modularity_csr_noalloc": (ct.c_int, [ct.c_uint32, _P, _P, _P, _P, ct.POINTER(ct.c_double),
                                              _P, _P]),
}

NOALLOC_MAX_VERTICES = 1 << 20


def modularity_csr_noalloc(n, offsets, indices, weights, membership, stream=None):
    """dfl_modularity_csr_noalloc on CUDA tensors (offsets int64/uint64,
    indices, weights and membership 32-bit), which the C function reads as
    device memory.  Returns (rc, q, num, den)."""
    lib = load()
    bufs = [_buf(offsets, np.uint64), _buf(indices, np.uint32), _buf(weights, np.uint32),
            _buf(membership, np.uint32)]  # kept alive (their keepalive objects) until the call returns
    if any(mk != MEM_DEVICE for _, mk, _ in bufs):
        raise TypeError("dfl_modularity_csr_noalloc takes device buffers only (CUDA tensors)")
    q = ct.c_double()
    parts = np.zeros(4, np.int64)
    rc = lib.dfl_modularity_csr_noalloc(int(n), bufs[0][0], bufs[1][0], bufs[2][0], bufs[3][0],
                                        ct.byref(q), parts.ctypes.data_as(ct.c_void_p),
                                        _stream_ptr(stream))
    del bufs
    return rc, q.value, _i128(int(parts[0]), int(parts[1])), _i128(int(parts[2]), int(parts[3]))


def test_fail_allocations(after: int) -> None:
    """Test hook: after `after` more device allocations every further one
    fails (DFL_ERR_NOMEM); a negative value lifts it (dfl_test_fail_allocations)."""
    load().dfl_test_fail_allocations(int(after))


def library_path() -> str:
    return _LIB


def load(path: str | None = None):
    """Load libdfl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        p = path or _LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libdfl.so not built ({p}); run __graft_entry__.build()")
        lib = ct.CDLL(p)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    load().dfl_default_options(ct.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _is_tensor(x) -> bool:
    return type(x).__module__.startswith("torch") and hasattr(x, "data_ptr")


_TENSOR_INT_WIDTH = {}  # torch integer dtype -> bytes, filled on the first tensor


def _tensor_int_width(dt) -> int:
    if not _TENSOR_INT_WIDTH:
        import torch
        for name in ("bool", "int8", "uint8", "int16", "uint16", "int32", "uint32", "int64", "uint64"):
            t = getattr(torch, name, None)
            if t is not None:
                _TENSOR_INT_WIDTH[t] = torch.empty(0, dtype=t).element_size()
    return _TENSOR_INT_WIDTH.get(dt, 0)


def _buf(x, dtype):
    """(pointer, mem_kind, keepalive) for a numpy array or a tensor (CUDA or
    host).  A tensor is passed as it is, so it must be contiguous and hold
    integers of `dtype`'s width (int32 or uint32 for uint32, ...); an array
    of another integer type is converted, one of floats is refused."""
    if x is None:
        return None, MEM_HOST, None
    want = np.dtype(dtype)
    if _is_tensor(x):
        if _tensor_int_width(x.dtype) != want.itemsize:
            raise TypeError(f"a tensor of {x.dtype} where {want.itemsize}-byte integers ({want}) are expected")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ct.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    if isinstance(x, np.ndarray) and x.dtype.kind not in "iub":
        raise TypeError(f"an array of {x.dtype} where integers ({want}) are expected")
    a = np.ascontiguousarray(x, dtype=dtype)
    return ct.c_void_p(a.ctypes.data), MEM_HOST, a


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return ct.c_void_p(stream.cuda_stream)
    return ct.c_void_p(int(stream))


def _i128(hi: int, lo: int) -> int:
    v = ((hi & 0xFFFFFFFFFFFFFFFF) << 64) | (lo & 0xFFFFFFFFFFFFFFFF)
    return v - (1 << 128) if v >> 127 else v


def save_checkpoint(path: str, ck: dict) -> None:
    """Write a Dfl.checkpoint() to an .npz file."""
    t = ck["tuning"]
    np.savez(path, n=np.uint64(ck["n"]), offsets=ck["offsets"], indices=ck["indices"], weights=ck["weights"],
             membership=ck["membership"], tuning_keys=np.array(list(t.keys())),
             tuning_values=np.array(list(t.values()), np.uint32))


def load_checkpoint(path: str) -> dict:
    """Read a checkpoint written by save_checkpoint."""
    z = np.load(path)
    return {"n": int(z["n"]), "offsets": z["offsets"], "indices": z["indices"], "weights": z["weights"],
            "membership": z["membership"],
            "tuning": {str(k): int(v) for k, v in zip(z["tuning_keys"], z["tuning_values"])}}


class Dfl:
    """One dynamic graph and its community state on the GPU."""

    def __init__(self, n, offsets, indices, weights, options: Options | None = None, stream=None):
        lib = load()
        self._lib = lib
        h = ct.c_void_p()
        off, mk, k0 = _buf(offsets, np.uint64)
        idx, _, k1 = _buf(indices, np.uint32)
        w, _, k2 = _buf(weights, np.uint32)
        nnz = int(indices.shape[0]) if hasattr(indices, "shape") else len(indices)
        self.n = int(n)
        rc = lib.dfl_create(ct.byref(h), self.n, off, idx, w, nnz, mk,
                            ct.byref(options) if options is not None else None, _stream_ptr(stream))
        if rc != 0:
            raise DflError(rc, "dfl_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dfl_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise DflError(rc, self._lib.dfl_last_error(self._h).decode())
        return rc

    @property
    def handle(self):
        return self._h

    def set_options(self, options: Options):
        self._check(self._lib.dfl_set_options(self._h, ct.byref(options)))

    def tuning(self) -> dict:
        t = Tuning()
        self._check(self._lib.dfl_get_tuning(self._h, ct.byref(t)))
        return t.as_dict()

    def set_tuning(self, **kw):
        t = Tuning()
        self._check(self._lib.dfl_get_tuning(self._h, ct.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        self._check(self._lib.dfl_set_tuning(self._h, ct.byref(t)))

    def autotune(self, mode: int = DF, reps: int = 3):
        """Pick the fastest launch shapes for the pending batch's frontier;
        returns (tuning dict, median decide ms)."""
        t = Tuning()
        ms = ct.c_double()
        self._check(self._lib.dfl_autotune(self._h, mode, reps, ct.byref(t), ct.byref(ms)))
        return t.as_dict(), ms.value

    def set_stream(self, stream):
        self._check(self._lib.dfl_set_stream(self._h, _stream_ptr(stream)))

    def static(self):
        self._check(self._lib.dfl_static(self._h))

    def apply_batch(self, dels, ins, check: bool = True) -> int:
        """dels/ins: (k, 3) uint32 arrays (u, v, w) or CUDA tensors (int32/uint32)."""
        d, mk1, k0 = _buf(dels, np.uint32)
        i, mk2, k1 = _buf(ins, np.uint32)
        nd = int(dels.shape[0]) if dels is not None else 0
        ni = int(ins.shape[0]) if ins is not None else 0
        mk = mk1 if nd else mk2
        rc = self._lib.dfl_apply_batch(self._h, d, nd, i, ni, mk)
        if check:
            self._check(rc)
        return rc

    def update(self, mode: int):
        self._check(self._lib.dfl_update(self._h, mode))

    def step(self, dels, ins, mode: int | None = None, check: bool = True) -> int:
        """apply_batch(dels, ins) then update(mode) in one call (dfl_step);
        mode defaults to DF."""
        d, mk1, k0 = _buf(dels, np.uint32)
        i, mk2, k1 = _buf(ins, np.uint32)
        nd = int(dels.shape[0]) if dels is not None else 0
        ni = int(ins.shape[0]) if ins is not None else 0
        mk = mk1 if nd else mk2
        rc = self._lib.dfl_step(self._h, d, nd, i, ni, mk, DF if mode is None else mode)
        if check:
            self._check(rc)
        return rc

    def membership(self, out=None):
        if out is None:
            out = np.zeros(self.n, np.uint32)
        p, mk, _ = _buf(out, np.uint32)
        self._check(self._lib.dfl_membership(self._h, p, mk))
        return out

    def modularity(self):
        q = ct.c_double()
        parts = np.zeros(4, np.int64)
        self._check(self._lib.dfl_modularity(self._h, ct.byref(q), parts.ctypes.data_as(ct.c_void_p)))
        return q.value, _i128(int(parts[0]), int(parts[1])), _i128(int(parts[2]), int(parts[3]))

    def weights(self):
        K = np.zeros(self.n, np.int64)
        S = np.zeros(self.n, np.int64)
        m2 = ct.c_int64()
        self._check(self._lib.dfl_weights(self._h, K.ctypes.data_as(ct.c_void_p),
                                          S.ctypes.data_as(ct.c_void_p), ct.byref(m2), MEM_HOST))
        return K, S, int(m2.value)

    def num_arcs(self) -> int:
        na = ct.c_uint64()
        self._check(self._lib.dfl_num_arcs(self._h, ct.byref(na)))
        return int(na.value)

    def graph(self):
        na = self.num_arcs()
        off = np.zeros(self.n + 1, np.uint64)
        idx = np.zeros(max(na, 1), np.uint32)
        w = np.zeros(max(na, 1), np.uint32)
        self._check(self._lib.dfl_graph(self._h, off.ctypes.data_as(ct.c_void_p),
                                        idx.ctypes.data_as(ct.c_void_p),
                                        w.ctypes.data_as(ct.c_void_p), MEM_HOST))
        return off, idx[:na], w[:na]

    def stats(self) -> dict:
        s = Stats()
        self._check(self._lib.dfl_stats(self._h, ct.byref(s)))
        return {"passes": s.passes, "iterations": list(s.iterations)[: s.passes],
                "affected_initial": s.affected_initial, "affected_ever": s.affected_ever,
                "kernel_launches": s.kernel_launches, "num_arcs": s.num_arcs,
                "arc_pool": s.arc_pool, "max_degree": s.max_degree,
                "num_communities": s.num_communities, "graph_captures": s.graph_captures,
                "graph_capture_ms": s.graph_capture_ms}

    def profile(self, reset: bool = False) -> dict:
        p = Profile()
        self._check(self._lib.dfl_profile(self._h, ct.byref(p), 1 if reset else 0))
        return {PROF_NAMES[k]: {"launches": p.launches[k], "ms": p.ms[k], "bytes": p.bytes[k]}
                for k in range(len(PROF_NAMES))}

    def trace(self):
        ln = ct.c_uint32()
        self._check(self._lib.dfl_trace(self._h, None, 0, ct.byref(ln)))
        out = np.zeros(4 * max(ln.value, 1), np.uint64)
        self._check(self._lib.dfl_trace(self._h, out.ctypes.data_as(ct.c_void_p), ln.value,
                                        ct.byref(ln)))
        return [(int(out[4 * k]), int(out[4 * k + 1]), (int(out[4 * k + 2]) << 64) | int(out[4 * k + 3]))
                for k in range(ln.value)]

    def set_membership(self, C):
        p, mk, _ = _buf(C, np.uint32)
        self._check(self._lib.dfl_set_membership(self._h, p, mk))

    def compact(self):
        """dfl_compact: rewrite the arc pool densely; (slots before, after)."""
        b, a = ct.c_uint64(), ct.c_uint64()
        self._check(self._lib.dfl_compact(self._h, ct.byref(b), ct.byref(a)))
        return int(b.value), int(a.value)

    def checkpoint(self) -> dict:
        """Everything later updates depend on, as host arrays: the graph
        (compact CSR, rows sorted), the membership and the launch tuning.  K
        and Sigma are functions of these and are recomputed on restore.  Take
        it between updates (a pending batch is not part of it)."""
        off, idx, w = self.graph()
        return {"n": self.n, "offsets": off, "indices": idx, "weights": w,
                "membership": self.membership().copy(), "tuning": self.tuning()}

    @classmethod
    def restore(cls, ck: dict, options: Options | None = None, stream=None) -> "Dfl":
        """A handle in the state a checkpoint recorded (dfl_create from its
        graph, then dfl_set_tuning and dfl_set_membership)."""
        h = cls(ck["n"], ck["offsets"], ck["indices"], ck["weights"], options=options, stream=stream)
        h.set_tuning(**{k: int(v) for k, v in ck["tuning"].items()})
        h.set_membership(np.ascontiguousarray(ck["membership"], np.uint32))
        return h

    def mark(self, mode: int):
        F = np.zeros(self.n, np.uint8)
        R = np.zeros(self.n, np.uint8)
        self._check(self._lib.dfl_mark(self._h, mode, F.ctypes.data_as(ct.c_void_p),
                                       R.ctypes.data_as(ct.c_void_p), MEM_HOST))
        return F, R

    def louvain_from(self, F0, R0):
        f, _, k0 = _buf(np.asarray(F0, np.uint8), np.uint8)
        r, _, k1 = _buf(np.asarray(R0, np.uint8), np.uint8)
        self._check(self._lib.dfl_louvain_from(self._h, f, r, MEM_HOST))

    def move_iteration(self, F, R):
        F = np.array(F, np.uint8)
        R = np.ascontiguousarray(R, np.uint8)
        moved = np.zeros(self.n, np.uint8)
        dq = np.zeros(2, np.int64)
        self._check(self._lib.dfl_move_iteration(self._h, F.ctypes.data_as(ct.c_void_p),
                                                 R.ctypes.data_as(ct.c_void_p),
                                                 moved.ctypes.data_as(ct.c_void_p),
                                                 dq.ctypes.data_as(ct.c_void_p), MEM_HOST))
        return F, moved, (int(dq[0]) << 64) | (int(dq[1]) & 0xFFFFFFFFFFFFFFFF)

    def aggregate(self):
        nv = ct.c_uint32()
        na = ct.c_uint64()
        self._check(self._lib.dfl_aggregate(self._h, ct.byref(nv), ct.byref(na), None, None, None))
        off = np.zeros(nv.value + 1, np.uint64)
        idx = np.zeros(max(na.value, 1), np.uint32)
        w = np.zeros(max(na.value, 1), np.uint64)
        self._check(self._lib.dfl_aggregate(self._h, ct.byref(nv), ct.byref(na),
                                            off.ctypes.data_as(ct.c_void_p),
                                            idx.ctypes.data_as(ct.c_void_p),
                                            w.ctypes.data_as(ct.c_void_p)))
        return off, idx[: na.value], w[: na.value]


class DflGroup(Dfl):
    """Many independent graphs in one handle (dfl_group_*): one launch per
    step covers every graph, each graph gets the result a Dfl of its own
    would.  graphs: list of (n, offsets, indices, weights) host CSR arrays."""

    def __init__(self, graphs, options: Options | None = None, stream=None):
        lib = load()
        self._lib = lib
        G = len(graphs)
        self.sizes = [int(g[0]) for g in graphs]
        self._keep = []
        ns = np.array(self.sizes, np.uint32)
        ptrs = {k: (ct.c_void_p * G)() for k in ("off", "idx", "w")}
        for g, (n, off, idx, w) in enumerate(graphs):
            a = np.ascontiguousarray(off, np.uint64)
            b = np.ascontiguousarray(idx, np.uint32)
            c = np.ascontiguousarray(w, np.uint32)
            self._keep += [a, b, c]
            ptrs["off"][g] = a.ctypes.data
            ptrs["idx"][g] = b.ctypes.data
            ptrs["w"][g] = c.ctypes.data
        h = ct.c_void_p()
        rc = lib.dfl_group_create(ct.byref(h), G, ns.ctypes.data_as(ct.c_void_p),
                                  ct.cast(ptrs["off"], ct.c_void_p), ct.cast(ptrs["idx"], ct.c_void_p),
                                  ct.cast(ptrs["w"], ct.c_void_p),
                                  ct.byref(options) if options is not None else None, _stream_ptr(stream))
        self._keep = []
        if rc != 0:
            raise DflError(rc, "dfl_group_create")
        self._h = h
        self.n = int(sum(self.sizes))
        self.ngraphs = G

    def static(self):
        self._check(self._lib.dfl_group_static(self._h))

    def apply_batches(self, dels, ins, check: bool = True) -> int:
        """dels/ins: per graph (k, 3) uint32 arrays with local vertex ids
        (host), or a pair (CUDA int32 tensor of all edges, offsets)."""
        if isinstance(dels, tuple):
            (d, doff), (i, ioff) = dels, ins
            dp, mk, k0 = _buf(d, np.uint32)
            ip, _, k1 = _buf(i, np.uint32)
        else:
            doff = np.concatenate([[0], np.cumsum([x.shape[0] for x in dels])]).astype(np.uint64)
            ioff = np.concatenate([[0], np.cumsum([x.shape[0] for x in ins])]).astype(np.uint64)
            d = np.concatenate([np.asarray(x, np.uint32).reshape(-1, 3) for x in dels]) if dels else np.zeros((0, 3), np.uint32)
            i = np.concatenate([np.asarray(x, np.uint32).reshape(-1, 3) for x in ins]) if ins else np.zeros((0, 3), np.uint32)
            dp, mk, k0 = _buf(d, np.uint32)
            ip, _, k1 = _buf(i, np.uint32)
        doff = np.ascontiguousarray(doff, np.uint64)
        ioff = np.ascontiguousarray(ioff, np.uint64)
        rc = self._lib.dfl_group_apply_batch(self._h, dp, doff.ctypes.data_as(ct.c_void_p), ip,
                                             ioff.ctypes.data_as(ct.c_void_p), mk)
        if check:
            self._check(rc)
        return rc

    def update(self, mode: int):
        self._check(self._lib.dfl_group_update(self._h, mode))

    def graph_membership(self, g: int, out=None):
        if out is None:
            out = np.zeros(self.sizes[g], np.uint32)
        p, mk, _ = _buf(out, np.uint32)
        self._check(self._lib.dfl_group_membership(self._h, g, p, mk))
        return out

    def graph_modularity(self, g: int):
        q = ct.c_double()
        parts = np.zeros(4, np.int64)
        self._check(self._lib.dfl_group_modularity(self._h, g, ct.byref(q),
                                                   parts.ctypes.data_as(ct.c_void_p)))
        return q.value, _i128(int(parts[0]), int(parts[1])), _i128(int(parts[2]), int(parts[3]))

    def graph_stats(self, g: int) -> dict:
        s = Stats()
        self._check(self._lib.dfl_group_stats(self._h, g, ct.byref(s)))
        return {"passes": s.passes, "iterations": list(s.iterations)[: s.passes],
                "num_communities": s.num_communities}


def __getattr__(name):
    # module-level access to the raw C functions under their C names
    if name in _SIGS:
        return getattr(load(), name)
    raise AttributeError(name)
