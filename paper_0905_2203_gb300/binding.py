"""ctypes binding of libfem.so (include/fem.h).

Argument marshalling only: every step of counting and mining runs in the
library's CUDA kernels.  Functions keep the C names (fem_*) and take either
numpy arrays (host memory) or CUDA torch tensors (device memory; their data
pointers are passed with the *_is_device flag set).  If libfem.so has not been
built this module raises ImportError: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfem.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with paper_0905_2203_gb300.build.build() "
        "(nvcc, sm_103a). The library has no CPU fallback.")

_lib = ctypes.CDLL(LIB_PATH)

FEM_OK = 0
FEM_ERR_INVAL = -1
FEM_ERR_UNSORTED = -2
FEM_ERR_DUP = -3
FEM_ERR_RANGE = -4
FEM_ERR_NOMEM = -5
FEM_ERR_TIMEOUT = -6
FEM_ERR_CUDA = -7
FEM_ERR_BUSY = -8
FEM_ERR_NOTFOUND = -9
FEM_MAX_NODES = 16

VP = ctypes.c_void_p
I32 = ctypes.c_int
I64 = ctypes.c_int64
U32 = ctypes.c_uint32
U64 = ctypes.c_uint64
SZ = ctypes.c_size_t


class fem_cands(ctypes.Structure):
    _fields_ = [("n_cand", I64), ("offs", VP), ("types", VP), ("lo", VP), ("hi", VP),
                ("ptr_is_device", I32)]


class fem_tuning(ctypes.Structure):
    _fields_ = [("lanes_per_cta", I32), ("segments", I32), ("tile_events", I32), ("prepass", I32),
                ("plain_path", I32), ("autotune", I32), ("kernel", I32), ("level_graph", I32),
                ("wait_polls", I32), ("track_last", I32)]


class fem_stats(ctypes.Structure):
    _fields_ = [("episode_events", ctypes.c_double), ("counted_episode_events", ctypes.c_double),
                ("relevant_events", ctypes.c_double),
                ("candidates_counted", I64), ("candidates_pruned", I64),
                ("fallback_recounts", I64), ("kernel_launches", I64), ("sparse_launches", I64),
                ("count_kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("levels", I32), ("graph_tails", I32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fem_job_info(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("finish_s", ctypes.c_double), ("n_events", I64), ("levels", I32),
                ("candidates_counted", I64), ("episode_events", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "fem_ctx_create": (I32, [I32, SZ, VP, ctypes.POINTER(VP)]),
    "fem_ctx_destroy": (None, [VP]),
    "fem_ctx_set_tuning": (I32, [VP, ctypes.POINTER(fem_tuning)]),
    "fem_ctx_last_stats": (I32, [VP, ctypes.POINTER(fem_stats)]),
    "fem_ctx_memory": (I32, [VP, ctypes.POINTER(SZ), ctypes.POINTER(SZ)]),
    "fem_ctx_set_autotune_cache": (I32, [VP, ctypes.c_char_p]),
    "fem_load_stream": (I32, [VP, VP, VP, I64, U32, I32, ctypes.POINTER(VP)]),
    "fem_stream_free": (None, [VP]),
    "fem_stream_info": (I32, [VP, ctypes.POINTER(I64), ctypes.POINTER(U32)]),
    "fem_stream_freq": (I32, [VP, VP, VP, I32]),
    "fem_count_episodes": (I32, [VP, VP, ctypes.POINTER(fem_cands), VP, I32]),
    "fem_count_batch": (I32, [VP, VP, I32, ctypes.POINTER(fem_cands), VP, VP, I32]),
    "fem_count_episodes_plain": (I32, [VP, VP, ctypes.POINTER(fem_cands), VP, I32]),
    "fem_upper_bound": (I32, [VP, VP, ctypes.POINTER(fem_cands), VP, I32]),
    "fem_upper_bound_coarse": (I32, [VP, VP, ctypes.POINTER(fem_cands), I32, VP, I32, ctypes.POINTER(I32)]),
    "fem_count_episodes_noalloc": (I32, [VP, VP, I64, VP, VP, VP, VP, I64, VP, VP]),
    "fem_mine_levelwise": (I32, [VP, VP, I32, VP, VP, I32, VP, I32, ctypes.POINTER(VP)]),
    "fem_result_level": (I32, [VP, I32, I32, ctypes.POINTER(I64), ctypes.POINTER(VP),
                               ctypes.POINTER(VP), ctypes.POINTER(VP), ctypes.POINTER(VP),
                               ctypes.POINTER(VP)]),
    "fem_result_stats": (I32, [VP, ctypes.POINTER(fem_stats)]),
    "fem_result_free": (None, [VP]),
    "fem_server_create": (I32, [I32, SZ, I32, ctypes.POINTER(VP)]),
    "fem_server_submit": (I32, [VP, VP, VP, I64, U32, VP, VP, I32, U32, I32,
                                ctypes.POINTER(U64)]),
    "fem_server_wait": (I32, [VP, U64, I32, ctypes.POINTER(VP), ctypes.POINTER(fem_job_info)]),
    "fem_server_destroy": (None, [VP]),
    "fem_session_create": (I32, [VP, ctypes.POINTER(fem_cands), U32, ctypes.POINTER(VP)]),
    "fem_session_append": (I32, [VP, VP, VP, I64, I32]),
    "fem_session_counts": (I32, [VP, VP, I32]),
    "fem_session_info": (I32, [VP, ctypes.POINTER(I64), ctypes.POINTER(I64)]),
    "fem_session_destroy": (None, [VP]),
    "fem_strerror": (ctypes.c_char_p, [I32]),
    "fem_version": (ctypes.c_char_p, []),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class FemError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = fem_strerror(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def check(status: int, what: str = "") -> None:
    if status != FEM_OK:
        raise FemError(status, what)


# ---------------------------------------------------------------------------
# Pointer marshalling

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, is_device, keepalive) for a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        import torch
        # same-width integer tensors are passed bit-for-bit (torch has few
        # unsigned kernels, so int16 / int32 tensors may carry uint16 / uint32)
        want = {np.uint16: (torch.uint16, torch.int16), np.int32: (torch.int32,),
                np.int64: (torch.int64,), np.uint32: (torch.uint32, torch.int32)}[dtype]
        if x.dtype not in want:
            raise TypeError(f"expected torch {want}, got {x.dtype}")
        x = x.contiguous()
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), 0, a


class Cands:
    """Candidate set in CSR form (numpy arrays or CUDA torch tensors)."""

    def __init__(self, offs, types, lo, hi):
        self.offs, d0, self._k0 = _ptr(offs, np.int64)
        self.types, d1, self._k1 = _ptr(types, np.uint16)
        self.lo, d2, self._k2 = _ptr(lo if len(lo) else np.zeros(1, np.int32), np.int32)
        self.hi, d3, self._k3 = _ptr(hi if len(hi) else np.zeros(1, np.int32), np.int32)
        if len({d0, d1, d2, d3}) != 1:
            raise ValueError("candidate arrays must all be host or all be device")
        self.is_device = d0
        self.n = int(len(offs) - 1)
        self.c = fem_cands(self.n, self.offs, self.types, self.lo, self.hi, d0)


class Context:
    """A library context on one device, optionally bound to a torch stream."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, cuda_stream=None):
        h = VP()
        st = None
        if cuda_stream is not None:
            st = VP(int(cuda_stream))
        check(fem_ctx_create(device, hbm_budget_bytes, st, ctypes.byref(h)), "fem_ctx_create")
        self.h = h
        self.device = device

    def close(self):
        if self.h:
            fem_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, lanes_per_cta=0, segments=0, tile_events=0, prepass=0, plain_path=0, autotune=0,
                   kernel=0, level_graph=0, wait_polls=0, track_last=0):
        t = fem_tuning(lanes_per_cta, segments, tile_events, prepass, plain_path, autotune, kernel, level_graph,
                       wait_polls, track_last)
        check(fem_ctx_set_tuning(self.h, ctypes.byref(t)), "fem_ctx_set_tuning")

    def reset_tuning(self):
        check(fem_ctx_set_tuning(self.h, None), "fem_ctx_set_tuning")

    def set_autotune_cache(self, path):
        check(fem_ctx_set_autotune_cache(self.h, None if path is None else str(path).encode()),
              "fem_ctx_set_autotune_cache")

    def last_stats(self) -> dict:
        s = fem_stats()
        check(fem_ctx_last_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def memory(self):
        u, b = SZ(), SZ()
        check(fem_ctx_memory(self.h, ctypes.byref(u), ctypes.byref(b)))
        return int(u.value), int(b.value)

    def load_stream(self, types, times, n_types: int) -> "Stream":
        tp, d0, k0 = _ptr(types, np.uint16)
        mp, d1, k1 = _ptr(times, np.int32)
        if d0 != d1:
            raise ValueError("types and times must both be host or both be device")
        h = VP()
        check(fem_load_stream(self.h, tp, mp, int(len(types)), int(n_types), d0, ctypes.byref(h)),
              "fem_load_stream")
        return Stream(self, h, int(len(types)), int(n_types))

    def _count(self, fn, stream, cands: Cands, out, what):
        if out is None:
            out = np.zeros(max(cands.n, 1), np.uint32)[: cands.n]
        op, od, keep = _ptr(out, np.uint32)
        check(fn(self.h, stream.h, ctypes.byref(cands.c), op, od), what)
        return keep

    def count_episodes(self, stream, cands: Cands, out=None):
        return self._count(fem_count_episodes, stream, cands, out, "fem_count_episodes")

    def count_episodes_plain(self, stream, cands: Cands, out=None):
        return self._count(fem_count_episodes_plain, stream, cands, out, "fem_count_episodes_plain")

    def upper_bound(self, stream, cands: Cands, out=None):
        return self._count(fem_upper_bound, stream, cands, out, "fem_upper_bound")

    def upper_bound_coarse(self, stream, cands: Cands, tick: int = 0, out=None):
        """Coarse-tick upper bound (fem_upper_bound_coarse): (ub, tick used)."""
        if out is None:
            out = np.zeros(max(cands.n, 1), np.uint32)[: cands.n]
        op, od, keep = _ptr(out, np.uint32)
        w = I32()
        check(fem_upper_bound_coarse(self.h, stream.h, ctypes.byref(cands.c), int(tick), op, od, ctypes.byref(w)),
              "fem_upper_bound_coarse")
        return keep, int(w.value)

    def count_batch(self, streams, cands: Cands, rec_id, out=None):
        arr = (VP * len(streams))(*[s.h for s in streams])
        rp, rd, rk = _ptr(rec_id, np.uint32)
        if rd != cands.is_device:
            raise ValueError("rec_id must live where the candidate arrays live")
        if out is None:
            out = np.zeros(max(cands.n, 1), np.uint32)[: cands.n]
        op, od, keep = _ptr(out, np.uint32)
        check(fem_count_batch(self.h, arr, len(streams), ctypes.byref(cands.c), rp, op, od),
              "fem_count_batch")
        return keep

    def session(self, cands: Cands, n_types: int) -> "Session":
        return Session(self, cands, n_types)

    def mine_levelwise(self, streams, bins, thresholds, max_size: int) -> "Result":
        arr = (VP * len(streams))(*[s.h for s in streams])
        blo = np.ascontiguousarray([b[0] for b in bins], np.int32)
        bhi = np.ascontiguousarray([b[1] for b in bins], np.int32)
        thr = np.ascontiguousarray(thresholds, np.uint32)
        h = VP()
        check(fem_mine_levelwise(self.h, arr, len(streams), VP(blo.ctypes.data), VP(bhi.ctypes.data),
                                 len(bins), VP(thr.ctypes.data), int(max_size), ctypes.byref(h)),
              "fem_mine_levelwise")
        return Result(h, len(streams), int(max_size))


class Session:
    """Exact counts of a fixed candidate set over a stream that grows by
    appends (fem_session_*): counts() equals count_episodes on the
    concatenation of every appended chunk."""

    def __init__(self, ctx: Context, cands: Cands, n_types: int):
        self.ctx, self.n = ctx, cands.n
        self.h = VP()
        check(fem_session_create(ctx.h, ctypes.byref(cands.c), int(n_types), ctypes.byref(self.h)),
              "fem_session_create")

    def append(self, types, times):
        tp, d0, k0 = _ptr(types, np.uint16)
        mp, d1, k1 = _ptr(times, np.int32)
        if d0 != d1:
            raise ValueError("types and times must both be host or both be device")
        check(fem_session_append(self.h, tp, mp, int(len(types)), d0), "fem_session_append")

    def counts(self, out=None):
        if out is None:
            out = np.zeros(max(self.n, 1), np.uint32)[: self.n]
        op, od, keep = _ptr(out, np.uint32)
        check(fem_session_counts(self.h, op, od), "fem_session_counts")
        return keep

    def info(self):
        seen, tail = I64(), I64()
        check(fem_session_info(self.h, ctypes.byref(seen), ctypes.byref(tail)), "fem_session_info")
        return int(seen.value), int(tail.value)

    def close(self):
        if self.h:
            fem_session_destroy(self.h)
            self.h = None


class Stream:
    def __init__(self, ctx: Context, h, n: int, n_types: int):
        self.ctx, self.h, self.n, self.n_types = ctx, h, n, n_types

    def free(self):
        if self.h:
            fem_stream_free(self.h)
            self.h = None

    def freq(self, out=None):
        if out is None:
            out = np.zeros(self.n_types, np.uint32)
        op, od, _ = _ptr(out, np.uint32)
        check(fem_stream_freq(self.ctx.h, self.h, op, od), "fem_stream_freq")
        return out


class Result:
    def __init__(self, h, n_recs: int, max_size: int):
        self.h, self.n_recs, self.max_size = h, n_recs, max_size

    def level_arrays(self, rec: int, level: int):
        """One recording's frequent episodes of one level as numpy arrays in
        the CSR layout of fem_result_level: (offs[n+1], types, lo, hi,
        counts[n]) -- copies of the result's arrays, no per-episode objects."""
        n = I64()
        po, pt, pl, ph, pc = VP(), VP(), VP(), VP(), VP()
        check(fem_result_level(self.h, rec, level, ctypes.byref(n), ctypes.byref(po),
                               ctypes.byref(pt), ctypes.byref(pl), ctypes.byref(ph),
                               ctypes.byref(pc)), "fem_result_level")
        n = int(n.value)
        if n == 0:
            z = np.zeros(0, np.int32)
            return np.zeros(1, np.int64), np.zeros(0, np.uint16), z, z.copy(), np.zeros(0, np.uint32)
        offs = np.ctypeslib.as_array(ctypes.cast(po, ctypes.POINTER(I64)), (n + 1,)).copy()
        nn = int(offs[-1])
        types = np.ctypeslib.as_array(ctypes.cast(pt, ctypes.POINTER(ctypes.c_uint16)), (nn,)).copy()
        ne = nn - n
        lo = (np.ctypeslib.as_array(ctypes.cast(pl, ctypes.POINTER(I32)), (ne,)).copy()
              if ne else np.zeros(0, np.int32))
        hi = (np.ctypeslib.as_array(ctypes.cast(ph, ctypes.POINTER(I32)), (ne,)).copy()
              if ne else np.zeros(0, np.int32))
        counts = np.ctypeslib.as_array(ctypes.cast(pc, ctypes.POINTER(U32)), (n,)).copy()
        return offs, types, lo, hi, counts

    def level(self, rec: int, level: int):
        """(list of (types, lo, hi) tuples, counts list) for one recording and level."""
        n = I64()
        po, pt, pl, ph, pc = VP(), VP(), VP(), VP(), VP()
        check(fem_result_level(self.h, rec, level, ctypes.byref(n), ctypes.byref(po),
                               ctypes.byref(pt), ctypes.byref(pl), ctypes.byref(ph),
                               ctypes.byref(pc)), "fem_result_level")
        n = int(n.value)
        if n == 0:
            return [], []
        offs = np.ctypeslib.as_array(ctypes.cast(po, ctypes.POINTER(I64)), (n + 1,)).copy()
        nn = int(offs[-1])
        types = np.ctypeslib.as_array(ctypes.cast(pt, ctypes.POINTER(ctypes.c_uint16)), (nn,)).copy()
        ne = nn - n
        lo = (np.ctypeslib.as_array(ctypes.cast(pl, ctypes.POINTER(I32)), (ne,)).copy()
              if ne else np.zeros(0, np.int32))
        hi = (np.ctypeslib.as_array(ctypes.cast(ph, ctypes.POINTER(I32)), (ne,)).copy()
              if ne else np.zeros(0, np.int32))
        counts = np.ctypeslib.as_array(ctypes.cast(pc, ctypes.POINTER(U32)), (n,)).copy()
        eps = []
        for c in range(n):
            o, p = int(offs[c]), int(offs[c + 1])
            eo = o - c
            eps.append((tuple(int(x) for x in types[o:p]), tuple(int(x) for x in lo[eo:eo + p - o - 1]),
                        tuple(int(x) for x in hi[eo:eo + p - o - 1])))
        return eps, [int(x) for x in counts]

    def stats(self) -> dict:
        s = fem_stats()
        check(fem_result_stats(self.h, ctypes.byref(s)))
        return s.as_dict()

    def free(self):
        if self.h:
            fem_result_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Serving loop for level-wise mining jobs (fem_server_*): admission by
    device memory, device-resident streams, continuous batching."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_jobs: int = 16):
        h = VP()
        check(fem_server_create(device, hbm_budget_bytes, max_jobs, ctypes.byref(h)), "fem_server_create")
        self.h = h

    def submit(self, types, times, n_types: int, bins, threshold: int, max_size: int) -> int:
        ty = np.ascontiguousarray(types, np.uint16)
        tm = np.ascontiguousarray(times, np.int32)
        blo = np.ascontiguousarray([b[0] for b in bins] or [0], np.int32)
        bhi = np.ascontiguousarray([b[1] for b in bins] or [1], np.int32)
        jid = U64()
        check(fem_server_submit(self.h, VP(ty.ctypes.data), VP(tm.ctypes.data), len(ty), int(n_types),
                                VP(blo.ctypes.data), VP(bhi.ctypes.data), len(bins), int(threshold),
                                int(max_size), ctypes.byref(jid)), "fem_server_submit")
        return int(jid.value)

    def wait(self, job_id: int, timeout_ms: int = -1):
        """(Result, info dict) of a finished job."""
        h = VP()
        info = fem_job_info()
        st = fem_server_wait(self.h, int(job_id), int(timeout_ms), ctypes.byref(h), ctypes.byref(info))
        check(st, "fem_server_wait")
        return Result(h, 1, 0), info.as_dict()

    def close(self):
        if self.h:
            fem_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def count_episodes_noalloc(types, times, offs, ep_types, lo, hi, out, cuda_stream=None):
    """Counts with no memory allocation (fem_count_episodes_noalloc): every
    argument is a CUDA torch tensor owned by the caller; `out` (uint32 or
    int32, n_cand) receives the counts.  Every tensor must sit on the current
    CUDA device; the work runs on `cuda_stream`, by default torch's current
    stream.  For callers that cannot allocate device memory at call time; see
    include/fem.h for the scratch limits and the rule that overlapping calls
    on one device must be serialised."""
    import torch
    ptrs = []
    cur = torch.cuda.current_device()
    for x, dt in ((types, np.uint16), (times, np.int32), (offs, np.int64), (ep_types, np.uint16),
                  (lo, np.int32), (hi, np.int32), (out, np.uint32)):
        p, dev, _ = _ptr(x, dt)
        if not dev:
            raise ValueError("fem_count_episodes_noalloc takes device tensors only")
        if x.device.index != cur:
            raise ValueError(f"fem_count_episodes_noalloc: tensor on {x.device}, current device is cuda:{cur}")
        ptrs.append(p)
    # default: torch's current stream, so the inputs written there are ordered
    # before the kernels (torch's streams do not synchronise with the legacy
    # default stream)
    if cuda_stream is None:
        cuda_stream = torch.cuda.current_stream(out.device).cuda_stream
    st = VP(int(cuda_stream)) if cuda_stream else None
    check(fem_count_episodes_noalloc(ptrs[0], ptrs[1], int(len(types)), ptrs[2], ptrs[3], ptrs[4], ptrs[5],
                                     int(len(offs) - 1), ptrs[6], st), "fem_count_episodes_noalloc")
    return out


def version() -> str:
    return fem_version().decode()
