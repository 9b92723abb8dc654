"""Error behaviour of the C ABI that needs no GPU: every entry point checks
its handles and pointers before touching the device, and returns
FEM_ERR_INVAL (or does nothing, for the void destructors) on a null one."""
import ctypes

import numpy as np

from paper_0905_2203_gb300 import binding as fb

INVAL = fb.FEM_ERR_INVAL


def _cands():
    offs = np.array([0, 2], np.int64)
    ty = np.array([0, 1], np.uint16)
    lo = np.array([0], np.int32)
    hi = np.array([5], np.int32)
    c = fb.Cands(offs, ty, lo, hi)
    return c


def test_null_handles_are_rejected():
    c = _cands()
    u32 = np.zeros(4, np.uint32)
    p = ctypes.c_void_p(u32.ctypes.data)
    out = ctypes.c_void_p()
    w = ctypes.c_int()
    i64 = ctypes.c_int64()
    assert fb.fem_ctx_set_tuning(None, None) == INVAL
    assert fb.fem_ctx_set_autotune_cache(None, None) == INVAL
    assert fb.fem_ctx_last_stats(None, None) == INVAL
    assert fb.fem_ctx_memory(None, None, None) == INVAL
    assert fb.fem_load_stream(None, p, p, 1, 2, 0, ctypes.byref(out)) == INVAL
    assert fb.fem_stream_info(None, None, None) == INVAL
    assert fb.fem_stream_freq(None, None, p, 0) == INVAL
    assert fb.fem_count_episodes(None, None, ctypes.byref(c.c), p, 0) == INVAL
    assert fb.fem_count_batch(None, None, 1, ctypes.byref(c.c), p, p, 0) == INVAL
    assert fb.fem_count_episodes_plain(None, None, ctypes.byref(c.c), p, 0) == INVAL
    assert fb.fem_upper_bound(None, None, ctypes.byref(c.c), p, 0) == INVAL
    assert fb.fem_upper_bound_coarse(None, None, ctypes.byref(c.c), 0, p, 0, ctypes.byref(w)) == INVAL
    assert fb.fem_mine_levelwise(None, None, 1, p, p, 1, p, 3, ctypes.byref(out)) == INVAL
    assert fb.fem_result_level(None, 0, 1, ctypes.byref(i64), None, None, None, None, None) == INVAL
    assert fb.fem_result_stats(None, None) == INVAL
    assert fb.fem_session_create(None, ctypes.byref(c.c), 2, ctypes.byref(out)) == INVAL
    assert fb.fem_session_append(None, p, p, 1, 0) == INVAL
    assert fb.fem_session_counts(None, p, 0) == INVAL
    assert fb.fem_session_info(None, None, None) == INVAL
    assert fb.fem_server_submit(None, p, p, 1, 2, p, p, 1, 1, 3, None) == INVAL
    assert fb.fem_server_wait(None, 0, 0, ctypes.byref(out), None) == INVAL
    # destructors take null
    fb.fem_stream_free(None)
    fb.fem_result_free(None)
    fb.fem_session_destroy(None)
    fb.fem_server_destroy(None)
    fb.fem_ctx_destroy(None)


def test_every_status_has_a_message():
    assert fb.fem_strerror(fb.FEM_OK) == b"ok"
    codes = [fb.FEM_ERR_INVAL, fb.FEM_ERR_UNSORTED, fb.FEM_ERR_DUP, fb.FEM_ERR_RANGE, fb.FEM_ERR_NOMEM,
             fb.FEM_ERR_TIMEOUT, fb.FEM_ERR_CUDA, fb.FEM_ERR_BUSY, fb.FEM_ERR_NOTFOUND]
    msgs = [fb.fem_strerror(c) for c in codes]
    assert all(m != b"unknown status" for m in msgs) and len(set(msgs)) == len(msgs)
    assert fb.fem_strerror(-1000) == b"unknown status"
