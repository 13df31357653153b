"""Thin ctypes binding of libjde (include/jde.h): same names, argument marshalling only.

Every computation happens in the CUDA library.  Device memory is passed as
raw pointers; ``torch`` tensors are accepted wherever a pointer is expected
(their ``data_ptr()`` is used), host numpy arrays where host memory is
expected.  Importing this module loads ``libjde.so`` and fails loudly if it
has not been built (``python -m paper_2011_03910_gb300._build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libjde.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libjde.so is not built ({_LIB_PATH}); run python -m paper_2011_03910_gb300._build")
lib = C.CDLL(_LIB_PATH)

JDE_OK = 0
JDE_FP32, JDE_BF16, JDE_FP8_E4M3 = 0, 1, 2
JDE_TRACK_TRACKED, JDE_TRACK_LOST, JDE_TRACK_UNCONFIRMED = 1, 2, 3
JDE_ROW, JDE_EMB, JDE_NUM_LAYERS = 518, 512, 78
STATUS = {0: "JDE_OK", 1: "JDE_ERR_INVALID_ARG", 2: "JDE_ERR_OOM", 3: "JDE_ERR_CUDA", 4: "JDE_ERR_CAPACITY",
          5: "JDE_ERR_ADMISSION", 6: "JDE_ERR_TIMEOUT", 7: "JDE_ERR_NOT_FOUND", 8: "JDE_ERR_WEIGHTS",
          9: "JDE_ERR_UNSUPPORTED"}


class jde_config(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_batch", C.c_int), ("max_in_w", C.c_int), ("max_in_h", C.c_int),
                ("max_src_w", C.c_int), ("max_src_h", C.c_int), ("max_cand", C.c_int), ("conf_thresh", C.c_float),
                ("nms_iou", C.c_float), ("assign_thresh", C.c_float), ("gate_chi2", C.c_double),
                ("lost_max_frames", C.c_int), ("emb_momentum", C.c_float), ("max_streams", C.c_int),
                ("max_tracks", C.c_int), ("max_track_dets", C.c_int), ("device", C.c_int),
                ("keep_layer_outputs", C.c_int), ("sparse_emb", C.c_int), ("assoc_cascade", C.c_int),
                ("motion_lambda", C.c_double), ("iou_cost2", C.c_double), ("iou_cost3", C.c_double),
                ("fuse_block1", C.c_int), ("dependent_launch", C.c_int)]


class jde_layer_desc(C.Structure):
    _fields_ = [("cin", C.c_int), ("cout", C.c_int), ("k", C.c_int), ("stride", C.c_int), ("has_bn", C.c_int),
                ("res_nblocks", C.c_int)]


class jde_dets(C.Structure):
    _fields_ = [("rows", C.c_void_p), ("count", C.c_void_p), ("anchor_index", C.c_void_p), ("cap", C.c_int),
                ("on_device", C.c_int)]


class jde_tracks(C.Structure):
    _fields_ = [("id", C.c_void_p), ("box", C.c_void_p), ("state", C.c_void_p), ("det", C.c_void_p),
                ("count", C.c_void_p), ("cap", C.c_int), ("on_device", C.c_int)]


_P = C.c_void_p


class jde_server_config(C.Structure):
    _fields_ = [("group", jde_config), ("src_w", C.c_int), ("src_h", C.c_int), ("max_streams_per_group", C.c_int),
                ("hbm_budget_bytes", C.c_size_t), ("det_cap", C.c_int), ("track_cap", C.c_int),
                ("caller_heads", C.c_int), ("collect_net_heads", C.c_int), ("use_graphs", C.c_int),
                ("prewarm", C.c_int)]


class jde_frame_out(C.Structure):
    _fields_ = [("track_id", _P), ("track_box", _P), ("track_state", _P), ("track_det", _P), ("rows", _P),
                ("net_det", _P * 3)]


class jde_frame_result(C.Structure):
    _fields_ = [("ticket", C.c_longlong), ("stream_id", C.c_int), ("n_dets", C.c_int), ("n_tracks", C.c_int),
                ("errors", C.c_int), ("done_ms", C.c_float)]


_sig = {
    "jde_default_config": (None, [C.POINTER(jde_config)]),
    "jde_layer_table": (C.c_int, [C.POINTER(jde_layer_desc), C.c_int]),
    "jde_create": (C.c_int, [C.POINTER(jde_config), _P, C.c_size_t, C.POINTER(_P)]),
    "jde_destroy": (None, [_P]),
    "jde_last_error": (C.c_char_p, [_P]),
    "jde_forward": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, _P]),
    "jde_postprocess": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(jde_dets), _P]),
    "jde_detect_batch": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(jde_dets), _P]),
    "jde_track_step": (C.c_int, [_P, C.c_int, _P, C.POINTER(jde_dets), C.POINTER(jde_tracks), _P]),
    "jde_stream_reset": (C.c_int, [_P, C.c_int, _P]),
    "jde_get_tensor": (C.c_int, [_P, C.c_int, _P, C.c_size_t, C.POINTER(C.c_int), C.POINTER(C.c_int), _P]),
    "jde_kernel_errors": (C.c_int, [_P, C.POINTER(C.c_int), _P]),
    "jde_autotune": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P]),
    "jde_tile_choice": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "jde_set_tile_choice": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "jde_set_act_amax": (C.c_int, [_P, C.POINTER(C.c_float), C.c_int]),
    "jde_act_amax": (C.c_int, [_P, C.POINTER(C.c_float), _P]),
    "jde_device_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t)]),
    "jde_estimate_device_bytes": (C.c_int, [C.POINTER(jde_config), C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "jde_launch_count": (C.c_ulonglong, []),
    "jde_set_profile_events": (C.c_int, [_P, _P, _P, _P]),
    "jde_set_dependent_launch": (C.c_int, [_P, C.c_int]),
    "jde_selftest_wait": (C.c_int, [_P, C.c_longlong, C.POINTER(C.c_int), _P]),
    "jde_postprocess_noalloc": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_float,
                                          C.c_int, C.POINTER(jde_dets), _P, C.c_char_p, C.c_size_t]),
    "jde_default_server_config": (None, [C.POINTER(jde_server_config)]),
    "jde_server_create": (C.c_int, [C.POINTER(jde_server_config), _P, C.c_size_t, C.POINTER(_P)]),
    "jde_server_destroy": (None, [_P]),
    "jde_server_last_error": (C.c_char_p, [_P]),
    "jde_server_reset_clock": (C.c_int, [_P]),
    "jde_stream_open": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "jde_stream_close": (C.c_int, [_P, C.c_int]),
    "jde_submit": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(jde_frame_out), C.POINTER(C.c_longlong)]),
    "jde_poll": (C.c_int, [_P, C.POINTER(jde_frame_result), C.c_int, C.POINTER(C.c_int)]),
    "jde_server_flush": (C.c_int, [_P]),
    "jde_server_group_cost": (C.c_int, [C.POINTER(jde_server_config), C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
    "jde_server_device_bytes": (C.c_int, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "jde_server_stats": (C.c_int, [_P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "jde_decoder_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(_P)]),
    "jde_decoder_destroy": (None, [_P]),
    "jde_decoder_last_error": (C.c_char_p, [_P]),
    "jde_decoder_backend": (C.c_int, [_P]),
    "jde_decode_jpeg": (C.c_int, [_P, _P, C.POINTER(C.c_size_t), C.c_int, C.c_int, C.c_int, _P, _P]),
    "jde_encode_jpeg": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P, C.POINTER(C.c_size_t), _P]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sig)


class JdeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def ptr(x) -> int | None:
    """Raw address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def stream_ptr(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(h, status):
    if status != JDE_OK:
        raise JdeError(status, lib.jde_last_error(h).decode(errors="replace"))


def jde_default_config() -> jde_config:
    cfg = jde_config()
    lib.jde_default_config(C.byref(cfg))
    return cfg


def jde_layer_table():
    """List of (cin, cout, k, stride, has_bn, res_nblocks) in weights-blob order."""
    n = lib.jde_layer_table(None, 0)
    arr = (jde_layer_desc * n)()
    lib.jde_layer_table(arr, n)
    return [(d.cin, d.cout, d.k, d.stride, bool(d.has_bn), d.res_nblocks) for d in arr]


def jde_create(cfg: jde_config, blob: bytes):
    h = _P()
    buf = C.create_string_buffer(blob, len(blob))
    _check(None, lib.jde_create(C.byref(cfg), buf, len(blob), C.byref(h)))
    return h


def jde_destroy(h) -> None:
    lib.jde_destroy(h)


def jde_last_error(h=None) -> str:
    return lib.jde_last_error(h).decode(errors="replace")


def jde_forward(h, frames, n, src_w, src_h, in_w, in_h, on_device=True, stream=None):
    _check(h, lib.jde_forward(h, ptr(frames), n, src_w, src_h, in_w, in_h, int(on_device), stream_ptr(stream)))


def make_dets(rows, count, anchor_index=None, cap=None, on_device=True) -> jde_dets:
    d = jde_dets()
    d.rows, d.count, d.anchor_index = ptr(rows), ptr(count), ptr(anchor_index)
    d.cap = int(cap if cap is not None else rows.shape[1])
    d.on_device = int(on_device)
    return d


def make_tracks(ids, box, state, det, count, cap=None, on_device=True) -> jde_tracks:
    t = jde_tracks()
    t.id, t.box, t.state, t.det, t.count = ptr(ids), ptr(box), ptr(state), ptr(det), ptr(count)
    t.cap = int(cap if cap is not None else ids.shape[1])
    t.on_device = int(on_device)
    return t


def jde_postprocess(h, heads, n, in_w, in_h, src_w, src_h, dets: jde_dets, stream=None):
    arr = None
    if heads is not None:
        arr = (_P * 6)(*[ptr(x) for x in heads])
    _check(h, lib.jde_postprocess(h, arr, n, in_w, in_h, src_w, src_h, C.byref(dets), stream_ptr(stream)))


def jde_detect_batch(h, frames, n, src_w, src_h, in_w, in_h, dets: jde_dets, on_device=True, stream=None):
    _check(h, lib.jde_detect_batch(h, ptr(frames), n, src_w, src_h, in_w, in_h, int(on_device), C.byref(dets),
                                   stream_ptr(stream)))


def jde_track_step(h, stream_ids, dets: jde_dets, tracks: jde_tracks, stream=None):
    ids = np.ascontiguousarray(stream_ids, dtype=np.int32)
    _check(h, lib.jde_track_step(h, len(ids), ids.ctypes.data, C.byref(dets), C.byref(tracks), stream_ptr(stream)))


def jde_stream_reset(h, stream_id, stream=None):
    _check(h, lib.jde_stream_reset(h, stream_id, stream_ptr(stream)))


def jde_get_tensor(h, tid, dst=None, dst_bytes=0, stream=None):
    """Returns ((n, h, w, c), dtype) and copies into dst (device) when given."""
    dims = (C.c_int * 4)()
    dt = C.c_int()
    _check(h, lib.jde_get_tensor(h, tid, ptr(dst), dst_bytes, dims, C.byref(dt), stream_ptr(stream)))
    return tuple(dims), dt.value


def jde_kernel_errors(h, stream=None) -> int:
    w = C.c_int()
    _check(h, lib.jde_kernel_errors(h, C.byref(w), stream_ptr(stream)))
    return w.value


def jde_autotune(h, n, in_w, in_h, stream=None) -> None:
    _check(h, lib.jde_autotune(h, n, in_w, in_h, stream_ptr(stream)))


def jde_tile_choice(h, n, in_w, in_h):
    k = lib.jde_layer_table(None, 0)
    arr = (C.c_int * k)()
    _check(h, lib.jde_tile_choice(h, n, in_w, in_h, arr))
    return list(arr)


def jde_set_tile_choice(h, n, in_w, in_h, codes) -> None:
    arr = (C.c_int * JDE_NUM_LAYERS)(*[int(c) for c in codes])
    _check(h, lib.jde_set_tile_choice(h, n, in_w, in_h, arr))


def jde_set_act_amax(h, amax) -> None:
    arr = (C.c_float * len(amax))(*[float(v) for v in amax])
    _check(h, lib.jde_set_act_amax(h, arr, len(amax)))


def jde_act_amax(h, stream=None):
    n = lib.jde_layer_table(None, 0)
    arr = (C.c_float * n)()
    _check(h, lib.jde_act_amax(h, arr, stream_ptr(stream)))
    return [float(v) for v in arr]


def jde_device_bytes(h) -> int:
    out = C.c_size_t()
    _check(h, lib.jde_device_bytes(h, C.byref(out)))
    return int(out.value)


def jde_estimate_device_bytes(cfg: jde_config, in_w: int, in_h: int) -> int:
    out = C.c_size_t()
    _check(None, lib.jde_estimate_device_bytes(C.byref(cfg), in_w, in_h, C.byref(out)))
    return int(out.value)


def jde_launch_count() -> int:
    return int(lib.jde_launch_count())


def jde_set_profile_events(h, forward_begin=None, conv_begin=None, conv_end=None):
    """Events are torch.cuda.Event objects (recorded by the library on the call's stream) or None."""
    ev = [None if e is None else e.cuda_event for e in (forward_begin, conv_begin, conv_end)]
    _check(h, lib.jde_set_profile_events(h, *ev))


def jde_set_dependent_launch(h, on):
    _check(h, lib.jde_set_dependent_launch(h, int(on)))


def jde_postprocess_noalloc(heads, n, in_w, in_h, src_w, src_h, conf_thresh, nms_iou, max_cand, dets: jde_dets,
                            stream=None):
    """Allocation-free post-processing (scratch from the library's fixed device array)."""
    arr = (_P * 6)(*[ptr(x) for x in heads])
    msg = C.create_string_buffer(512)
    st = lib.jde_postprocess_noalloc(arr, n, in_w, in_h, src_w, src_h, conf_thresh, nms_iou, max_cand,
                                     C.byref(dets), stream_ptr(stream), msg, len(msg))
    if st != JDE_OK:
        raise JdeError(st, msg.value.decode(errors="replace"))


def jde_selftest_wait(h, limit_cycles, stream=None) -> tuple[int, int]:
    """Run the bounded-wait self-test; returns (status, error word) without raising for JDE_ERR_TIMEOUT."""
    w = C.c_int()
    st = lib.jde_selftest_wait(h, int(limit_cycles), C.byref(w), stream_ptr(stream))
    if st not in (JDE_OK, 6):
        _check(h, st)
    return st, w.value


# ----------------------------------------------------------------------------- server
def _check_server(s, status):
    if status != JDE_OK:
        msg = lib.jde_server_last_error(s).decode(errors="replace") if s else "invalid argument"
        raise JdeError(status, msg)


def jde_default_server_config() -> jde_server_config:
    cfg = jde_server_config()
    lib.jde_default_server_config(C.byref(cfg))
    return cfg


def jde_server_create(cfg: jde_server_config, blob: bytes):
    out = _P()
    buf = C.create_string_buffer(blob, len(blob))
    st = lib.jde_server_create(C.byref(cfg), buf, len(blob), C.byref(out))
    if st != JDE_OK:
        raise JdeError(st, "jde_server_create")
    return out


def jde_server_destroy(s) -> None:
    lib.jde_server_destroy(s)


def jde_server_reset_clock(s) -> None:
    _check_server(s, lib.jde_server_reset_clock(s))


def jde_stream_open(s, in_w, in_h) -> int:
    """Returns the stream id; raises JdeError (status JDE_ERR_ADMISSION = 5 when refused)."""
    sid = C.c_int()
    _check_server(s, lib.jde_stream_open(s, in_w, in_h, C.byref(sid)))
    return sid.value


def jde_stream_close(s, stream_id) -> None:
    _check_server(s, lib.jde_stream_close(s, stream_id))


def make_frame_out(track_id=None, track_box=None, track_state=None, track_det=None, rows=None, net_det=None):
    """jde_frame_out over host numpy arrays (kept alive by the caller until the frame's result is polled)."""
    nd = list(net_det) if net_det is not None else [None, None, None]
    return jde_frame_out(ptr(track_id), ptr(track_box), ptr(track_state), ptr(track_det), ptr(rows),
                         (_P * 3)(*[ptr(x) for x in nd]))


def jde_submit(s, stream_id, frame, heads=None, out: jde_frame_out | None = None, ready=None) -> int:
    """ready: a torch.cuda.Event recorded after the frame's inputs were written (or None)."""
    hp = None if heads is None else (_P * 6)(*[ptr(x) for x in heads])
    t = C.c_longlong()
    ev = None if ready is None else ready.cuda_event
    _check_server(s, lib.jde_submit(s, stream_id, ptr(frame), hp, ev, None if out is None else C.byref(out),
                                    C.byref(t)))
    return t.value


def jde_poll(s, cap=256):
    """Results of finished frames (jde_frame_result structures), at most cap."""
    arr = (jde_frame_result * cap)()
    n = C.c_int()
    _check_server(s, lib.jde_poll(s, arr, cap, C.byref(n)))
    return [arr[i] for i in range(n.value)]


def jde_server_flush(s) -> None:
    _check_server(s, lib.jde_server_flush(s))


def jde_server_group_cost(cfg: jde_server_config, in_w, in_h) -> int:
    out = C.c_size_t()
    st = lib.jde_server_group_cost(C.byref(cfg), in_w, in_h, C.byref(out))
    if st != JDE_OK:
        raise JdeError(st, f"jde_server_group_cost({in_w}, {in_h})")
    return int(out.value)


def jde_server_device_bytes(s) -> tuple[int, int]:
    a, b = C.c_size_t(), C.c_size_t()
    _check_server(s, lib.jde_server_device_bytes(s, C.byref(a), C.byref(b)))
    return int(a.value), int(b.value)


def jde_server_stats(s) -> tuple[int, int, int]:
    """(batches launched eagerly, graphs captured, graph replays)."""
    e, c, r = C.c_longlong(), C.c_longlong(), C.c_longlong()
    _check_server(s, lib.jde_server_stats(s, C.byref(e), C.byref(c), C.byref(r)))
    return e.value, c.value, r.value


# ----------------------------------------------------------------------------- device decode
JDE_DECODE_HARDWARE, JDE_DECODE_GPU_HYBRID = 1, 2


def _check_decoder(d, status):
    if status != JDE_OK:
        raise JdeError(status, lib.jde_decoder_last_error(d).decode(errors="replace") if d else "decoder")


def jde_decoder_create(device=0, max_batch=16, hardware=True):
    out = _P()
    st = lib.jde_decoder_create(device, max_batch, 1 if hardware else 0, C.byref(out))
    if st != JDE_OK:
        raise JdeError(st, "jde_decoder_create (nvJPEG unavailable or set-up failed)")
    return out


def jde_decoder_destroy(d) -> None:
    lib.jde_decoder_destroy(d)


def jde_decoder_backend(d) -> int:
    return int(lib.jde_decoder_backend(d))


def jde_decode_jpeg(d, bitstreams, w, h, frames, stream=None) -> None:
    """bitstreams: list of host byte buffers (bytes or uint8 numpy arrays); frames: device tensor
    [n, h, w, 3] uint8."""
    n = len(bitstreams)
    arrs = [np.frombuffer(b, np.uint8) if isinstance(b, (bytes, bytearray)) else b for b in bitstreams]
    ptrs = (_P * n)(*[a.ctypes.data for a in arrs])
    lens = (C.c_size_t * n)(*[a.nbytes for a in arrs])
    _check_decoder(d, lib.jde_decode_jpeg(d, ptrs, lens, n, w, h, ptr(frames), stream_ptr(stream)))


def jde_encode_jpeg(d, frames, n, w, h, quality=90, stream=None):
    """Encode n device frames [n, h, w, 3] uint8; returns a list of n uint8 numpy bitstreams."""
    cap = max(1 << 16, w * h * 3 // 2)
    for _ in range(3):
        bufs = [np.empty(cap, np.uint8) for _ in range(n)]
        ptrs = (_P * n)(*[b.ctypes.data for b in bufs])
        lens = (C.c_size_t * n)(*([cap] * n))
        st = lib.jde_encode_jpeg(d, ptr(frames), n, w, h, quality, ptrs, lens, stream_ptr(stream))
        if st == 4:        # JDE_ERR_CAPACITY: one frame needs a larger buffer
            cap = max(int(lens[i]) for i in range(n)) + 1024
            continue
        _check_decoder(d, st)
        return [bufs[i][:int(lens[i])].copy() for i in range(n)]
    raise JdeError(4, "jde_encode_jpeg: bitstream buffers")
