"""Python binding of the C ABI in ``include/glassnet.h`` (argument marshalling only).

Every function here converts Python / torch arguments to plain pointers and
sizes and calls the entry point of the same name in ``libglassnet.so``; all
network arithmetic runs in the library's CUDA kernels.  If the library cannot
be loaded, every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import struct

import numpy as np

from . import build as _build

GN_OK = 0
GN_EINVAL = -1
GN_ENOMEM = -2
GN_ECUDA = -3
GN_EFORMAT = -4
GN_ETIMEOUT = -5
GN_EUNSUPPORTED = -6
GN_ERANGE = -7
GN_ESATURATED = -8
GN_FP8_SCALES = 32
GN_SCHEDULE_SORTED = 0
GN_SCHEDULE_COMPACT = 1

GN_FP32_PLAIN = 0
GN_BF16_FUSED = 1
GN_FP8_FUSED = 2
GN_POOL_MAX_MEAN = 0
GN_POOL_SUM = 1

BLOB_MAGIC = 0x544E4C47
BLOB_VERSION = 1
HEADER_FMT = "<8I2Q"  # magic, version, H, Z, scene, tbuf ch, gbuf ch, out ch, floats, checksum
LAYER_ORDER = ("F1", "F2", "phi1", "phi2", "rho", "B1", "B2", "R1", "R2")

# Every entry point the header declares: name -> (restype, argtypes).
_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGNATURES = {
    "glassnet_load_weights": (_I, [_P, ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "glassnet_model_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "glassnet_load_weights_ex": (_I, [_P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "glassnet_model_config": (_I, [_P, _P]),
    "glassnet_encode_scene": (_I, [_P, _P, ctypes.POINTER(_P), _P]),
    "glassnet_encode_scene_device": (_I, [_P, _P, _P, _P]),
    "glassnet_latent_read": (_I, [_P, _P, _P, _P, _P]),
    "glassnet_render": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P, _P]),
    "glassnet_workspace_bytes": (_I, [_P, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "glassnet_render_ws": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P, _P, ctypes.c_size_t, _P]),
    "glassnet_render_host": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P, _P]),
    "glassnet_render_batch": (_I, [_P, _P, _I, _P]),
    "glassnet_check": (_I, [_P, _P]),
    "glassnet_debug_stall_next_render": (_I, [_P, ctypes.c_uint64]),
    "glassnet_set_layer_schedule": (_I, [_P, _I]),
    "glassnet_render_fp32_static": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P, _P]),
    "glassnet_calibrate_fp8": (_I, [_P, _P, _P, _P, _P, _I, _I, _I, _P]),
    "glassnet_fp8_scales": (_I, [_P, _P]),
    "glassnet_server_create": (_I, [_P, _P, ctypes.POINTER(_P)]),
    "glassnet_server_add_scene": (_I, [_P, _P, ctypes.POINTER(_I)]),
    "glassnet_server_prepare": (_I, [_P, _I, _I, _I]),
    "glassnet_server_submit": (_I, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "glassnet_server_wait": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "glassnet_server_wait_times": (_I, [_P, ctypes.c_uint64, _P]),
    "glassnet_server_stats": (_I, [_P, _P]),
    "glassnet_server_destroy": (None, [_P]),
    "glassnet_pool_create": (_I, [_P, _I, _I, ctypes.POINTER(_P)]),
    "glassnet_pool_reset": (_I, [_P, _P]),
    "glassnet_accumulate_layer": (_I, [_P, _P, _P, _P, _P, _P]),
    "glassnet_resolve": (_I, [_P, _P, _P, _P, _P, _P]),
    "glassnet_pool_free": (None, [_P]),
    "glassnet_graph_create": (_I, [_P, _P, _I, ctypes.POINTER(_P)]),
    "glassnet_graph_launch": (_I, [_P, _P]),
    "glassnet_graph_update": (_I, [_P, _P, _I]),
    "glassnet_graph_free": (None, [_P]),
    "glassnet_free_latent": (None, [_P]),
    "glassnet_free_model": (None, [_P]),
    "glassnet_last_error": (ctypes.c_char_p, []),
}

_LIB = None


class GlassNetError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"glassnet error {code}: {message}")
        self.code = code


def load_library(path: str | None = None, build: bool = True):
    """Loads libglassnet.so (building it first if needed) and binds every symbol."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    if path is None:
        path = _build.build() if build else _build.lib_path()
    if not os.path.exists(path):
        raise GlassNetError(GN_EINVAL, f"CUDA library not found at {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _lib():
    return _LIB if _LIB is not None else load_library()


def _check(rc: int):
    if rc != GN_OK:
        raise GlassNetError(rc, _lib().glassnet_last_error().decode())


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ------------------------------------------------------------------- blobs

def pack_blob(weights: dict) -> bytes:
    """Serialises {name: (W [out][in], b [out])} into the weight-blob format."""
    H = int(np.shape(weights["phi2"][0])[0])
    Z = int(np.shape(weights["F2"][0])[0])
    parts = []
    for name in LAYER_ORDER:
        W, b = weights[name]
        parts.append(np.ascontiguousarray(W, dtype=np.float32).reshape(-1))
        parts.append(np.ascontiguousarray(b, dtype=np.float32).reshape(-1))
    payload = np.concatenate(parts).astype("<f4").tobytes()
    h = 0xCBF29CE484222325
    prime = 0x100000001B3
    arr = np.frombuffer(payload, dtype=np.uint8)
    for byte in arr.tolist():  # FNV-1a 64
        h = ((h ^ byte) * prime) & 0xFFFFFFFFFFFFFFFF
    header = struct.pack(HEADER_FMT, BLOB_MAGIC, BLOB_VERSION, H, Z, 32, 12, 14, 3,
                         len(payload) // 4, h)
    return header + payload


# ------------------------------------------------- entry points (same names)

def glassnet_load_weights(blob: bytes, precision: int) -> int:
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib().glassnet_load_weights(buf, len(blob), precision, ctypes.byref(out)))
    return out.value


class ModelConfig(ctypes.Structure):
    """gn_model_config."""
    _fields_ = [("precision", ctypes.c_int), ("pooling", ctypes.c_int), ("pe_freqs", ctypes.c_int),
                ("r_kernel", ctypes.c_int)]


def glassnet_load_weights_ex(blob: bytes, precision: int, pooling: int = 0, pe_freqs: int = 0,
                             r_kernel: int = 1) -> int:
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    cfg = ModelConfig(precision, pooling, pe_freqs, r_kernel)
    _check(_lib().glassnet_load_weights_ex(buf, len(blob), ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def glassnet_model_info(model: int):
    h, z, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib().glassnet_model_info(model, ctypes.byref(h), ctypes.byref(z), ctypes.byref(p)))
    return h.value, z.value, p.value


def glassnet_model_config(model: int) -> ModelConfig:
    cfg = ModelConfig()
    _check(_lib().glassnet_model_config(model, ctypes.byref(cfg)))
    return cfg


def glassnet_encode_scene(model: int, scene, stream=None) -> int:
    s = np.ascontiguousarray(scene, dtype=np.float32)
    if s.size != 32:
        raise GlassNetError(GN_EINVAL, "scene vector must hold 32 floats")
    out = ctypes.c_void_p()
    _check(_lib().glassnet_encode_scene(model, s.ctypes.data, ctypes.byref(out), _stream(stream)))
    return out.value


def glassnet_encode_scene_device(model: int, scene_dev, latent: int, stream=None):
    _check(_lib().glassnet_encode_scene_device(model, _ptr(scene_dev), latent, _stream(stream)))


def glassnet_latent_read(latent: int, sigma=None, c_phi=None, c_b=None, stream=None):
    _check(_lib().glassnet_latent_read(latent, _ptr(sigma), _ptr(c_phi), _ptr(c_b), _stream(stream)))


def glassnet_render(model, latent, gbuf, tbuf, layer_count, K, h, w, out, stream=None):
    _check(_lib().glassnet_render(model, latent, _ptr(gbuf), _ptr(tbuf), _ptr(layer_count),
                                  K, h, w, _ptr(out), _stream(stream)))


def glassnet_workspace_bytes(model, K, h, w) -> int:
    n = ctypes.c_size_t()
    _check(_lib().glassnet_workspace_bytes(model, K, h, w, ctypes.byref(n)))
    return n.value


def glassnet_render_ws(model, latent, gbuf, tbuf, layer_count, K, h, w, out, workspace,
                       workspace_bytes, stream=None):
    _check(_lib().glassnet_render_ws(model, latent, _ptr(gbuf), _ptr(tbuf), _ptr(layer_count),
                                     K, h, w, _ptr(out), _ptr(workspace), workspace_bytes,
                                     _stream(stream)))


def glassnet_render_host(model, latent, gbuf_h, tbuf_h, count_h, K, h, w, out_h, stream=None):
    """Host tensors (ideally pinned) in and out; returns after the result is in out_h."""
    _check(_lib().glassnet_render_host(model, latent, gbuf_h.data_ptr(),
                                       tbuf_h.data_ptr() if tbuf_h is not None else None,
                                       count_h.data_ptr(), K, h, w, out_h.data_ptr(),
                                       _stream(stream)))


class GnFrame(ctypes.Structure):
    _fields_ = [("latent", ctypes.c_void_p), ("gbuf", ctypes.c_void_p), ("tbuf", ctypes.c_void_p),
                ("layer_count", ctypes.c_void_p), ("K", ctypes.c_int), ("h", ctypes.c_int),
                ("w", ctypes.c_int), ("out", ctypes.c_void_p)]


def glassnet_render_batch(model, frames, stream=None):
    """frames: list of dicts with latent, gbuf, tbuf, layer_count, K, h, w, out."""
    _check(_lib().glassnet_render_batch(model, _frame_array(frames), len(frames), _stream(stream)))


def glassnet_calibrate_fp8(model, latent, gbuf, tbuf, layer_count, K, h, w, stream=None):
    _check(_lib().glassnet_calibrate_fp8(model, latent, _ptr(gbuf), _ptr(tbuf), _ptr(layer_count),
                                         K, h, w, _stream(stream)))


def glassnet_fp8_scales(model) -> np.ndarray:
    out = np.zeros(GN_FP8_SCALES, dtype=np.float32)
    _check(_lib().glassnet_fp8_scales(model, out.ctypes.data))
    return out


def _frame_array(frames):
    arr = (GnFrame * len(frames))()
    for i, f in enumerate(frames):
        arr[i] = GnFrame(f["latent"], _ptr(f["gbuf"]), _ptr(f.get("tbuf")), _ptr(f["layer_count"]),
                         f["K"], f["h"], f["w"], _ptr(f["out"]))
    return arr


def glassnet_graph_create(model, frames) -> int:
    """Captures the batched launch of `frames` (same dicts as glassnet_render_batch)."""
    out = ctypes.c_void_p()
    _check(_lib().glassnet_graph_create(model, _frame_array(frames), len(frames), ctypes.byref(out)))
    return out.value


def glassnet_pool_create(model, h, w) -> int:
    """Streaming pool for h x w frames (GN_BF16_FUSED models), empty."""
    out = ctypes.c_void_p()
    _check(_lib().glassnet_pool_create(model, h, w, ctypes.byref(out)))
    return out.value


def glassnet_pool_reset(pool, stream=None):
    _check(_lib().glassnet_pool_reset(pool, _stream(stream)))


def glassnet_accumulate_layer(model, latent, pool, layer, covered=None, stream=None):
    """layer: device [12][h][w] f32; covered: device [h][w] u8 (0 / 1) or None (all)."""
    _check(_lib().glassnet_accumulate_layer(model, latent, pool, _ptr(layer), _ptr(covered),
                                            _stream(stream)))


def glassnet_resolve(model, latent, pool, gbuf, out, stream=None):
    _check(_lib().glassnet_resolve(model, latent, pool, _ptr(gbuf), _ptr(out), _stream(stream)))


def glassnet_pool_free(pool):
    _lib().glassnet_pool_free(pool)


def glassnet_graph_launch(graph, stream=None):
    _check(_lib().glassnet_graph_launch(graph, _stream(stream)))


def glassnet_graph_update(graph, frames):
    _check(_lib().glassnet_graph_update(graph, _frame_array(frames), len(frames)))


def glassnet_graph_free(graph):
    _lib().glassnet_graph_free(graph)


class GnServerConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int), ("max_scenes", ctypes.c_int),
                ("budget_bytes", ctypes.c_size_t), ("max_h", ctypes.c_int), ("max_w", ctypes.c_int),
                ("max_K", ctypes.c_int)]


class GnRequest(ctypes.Structure):
    _fields_ = [("scene", ctypes.c_int), ("gbuf", ctypes.c_void_p), ("tbuf", ctypes.c_void_p),
                ("layer_count", ctypes.c_void_p), ("K", ctypes.c_int), ("h", ctypes.c_int),
                ("w", ctypes.c_int), ("out", ctypes.c_void_p)]


class GnServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("pixels", ctypes.c_double)]


def glassnet_server_create(model, n_streams=4, max_scenes=32, budget_bytes=40 << 30, max_h=1024,
                           max_w=1024, max_K=8) -> int:
    cfg = GnServerConfig(n_streams, max_scenes, budget_bytes, max_h, max_w, max_K)
    out = ctypes.c_void_p()
    _check(_lib().glassnet_server_create(model, ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def glassnet_server_add_scene(server, scene) -> int:
    s = np.ascontiguousarray(scene, dtype=np.float32)
    sid = ctypes.c_int()
    _check(_lib().glassnet_server_add_scene(server, s.ctypes.data, ctypes.byref(sid)))
    return sid.value


def glassnet_server_prepare(server, h, w, K):
    _check(_lib().glassnet_server_prepare(server, h, w, K))


def glassnet_server_submit(server, scene_id, gbuf, tbuf, layer_count, K, h, w, out) -> int:
    """Host tensors (page-locked for full bandwidth) that stay alive until the wait."""
    req = GnRequest(scene_id, gbuf.data_ptr(), tbuf.data_ptr() if tbuf is not None and K > 0 else None,
                    layer_count.data_ptr(), K, h, w, out.data_ptr())
    t = ctypes.c_uint64()
    _check(_lib().glassnet_server_submit(server, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def glassnet_server_wait(server, ticket) -> float:
    lat = ctypes.c_double()
    _check(_lib().glassnet_server_wait(server, ticket, ctypes.byref(lat)))
    return lat.value


class GnRequestTimes(ctypes.Structure):
    _fields_ = [("queue_ms", ctypes.c_double), ("enqueue_ms", ctypes.c_double),
                ("device_ms", ctypes.c_double), ("total_ms", ctypes.c_double),
                ("copy_in_ms", ctypes.c_double), ("render_ms", ctypes.c_double),
                ("copy_out_ms", ctypes.c_double)]


def glassnet_server_wait_times(server, ticket) -> dict:
    """As glassnet_server_wait, returning the latency's parts (milliseconds)."""
    t = GnRequestTimes()
    _check(_lib().glassnet_server_wait_times(server, ticket, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in GnRequestTimes._fields_}


def glassnet_server_stats(server) -> dict:
    st = GnServerStats()
    _check(_lib().glassnet_server_stats(server, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in GnServerStats._fields_}


def glassnet_server_destroy(server):
    _lib().glassnet_server_destroy(server)


def glassnet_render_fp32_static(model, latent, gbuf, tbuf, layer_count, K, h, w, out,
                                stream=None):
    """FP32 plain render whose scratch is the library's static device array (no allocation)."""
    _check(_lib().glassnet_render_fp32_static(model, latent, _ptr(gbuf), _ptr(tbuf),
                                              _ptr(layer_count), K, h, w, _ptr(out),
                                              _stream(stream)))


def glassnet_check(model, stream=None):
    _check(_lib().glassnet_check(model, _stream(stream)))


def glassnet_debug_stall_next_render(model, stall_ns: int):
    _check(_lib().glassnet_debug_stall_next_render(model, int(stall_ns)))


def glassnet_set_layer_schedule(model, schedule: int):
    _check(_lib().glassnet_set_layer_schedule(model, int(schedule)))


def glassnet_check_code(model, stream=None) -> int:
    """Like glassnet_check but returns the status code instead of raising."""
    return _lib().glassnet_check(model, _stream(stream))


def glassnet_free_latent(latent):
    _lib().glassnet_free_latent(latent)


def glassnet_free_model(model):
    _lib().glassnet_free_model(model)


def glassnet_last_error() -> str:
    return _lib().glassnet_last_error().decode()


# ----------------------------------------------------------- conveniences

class Model:
    """Owns a gn_model handle."""

    def __init__(self, weights_or_blob, precision: int = GN_BF16_FUSED,
                 pooling: int = GN_POOL_MAX_MEAN, pe_freqs=None, r_kernel=None):
        """``pe_freqs`` and ``r_kernel`` default to the weight dict's keys of
        those names (0 and 1 for a blob)."""
        is_blob = isinstance(weights_or_blob, (bytes, bytearray))
        if pe_freqs is None:
            pe_freqs = 0 if is_blob else int(weights_or_blob.get("pe_freqs", 0))
        if r_kernel is None:
            r_kernel = 1 if is_blob else int(weights_or_blob.get("r_kernel", 1))
        blob = weights_or_blob if is_blob else pack_blob(weights_or_blob)
        self.handle = glassnet_load_weights_ex(bytes(blob), precision, pooling, pe_freqs, r_kernel)
        self.hidden, self.latent_width, self.precision = glassnet_model_info(self.handle)
        cfg = glassnet_model_config(self.handle)
        self.pooling, self.pe_freqs, self.r_kernel = cfg.pooling, cfg.pe_freqs, cfg.r_kernel

    def encode(self, scene, stream=None) -> "Latent":
        return Latent(glassnet_encode_scene(self.handle, scene, stream))

    def render(self, latent: "Latent", gbuf, tbuf, counts, out, stream=None):
        K = 0 if tbuf is None else int(tbuf.shape[0])
        h, w = int(gbuf.shape[-2]), int(gbuf.shape[-1])
        glassnet_render(self.handle, latent.handle, gbuf, tbuf, counts, K, h, w, out, stream)

    def check(self, stream=None):
        glassnet_check(self.handle, stream)

    def close(self):
        if getattr(self, "handle", None):
            glassnet_free_model(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Latent:
    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            glassnet_free_latent(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
