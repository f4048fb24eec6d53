"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point the header declares, and rejects bad arguments and bad
weight blobs before touching the device."""
import ctypes
import os
import re
import struct

import numpy as np
import pytest

from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glassnet.h")


@pytest.fixture(scope="module")
def lib():
    return gl.load_library()


def _declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glassnet_\w+)\s*\(", text)))


def test_header_declarations_are_bound():
    decl = _declared_symbols()
    assert len(decl) >= 14
    assert set(decl) == set(gl._SIGNATURES), set(decl) ^ set(gl._SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_last_error_starts_empty_or_string(lib):
    assert isinstance(gl.glassnet_last_error(), str)


def _blob(widths=synth.BASE_WIDTHS):
    return gl.pack_blob(synth.make_weights(widths, seed=0))


def _load(lib, blob, precision=gl.GN_BF16_FUSED):
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    rc = lib.glassnet_load_weights(buf, len(blob), precision, ctypes.byref(out))
    return rc, out.value


def test_blob_header_layout():
    blob = _blob()
    fields = struct.unpack(gl.HEADER_FMT, blob[:48])
    assert fields[0] == 0x544E4C47 and blob[:4] == b"GLNT"
    assert fields[1:8] == (1, 64, 128, 32, 12, 14, 3)
    assert fields[8] * 4 == len(blob) - 48


def test_blob_checksum_is_fnv1a64():
    blob = _blob()
    payload = blob[48:]
    h = 0xCBF29CE484222325
    for byte in payload:
        h ^= byte
        h = (h * 0x100000001B3) % (1 << 64)
    assert struct.unpack("<Q", blob[40:48])[0] == h


@pytest.mark.parametrize("mutate,code", [
    (lambda b: b[:20], gl.GN_EFORMAT),                                   # truncated header
    (lambda b: b"XXXX" + b[4:], gl.GN_EFORMAT),                          # magic
    (lambda b: b[:4] + struct.pack("<I", 9) + b[8:], gl.GN_EFORMAT),     # version
    (lambda b: b[:-4], gl.GN_EFORMAT),                                   # truncated payload
    (lambda b: b[:100] + bytes([b[100] ^ 1]) + b[101:], gl.GN_EFORMAT),  # checksum
    (lambda b: b[:16] + struct.pack("<I", 13) + b[20:], gl.GN_EFORMAT),  # scene dim
])
def test_corrupt_blobs_rejected(lib, mutate, code):
    rc, handle = _load(lib, mutate(_blob()))
    assert rc == code and not handle
    assert gl.glassnet_last_error()


def test_unsupported_widths_rejected(lib):
    w = synth.make_weights(synth.Widths(hidden=32, latent=64), seed=0)
    rc, handle = _load(lib, gl.pack_blob(w))
    assert rc == gl.GN_EUNSUPPORTED and not handle


def test_unknown_precision_rejected(lib):
    rc, _ = _load(lib, _blob(), precision=7)
    assert rc == gl.GN_EINVAL


def test_pooling_arguments_checked_before_any_device_work(lib):
    """Unknown pooling or frequency count -> EINVAL; positional encoding in
    FP8 beyond the 4 frequencies its operands hold -> EUNSUPPORTED; all
    rejected on the host, before the blob reaches the device."""
    blob = _blob()
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))

    def load(precision, pooling, pe):
        cfg = gl.ModelConfig(precision, pooling, pe)
        return lib.glassnet_load_weights_ex(buf, len(blob), ctypes.byref(cfg), ctypes.byref(out))

    assert load(gl.GN_BF16_FUSED, 2, 0) == gl.GN_EINVAL
    assert load(gl.GN_BF16_FUSED, 0, -1) == gl.GN_EINVAL
    assert load(gl.GN_BF16_FUSED, 0, 11) == gl.GN_EINVAL
    assert load(gl.GN_FP8_FUSED, 0, 5) == gl.GN_EUNSUPPORTED
    assert "positional encoding" in gl.glassnet_last_error()
    assert load(gl.GN_FP8_FUSED, 0, 2) == gl.GN_EFORMAT  # a plain blob read as L = 2
    # a plain (L = 0) blob read as L = 1 has the wrong payload size
    assert load(gl.GN_BF16_FUSED, 0, 1) == gl.GN_EFORMAT
    assert "pe_freqs 1" in gl.glassnet_last_error()
    assert not out.value
    assert lib.glassnet_load_weights_ex(None, 10, None, ctypes.byref(out)) == gl.GN_EINVAL
    assert lib.glassnet_model_config(None, None) == gl.GN_EINVAL


def test_r_kernel_checked_on_the_host(lib):
    """r_kernel must be 0, 1 or 3; a 1x1 blob read as 3x3 has the wrong
    payload size.  All refused before any device work."""
    blob = _blob()
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    for precision, rk, code in [(gl.GN_BF16_FUSED, 2, gl.GN_EINVAL), (gl.GN_BF16_FUSED, 5, gl.GN_EINVAL),
                                (gl.GN_FP8_FUSED, 3, gl.GN_EFORMAT), (gl.GN_BF16_FUSED, 3, gl.GN_EFORMAT),
                                (gl.GN_FP32_PLAIN, 3, gl.GN_EFORMAT)]:
        cfg = gl.ModelConfig(precision, 0, 0, rk)
        assert lib.glassnet_load_weights_ex(buf, len(blob), ctypes.byref(cfg), ctypes.byref(out)) == code, rk
        assert not out.value


def test_positional_encoding_limits_checked_on_the_host(lib):
    """The fused kernel's encoded operands hold L <= 4 frequencies at both
    widths: larger forms are refused before the blob reaches the device."""
    out = ctypes.c_void_p()
    for widths, pe, code in [(synth.Widths(hidden=128, latent=256, pe_freqs=5), 5, gl.GN_EUNSUPPORTED),
                             (synth.Widths(hidden=64, latent=128, pe_freqs=5), 5, gl.GN_EUNSUPPORTED)]:
        blob = gl.pack_blob(synth.make_weights(widths, seed=0))
        buf = ctypes.create_string_buffer(blob, len(blob))
        cfg = gl.ModelConfig(gl.GN_BF16_FUSED, 0, pe)
        assert lib.glassnet_load_weights_ex(buf, len(blob), ctypes.byref(cfg), ctypes.byref(out)) == code
        assert "pe_freqs 1..4" in gl.glassnet_last_error()
        assert not out.value


def test_null_arguments_rejected(lib):
    out = ctypes.c_void_p()
    assert lib.glassnet_load_weights(None, 10, 1, ctypes.byref(out)) == gl.GN_EINVAL
    assert lib.glassnet_render(None, None, None, None, None, 1, 8, 8, None, None) == gl.GN_EINVAL
    assert lib.glassnet_render_batch(None, None, 1, None) == gl.GN_EINVAL
    assert lib.glassnet_encode_scene(None, None, ctypes.byref(out), None) == gl.GN_EINVAL
    assert lib.glassnet_check(None, None) == gl.GN_EINVAL
    n = ctypes.c_size_t()
    assert lib.glassnet_workspace_bytes(None, 1, 1, 1, ctypes.byref(n)) == gl.GN_EINVAL
    lib.glassnet_free_model(None)
    lib.glassnet_free_latent(None)
    assert lib.glassnet_graph_create(None, None, 1, ctypes.byref(out)) == gl.GN_EINVAL
    assert lib.glassnet_graph_create(None, None, 1, None) == gl.GN_EINVAL
    assert lib.glassnet_graph_launch(None, None) == gl.GN_EINVAL
    assert lib.glassnet_graph_update(None, None, 1) == gl.GN_EINVAL
    lib.glassnet_graph_free(None)
    assert lib.glassnet_server_create(None, None, ctypes.byref(out)) == gl.GN_EINVAL
    t = ctypes.c_uint64()
    assert lib.glassnet_server_submit(None, None, ctypes.byref(t)) == gl.GN_EINVAL
    assert lib.glassnet_server_wait(None, 1, None) == gl.GN_EINVAL
    assert lib.glassnet_server_stats(None, None) == gl.GN_EINVAL
    lib.glassnet_server_destroy(None)
    assert lib.glassnet_pool_create(None, 8, 8, ctypes.byref(out)) == gl.GN_EINVAL
    assert lib.glassnet_pool_reset(None, None) == gl.GN_EINVAL
    assert lib.glassnet_accumulate_layer(None, None, None, None, None, None) == gl.GN_EINVAL
    assert lib.glassnet_resolve(None, None, None, None, None, None) == gl.GN_EINVAL
    lib.glassnet_pool_free(None)


def test_python_binding_raises_with_message(lib):
    with pytest.raises(gl.GlassNetError) as ei:
        gl.glassnet_load_weights(b"short", gl.GN_BF16_FUSED)
    assert ei.value.code == gl.GN_EFORMAT


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: a library that is not there is an error, not a
    silent substitute."""
    with pytest.raises(gl.GlassNetError) as ei:
        gl.load_library(path=str(tmp_path / "libglassnet_absent.so"))
    assert "not found" in str(ei.value)


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: nothing in the product package
    imports it or any numpy / torch math path that could stand in for the
    CUDA library."""
    import pathlib
    pkg = pathlib.Path(gl.__file__).parent
    for f in pkg.rglob("*.py"):
        text = f.read_text()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "glassnet_oracle" not in text, f


def test_edge_frame_sizes_of_the_gpu_tests_are_the_documented_limit():
    """The frames of test_gpu_max_size.py sit at glassnet_render's limit
    12 max(K, 1) h w < 2^31: accepted as they are, refused one column wider."""
    for K, h, w in ((8, 4729, 4730), (0, 13377, 13377)):
        assert 12 * max(K, 1) * h * w < 1 << 31
        assert 12 * max(K, 1) * h * (w + 1) >= 1 << 31
