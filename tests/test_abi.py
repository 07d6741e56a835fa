"""The C-ABI library loads and exports every entry point include/ugp.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ugp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(ugp_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libugp():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    from paper_2406_09733_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for must in ("ugp_build_bvh", "ugp_trace_transmittance", "ugp_sample_free_flight"):
        assert must in names


def test_every_declared_symbol_is_exported(libugp):
    missing = [n for n in declared_functions() if not hasattr(libugp, n)]
    assert not missing, missing


def test_status_strings_and_errors_without_gpu(libugp):
    libugp.ugp_status_string.restype = ctypes.c_char_p
    libugp.ugp_last_error.restype = ctypes.c_char_p
    assert libugp.ugp_status_string(0) == b"ok"
    assert libugp.ugp_status_string(6).startswith(b"BVH")
    # argument validation happens on the host before any device work
    libugp.ugp_trace_transmittance.restype = ctypes.c_int
    st = libugp.ugp_trace_transmittance(None, ctypes.c_int64(1), None, None, None, None, None,
                                        None, None, None)
    assert st == 6
    assert b"invalid BVH" in libugp.ugp_last_error()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2406_09733_gb300 import ugp, build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(ugp, "_LIB", None)
    with pytest.raises(ugp.UgpError):
        ugp.lib()


def test_radiance_field_entry_point_validates_on_host(libugp):
    libugp.ugp_render_radiance_field_workspace_size.restype = ctypes.c_size_t
    libugp.ugp_render_radiance_field_workspace_size.argtypes = [ctypes.c_int64]
    libugp.ugp_last_error.restype = ctypes.c_char_p
    ff = libugp.ugp_sample_free_flight_workspace_size
    ff.restype = ctypes.c_size_t
    ff.argtypes = [ctypes.c_int64]
    # the free-flight pass's scratch plus six per-ray columns
    assert libugp.ugp_render_radiance_field_workspace_size(1000) >= ff(1000) + 6 * 1000
    assert libugp.ugp_render_radiance_field_workspace_size(-1) == 0
    st = libugp.ugp_render_radiance_field(None, ctypes.c_int64(4), None, None, None, None, None, None, None, None,
                                          None, ctypes.c_size_t(0), None)
    assert st == 6 and b"invalid BVH handle" in libugp.ugp_last_error()   # UGP_ERR_NOT_BUILT


def test_exponential_entry_points_validate_on_host(libugp):
    libugp.ugp_last_error.restype = ctypes.c_char_p
    st = libugp.ugp_sample_free_flight_exponential(None, ctypes.c_int64(4), None, None, None, None, None, None,
                                                   None, None, None, None)
    assert st == 6 and b"invalid BVH handle" in libugp.ugp_last_error()
    st = libugp.ugp_trace_transmittance_exponential(None, ctypes.c_int64(4), None, None, None, None, None, None,
                                                    None, None)
    assert st == 6 and b"invalid BVH handle" in libugp.ugp_last_error()


def test_emitter_table_entry_points_validate_on_host(libugp):
    libugp.ugp_last_error.restype = ctypes.c_char_p
    libugp.ugp_emitter_table_size.restype = ctypes.c_size_t
    libugp.ugp_emitter_table_size.argtypes = [ctypes.c_int64]
    assert libugp.ugp_emitter_table_size(1000) >= 76 * 1000
    assert libugp.ugp_emitter_table_size(-1) == 0
    st = libugp.ugp_build_emitter_table(None, None, None, ctypes.c_size_t(0), None)
    assert st == 6 and b"invalid BVH handle" in libugp.ugp_last_error()


def test_guide_entry_points_validate_on_host(libugp):
    libugp.ugp_guide_workspace_size.restype = ctypes.c_size_t
    libugp.ugp_render_guided_workspace_size.restype = ctypes.c_size_t
    libugp.ugp_render_workspace_size.restype = ctypes.c_size_t
    libugp.ugp_last_error.restype = ctypes.c_char_p
    assert libugp.ugp_guide_workspace_size() > 42240
    plain = libugp.ugp_render_workspace_size(4, 4)
    guided = libugp.ugp_render_guided_workspace_size(4, 4, 3)
    assert guided > plain > 0
    assert libugp.ugp_render_guided_workspace_size(4, 4, 15) == 0
    st = libugp.ugp_guide_forward(None, ctypes.c_int64(4), None, None, None, None, None, ctypes.c_size_t(0), None)
    assert st == 1 and b"NULL guide" in libugp.ugp_last_error()
    st = libugp.ugp_guide_adam_step(None, None, None)
    assert st == 1
    st = libugp.ugp_guide_mixture_pdf(ctypes.c_int64(-1), None, None, None, None)
    assert st == 1


def test_guide_struct_layouts_match_the_header():
    """The ctypes mirrors have the C layout (offsets follow the header's field order)."""
    from paper_2406_09733_gb300 import ugp
    assert ctypes.sizeof(ugp.UgpGuide) == 88
    assert ugp.UgpGuide.kappa_max.offset == 76 and ugp.UgpGuide.train_target.offset == 80
    assert ctypes.sizeof(ugp.UgpRenderParams) == 56
    assert ugp.UgpRenderParams.guide.offset == 32 and ugp.UgpRenderParams.guide_alpha.offset == 40
    assert ugp.UgpRenderParams.guide_min_roughness.offset == 44
    assert ugp.UgpRenderParams.emitters.offset == 48


def test_batch_entry_points_validate_on_host(libugp):
    from paper_2406_09733_gb300 import ugp
    libugp.ugp_render_batch_workspace_size.restype = ctypes.c_size_t
    cfg = ugp.UgpBatchConfig(16, 12, 1, 0)
    assert libugp.ugp_render_batch_workspace_size(4, ctypes.byref(cfg)) > (1 << 12) * 24 * 4
    bad = ugp.UgpBatchConfig(12, 12, 1, 0)
    st = libugp.ugp_render_batch(0, None, ctypes.byref(bad), 4, None, ctypes.c_size_t(0), None, None, None)
    assert st == 1
    assert ctypes.sizeof(ugp.UgpRequest) == 168 and ugp.UgpRequest.seed.offset == 144


def test_binding_rejects_host_tensors():
    """The binding has no CPU path: host tensors are refused before the library is called."""
    torch = pytest.importorskip("torch")
    from paper_2406_09733_gb300 import ugp

    class FakeBvh:
        handle = 0
        n = 1
        workspace = torch.zeros(1)

    o = torch.zeros((4, 3))
    d = torch.zeros((4, 3))
    t = torch.zeros(4)
    for call in (lambda: ugp.trace_transmittance(FakeBvh(), o, d, t, t),
                 lambda: ugp.trace_transmittance_exponential(FakeBvh(), o, d, t, t),
                 lambda: ugp.sample_free_flight_exponential(FakeBvh(), o, d, t, t, t),
                 lambda: ugp.collect_hits(FakeBvh(), o, d, t, t, 4)):
        with pytest.raises(TypeError, match="CUDA tensor"):
            call()


def test_binding_checks_lengths_and_devices():
    """Per-ray arrays shorter than the ray count, and a workspace on another device than the
    rays, are refused before the library is called (the kernels would read or write past the
    array, or write through a host pointer)."""
    torch = pytest.importorskip("torch")
    from paper_2406_09733_gb300 import ugp

    class FakeBvh:
        handle = 0
        n = 4
        workspace = torch.zeros(1)

    o, d, t = torch.zeros((4, 3)), torch.zeros((4, 3)), torch.zeros(4)
    short, d_short = torch.zeros(3), torch.zeros((3, 3))
    ex_short = torch.zeros(3, dtype=torch.int32)
    for call in (lambda: ugp.trace_transmittance(FakeBvh(), o, d, short, t),
                 lambda: ugp.trace_transmittance(FakeBvh(), o, d_short, t, t),
                 lambda: ugp.trace_transmittance(FakeBvh(), o, d, t, t, exclude=ex_short),
                 lambda: ugp.sample_free_flight(FakeBvh(), o, d, t, t, t, short),
                 lambda: ugp.sample_free_flight_exponential(FakeBvh(), o, d, t, t, short),
                 lambda: ugp.collect_hits(FakeBvh(), o, d, t, short, 4)):
        with pytest.raises(ValueError, match="must hold"):
            call()
    host_ws = torch.zeros(1 << 12, dtype=torch.uint8)
    with pytest.raises(ValueError, match="expected cuda"):
        ugp._workspace(host_ws, 256, torch.device("cuda", 0))
    with pytest.raises(TypeError, match="uint8"):
        ugp._workspace(torch.zeros(1 << 12), 256, torch.device("cuda", 0))


def test_render_workspace_matches_the_documented_size(libugp):
    """ugp_render_workspace_size against the header's account: 1284 bytes per pixel (path
    state, queues, shadow queues, finish table, slot lists), one 73,728-byte interval slot of
    the finish per 64 pixels (4 to 2432 of them), plus 256-byte alignment of each column and a
    few headers."""
    libugp.ugp_render_workspace_size.restype = ctypes.c_size_t
    libugp.ugp_render_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int32]
    for w, h in ((1920, 1080), (1024, 1024), (64, 64), (7, 3)):
        n = w * h
        slots = min(max(n // 64, 4), 2432)
        expect = 1284 * n + slots * 73728
        got = libugp.ugp_render_workspace_size(w, h)
        assert expect <= got <= expect + 400 * 256 + 4096, (w, h, got, expect)
    assert libugp.ugp_render_workspace_size(0, 5) == 0
    assert libugp.ugp_render_workspace_size(1 << 16, 1 << 16) == 0


def test_free_flight_workspace_matches_the_documented_size(libugp):
    libugp.ugp_sample_free_flight_workspace_size.restype = ctypes.c_size_t
    libugp.ugp_sample_free_flight_workspace_size.argtypes = [ctypes.c_int64]
    for n in (1, 1000, 65536, 2073600):
        slots = min(max(n // 64, 4), 2432)
        expect = 1100 * n + slots * 73728
        got = libugp.ugp_sample_free_flight_workspace_size(n)
        assert expect <= got <= expect + 30 * 256 + 256, (n, got, expect)
    assert libugp.ugp_sample_free_flight_workspace_size(-1) == 0
