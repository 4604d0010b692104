"""libvg.so without a GPU: it builds, loads, exports every entry point that
include/vg.h declares, its host-only helpers agree with the oracle and the
paper, and compute calls fail loudly (no CPU fallback) when no device is
present."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def vg():
    from paper_2112_13169_gb300 import build
    build.build()
    from paper_2112_13169_gb300 import vg as vgmod
    vgmod.load()
    return vgmod


def _declared():
    src = open(os.path.join(ROOT, "include", "vg.h")).read()
    return sorted(set(re.findall(r"VG_API\s+[\w\s\*]+?\b(vg_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("vg_create", "vg_integrate_depth", "vg_integrate_points", "vg_shift",
                     "vg_read", "vg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(vg):
    lib = C.CDLL(vg.LIB_PATH)
    names = _declared()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(vg.EXPORTS) == names


def test_exports_nothing_else(vg):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", vg.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    text = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert sorted(text) == _declared()


@pytest.mark.parametrize("cfg", [
    ((100, 100, 20), 0.15, 85.0, 101.0, 6.5, 2),
    ((80, 80, 40), 0.1, 87.0, 58.0, 4.0, 1),
    ((200, 200, 100), 0.05, 87.0, 58.0, 5.0, 2),
    ((400, 400, 120), 0.05, 90.0, 60.0, 6.0, 2),
    ((7, 5, 3), 0.2, 30.0, 150.0, 1.3, 0),
])
def test_ray_bundle_matches_oracle(vg, orc, cfg):
    from oracle import OracleParams
    p = vg.make_params(*cfg)
    got, n = vg.vg_ray_bundle(p)
    want, wn = orc.ray_bundle(OracleParams(*cfg))
    assert tuple(got) == tuple(want) and n == wn


def test_paper_standard_setup_ray_count(vg):
    import json
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_standard_setup.json")))
    n = [int(round(m / g["vox_size_m"])) for m in g["grid_size_m"]]
    p = vg.make_params(n, g["vox_size_m"], g["fov_x_deg"], g["fov_y_deg"], g["depth_m"], g["vox_inf"])
    _, nrays = vg.vg_ray_bundle(p)
    assert abs(nrays - g["printed_rays_approx"]) / g["printed_rays_approx"] <= g["rays_rel_tolerance"]
    assert n[0] * n[1] * n[2] == g["printed_voxels"]


def test_grid_bytes(vg):
    p = vg.make_params((200, 200, 100), 0.05, 87, 58, 5.0, 2)
    b = vg.vg_grid_bytes(p)
    # two loc buffers of N bytes and four bit planes of 8 words x 200 x 100
    assert b >= 2 * (4_000_000 + 16) + 4 * 8 * 4 * 200 * 100
    assert b < 2 * 4_000_000 + 4 * 8 * 4 * 200 * 100 + 4096
    bad = vg.make_params((0, 10, 10), 0.05, 87, 58, 5.0, 2)
    assert vg.vg_grid_bytes(bad) == 0


def test_kernel_ids_match_the_header(vg):
    # the binding sizes vg_profile_read's arrays from its kernel list
    hdr = open(os.path.join(ROOT, "include", "vg.h")).read()
    ids = dict(re.findall(r"VG_K_(\w+) = (\d+)", hdr))
    n = int(re.search(r"VG_NKERNELS = (\d+)", hdr).group(1))
    assert n == len(vg.KERNELS) == len(ids)
    assert sorted(int(v) for v in ids.values()) == list(range(n))
    for name, v in ids.items():
        assert vg.KERNELS[int(v)] == name.lower(), (name, v)


def test_grid_bytes_of_literal_flags(vg):
    args = ((200, 200, 100), 0.05, 87, 58, 5.0, 2)
    base = vg.vg_grid_bytes(vg.make_params(*args))
    # the loc_grid reading holds one more bit plane; the others none
    assert vg.vg_grid_bytes(vg.make_params(*args, flags=vg.VG_FLAG_LIT_LOC_OCCUPANCY)) == base + 8 * 4 * 200 * 100
    for f in (vg.VG_FLAG_LIT_INFLATE_AFTER_TRACE, vg.VG_FLAG_LIT_SKIP_START_VOXEL, vg.VG_FLAG_STATS):
        assert vg.vg_grid_bytes(vg.make_params(*args, flags=f)) == base
    # exclusive readings, and unknown bits, are invalid parameters
    both = vg.VG_FLAG_LIT_INFLATE_AFTER_TRACE | vg.VG_FLAG_LIT_LOC_OCCUPANCY
    assert vg.vg_grid_bytes(vg.make_params(*args, flags=both)) == 0
    assert vg.vg_grid_bytes(vg.make_params(*args, flags=1 << 7)) == 0


@pytest.mark.parametrize("field,value", [
    ("grid_size", (0, 10, 10)), ("vox_size", 0.0), ("vox_size", float("nan")), ("fov_x_deg", 180.0),
    ("fov_y_deg", 0.0), ("depth", -1.0), ("vox_inf", 16), ("vox_inf", -1), ("grid_size", (2048, 2048, 1024)),
    ("grid_size", (1, 65536, 512)),   # 2^27 plane words: beyond K3's 32-bit plane bit index
])
def test_create_rejects_bad_params(vg, field, value):
    kw = dict(n=(10, 10, 10), vox_size=0.1, fov_x_deg=87, fov_y_deg=58, depth=4.0, vox_inf=1)
    key = {"grid_size": "n"}.get(field, field)
    kw[key] = value
    p = vg.make_params(kw["n"], kw["vox_size"], kw["fov_x_deg"], kw["fov_y_deg"], kw["depth"], kw["vox_inf"])
    with pytest.raises(vg.VGError) as e:
        vg.vg_create(p, (0.0, 0.0, 0.0), stream=0)
    assert e.value.status == vg.VG_EINVAL


@pytest.mark.parametrize("pos", [(0.0, float("inf"), 0.0), (0.0, 0.0, float("nan")), (2.0e8, 0.0, 0.0)])
def test_create_rejects_unusable_position(vg, pos):
    # not finite, or an origin index (pos / vox_size) of 2^30 or more
    p = vg.make_params((10, 10, 10), 0.1, 87, 58, 4.0, 1)
    with pytest.raises(vg.VGError) as e:
        vg.vg_create(p, pos, stream=0)
    assert e.value.status == vg.VG_EINVAL


def test_no_gpu_means_an_error_not_a_fallback(vg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = vg.make_params((10, 10, 10), 0.1, 87, 58, 4.0, 1)
    with pytest.raises(vg.VGError) as e:
        vg.vg_create(p, (0.0, 0.0, 0.0), stream=0)
    assert e.value.status == vg.VG_ECUDA


def test_null_handles_are_rejected(vg):
    L = vg.load()
    T = np.eye(4).ravel()
    assert L.vg_integrate_depth(None, None, 0, 4, 4, 0, 1.0, T.ctypes.data, None) == vg.VG_EINVAL
    assert L.vg_shift(None, np.zeros(3).ctypes.data, None) == vg.VG_EINVAL
    assert L.vg_read(None, None, 0, 0, None, None) == vg.VG_EINVAL
    assert L.vg_tune(None, 0, 8) == vg.VG_EINVAL
    L.vg_destroy(None)
    assert vg.strerror(vg.VG_EINVAL) == "invalid argument"


@pytest.mark.parametrize("field,value", [("max_batch", 0), ("queue_depth", 0), ("queue_depth", 9),
                                         ("pending_frames", 1), ("memory_budget", 0), ("plain_max", -1),
                                         ("plain_max", 5000), ("max_width", 0)])
def test_server_rejects_bad_params_before_any_device_work(vg, field, value):
    p = vg.vg_server_params()
    p.memory_budget, p.max_batch, p.max_width, p.max_height = 1 << 30, 8, 640, 480
    p.queue_depth, p.pending_frames, p.plain_max = 2, 16, 0
    setattr(p, field, value)
    h = C.c_void_p()
    assert vg.load().vg_server_create(C.byref(p), C.byref(h)) == vg.VG_EINVAL
    assert not h.value


def test_batch_and_server_null_handles(vg):
    L = vg.load()
    assert L.vg_batch_prepare(None, None, 1) == vg.VG_EINVAL
    assert L.vg_batch_enqueue(None, None) == vg.VG_EINVAL
    assert L.vg_batch_status(None) == vg.VG_EINVAL
    assert L.vg_server_wait(None, 0, 0) == vg.VG_EINVAL
    st = vg.vg_server_stats_t()
    assert L.vg_server_stats(None, C.byref(st), 0) == vg.VG_EINVAL
    L.vg_batch_destroy(None)
    L.vg_server_destroy(None)


def test_current_stream_lookup_falls_back_to_the_public_call(vg):
    # the binding reads torch's current stream through torch's raw getter
    # where it exists (the handle of the current device's current stream),
    # else through torch.cuda.current_stream(); both give the same integer
    import types
    calls = []

    class FakeCuda:
        @staticmethod
        def current_device():
            return 3

        @staticmethod
        def current_stream():
            calls.append("public")
            return types.SimpleNamespace(cuda_stream=0xabc)

    with_raw = types.SimpleNamespace(cuda=FakeCuda, _C=types.SimpleNamespace(
        _cuda_getCurrentRawStream=lambda dev: calls.append(("raw", dev)) or 0xabc))
    without_raw = types.SimpleNamespace(cuda=FakeCuda, _C=types.SimpleNamespace())
    assert vg._current_stream_getter(with_raw)() == 0xabc
    assert calls == [("raw", 3)]
    assert vg._current_stream_getter(without_raw)() == 0xabc
    assert calls == [("raw", 3), "public"]
    # explicit streams pass through unchanged
    assert vg._stream(0x1234) == 0x1234
    assert vg._stream(types.SimpleNamespace(cuda_stream=0x99)) == 0x99
