"""Served form: continuous batching of frames from many cameras.

A camera's grid must come out the same, voxel for voxel, whether its frames
are served alone or mixed with many other cameras' frames arriving from
several threads, and the same as the CPU oracle driven with that camera's
frames (integrate, then re-centre).  The mix covers every camera of the
served configuration: 320x240, 640x480 and 1280x720 depth, float32 and
uint16, into grids of 80x80x40 up to 400x400x120.
"""
import threading

import numpy as np
import pytest

from gridcheck import assert_grid, oracle_grid
from synth import make
from synth.scenes import CAMERA_KINDS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_13169_gb300 import build
    build.build()
    from paper_2112_13169_gb300 import vg as vgmod
    vgmod.load()
    return vgmod


def _add(server, w):
    g = w.grid
    return server.add_camera(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)


def _read(server, cam, w):
    out = np.empty(w.nvox, np.uint8)
    o = server.read(cam, out)
    return out, o


def _oracle(w):
    """The oracle grid after all of w's frames, each followed by its re-centre."""
    og = oracle_grid(w)
    for f in w.frames:
        og.integrate_depth(f.T_wc, f.depth, w.cam.scale)
        og.shift(f.robot_pos)
    return og


def _check(server, cam, w, og, what):
    got, o = _read(server, cam, w)
    assert_grid(got, o, og, "%s (%dx%d %s, grid %s)" % (what, w.cam.W, w.cam.H, w.cam.dtype, w.grid.n))


@pytest.fixture(scope="module")
def mix():
    """Two cameras of every kind of the served configuration, three frames
    each, with their oracle grids."""
    ws = [make("camera", robot=600 + i, frames=3, spec=i % CAMERA_KINDS) for i in range(2 * CAMERA_KINDS)]
    return ws, [_oracle(w) for w in ws]


def _submit_all(server, cam, w, tickets):
    for f in w.frames:
        while True:
            t = server.submit(cam, f.depth, f.T_wc, f.robot_pos, w.cam.scale)
            if t is not None:
                tickets.append(t)
                break
            threading.Event().wait(0.001)   # pool full: retry


@pytest.mark.parametrize("plain_max,queue_depth", [(1, 1), (4096, 3)], ids=["fused-and-chains", "chains-only"])
def test_same_result_alone_and_in_the_mix(vg, mix, plain_max, queue_depth):
    # plain_max 1: single-frame batches run as per-frame chains and larger
    # ones as fused launches, so a camera's frames alternate between the two
    # (one launch at a time, so frames queue up and share launches);
    # 4096: every batch runs as per-frame chains on the lane streams, with
    # up to three launches, possibly holding frames of one camera, in flight
    ws, oracles = mix
    kinds = {(w.cam.W, w.cam.H, w.cam.dtype) for w in ws}
    assert {(k[0], k[1]) for k in kinds} == {(320, 240), (640, 480), (1280, 720)}
    assert {k[2] for k in kinds} == {"f32", "u16"} and max(w.nvox for w in ws) == 400 * 400 * 120
    target = ws[5]   # 1280x720 f32 into a 400x400x120 grid

    # alone
    s1 = vg.Server(8 << 30, max_batch=16)
    cam = _add(s1, target)
    tickets = []
    _submit_all(s1, cam, target, tickets)
    assert all(s1.wait(t) == vg.VG_OK for t in tickets)
    _check(s1, cam, target, oracles[5], "served alone")
    s1.close()

    # in the mix: four client threads interleave all cameras' frames.  With
    # one launch at a time frames queue up and share launches whenever they
    # arrive faster than the server serves them; arrival times depend on the
    # host, so a run in which no launch happened to hold two frames is
    # repeated (at most three runs) before that counts as a failure
    for attempt in range(3):
        s2 = vg.Server(12 << 30, max_batch=8, queue_depth=queue_depth, pending_frames=24, plain_max=plain_max)
        cams = [_add(s2, w) for w in ws]
        tickets = []
        lock = threading.Lock()

        def client(idx):
            local = []
            rng = np.random.default_rng(idx)
            pos = {k: 0 for k in idx}
            while any(pos[k] < len(ws[k].frames) for k in idx):
                k = rng.choice([k for k in idx if pos[k] < len(ws[k].frames)])
                f = ws[k].frames[pos[k]]
                t = s2.submit(cams[k], f.depth, f.T_wc, f.robot_pos, ws[k].cam.scale)
                if t is None:
                    threading.Event().wait(0.001)
                    continue
                local.append(t)
                pos[k] += 1
            with lock:
                tickets.extend(local)

        threads = [threading.Thread(target=client, args=(list(range(i, len(ws), 4)),)) for i in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        assert all(s2.wait(t) == vg.VG_OK for t in tickets)
        st = s2.stats()
        assert st["completed"] == st["submitted"] == sum(len(w.frames) for w in ws)
        for k, (w, og) in enumerate(zip(ws, oracles)):
            _check(s2, cams[k], w, og, "camera %d in the mix" % k)
        s2.close()
        if queue_depth != 1 or st["mean_batch"] > 1.0:
            break
    if queue_depth == 1:
        assert st["mean_batch"] > 1.0, st       # frames did share launches


def test_admission_by_memory_budget(vg):
    w = make("robot", robot=50, frames=1)
    g = w.grid
    per_grid = vg.vg_grid_bytes(vg.make_params(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf))
    # the server's own frame pool (16 pending frames of 1280x720x4, the
    # default 4 x max_batch) and 2 launch tables, plus room for two grids
    fixed = 16 * ((1280 * 720 * 4 + 255) // 256 * 256) + 2 * (4 * 1024 + 4096)
    s = vg.Server(fixed + 2 * per_grid + per_grid // 2, max_batch=4)
    a = _add(s, w)
    b = _add(s, w)
    with pytest.raises(vg.VGError) as e:
        _add(s, w)
    assert e.value.status == vg.VG_ENOMEM
    s.remove_camera(a)
    c = _add(s, w)                                 # the freed memory is admitted again
    assert c != a and s.stats()["cameras"] == 2
    with pytest.raises(vg.VGError):
        s.submit(a, w.frames[0].depth, w.frames[0].T_wc)   # removed camera
    s.close()
    del b


def test_backpressure_and_latency_counters(vg):
    # 1280x720 frames on a 400x400x120 grid take the device longer than a
    # submit takes, and two threads submit at once, so a 4-frame pool fills
    w = make("hires", frames=1)
    s = vg.Server(4 << 30, max_batch=4, queue_depth=1, pending_frames=4)
    cam = _add(s, w)
    f = w.frames[0]
    tickets, busy = [], [0, 0]

    def client(i):
        for _ in range(48):
            t = s.submit(cam, f.depth, f.T_wc, None, w.cam.scale)
            if t is None:
                busy[i] += 1
            else:
                tickets.append(t)

    threads = [threading.Thread(target=client, args=(i,)) for i in range(2)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert sum(busy) > 0, "a 4-frame pool never filled"
    assert all(s.wait(t) == vg.VG_OK for t in tickets)
    st = s.stats()
    assert st["completed"] == len(tickets) and st["latency_p50_us"] > 0 and st["latency_p99_us"] >= st["latency_p50_us"]
    # per-ticket stamps on the host's monotonic clock (time.monotonic's)
    import time
    now = time.monotonic()
    lat = []
    for t in tickets:
        rc, sub, done = s.ticket_times(t)
        assert rc == vg.VG_OK and sub <= done <= now, (rc, sub, done, now)
        lat.append(done - sub)
    assert abs(np.percentile(lat, 50) * 1e6 - st["latency_p50_us"]) <= 0.1 * st["latency_p50_us"] + 50
    with pytest.raises(vg.VGError):
        s.ticket_times(10 ** 9)
    with pytest.raises(vg.VGError):
        s.submit(cam, np.zeros((800, 1400), np.float32), f.T_wc)   # larger than the server's frames
    s.close()


def test_cameras_added_while_frames_are_served(vg):
    # cameras admitted from one thread while another submits frames of
    # earlier cameras: the server must keep serving every grid it admitted
    # (its camera table grows meanwhile), and each grid must match the
    # oracle
    first = [make("robot", robot=70 + i, frames=3) for i in range(3)]
    late = [make("robot", robot=80 + i, frames=1) for i in range(24)]
    s = vg.Server(8 << 30, max_batch=4, queue_depth=3, pending_frames=12, plain_max=2)
    cams = [_add(s, w) for w in first]
    added = []

    def adder():
        for w in late:
            added.append((_add(s, w), w))

    th = threading.Thread(target=adder)
    th.start()
    tickets = []
    for k in range(3):
        for cam, w in zip(cams, first):
            _submit_all(s, cam, type(w)(w.name, w.cam, w.grid, [w.frames[k]], w.prims), tickets)
    th.join()
    for cam, w in added:
        _submit_all(s, cam, w, tickets)
    assert all(s.wait(t) == vg.VG_OK for t in tickets)
    for cam, w in list(zip(cams, first)) + added[:4]:
        _check(s, cam, w, _oracle(w), "camera %d" % cam)
    assert s.stats()["cameras"] == len(first) + len(late)
    s.close()


@pytest.mark.parametrize("page_locked", [False, True], ids=["pageable", "page-locked"])
@pytest.mark.parametrize("robot", [89, 90], ids=["320x240", "848x480"])
def test_caller_may_reuse_its_buffer_when_submit_returns(vg, page_locked, robot):
    # a submit copies the frame before it returns: the client overwrites its
    # one buffer with the next frame (or garbage) at once, and the grid must
    # still match the oracle, whether the buffer is pageable or
    # page-locked (a copy from page-locked memory would otherwise still be
    # in flight)
    w = make("robot", robot=robot, frames=4)
    s = vg.Server(4 << 30, max_batch=4, queue_depth=2, pending_frames=8)
    cam = _add(s, w)
    shape, dt = w.frames[0].depth.shape, w.frames[0].depth.dtype
    if page_locked:
        buf = torch.empty(shape, dtype=torch.float32 if dt == np.float32 else torch.uint16).pin_memory().numpy()
    else:
        buf = np.empty(shape, dt)
    tickets = []
    for f in w.frames:
        np.copyto(buf, f.depth)
        while True:
            t = s.submit(cam, buf, f.T_wc, f.robot_pos, w.cam.scale)
            if t is not None:
                break
            threading.Event().wait(0.001)
        tickets.append(t)
        buf.fill(0.5 if dt == np.float32 else 7)   # the caller's next use of its buffer
    assert all(s.wait(t) == vg.VG_OK for t in tickets)
    _check(s, cam, w, _oracle(w), "buffer reused after each submit")
    s.close()
