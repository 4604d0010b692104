"""Served form: continuous batching of frames from many cameras.

A camera's grid must come out the same, voxel for voxel, whether its frames
are served alone or mixed with many other cameras' frames arriving from
several threads, and the same as the plain frame-by-frame path.
"""
import threading

import numpy as np
import pytest

from synth import make

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


def _plain(vg, w):
    g = w.grid
    grid = vg.Grid(g.n, g.vox_size, w.cam.fov_x, w.cam.fov_y, g.depth, g.vox_inf, w.frames[0].robot_pos)
    for f in w.frames:
        grid.integrate_depth(torch.from_numpy(f.depth).cuda(), f.T_wc, w.cam.scale)
        grid.shift(f.robot_pos)
    out = torch.empty(grid.nvox, dtype=torch.uint8, device="cuda")
    o = grid.read(out)
    torch.cuda.synchronize()
    grid.close()
    return out.cpu().numpy(), o


def _submit_all(server, cam, w, tickets):
    for f in w.frames:
        while True:
            t = server.submit(cam, f.depth, f.T_wc, f.robot_pos, w.cam.scale)
            if t is not None:
                tickets.append(t)
                break
            threading.Event().wait(0.001)   # pool full: retry


@pytest.mark.parametrize("plain_max,queue_depth", [(1, 1), (4096, 3)], ids=["fused-and-chains", "chains-only"])
def test_same_result_alone_and_in_the_mix(vg, plain_max, queue_depth):
    # plain_max 1: single-frame batches run as per-frame chains and larger
    # ones as fused launches, so a camera's frames alternate between the two
    # (one launch at a time, so frames queue up and share launches);
    # 4096: every batch runs as per-frame chains on the lane streams, with
    # up to three launches, possibly holding frames of one camera, in flight
    target = make("robot", robot=30, frames=4)
    others = [make("robot", robot=40 + i, frames=3) for i in range(10)] + [make("hires", frames=2)]

    # alone
    s1 = vg.Server(8 << 30, max_batch=16)
    cam = _add(s1, target)
    tickets = []
    _submit_all(s1, cam, target, tickets)
    assert all(s1.wait(t) == vg.VG_OK for t in tickets)
    alone, o_alone = _read(s1, cam, target)
    s1.close()

    # in the mix: four client threads interleave all cameras' frames.  With
    # one launch at a time frames queue up and share launches whenever they
    # arrive faster than the server serves them; arrival times depend on the
    # host, so a run in which no launch happened to hold two frames is
    # repeated (at most three runs) before that counts as a failure
    ws = [target] + others
    for attempt in range(3):
        s2 = vg.Server(8 << 30, max_batch=8, queue_depth=queue_depth, pending_frames=24, plain_max=plain_max)
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
        mixed, o_mixed = _read(s2, cams[0], target)
        st = s2.stats()
        assert st["completed"] == st["submitted"] == sum(len(w.frames) for w in ws)
        for k in range(1, len(ws)):
            got, o = _read(s2, cams[k], ws[k])
            want, ow = _plain(vg, ws[k])
            assert list(o) == list(ow) and np.array_equal(got, want), "camera %d differs from the plain path" % k
        s2.close()
        assert list(o_alone) == list(o_mixed)
        assert np.array_equal(alone, mixed), "%d voxels differ alone vs mixed" % np.count_nonzero(alone != mixed)
        if queue_depth != 1 or st["mean_batch"] > 1.0:
            break
    if queue_depth == 1:
        assert st["mean_batch"] > 1.0, st       # frames did share launches
    want, ow = _plain(vg, target)
    assert list(o_alone) == list(ow) and np.array_equal(alone, want)


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
    with pytest.raises(vg.VGError):
        s.submit(cam, np.zeros((800, 1400), np.float32), f.T_wc)   # larger than the server's frames
    s.close()


def test_cameras_added_while_frames_are_served(vg):
    # cameras admitted from one thread while another submits frames of
    # earlier cameras: the server must keep serving every grid it admitted
    # (its camera table grows meanwhile), and each grid must match the
    # plain path
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
        got, o = _read(s, cam, w)
        want, ow = _plain(vg, w)
        assert list(o) == list(ow) and np.array_equal(got, want)
    assert s.stats()["cameras"] == len(first) + len(late)
    s.close()


@pytest.mark.parametrize("page_locked", [False, True], ids=["pageable", "page-locked"])
@pytest.mark.parametrize("robot", [89, 90], ids=["320x240", "848x480"])
def test_caller_may_reuse_its_buffer_when_submit_returns(vg, page_locked, robot):
    # a submit copies the frame before it returns: the client overwrites its
    # one buffer with the next frame (or garbage) at once, and the grid must
    # still match the plain path, whether the buffer is pageable or
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
    got, o = _read(s, cam, w)
    want, ow = _plain(vg, w)
    assert list(o) == list(ow) and np.array_equal(got, want)
    s.close()
