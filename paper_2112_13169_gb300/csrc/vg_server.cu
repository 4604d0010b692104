// vg_server.cu -- the served form: continuous batching of measurements from
// many cameras (declared in include/vg.h).
//
// Client threads submit frames into one arrival-ordered queue.  Each frame
// is copied from the caller's host memory (pageable or page-locked) into a
// slot of a device pool on one of a few copy streams, and the submit
// returns once that copy has ended.  The server thread repeatedly
//   - polls the completion events of the launches in flight, stamping each
//     frame's completion time as soon as its work has ended, and retires a
//     launch (status, latencies, pool slots, launch slot) once all of its
//     frames have ended,
//   - forms a batch when a launch slot is free: the oldest queued frames,
//     at most one per camera, skipping cameras being read,
//   - issues the batch in one of two ways:
//       small batches (at most plain_max frames): each frame runs the
//       per-frame kernel chain (K1..K4, PDL-chained) on its camera's lane
//       stream, K1 reading the frame from its pool slot; frames of
//       different cameras overlap on the device;
//       larger batches: one fused cooperative launch (vg_batch_prepare +
//       vg_batch_enqueue) on the fused stream, reading the pool slots too.
// Frames of one camera apply in submission order: one per launch, launches
// issued in order, a camera always on the same lane stream, and every fused
// launch fenced both ways against the lanes (it waits for the lanes' work
// issued before it, and lane work issued after it waits for it).  The fence
// also means a cooperative launch never shares the device with this
// server's other kernels, so its CTAs are all resident together.
//
// While launches are in flight the server thread spins on their events
// (cudaEventQuery) instead of sleeping, so a completion is seen within
// microseconds; with nothing in flight it sleeps on the condition variable.
// The server's mutex is never held across a CUDA call (a copy stream's own
// mutex is, for one submit's copy), and the server's streams are
// non-blocking so a synchronous copy elsewhere does not wait for them.
#include "vg.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

namespace {

using Clock = std::chrono::steady_clock;

// Lane streams for small batches; a camera always uses lane camera % kLanes.
constexpr int kLanes = 8;
// Default largest batch issued as per-frame chains (vg_server_params.plain_max == 0).
constexpr int kDefaultPlainMax = 4;
// Streams that copy submitted frames into the pool; concurrent submits take
// them in turn.
constexpr int kCopyStreams = 4;

struct Request {
    uint64_t ticket;
    vg_grid *grid;   // the camera's grid, captured under the lock when the batch is formed
    int32_t camera, slot, width, height, dtype, recentre;
    float scale;
    double T_wc[16], pos[3];
    Clock::time_point arrival;
    Clock::time_point done_at;
    int status;      // VG_OK, or the frame's error
    bool ended;      // its device work has ended (or never started)
};

struct Camera {
    vg_grid *grid = nullptr;
    int64_t bytes = 0;
    bool removed = false;
    bool reading = false;
    int32_t pending = 0;   // queued or in flight
};

struct Launch {
    vg_batch *batch = nullptr;
    cudaEvent_t done = nullptr;   // end of a fused launch
    std::vector<cudaEvent_t> ev;  // end of each frame's chain (per-frame launches)
    std::vector<Request> reqs;
    bool busy = false;     // formed, not yet retired
    bool issued = false;   // its device work has been enqueued
    bool fused = false;
    int remaining = 0;     // frames whose device work has not been seen to end
};

}  // namespace

struct vg_server {
    vg_server_params p;
    int plain_max = kDefaultPlainMax;
    int device = 0;
    size_t frame_bytes = 0;
    cudaStream_t compute = nullptr, admin = nullptr;
    cudaStream_t copies[kCopyStreams] = {};
    std::mutex copy_mu[kCopyStreams];     // one submit at a time per copy stream
    std::atomic<unsigned> next_copy{0};
    cudaStream_t lanes[kLanes] = {};
    cudaEvent_t lane_tail[kLanes] = {};   // a lane's work before a fused launch
    bool lane_dirty[kLanes] = {};         // work issued on the lane since the last fused fence
    bool lane_behind[kLanes] = {};        // a fused launch was issued since the lane's last work
    cudaEvent_t fused_tail = nullptr;     // end of the last fused launch
    uint8_t *slots = nullptr;             // device pool: pending_frames frames of frame_bytes
    std::vector<int32_t> free_slots;
    std::vector<Camera> cams;
    std::deque<Request> queue;
    std::vector<Launch> launches;
    int32_t inflight = 0;
    int64_t fixed_bytes = 0, grid_bytes = 0;
    std::vector<uint8_t> status;   // per ticket: 0 pending, 1 done, 2 failed
    std::vector<double> t_submit;  // per ticket: submission and completion, monotonic clock seconds
    std::vector<double> t_done;
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_frames = 0;
    std::vector<float> lat_us;
    std::mutex mu;
    std::condition_variable cv;
    std::thread th;
    bool stop = false;
};

namespace {

bool can_launch(const vg_server *S) {
    if (S->inflight >= S->p.queue_depth) return false;
    for (const Request &r : S->queue)
        if (!S->cams[r.camera].reading) return true;
    return false;
}

// Under the lock: retire a launch all of whose frames have ended.
double seconds(Clock::time_point t) { return std::chrono::duration<double>(t.time_since_epoch()).count(); }

void finish(vg_server *S, Launch &L) {
    for (const Request &r : L.reqs) {
        S->status[r.ticket] = r.status == VG_OK ? 1 : 2;
        S->t_done[r.ticket] = seconds(r.done_at);
        if (r.status == VG_OK) {
            ++S->completed;
            S->lat_us.push_back((float)std::chrono::duration<double, std::micro>(r.done_at - r.arrival).count());
        } else {
            ++S->failed;
        }
        --S->cams[r.camera].pending;
        S->free_slots.push_back(r.slot);
    }
    ++S->batches;
    S->batched_frames += L.reqs.size();
    L.reqs.clear();
    L.busy = false;
    L.issued = false;
    --S->inflight;
    S->cv.notify_all();
}

void end_frame(Request &r, int st, Clock::time_point when, int &remaining) {
    if (r.ended) return;
    r.ended = true;
    r.status = st;
    r.done_at = when;
    --remaining;
}

// Server thread, no lock: notes which frames of an issued launch have ended.
void poll(Launch &L) {
    if (L.fused) {
        const cudaError_t e = cudaEventQuery(L.done);
        if (e == cudaErrorNotReady) return;
        const Clock::time_point now = Clock::now();
        const int st = e != cudaSuccess ? VG_ECUDA : vg_batch_status(L.batch);   // ended: no wait
        for (Request &r : L.reqs) end_frame(r, st, now, L.remaining);
        return;
    }
    for (size_t k = 0; k < L.reqs.size(); ++k) {
        Request &r = L.reqs[k];
        if (r.ended) continue;
        const cudaError_t e = cudaEventQuery(L.ev[k]);
        if (e == cudaErrorNotReady) continue;
        end_frame(r, e == cudaSuccess ? VG_OK : VG_ECUDA, Clock::now(), L.remaining);
    }
}

// Per-frame chains: each frame on its camera's lane, K1 reading its pool
// slot.  A frame whose work could not be enqueued ends now with its error.
void issue_lanes(vg_server *S, Launch &L) {
    for (size_t k = 0; k < L.reqs.size(); ++k) {
        Request &r = L.reqs[k];
        const int lane = r.camera % kLanes;
        cudaStream_t st = S->lanes[lane];
        int rc = VG_OK;
        if (S->lane_behind[lane]) {
            if (cudaStreamWaitEvent(st, S->fused_tail, 0) != cudaSuccess) rc = VG_ECUDA;
            else S->lane_behind[lane] = false;
        }
        S->lane_dirty[lane] = true;
        vg_grid *grid = r.grid;
        if (rc == VG_OK)
            rc = vg_integrate_depth(grid, S->slots + (size_t)r.slot * S->frame_bytes, VG_MEM_DEVICE, r.width,
                                    r.height, r.dtype, r.scale, r.T_wc, st);
        if (rc == VG_OK && r.recentre) rc = vg_shift(grid, r.pos, st);
        if (rc == VG_OK && cudaEventRecord(L.ev[k], st) != cudaSuccess) rc = VG_ECUDA;
        if (rc != VG_OK) end_frame(r, rc, Clock::now(), L.remaining);
    }
}

// One fused launch, fenced against the lanes.  Returns VG_OK once enqueued.
int issue_fused(vg_server *S, Launch &L) {
    const size_t n = L.reqs.size();
    for (int i = 0; i < kLanes; ++i) {
        if (!S->lane_dirty[i]) continue;
        if (cudaEventRecord(S->lane_tail[i], S->lanes[i]) != cudaSuccess ||
            cudaStreamWaitEvent(S->compute, S->lane_tail[i], 0) != cudaSuccess)
            return VG_ECUDA;
        S->lane_dirty[i] = false;
    }
    std::vector<vg_frame> fr(n);
    for (size_t k = 0; k < n; ++k) {
        const Request &r = L.reqs[k];
        vg_frame &f = fr[k];
        std::memset(&f, 0, sizeof(f));
        f.grid = r.grid;
        f.depth = S->slots + (size_t)r.slot * S->frame_bytes;
        f.width = r.width;
        f.height = r.height;
        f.dtype = r.dtype;
        f.depth_scale = r.scale;
        std::memcpy(f.T_wc, r.T_wc, sizeof(f.T_wc));
        f.recentre = r.recentre;
        std::memcpy(f.robot_pos_w, r.pos, sizeof(f.robot_pos_w));
    }
    int rc = vg_batch_prepare(L.batch, fr.data(), (int32_t)n);
    if (rc == VG_OK) rc = vg_batch_enqueue(L.batch, S->compute);
    if (rc != VG_OK) return rc;
    if (cudaEventRecord(S->fused_tail, S->compute) != cudaSuccess) return VG_ECUDA;
    for (int i = 0; i < kLanes; ++i) S->lane_behind[i] = true;
    return cudaEventRecord(L.done, S->compute) == cudaSuccess ? VG_OK : VG_ECUDA;
}

void issue(vg_server *S, Launch &L) {
    L.remaining = (int)L.reqs.size();
    for (Request &r : L.reqs) r.ended = false;
    L.fused = (int)L.reqs.size() > S->plain_max;
    if (!L.fused) {
        issue_lanes(S, L);
        return;
    }
    const int rc = issue_fused(S, L);
    if (rc != VG_OK) {
        // nothing of this batch is waited for: end it here
        const Clock::time_point now = Clock::now();
        for (Request &r : L.reqs) end_frame(r, rc, now, L.remaining);
    }
}

void server_loop(vg_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool in_flight = false;
        std::vector<Launch *> done;
        for (Launch &L : S->launches) {
            if (!L.busy || !L.issued) continue;
            if (L.remaining > 0) poll(L);
            if (L.remaining == 0) done.push_back(&L);
            else in_flight = true;
        }
        Launch *next = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            for (Launch *L : done) finish(S, *L);
            auto idle_exit = [&] { return S->stop && S->queue.empty() && S->inflight == 0; };
            if (!in_flight && !can_launch(S)) {
                if (idle_exit()) return;
                S->cv.wait(lk, [&] { return can_launch(S) || idle_exit(); });
                if (!can_launch(S)) return;   // idle_exit
            }
            if (can_launch(S)) {
                for (Launch &L : S->launches)
                    if (!L.busy) {
                        next = &L;
                        break;
                    }
                // the oldest frames, at most one per camera, none of a camera being read
                std::vector<char> used(S->cams.size(), 0);
                for (auto it = S->queue.begin();
                     it != S->queue.end() && next->reqs.size() < (size_t)S->p.max_batch;) {
                    if (used[it->camera] || S->cams[it->camera].reading) {
                        ++it;
                        continue;
                    }
                    used[it->camera] = 1;
                    next->reqs.push_back(*it);
                    // the camera vector may grow (and move) under a concurrent
                    // vg_server_add_camera once the lock is released; the grid
                    // itself lives until the camera has no pending frame
                    next->reqs.back().grid = S->cams[it->camera].grid;
                    it = S->queue.erase(it);
                }
                next->busy = true;
                ++S->inflight;
            }
        }
        if (next) {
            issue(S, *next);
            next->issued = true;
        } else if (in_flight) {
            std::this_thread::yield();
        }
    }
}

}  // namespace

extern "C" {

int vg_server_create(const vg_server_params *p, vg_server **out) {
    if (!out) return VG_EINVAL;
    *out = nullptr;
    if (!p || p->max_batch < 1 || p->max_batch > 4096 || p->queue_depth < 1 || p->queue_depth > 8 ||
        p->max_width < 1 || p->max_height < 1 || (int64_t)p->max_width * p->max_height >= (int64_t(1) << 31) ||
        p->pending_frames < p->max_batch || p->memory_budget <= 0 || p->plain_max < 0 || p->plain_max > 4096)
        return VG_EINVAL;
    vg_server *S = new (std::nothrow) vg_server();
    if (!S) return VG_ENOMEM;
    S->p = *p;
    S->plain_max = p->plain_max ? p->plain_max : kDefaultPlainMax;
    S->frame_bytes = ((size_t)p->max_width * p->max_height * 4 + 255) & ~size_t(255);
    // the frame pool and a generous bound on each launch's descriptor table
    S->fixed_bytes = (int64_t)(S->frame_bytes * (size_t)p->pending_frames) +
                     (int64_t)((size_t)p->max_batch * 1024 + 4096) * p->queue_depth;
    if (S->fixed_bytes > p->memory_budget) {
        delete S;
        return VG_ENOMEM;
    }
    cudaError_t e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->compute, cudaStreamNonBlocking);
    for (int i = 0; i < kCopyStreams && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&S->copies[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->admin, cudaStreamNonBlocking);
    for (int i = 0; i < kLanes && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&S->lanes[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->lane_tail[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->fused_tail, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void **)&S->slots, S->frame_bytes * (size_t)p->pending_frames);
    int rc = e == cudaSuccess ? VG_OK : (e == cudaErrorMemoryAllocation ? VG_ENOMEM : VG_ECUDA);
    S->launches.resize((size_t)p->queue_depth);
    for (Launch &L : S->launches) {
        if (rc != VG_OK) break;
        rc = vg_batch_create(p->max_batch, &L.batch);
        if (rc == VG_OK && cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess) rc = VG_ECUDA;
        const int nev = std::min(S->plain_max, p->max_batch);
        for (int k = 0; k < nev && rc == VG_OK; ++k) {
            cudaEvent_t ev = nullptr;
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) rc = VG_ECUDA;
            else L.ev.push_back(ev);
        }
    }
    if (rc != VG_OK) {
        vg_server_destroy(S);
        return rc;
    }
    for (int32_t i = p->pending_frames - 1; i >= 0; --i) S->free_slots.push_back(i);
    try {
        S->th = std::thread(server_loop, S);
    } catch (...) {
        vg_server_destroy(S);
        return VG_ENOMEM;
    }
    *out = S;
    return VG_OK;
}

void vg_server_destroy(vg_server *S) {
    if (!S) return;
    if (S->th.joinable()) {
        {
            std::lock_guard<std::mutex> g(S->mu);
            S->stop = true;
            S->cv.notify_all();
        }
        S->th.join();
    }
    cudaSetDevice(S->device);
    if (S->compute) cudaStreamSynchronize(S->compute);
    for (int i = 0; i < kLanes; ++i)
        if (S->lanes[i]) cudaStreamSynchronize(S->lanes[i]);
    for (Launch &L : S->launches) {
        vg_batch_destroy(L.batch);
        if (L.done) cudaEventDestroy(L.done);
        for (cudaEvent_t ev : L.ev) cudaEventDestroy(ev);
    }
    for (int i = 0; i < kLanes; ++i) {
        if (S->lanes[i]) cudaStreamDestroy(S->lanes[i]);
        if (S->lane_tail[i]) cudaEventDestroy(S->lane_tail[i]);
    }
    if (S->fused_tail) cudaEventDestroy(S->fused_tail);
    for (Camera &c : S->cams)
        if (c.grid) vg_destroy(c.grid);
    cudaFree(S->slots);
    if (S->compute) cudaStreamDestroy(S->compute);
    for (int i = 0; i < kCopyStreams; ++i)
        if (S->copies[i]) cudaStreamDestroy(S->copies[i]);
    if (S->admin) cudaStreamDestroy(S->admin);
    delete S;
}

int vg_server_add_camera(vg_server *S, const vg_params *params, const double robot_pos_w[3], int32_t *camera) {
    if (!S || !params || !robot_pos_w || !camera || params->vox_inf > 3) return VG_EINVAL;
    if (params->flags & (VG_FLAG_LIT_INFLATE_AFTER_TRACE | VG_FLAG_LIT_SKIP_START_VOXEL | VG_FLAG_LIT_LOC_OCCUPANCY))
        return VG_EINVAL;   // literal readings take the plain path only
    const int64_t bytes = vg_grid_bytes(params);
    if (bytes <= 0) return VG_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->fixed_bytes + S->grid_bytes + bytes > S->p.memory_budget) return VG_ENOMEM;
        S->grid_bytes += bytes;   // reserved while the grid is made
    }
    vg_grid *grid = nullptr;
    int rc = vg_create(params, robot_pos_w, S->admin, &grid);
    std::lock_guard<std::mutex> g(S->mu);
    if (rc != VG_OK) {
        S->grid_bytes -= bytes;
        return rc;
    }
    Camera c;
    c.grid = grid;
    c.bytes = bytes;
    S->cams.push_back(c);
    *camera = (int32_t)S->cams.size() - 1;
    return VG_OK;
}

int vg_server_remove_camera(vg_server *S, int32_t camera) {
    if (!S) return VG_EINVAL;
    vg_grid *grid = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        if (camera < 0 || camera >= (int32_t)S->cams.size() || S->cams[camera].removed) return VG_EINVAL;
        S->cams[camera].removed = true;
        S->cv.wait(lk, [&] { return S->cams[camera].pending == 0; });
        grid = S->cams[camera].grid;
        S->cams[camera].grid = nullptr;
        S->grid_bytes -= S->cams[camera].bytes;
    }
    vg_destroy(grid);
    return VG_OK;
}

int vg_server_submit(vg_server *S, int32_t camera, const void *depth, int32_t width, int32_t height, int32_t dtype,
                     float depth_scale, const double T_wc[16], int32_t recentre, const double robot_pos_w[3],
                     uint64_t *ticket) {
    const Clock::time_point arrival = Clock::now();
    if (!S || !depth || !T_wc || width < 1 || height < 1 || width > S->p.max_width || height > S->p.max_height)
        return VG_EINVAL;
    if (dtype != VG_DEPTH_F32 && dtype != VG_DEPTH_U16) return VG_EINVAL;
    if (dtype == VG_DEPTH_U16 && !(depth_scale > 0.0f && depth_scale < 1e30f)) return VG_EINVAL;
    if (recentre && !robot_pos_w) return VG_EINVAL;
    for (int i = 0; i < 16; ++i)
        if (!(T_wc[i] == T_wc[i]) || T_wc[i] > 1e300 || T_wc[i] < -1e300) return VG_EINVAL;
    Request r;
    r.camera = camera;
    r.width = width;
    r.height = height;
    r.dtype = dtype;
    r.scale = depth_scale;
    r.recentre = recentre != 0;
    std::memcpy(r.T_wc, T_wc, sizeof(r.T_wc));
    if (recentre) std::memcpy(r.pos, robot_pos_w, sizeof(r.pos));
    else std::memset(r.pos, 0, sizeof(r.pos));
    r.arrival = arrival;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (camera < 0 || camera >= (int32_t)S->cams.size() || S->cams[camera].removed) return VG_EINVAL;
        if (S->free_slots.empty()) return VG_EBUSY;
        r.slot = S->free_slots.back();
        S->free_slots.pop_back();
        ++S->cams[camera].pending;   // keeps the camera alive while the frame is copied in
    }
    // the frame goes straight into its device slot, whether the caller's
    // memory is pageable or page-locked, and the call returns once the copy
    // has ended, so the caller may reuse its buffer at once
    const size_t bytes = (size_t)width * height * (dtype == VG_DEPTH_F32 ? 4 : 2);
    cudaError_t e = cudaSuccess;
    {
        int prev = -1;
        e = cudaGetDevice(&prev);
        if (e == cudaSuccess && prev != S->device) e = cudaSetDevice(S->device);
        const unsigned c = S->next_copy.fetch_add(1u, std::memory_order_relaxed) % kCopyStreams;
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> cg(S->copy_mu[c]);
            e = cudaMemcpyAsync(S->slots + (size_t)r.slot * S->frame_bytes, depth, bytes, cudaMemcpyHostToDevice,
                                S->copies[c]);
            if (e == cudaSuccess) e = cudaStreamSynchronize(S->copies[c]);
        }
        if (prev >= 0 && prev != S->device) cudaSetDevice(prev);
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (e != cudaSuccess) {
        S->free_slots.push_back(r.slot);
        --S->cams[camera].pending;
        S->cv.notify_all();
        return VG_ECUDA;
    }
    r.ticket = S->status.size();
    S->status.push_back(0);
    S->t_submit.push_back(seconds(arrival));
    S->t_done.push_back(0.0);
    ++S->submitted;
    S->queue.push_back(r);
    if (ticket) *ticket = r.ticket;
    S->cv.notify_all();
    return VG_OK;
}

int vg_server_wait(vg_server *S, uint64_t ticket, int64_t timeout_us) {
    if (!S) return VG_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (ticket >= S->status.size()) return VG_EINVAL;
    auto ready = [&] { return S->status[ticket] != 0; };
    if (timeout_us < 0) S->cv.wait(lk, ready);
    else if (!S->cv.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) return VG_ETIMEOUT;
    return S->status[ticket] == 1 ? VG_OK : VG_ECUDA;
}

int vg_server_ticket_times(vg_server *S, uint64_t ticket, double *submitted_s, double *completed_s) {
    if (!S) return VG_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    if (ticket >= S->status.size()) return VG_EINVAL;
    if (submitted_s) *submitted_s = S->t_submit[ticket];
    if (S->status[ticket] == 0) return VG_ETIMEOUT;
    if (completed_s) *completed_s = S->t_done[ticket];
    return S->status[ticket] == 1 ? VG_OK : VG_ECUDA;
}

int vg_server_read(vg_server *S, int32_t camera, uint8_t *dst, int32_t dst_mem, int64_t dst_bytes,
                   int32_t origin[3]) {
    if (!S) return VG_EINVAL;
    vg_grid *grid = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        if (camera < 0 || camera >= (int32_t)S->cams.size() || S->cams[camera].removed) return VG_EINVAL;
        S->cv.wait(lk, [&] { return S->cams[camera].pending == 0 && !S->cams[camera].reading; });
        S->cams[camera].reading = true;   // the server leaves the grid alone meanwhile
        grid = S->cams[camera].grid;
    }
    int rc = vg_read(grid, dst, dst_mem, dst_bytes, origin, S->admin);
    if (rc == VG_OK && cudaStreamSynchronize(S->admin) != cudaSuccess) rc = VG_ECUDA;
    std::lock_guard<std::mutex> g(S->mu);
    S->cams[camera].reading = false;
    S->cv.notify_all();
    return rc;
}

int vg_server_stats(vg_server *S, vg_server_stats_t *out, int32_t reset) {
    if (!S || !out) return VG_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->batches = S->batches;
    out->mean_batch = S->batches ? (double)S->batched_frames / (double)S->batches : 0.0;
    if (!S->lat_us.empty()) {
        std::vector<float> v(S->lat_us);
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return (double)v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        out->latency_p50_us = pct(0.50);
        out->latency_p99_us = pct(0.99);
        out->latency_max_us = v.back();
    }
    out->bytes_in_use = S->fixed_bytes + S->grid_bytes;
    int32_t live = 0;
    for (const Camera &c : S->cams) live += c.removed ? 0 : 1;
    out->cameras = live;
    if (reset) {
        S->submitted = S->completed = S->failed = S->batches = S->batched_frames = 0;
        S->lat_us.clear();
    }
    return VG_OK;
}

}  // extern "C"
