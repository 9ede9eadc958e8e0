// serve.cu -- a continuous-batching request server around the renderer.
//
// Several scenes stay resident; camera and LiDAR render requests of any size
// arrive through sg_server_submit.  n_slots worker threads each own a CUDA
// stream and a render workspace (frame).  A request is admitted, in arrival
// order, as soon as a slot is free and its estimated workspace fits in the
// device-memory budget next to the requests already in flight; admitted
// requests run concurrently on their own streams, so one request's
// projection and sort overlap another's compositing on the GPU.  Latency is
// measured from submission to the completion of the request's last kernel.
//
// With graphs on, each slot keeps one captured CUDA graph per (scene,
// sensor, options) combination: the render in capacity mode (pair buffers
// sized ahead, no host wait for the pair count), replayed with one launch
// per request.  The request's pose and its output / pose pointers reach the
// replay through the frame's pinned RenderDesc, which the graph's first node
// copies to the device.  A graph is dropped when one of the frame's buffers
// has been reallocated since its capture, and after a replay that ran out of
// pair capacity (that request is rendered again exactly).
//
// FIFO priority: each slot has one stream per CUDA stream-priority level
// (up to n_slots levels); a request admitted while k others are in flight is
// launched on the k-th level, so that the block scheduler serves the older
// requests first and newer ones fill the SMs they leave idle, instead of
// every request in flight sharing the GPU equally.
//
// Every wait here is a host-side condition-variable wait with a timeout; no
// kernel waits on another.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

extern "C" {
sg_status sg_render_camera(sg_scene scene, sg_camera cam, const float h_c2w[12],
                           const sg_render_opts *opts, sg_frame frame, float *d_rgb,
                           float *d_alpha, float *d_depth, void *stream);
sg_status sg_render_lidar(sg_scene scene, sg_lidar lidar, const float *d_col_c2w,
                          const sg_render_opts *opts, sg_frame frame, float *d_range,
                          float *d_intensity, float *d_drop, float *d_alpha, void *stream);
}

namespace sg {

using Clock = std::chrono::steady_clock;

struct Job {
    uint64_t ticket;
    sg_request req;
    size_t bytes;               // admission estimate
    Clock::time_point arrival;
};

struct Result {
    bool done = false;
    sg_status status = SG_OK;
    double latency_ms = 0;
    std::string message;   // the worker's error message when status != SG_OK
};

// A captured render of one (scene, sensor, options) combination on one slot.
struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;          // kernel nodes, counted as launches per replay
    int64_t cap = 0;              // pair capacity the graph was captured with
    std::vector<void *> bufs;     // the frame's buffers at capture
};

static std::string graph_key(const sg_request &r)
{
    std::string k;
    const uint64_t ids[3] = {(uint64_t)r.kind, r.scene ? r.scene->uid : 0,
                             r.kind == SG_REQ_CAMERA ? (r.camera ? r.camera->uid : 0)
                                                     : (r.lidar ? r.lidar->uid : 0)};
    k.append((const char *)ids, sizeof(ids));
    k.append((const char *)&r.opts, sizeof(r.opts));
    return k;
}

static std::vector<void *> frame_bufs(Frame &f)
{
    std::vector<void *> v;
    for_each_buf(f, [&](Buf &b) { v.push_back(b.p); });
    return v;
}

static int64_t count_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int64_t k = 0;
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// Workspace estimate of one request for admission: sg_workspace_bytes of
// its scene and sensor.
static size_t request_bytes(const sg_request &r)
{
    int64_t rays = 0;
    if (r.kind == SG_REQ_CAMERA && r.camera)
        rays = (int64_t)r.camera->c.width * r.camera->c.height;
    else if (r.kind == SG_REQ_LIDAR && r.lidar)
        rays = (int64_t)r.lidar->l.n_beams * r.lidar->l.n_cols;
    size_t b = 0;
    if (!r.scene || sg_workspace_bytes(r.scene, r.kind, rays, &b) != SG_OK) return 0;
    return b;
}

}  // namespace sg

using namespace sg;

struct sg_server_s {
    sg_server_config cfg;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> queue;
    std::unordered_map<uint64_t, Result> results;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;   // [slot * n_prio + level], level 0 the highest
    int n_prio = 1, prio_hi = 0;
    // per slot and batch position: a frame and a view stream (forked from the
    // slot's stream for batches of several requests), and the fork / join events
    std::vector<std::vector<sg_frame>> frames;
    std::vector<std::vector<cudaStream_t>> vstreams;
    std::vector<cudaEvent_t> fork_ev;
    std::vector<std::vector<cudaEvent_t>> join_ev;
    // batches: timed events at the start and at each request's end (recorded
    // as graph nodes in captures), for each request's own completion time
    std::vector<cudaEvent_t> start_ev;
    std::vector<std::vector<cudaEvent_t>> done_ev;
    size_t bytes_in_flight = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    int in_flight = 0;
    // graphs: per slot, per (combination, batch size); largest pair count seen
    // per combination
    std::vector<std::unordered_map<std::string, GraphEntry>> graphs;
    std::unordered_map<std::string, int64_t> max_pairs;
    // statistics
    std::vector<double> latencies;
    int64_t completed = 0, failed = 0, rays = 0, busy_peak = 0;
    int64_t replays = 0, captures = 0, overflows = 0, batches = 0, batched = 0;
    Clock::time_point t_first, t_last;
    bool any = false;
};

static sg_status render_plain(const sg_request &r, sg_frame fr, cudaStream_t st)
{
    if (r.kind == SG_REQ_CAMERA)
        return sg_render_camera(r.scene, r.camera, r.c2w, &r.opts, fr, r.d_out[0], r.d_out[1],
                                r.d_out[2], st);
    return sg_render_lidar(r.scene, r.lidar, r.d_col_c2w, &r.opts, fr, r.d_out[0], r.d_out[1],
                           r.d_out[2], r.d_out[3], st);
}

// A batch of requests of one combination (same scene, sensor and options),
// request i on the slot's frame i.  One request renders on `st` itself;
// several are forked onto the slot's view streams (waiting for `st`), cameras
// as one sg_render_cameras call (their pair counts all on the way before the
// host waits for one), LiDAR sweeps one after another, and joined back into
// `st`.  The same sequence is what a captured graph of the batch holds.
static sg_status render_batch(sg_server S, int slot, const std::vector<const sg_request *> &rs,
                              cudaStream_t st)
{
    const size_t B = rs.size();
    const std::vector<sg_frame> &F = S->frames[slot];
    if (B == 1) return render_plain(*rs[0], F[0], st);
    const std::vector<cudaStream_t> &V = S->vstreams[slot];
    // the timing events become graph nodes when the batch is being captured
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    SG_CUDA(cudaStreamIsCapturing(st, &cap_st));
    const unsigned rec_flags =
        cap_st == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    SG_CUDA(cudaEventRecordWithFlags(S->start_ev[slot], st, rec_flags));
    SG_CUDA(cudaEventRecord(S->fork_ev[slot], st));
    for (size_t i = 0; i < B; ++i) SG_CUDA(cudaStreamWaitEvent(V[i], S->fork_ev[slot], 0));
    sg_status s = SG_OK;
    if (rs[0]->kind == SG_REQ_CAMERA) {
        std::vector<sg_camera_view> views(B);
        for (size_t i = 0; i < B; ++i) {
            const sg_request &r = *rs[i];
            sg_camera_view &v = views[i];
            memset(&v, 0, sizeof(v));
            v.camera = r.camera;
            memcpy(v.c2w, r.c2w, sizeof(v.c2w));
            v.frame = F[i];
            v.rgb = r.d_out[0];
            v.alpha = r.d_out[1];
            v.depth = r.d_out[2];
            v.stream = V[i];
        }
        s = sg_render_cameras(rs[0]->scene, (int)B, views.data(), &rs[0]->opts, 0);
    } else {
        for (size_t i = 0; i < B && s == SG_OK; ++i) s = render_plain(*rs[i], F[i], V[i]);
    }
    // join every view stream (also after an error: nothing is left forked)
    for (size_t i = 0; i < B; ++i) {
        cudaError_t e = cudaEventRecordWithFlags(S->done_ev[slot][i], V[i], rec_flags);
        if (e == cudaSuccess) e = cudaEventRecord(S->join_ev[slot][i], V[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, S->join_ev[slot][i], 0);
        if (e != cudaSuccess && s == SG_OK) s = cuda_status(e, "joining a batch's streams");
    }
    return s;
}

// Wait for the batch's renders on `st` and check their device status words:
// a capacity-mode render copies its word with its scalars; after an exact
// render it is copied here.
static sg_status finish(const std::vector<sg_frame> &F, size_t B, cudaEvent_t ev, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < B && e == cudaSuccess; ++i) {
        Frame &fr = F[i]->f;
        if (fr.k_cap == 0)
            e = cudaMemcpyAsync(fr.h_scalars + kHostStatusQuery,
                                (const uint32_t *)fr.scalars.p + kScalStatus, 4,
                                cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev);
    if (e != cudaSuccess) return cuda_status(e, "request completion");
    for (size_t i = 0; i < B; ++i) {
        const Frame &fr = F[i]->f;
        if (fr.h_scalars[fr.k_cap == 0 ? kHostStatusQuery : kScalStatus]) {
            set_error("a bounded device wait (sort look-back or projection bulk copy) gave up in this request's render");
            return SG_ERR_TIMEOUT;
        }
    }
    return SG_OK;
}

static void note_pairs(sg_server S, const std::string &key, int64_t K)
{
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t &m = S->max_pairs[key];
    if (K > m) m = K;
}

static void drop_graph(GraphEntry &g)
{
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = GraphEntry();
}

static std::vector<void *> batch_bufs(const std::vector<sg_frame> &F, size_t B)
{
    std::vector<void *> v;
    for (size_t i = 0; i < B; ++i) {
        std::vector<void *> b = frame_bufs(F[i]->f);
        v.insert(v.end(), b.begin(), b.end());
    }
    return v;
}

static void set_capacity(const std::vector<sg_frame> &F, size_t B, int64_t cap)
{
    for (size_t i = 0; i < B; ++i) F[i]->f.k_cap = cap;
}

// A batch of requests of one combination on `slot`, with graphs: replay the
// graph of (combination, batch size), or warm up and capture it.  The first
// batch of a combination renders exactly; the next one in capacity mode
// (room for 1.25x the largest pair count seen plus 64K) and is captured.
static sg_status render_graphed(sg_server S, int slot, const std::vector<const sg_request *> &rs,
                                cudaStream_t st, cudaEvent_t ev)
{
    const size_t B = rs.size();
    const std::vector<sg_frame> &F = S->frames[slot];
    const std::string key = graph_key(*rs[0]);
    GraphEntry &g = S->graphs[slot][key + "#" + std::to_string(B)];
    sg_status s;
    auto pairs_needed = [&]() {
        int64_t need = 0;
        for (size_t i = 0; i < B; ++i) {
            const Frame &fr = F[i]->f;
            const int64_t n = fr.k_cap > 0 ? (int64_t)fr.h_scalars[1] + fr.h_scalars[3] : fr.n_pairs;
            need = std::max(need, n);
        }
        return need;
    };
    auto dropped_any = [&]() {
        for (size_t i = 0; i < B; ++i)
            if (F[i]->f.h_scalars[3] != 0) return true;
        return false;
    };
    if (g.exec && g.bufs == batch_bufs(F, B)) {
        // replay: each request's parameters through its frame's pinned descriptor
        for (size_t i = 0; i < B; ++i) {
            const sg_request &r = *rs[i];
            Frame &fr = F[i]->f;
            RenderDesc &D = *fr.h_desc;
            if (r.kind == SG_REQ_CAMERA) {
                memcpy(D.c2w, r.c2w, sizeof(D.c2w));
                D.poses = nullptr;
                for (int k = 0; k < 3; ++k) D.out[k] = r.d_out[k];
                D.out[3] = nullptr;
                memcpy(fr.c2w, r.c2w, sizeof(fr.c2w));
            } else {
                memset(D.c2w, 0, sizeof(D.c2w));
                D.poses = r.d_col_c2w;
                for (int k = 0; k < 4; ++k) D.out[k] = r.d_out[k];
                fr.d_lidar_poses = r.d_col_c2w;
            }
        }
        set_capacity(F, B, g.cap);
        cudaError_t e = cudaGraphLaunch(g.exec, st);
        if (e != cudaSuccess) return cuda_status(e, "cudaGraphLaunch");
        count_launches(g.kernels);
        if ((s = finish(F, B, ev, st)) != SG_OK) return s;
        if (!dropped_any()) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->replays += (int64_t)B;
            return SG_OK;
        }
        // out of pair capacity: render exactly, capture anew next time
        const int64_t need = pairs_needed();
        drop_graph(g);
        set_capacity(F, B, 0);
        if ((s = render_batch(S, slot, rs, st)) != SG_OK) return s;
        if ((s = finish(F, B, ev, st)) != SG_OK) return s;
        note_pairs(S, key, std::max(need, pairs_needed()));
        std::lock_guard<std::mutex> lk(S->mu);
        S->overflows++;
        return SG_OK;
    }
    drop_graph(g);
    int64_t known = -1;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->max_pairs.find(key);
        if (it != S->max_pairs.end()) known = it->second;
    }
    if (known < 0) {    // first sight of this combination: exact render
        set_capacity(F, B, 0);
        if ((s = render_batch(S, slot, rs, st)) != SG_OK) return s;
        if ((s = finish(F, B, ev, st)) != SG_OK) return s;
        note_pairs(S, key, pairs_needed());
        return SG_OK;
    }
    // capacity-mode render (grows the workspace as needed), then capture
    const int64_t cap = std::min<int64_t>(known + known / 4 + 65536, 0x7fffffffLL);
    set_capacity(F, B, cap);
    if ((s = render_batch(S, slot, rs, st)) != SG_OK) return s;
    if ((s = finish(F, B, ev, st)) != SG_OK) return s;
    if (dropped_any()) {
        const int64_t need = pairs_needed();
        set_capacity(F, B, 0);
        if ((s = render_batch(S, slot, rs, st)) != SG_OK) return s;
        if ((s = finish(F, B, ev, st)) != SG_OK) return s;
        note_pairs(S, key, need);
        return SG_OK;
    }
    cudaGraph_t graph = nullptr;
    capture_guard() = true;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    sg_status cs = e == cudaSuccess ? render_batch(S, slot, rs, st) : SG_ERR_CUDA;
    if (e == cudaSuccess) e = cudaStreamEndCapture(st, &graph);
    capture_guard() = false;
    if (cs == SG_OK && e == cudaSuccess && graph) {
        cudaGraphExec_t exec = nullptr;
        if (cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            g.exec = exec;
            g.kernels = count_kernel_nodes(graph);
            g.cap = cap;
            g.bufs = batch_bufs(F, B);
            std::lock_guard<std::mutex> lk(S->mu);
            S->captures++;
        }
    }
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();   // a failed capture leaves no graph; the result is complete
    return SG_OK;
}

static int64_t request_rays(const sg_request &r)
{
    return r.kind == SG_REQ_CAMERA ? (int64_t)r.camera->c.width * r.camera->c.height
                                   : (int64_t)r.lidar->l.n_beams * r.lidar->l.n_cols;
}

static void worker_main(sg_server S, int slot)
{
    cudaSetDevice(S->device);
    const cudaStream_t *slot_streams = &S->streams[(size_t)slot * S->n_prio];
    const std::vector<sg_frame> &F = S->frames[slot];
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // admit the oldest request once it fits next to the work in flight
        S->cv_work.wait(lk, [&] {
            if (S->stop) return true;
            if (S->queue.empty()) return false;
            const Job &j = S->queue.front();
            return S->cfg.memory_budget == 0 || S->in_flight == 0 ||
                   S->bytes_in_flight + j.bytes <= S->cfg.memory_budget;
        });
        if (S->stop) break;   // requests not yet started are dropped
        std::vector<Job> jobs(1, S->queue.front());
        S->queue.pop_front();
        size_t bytes = jobs[0].bytes;
        // batching: queued requests of the same combination join it, up to
        // max_batch, as far as the memory budget allows (a look at the first
        // kBatchScan waiting requests; the others keep their order)
        constexpr int kBatchScan = 32;
        if (S->cfg.max_batch > 1 && !S->queue.empty()) {
            const std::string k0 = graph_key(jobs[0].req);
            int scanned = 0;
            for (auto it = S->queue.begin();
                 it != S->queue.end() && (int)jobs.size() < S->cfg.max_batch && scanned < kBatchScan;
                 ++scanned) {
                const bool fits = S->cfg.memory_budget == 0 ||
                                  S->bytes_in_flight + bytes + it->bytes <= S->cfg.memory_budget;
                if (fits && graph_key(it->req) == k0) {
                    bytes += it->bytes;
                    jobs.push_back(*it);
                    it = S->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        const int B = (int)jobs.size();
        S->bytes_in_flight += bytes;
        // FIFO priority: a batch admitted behind k others in flight runs at
        // the k-th priority level, so the oldest ones take the SMs first
        const int level = S->cfg.fifo_priority ? std::min(S->in_flight, S->n_prio - 1) : 0;
        const cudaStream_t st = slot_streams[level];
        S->in_flight += B;
        S->busy_peak = std::max<int64_t>(S->busy_peak, S->in_flight);
        if (B > 1) {
            S->batches++;
            S->batched += B;
        }
        lk.unlock();
        S->cv_work.notify_all();

        std::vector<const sg_request *> rs;
        for (const Job &j : jobs) rs.push_back(&j.req);
        sg_status s;
        if (S->cfg.use_graphs) {
            s = render_graphed(S, slot, rs, st, ev);
        } else {
            set_capacity(F, (size_t)B, 0);
            s = render_batch(S, slot, rs, st);
            if (s == SG_OK) s = finish(F, (size_t)B, ev, st);
        }
        const Clock::time_point t_done = Clock::now();
        // in a batch each request completes with its own view: its end, on
        // the device clock, against the batch's last one
        std::vector<double> early_ms((size_t)B, 0.0);
        if (B > 1 && s == SG_OK) {
            std::vector<float> at((size_t)B, 0.f);
            bool ok = true;
            for (int i = 0; i < B && ok; ++i)
                ok = cudaEventElapsedTime(&at[i], S->start_ev[slot], S->done_ev[slot][i]) ==
                     cudaSuccess;
            if (ok) {
                const float last = *std::max_element(at.begin(), at.end());
                for (int i = 0; i < B; ++i) early_ms[i] = (double)(last - at[i]);
            } else {
                cudaGetLastError();
            }
        }

        lk.lock();
        S->bytes_in_flight -= bytes;
        S->in_flight -= B;
        for (int bi = 0; bi < B; ++bi) {
            const Job &job = jobs[bi];
            Result &res = S->results[job.ticket];
            res.done = true;
            res.status = s;
            if (s != SG_OK) res.message = sg_last_error();
            res.latency_ms =
                std::chrono::duration<double, std::milli>(t_done - job.arrival).count() -
                early_ms[bi];
            if (s == SG_OK) {
                S->completed++;
                S->rays += request_rays(job.req);
                S->latencies.push_back(res.latency_ms);
            } else {
                S->failed++;
            }
            if (!S->any) { S->t_first = job.arrival; S->any = true; }
        }
        S->t_last = t_done;
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    lk.unlock();
    cudaEventDestroy(ev);
}

extern "C" {

sg_server_config sg_default_server_config(void)
{
    sg_server_config c;
    memset(&c, 0, sizeof(c));
    c.n_slots = 4;
    c.memory_budget = 0;
    c.queue_capacity = 4096;
    c.use_graphs = 1;
    c.fifo_priority = 1;
    c.max_batch = 4;
    return c;
}

sg_status sg_server_create(const sg_server_config *cfg, sg_server *out)
{
    if (!cfg || !out) { set_error("NULL argument"); return SG_ERR_INVALID; }
    *out = nullptr;
    if (cfg->n_slots < 1 || cfg->n_slots > 64 || cfg->queue_capacity < 1 ||
        cfg->max_batch < 1 || cfg->max_batch > 16) {
        set_error("sg_server_create: n_slots must be in 1..64, queue_capacity >= 1 and "
                  "max_batch in 1..16");
        return SG_ERR_INVALID;
    }
    sg_server S = new (std::nothrow) sg_server_s;
    if (!S) { set_error("host allocation failed"); return SG_ERR_OOM; }
    S->cfg = *cfg;
    S->graphs.resize(cfg->n_slots);
    cudaGetDevice(&S->device);
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    S->n_prio = cfg->fifo_priority ? std::max(1, std::min(cfg->n_slots, least - greatest + 1)) : 1;
    S->prio_hi = greatest;
    for (int i = 0; i < cfg->n_slots; ++i) {
        for (int k = 0; k < S->n_prio; ++k) {
            cudaStream_t st;
            cudaError_t e = cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking,
                                                         std::min(least, greatest + k));
            if (e != cudaSuccess) {
                sg_status r = cuda_status(e, "cudaStreamCreateWithPriority");
                sg_server_destroy(S);
                return r;
            }
            S->streams.push_back(st);
        }
        // a frame and a view stream per batch position, fork and join events
        S->frames.emplace_back();
        S->vstreams.emplace_back();
        S->join_ev.emplace_back();
        S->done_ev.emplace_back();
        S->fork_ev.push_back(nullptr);
        S->start_ev.push_back(nullptr);
        cudaError_t e = cudaEventCreateWithFlags(&S->fork_ev.back(), cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreate(&S->start_ev.back());
        for (int b = 0; b < cfg->max_batch && e == cudaSuccess; ++b) {
            sg_frame f = nullptr;
            if (sg_frame_create(&f) != SG_OK) {
                sg_server_destroy(S);
                return SG_ERR_OOM;
            }
            f->f.keep_state = false;   // no backward follows a served render
            S->frames.back().push_back(f);
            cudaStream_t vs = nullptr;
            e = cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking);
            if (e == cudaSuccess) S->vstreams.back().push_back(vs);
            cudaEvent_t je = nullptr;
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&je, cudaEventDisableTiming);
            if (e == cudaSuccess) S->join_ev.back().push_back(je);
            cudaEvent_t de = nullptr;
            if (e == cudaSuccess) e = cudaEventCreate(&de);
            if (e == cudaSuccess) S->done_ev.back().push_back(de);
        }
        if (e != cudaSuccess) {
            sg_status r = cuda_status(e, "server streams and events");
            sg_server_destroy(S);
            return r;
        }
    }
    for (int i = 0; i < cfg->n_slots; ++i) S->workers.emplace_back(worker_main, S, i);
    *out = S;
    return SG_OK;
}

sg_status sg_server_submit(sg_server S, const sg_request *req, uint64_t *ticket)
{
    if (!S || !req || !ticket) { set_error("NULL argument"); return SG_ERR_INVALID; }
    if (!req->scene || (req->kind == SG_REQ_CAMERA && !req->camera) ||
        (req->kind == SG_REQ_LIDAR &&
         (!req->lidar || !req->d_col_c2w || (uintptr_t)req->d_col_c2w % 16 != 0)) ||
        (req->kind != SG_REQ_CAMERA && req->kind != SG_REQ_LIDAR)) {
        set_error("sg_server_submit: incomplete request");
        return SG_ERR_INVALID;
    }
    Job j;
    j.req = *req;
    j.bytes = request_bytes(*req);
    if (S->cfg.memory_budget && j.bytes > S->cfg.memory_budget) {
        set_error("sg_server_submit: the request's workspace (%zu bytes) exceeds the budget",
                  j.bytes);
        return SG_ERR_INVALID;
    }
    j.arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if ((int)S->queue.size() >= S->cfg.queue_capacity) {
            set_error("sg_server_submit: queue full");
            return SG_ERR_BUSY;
        }
        j.ticket = S->next_ticket++;
        S->results[j.ticket] = Result();
        S->queue.push_back(j);
        *ticket = j.ticket;
    }
    S->cv_work.notify_all();
    return SG_OK;
}

sg_status sg_server_wait(sg_server S, uint64_t ticket, double timeout_s, double *latency_ms)
{
    if (!S) { set_error("NULL server"); return SG_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return SG_ERR_INVALID; }
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    if (!S->cv_done.wait_until(lk, deadline, [&] { return S->results[ticket].done; })) {
        set_error("sg_server_wait: ticket %llu not done within %.3f s", (unsigned long long)ticket,
                  timeout_s);
        return SG_ERR_TIMEOUT;
    }
    Result r = S->results[ticket];
    S->results.erase(ticket);
    if (latency_ms) *latency_ms = r.latency_ms;
    if (r.status != SG_OK)
        set_error("request %llu failed (status %d): %s", (unsigned long long)ticket, r.status,
                  r.message.c_str());
    return r.status;
}

sg_status sg_server_drain(sg_server S, double timeout_s)
{
    if (!S) { set_error("NULL server"); return SG_ERR_INVALID; }
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    if (!S->cv_done.wait_until(lk, deadline, [&] { return S->queue.empty() && S->in_flight == 0; })) {
        set_error("sg_server_drain: work left after %.3f s", timeout_s);
        return SG_ERR_TIMEOUT;
    }
    return SG_OK;
}

sg_status sg_server_stats(sg_server S, sg_server_report *out)
{
    if (!S || !out) { set_error("NULL argument"); return SG_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    out->completed = S->completed;
    out->failed = S->failed;
    out->rays = S->rays;
    out->peak_in_flight = S->busy_peak;
    out->queued = (int64_t)S->queue.size();
    out->graph_replays = S->replays;
    out->graph_captures = S->captures;
    out->overflow_rerenders = S->overflows;
    out->batches = S->batches;
    out->batched_requests = S->batched;
    std::vector<double> l = S->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double p) {
            double idx = p * (double)(l.size() - 1);
            size_t i = (size_t)floor(idx);
            size_t k = std::min(i + 1, l.size() - 1);
            return l[i] + (l[k] - l[i]) * (idx - (double)i);
        };
        double s = 0;
        for (double v : l) s += v;
        out->latency_mean_ms = s / (double)l.size();
        out->latency_p50_ms = q(0.50);
        out->latency_p99_ms = q(0.99);
        out->latency_max_ms = l.back();
    }
    if (S->any) {
        out->span_s = std::chrono::duration<double>(S->t_last - S->t_first).count();
        out->mrays_per_s = out->span_s > 0 ? (double)S->rays / out->span_s / 1e6 : 0.0;
    }
    return SG_OK;
}

sg_status sg_server_reset_stats(sg_server S)
{
    if (!S) { set_error("NULL server"); return SG_ERR_INVALID; }
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies.clear();
    S->completed = S->failed = S->rays = S->busy_peak = 0;
    S->replays = S->captures = S->overflows = S->batches = S->batched = 0;
    S->any = false;
    return SG_OK;
}

void sg_server_destroy(sg_server S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto &t : S->workers)
        if (t.joinable()) t.join();
    for (auto &m : S->graphs)
        for (auto &kv : m) drop_graph(kv.second);
    for (auto st : S->streams) cudaStreamDestroy(st);
    for (auto &v : S->vstreams)
        for (auto st : v) cudaStreamDestroy(st);
    for (auto e : S->fork_ev)
        if (e) cudaEventDestroy(e);
    for (auto &v : S->join_ev)
        for (auto e : v) cudaEventDestroy(e);
    for (auto e : S->start_ev)
        if (e) cudaEventDestroy(e);
    for (auto &v : S->done_ev)
        for (auto e : v) cudaEventDestroy(e);
    for (auto &v : S->frames)
        for (auto f : v) sg_frame_destroy(f);
    delete S;
}

}  // extern "C"
