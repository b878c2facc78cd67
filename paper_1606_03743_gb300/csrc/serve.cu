// serve.cu -- continuous batching of field-point queries on a device-resident
// mesh (bem_server_*).
//
// A particle tracker asks for phi and E at the successive positions of its
// tracks, in requests of very uneven size.  The server keeps the mesh on the
// GPU and runs a host thread that forms "ticks":
//  * requests wait in a queue; a tick takes points up to the capacity of its
//    device buffers (the memory admitted per tick): first every waiting
//    small request (at most 1/8 of a tick) in arrival order, whole, then the
//    other requests in arrival order, a request larger than the space left
//    being split -- its next piece goes into this tick, the rest into later
//    ones.  At most one tick holding pieces of large requests is on the GPU
//    at a time, so a small request never waits behind more than one such
//    tick;
//  * the points are packed into pinned host memory, copied to the device,
//    and one CUDA graph -- the whole evaluation (spatial sort, the persistent
//    far-field kernel over (point tile x element chunk) work items, the
//    near-pair scan and analytic pass, finalisation) captured once at
//    creation, with the point count read on the device -- is replayed;
//  * the results are copied back and handed to their requests.
// Two such slots alternate: while one tick runs on the GPU, requests that
// arrive meanwhile are admitted into the other slot, whose copies and
// kernels are queued behind it, so new work overlaps work already on the
// device.  Every point's result depends only on the point and the mesh, so
// a request gets bit-identical results alone or in any mix.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bem_internal.cuh"

namespace bem {
namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { kPending = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Req {
    uint64_t ticket = 0;
    int64_t n = 0;
    std::vector<double> pts;  // host copy, n x 3
    std::vector<double> phi;  // n
    std::vector<double> E;    // n x 3
    Clock::time_point t_submit, t_done;
    int state = kPending;
    int status = BEM_OK;
    bool cancelled = false;
    bool queued = true;     // still in the pending queue (points not yet admitted)
    int64_t next = 0;       // points [0, next) have been admitted into ticks
    int64_t done_pts = 0;   // points whose results have come back
    int in_flight = 0;      // pieces on the GPU
};

// A contiguous run of one request's points inside a tick.
struct Piece {
    Req* r;
    int64_t roff;  // first point within the request
    int64_t n;     // points
    int64_t soff;  // first point within the tick
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bem_mesh view;  // the mesh with this slot's scratch in view.w
    double *d_pts = nullptr, *d_phi = nullptr, *d_E = nullptr;
    int* d_n = nullptr;
    double *h_pts = nullptr, *h_phi = nullptr, *h_E = nullptr;  // pinned
    int* h_n = nullptr;
    unsigned long long* h_near = nullptr;
    std::vector<Piece> pieces;
    int64_t n = 0;
    bool busy = false;
    bool large = false;  // holds pieces of requests larger than a small one
    std::vector<void*> dev_allocs;
};

}  // namespace
}  // namespace bem

struct bem_server {
    bem_mesh* mesh = nullptr;
    int64_t cap = 0;        // points per tick
    size_t near_cap = 0;    // near pairs per tick
    size_t dev_bytes = 0;
    bem::Slot slot[2];
    cudaStream_t side = nullptr;  // for the rare fallback evaluations
    std::thread thr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<bem::Req*> pending;
    std::unordered_map<uint64_t, bem::Req*> reqs;
    uint64_t next_ticket = 1;
    bool stop = false, paused = false;
    std::vector<double> lat_ms;
    std::vector<int64_t> lat_n;  // points of each request in lat_ms
    int64_t ticks = 0, points_done = 0, fallbacks = 0, graph_launches = 0;
    std::string thread_error;
};

namespace bem {
namespace {

constexpr size_t kCountersN = 24;

template <typename T>
int slot_alloc(bem_server* sv, Slot& sl, T** p, size_t count) {
    const cudaError_t e = dev_malloc((void**)p, sizeof(T) * (count ? count : 1));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("bem_server_create: cudaMalloc of %zu bytes failed: %s", sizeof(T) * count, cudaGetErrorString(e));
        *p = nullptr;
        return BEM_ERR_OOM;
    }
    sl.dev_allocs.push_back(*p);
    sv->dev_bytes += sizeof(T) * count;
    return BEM_OK;
}

// The evaluation of up to sv->cap points whose count is in sl.d_n.
int enqueue_pipeline(bem_server* sv, Slot& sl) {
    bem_mesh* m = &sl.view;
    Work& w = m->w;
    const int cap = (int)sv->cap;
    cudaStream_t s = sl.stream;
    BEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, kCountersN * sizeof(unsigned long long), s));
    int rc = launch_sort_points(m, sl.d_pts, cap, s, sl.d_n);
    if (rc) return rc;
    FarArgs a{};
    a.pts = sl.d_pts;
    a.perm = w.perm;
    a.n_pts = cap;
    a.n_dev = sl.d_n;
    a.sigma = m->d.sigma;
    a.slope = eval_slope(m, m->d.sigma);
    far_args_from_work(a, w, m->n_chunks);
    a.work = reinterpret_cast<int*>(w.counters + 14);
    a.near_rec = w.near_rec;
    a.counters = w.counters;
    a.near_cap = w.cap_near;
    a.kc = m->kc;
    a.want_e = 1;
    a.bbox = reinterpret_cast<const unsigned*>(w.bbox);
    if ((rc = launch_far(m, a, s))) return rc;
    // entries past the tick's points are stale but only shift offsets after them
    if ((rc = launch_exclusive_scan(w.near_tot, w.near_off, cap, w.scan_tmp, s))) return rc;
    if ((rc = launch_near_eval(m, sl.d_pts, w.perm, cap, m->d.sigma, 0, s, eval_slope(m, m->d.sigma)))) return rc;
    return launch_finalize(m, w.perm, cap, sl.d_phi, sl.d_E, 0, s, sl.d_n);
}

int slot_setup(bem_server* sv, Slot& sl) {
    bem_mesh* mesh = sv->mesh;
    sl.view = *mesh;
    memset(&sl.view.w, 0, sizeof sl.view.w);
    sl.view.stats = false;
    sl.view.timing = false;
    Work& w = sl.view.w;
    const size_t cap = (size_t)sv->cap;
    const size_t capt = (cap + 127) / 128 * 128;  // whole tiles of the far pass
    const size_t ns = capt * (size_t)mesh->n_chunks;
    const size_t cells = size_t(1) << 21;
    int rc;
    if ((rc = slot_alloc(sv, sl, &sl.d_pts, 3 * cap)) || (rc = slot_alloc(sv, sl, &sl.d_phi, cap)) ||
        (rc = slot_alloc(sv, sl, &sl.d_E, 3 * cap)) || (rc = slot_alloc(sv, sl, &sl.d_n, 1)) ||
        (rc = slot_alloc(sv, sl, &w.perm, cap)) || (rc = slot_alloc(sv, sl, &w.key, cap)) ||
        (rc = slot_alloc(sv, sl, &w.cell_cnt, cells)) || (rc = slot_alloc(sv, sl, &w.cell_off, cells)) ||
        (rc = slot_alloc(sv, sl, &w.part, ns)) || (rc = slot_alloc(sv, sl, &w.near_cnt, ns)) ||
        (rc = slot_alloc(sv, sl, &w.near_rows, ns)) || (rc = slot_alloc(sv, sl, &w.far, capt)) ||
        (rc = slot_alloc(sv, sl, &w.near_tot, capt)) || (rc = slot_alloc(sv, sl, &w.near_row, capt)) ||
        (rc = slot_alloc(sv, sl, &w.near_off, capt)) || (rc = slot_alloc(sv, sl, &w.tile_done, tile_done_ints(capt))) ||
        (rc = slot_alloc(sv, sl, &w.scan_tmp, scan_tmp_ints((int)std::max(capt, cells)))) ||
        (rc = slot_alloc(sv, sl, &w.near_rec, sv->near_cap)) || (rc = slot_alloc(sv, sl, &w.near_val, sv->near_cap)) ||
        (rc = slot_alloc(sv, sl, &w.counters, kCountersN)) || (rc = slot_alloc(sv, sl, &w.bbox, 2)))
        return rc;
    w.cap_pts = cap;
    w.cap_near = sv->near_cap;
    BEM_CUDA_TRY(pinned_malloc((void**)&sl.h_pts, sizeof(double) * 3 * cap));
    BEM_CUDA_TRY(pinned_malloc((void**)&sl.h_phi, sizeof(double) * cap));
    BEM_CUDA_TRY(pinned_malloc((void**)&sl.h_E, sizeof(double) * 3 * cap));
    BEM_CUDA_TRY(pinned_malloc((void**)&sl.h_n, sizeof(int)));
    BEM_CUDA_TRY(pinned_malloc((void**)&sl.h_near, 3 * sizeof(unsigned long long)));
    BEM_CUDA_TRY(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking));
    BEM_CUDA_TRY(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));

    // one eager run (one point) sets up everything the launchers initialise
    // on first use, then the sequence is captured as a graph
    for (int k = 0; k < 3; ++k) sl.h_pts[k] = 0.0;
    *sl.h_n = 1;
    BEM_CUDA_TRY(cudaMemcpyAsync(sl.d_n, sl.h_n, sizeof(int), cudaMemcpyHostToDevice, sl.stream));
    BEM_CUDA_TRY(cudaMemcpyAsync(sl.d_pts, sl.h_pts, sizeof(double) * 3, cudaMemcpyHostToDevice, sl.stream));
    if ((rc = enqueue_pipeline(sv, sl))) return rc;
    BEM_CUDA_TRY(cudaStreamSynchronize(sl.stream));
    BEM_CUDA_TRY(cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal));
    rc = enqueue_pipeline(sv, sl);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(sl.stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    sl.graph = g;
    BEM_CUDA_TRY(cudaGraphInstantiate(&sl.exec, sl.graph, 0));
    return BEM_OK;
}

void slot_free(Slot& sl) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (sl.graph) cudaGraphDestroy(sl.graph);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    for (void* p : sl.dev_allocs) cudaFree(p);
    sl.dev_allocs.clear();
    cudaFreeHost(sl.h_pts);
    cudaFreeHost(sl.h_phi);
    cudaFreeHost(sl.h_E);
    cudaFreeHost(sl.h_n);
    cudaFreeHost(sl.h_near);
}

// Drop a request that is neither queued nor on the GPU.  Lock held.
void forget(bem_server* sv, Req* r) {
    sv->reqs.erase(r->ticket);
    delete r;
}

// A request has failed: no further piece of it is admitted.  Lock held.
void fail_request(bem_server* sv, Req* r, int status) {
    r->state = kFailed;
    r->status = status;
    if (r->queued) {
        sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), r));
        r->queued = false;
    }
}

// Its results are complete, or it failed and nothing of it is left on the GPU.
bool finished(const Req* r) { return r->state == kDone || (r->state == kFailed && r->in_flight == 0 && !r->queued); }

// Requests of at most this many points are small: admitted whole, ahead of
// the pieces of larger ones.
int64_t small_limit(const bem_server* sv) { return std::max<int64_t>(1, sv->cap / 8); }

// Admit points of waiting requests into a free slot and launch the tick
// (policy at the top of this file).  Called with the lock held; returns false
// if nothing was admitted.
bool fill_and_launch(bem_server* sv, Slot& sl, bool allow_large, std::unique_lock<std::mutex>& lk) {
    sl.pieces.clear();
    sl.large = false;
    const int64_t small = small_limit(sv);
    int64_t n = 0;
    auto admit = [&](Req* r, int64_t take) {
        sl.pieces.push_back(Piece{r, r->next, take, n});
        r->next += take;
        ++r->in_flight;
        r->state = kRunning;
        n += take;
        if (r->n > small) sl.large = true;
    };
    // small requests first, whole, in arrival order
    for (Req* r : sv->pending) {
        if (r->cancelled || r->n > small) continue;
        const int64_t rem = r->n - r->next;
        if (rem > 0 && n + rem <= sv->cap) admit(r, rem);
    }
    // then the rest in arrival order, the last one split to fill the tick
    if (allow_large) {
        for (Req* r : sv->pending) {
            if (n >= sv->cap) break;
            if (r->cancelled) continue;
            const int64_t rem = r->n - r->next;
            if (rem > 0) admit(r, std::min(rem, sv->cap - n));
        }
    }
    // fully admitted requests leave the queue
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
        if ((*it)->next == (*it)->n || (*it)->cancelled) {
            (*it)->queued = false;
            it = sv->pending.erase(it);
        } else {
            ++it;
        }
    }
    if (sl.pieces.empty()) return false;
    sl.n = n;
    lk.unlock();
    NvtxRange range("bem.tick");
    for (const Piece& pc : sl.pieces)
        memcpy(sl.h_pts + 3 * pc.soff, pc.r->pts.data() + 3 * pc.roff, sizeof(double) * 3 * pc.n);
    *sl.h_n = (int)n;
    cudaError_t e = cudaMemcpyAsync(sl.d_n, sl.h_n, sizeof(int), cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.d_pts, sl.h_pts, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(sl.exec, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_phi, sl.d_phi, sizeof(double) * n, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_E, sl.d_E, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sl.h_near, sl.view.w.counters + kPairCounter, 3 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
    lk.lock();
    if (e != cudaSuccess) {
        sv->thread_error = cudaGetErrorString(e);
        for (const Piece& pc : sl.pieces) {
            --pc.r->in_flight;
            fail_request(sv, pc.r, BEM_ERR_CUDA);
        }
        sl.pieces.clear();
        sv->cv_done.notify_all();
        return false;
    }
    sl.busy = true;
    ++sv->ticks;
    ++sv->graph_launches;
    return true;
}


// Hand a finished tick's results to its requests.  Called without the lock.
void harvest(bem_server* sv, Slot& sl) {
    // h_near: the pair counter and, two further on, the checked build's flags
    static_assert(kCheckCounter == kPairCounter + 2, "counter layout");
    const bool overflow = sl.h_near[0] > sl.view.w.cap_near;
    const int checked = check_flags(sl.h_near[2], "bem_server tick");
    std::vector<int> status(sl.pieces.size(), checked);
    for (size_t i = 0; i < sl.pieces.size() && checked == BEM_OK; ++i) {
        const Piece& pc = sl.pieces[i];
        Req* r = pc.r;  // its result arrays were sized at submission; pieces write disjoint ranges
        if (!overflow) {
            memcpy(r->phi.data() + pc.roff, sl.h_phi + pc.soff, sizeof(double) * pc.n);
            memcpy(r->E.data() + 3 * pc.roff, sl.h_E + 3 * pc.soff, sizeof(double) * 3 * pc.n);
        } else {
            // the tick's near-pair list overflowed: evaluate this piece on its own
            status[i] = bem_eval(sv->mesh, r->pts.data() + 3 * pc.roff, pc.n, r->phi.data() + pc.roff,
                                 r->E.data() + 3 * pc.roff, sv->side);
        }
    }
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (overflow) ++sv->fallbacks;
    for (size_t i = 0; i < sl.pieces.size(); ++i) {
        const Piece& pc = sl.pieces[i];
        Req* r = pc.r;
        --r->in_flight;
        if (status[i] != BEM_OK) fail_request(sv, r, status[i]);
        r->done_pts += pc.n;
        if (r->state != kFailed && r->done_pts == r->n) {
            r->t_done = now;
            r->state = kDone;
            sv->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
            sv->lat_n.push_back(r->n);
            sv->points_done += r->n;
        }
        if (r->cancelled && r->in_flight == 0 && !r->queued) forget(sv, r);
    }
    sl.pieces.clear();
    sl.busy = false;
    sv->cv_done.notify_all();
}

void server_loop(bem_server* sv) {
    cudaSetDevice(sv->mesh->device);
    int next = 0;  // slot to fill next
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // harvest finished ticks
        for (int k = 0; k < 2; ++k) {
            Slot& sl = sv->slot[k];
            if (sl.busy && cudaEventQuery(sl.done) == cudaSuccess) {
                lk.unlock();
                harvest(sv, sl);
                lk.lock();
            }
        }
        if (sv->stop && sv->pending.empty() && !sv->slot[0].busy && !sv->slot[1].busy) break;
        // launch into the free slot (ticks run in submission order); pieces of
        // large requests only while the other slot holds none
        bool launched = false;
        Slot& sl = sv->slot[next];
        const Slot& other = sv->slot[next ^ 1];
        if (!sl.busy && !sv->paused && !sv->pending.empty()) {
            launched = fill_and_launch(sv, sl, !(other.busy && other.large), lk);
            if (launched) next ^= 1;
        }
        if (launched) continue;
        if (sv->slot[0].busy || sv->slot[1].busy) {
            // a tick is on the GPU: poll it, and take new requests meanwhile
            sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
        } else {
            sv->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

double percentile(std::vector<double> v, double q) {
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - i;
    return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" {

int bem_server_create(bem_mesh* mesh, const bem_server_options* opt, bem_server** out) {
    if (!out || !mesh) {
        set_error("bem_server_create: mesh or out is NULL");
        return BEM_ERR_INVALID;
    }
    *out = nullptr;
    bem_server* sv = new (std::nothrow) bem_server();
    if (!sv) {
        set_error("bem_server_create: out of host memory");
        return BEM_ERR_OOM;
    }
    sv->mesh = mesh;
    int64_t cap = opt && opt->max_points_per_tick > 0 ? opt->max_points_per_tick : 131072;
    sv->near_cap = opt && opt->max_near_pairs_per_tick > 0 ? (size_t)opt->max_near_pairs_per_tick : (size_t(1) << 21);
    size_t budget = opt && opt->device_mem_budget ? opt->device_mem_budget : (size_t(2) << 30);
    // admission by device memory: the budget, but no more than 3/4 of what the device has free now
    // (the slots' buffers are all allocated here; ticks allocate nothing)
    {
        size_t free_b = 0, total_b = 0;
        if (cudaSetDevice(mesh->device) == cudaSuccess && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
            budget = std::min(budget, free_b / 4 * 3);
        cudaGetLastError();
    }
    // shrink the per-tick capacity until both slots fit
    auto need = [&](int64_t c) {
        const size_t ns = (size_t)c * mesh->n_chunks;
        return 2 * (sizeof(double) * 11 * c + sizeof(int) * 5 * c + 40 * ns + 48 * sv->near_cap + (size_t(17) << 20));
    };
    while (cap > 1024 && need(cap) > budget) cap /= 2;
    if (cap < 1 || cap > (int64_t(1) << 24) || need(cap) > budget) {
        set_error("bem_server_create: device_mem_budget (or 3/4 of the free device memory, %zu bytes) too small "
                  "for one tick", budget);
        delete sv;
        return BEM_ERR_OOM;
    }
    sv->cap = cap;
    int rc = BEM_OK;
    cudaError_t ce = cudaSetDevice(mesh->device);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaSetDevice");
    if (!rc) {
        ce = cudaStreamCreateWithFlags(&sv->side, cudaStreamNonBlocking);
        if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaStreamCreate");
    }
    for (int k = 0; k < 2 && !rc; ++k) rc = slot_setup(sv, sv->slot[k]);
    if (rc) {
        for (int k = 0; k < 2; ++k) slot_free(sv->slot[k]);
        if (sv->side) cudaStreamDestroy(sv->side);
        delete sv;
        return rc;
    }
    sv->thr = std::thread(server_loop, sv);
    *out = sv;
    return BEM_OK;
}

void bem_server_destroy(bem_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        sv->paused = false;
    }
    sv->cv_work.notify_all();
    if (sv->thr.joinable()) sv->thr.join();
    cudaSetDevice(sv->mesh->device);
    for (int k = 0; k < 2; ++k) slot_free(sv->slot[k]);
    if (sv->side) cudaStreamDestroy(sv->side);
    for (auto& kv : sv->reqs) delete kv.second;
    delete sv;
}

int bem_submit(bem_server* sv, const double* points, int64_t n, uint64_t* ticket) {
    if (!sv || !ticket || (n > 0 && !points) || n < 1) {
        set_error("bem_submit: bad arguments (n = %lld)", (long long)n);
        return BEM_ERR_INVALID;
    }
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(points[i]) || fabs(points[i]) >= 1e30) {
            set_error("bem_submit: point %lld has a non-finite coordinate", (long long)(i / 3));
            return BEM_ERR_INVALID;
        }
    Req* r = new (std::nothrow) Req();
    if (!r) {
        set_error("bem_submit: out of host memory");
        return BEM_ERR_OOM;
    }
    r->n = n;
    try {
        r->pts.assign(points, points + 3 * n);
        r->phi.resize(n);
        r->E.resize(3 * n);
    } catch (const std::bad_alloc&) {
        delete r;
        set_error("bem_submit: out of host memory for %lld points", (long long)n);
        return BEM_ERR_OOM;
    }
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stop) {
            delete r;
            set_error("bem_submit: server is shutting down");
            return BEM_ERR_INVALID;
        }
        r->ticket = sv->next_ticket++;
        sv->reqs[r->ticket] = r;
        sv->pending.push_back(r);
        *ticket = r->ticket;
    }
    sv->cv_work.notify_one();
    return BEM_OK;
}

// Copies the results of a finished request and forgets it.  Lock held.
static int take_result(bem_server* sv, Req* r, double* phi, double* E) {
    const int st = r->status;
    if (r->state == kDone) {
        if (phi) memcpy(phi, r->phi.data(), sizeof(double) * r->n);
        if (E) memcpy(E, r->E.data(), sizeof(double) * 3 * r->n);
    } else {
        set_error("request %llu failed (status %d): %s", (unsigned long long)r->ticket, st, sv->thread_error.c_str());
    }
    sv->reqs.erase(r->ticket);
    delete r;
    return st;
}

int bem_poll(bem_server* sv, uint64_t ticket, double* phi, double* E, int32_t* done) {
    if (!sv || !done) {
        set_error("bem_poll: bad arguments");
        return BEM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end() || it->second->cancelled) {
        set_error("bem_poll: unknown ticket %llu", (unsigned long long)ticket);
        return BEM_ERR_NOT_FOUND;
    }
    Req* r = it->second;
    if (!finished(r)) {
        *done = 0;
        return BEM_OK;
    }
    *done = 1;
    return take_result(sv, r, phi, E);
}

int bem_wait(bem_server* sv, uint64_t ticket, double timeout_s, double* phi, double* E) {
    if (!sv) {
        set_error("bem_wait: server is NULL");
        return BEM_ERR_INVALID;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end() || it->second->cancelled) {
        set_error("bem_wait: unknown ticket %llu", (unsigned long long)ticket);
        return BEM_ERR_NOT_FOUND;
    }
    Req* r = it->second;
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0.0));
    while (!finished(r)) {
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !finished(r)) {
            set_error("bem_wait: request %llu not finished after %.3f s", (unsigned long long)ticket, timeout_s);
            return BEM_ERR_TIMEOUT;
        }
    }
    return take_result(sv, r, phi, E);
}

int bem_cancel(bem_server* sv, uint64_t ticket) {
    if (!sv) {
        set_error("bem_cancel: server is NULL");
        return BEM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end() || it->second->cancelled) {
        set_error("bem_cancel: unknown ticket %llu", (unsigned long long)ticket);
        return BEM_ERR_NOT_FOUND;
    }
    Req* r = it->second;
    if (r->queued) {
        sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), r));
        r->queued = false;
    }
    if (r->in_flight > 0) {
        r->cancelled = true;  // dropped when its last piece's tick finishes
    } else {
        forget(sv, r);
    }
    return BEM_OK;
}

int bem_server_pause(bem_server* sv, int32_t paused) {
    if (!sv) {
        set_error("bem_server_pause: server is NULL");
        return BEM_ERR_INVALID;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->paused = paused != 0;
    }
    sv->cv_work.notify_all();
    return BEM_OK;
}

int bem_server_stats(bem_server* sv, int32_t reset, double* out) {
    if (!sv || !out) {
        set_error("bem_server_stats: bad arguments");
        return BEM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    const size_t n = sv->lat_ms.size();
    double mean = 0.0;
    for (double v : sv->lat_ms) mean += v;
    out[0] = (double)n;
    out[1] = percentile(sv->lat_ms, 0.50);
    out[2] = percentile(sv->lat_ms, 0.99);
    out[3] = n ? mean / n : 0.0;
    out[4] = (double)sv->ticks;
    out[5] = (double)sv->points_done;
    out[6] = (double)sv->fallbacks;
    out[7] = (double)sv->cap;
    out[8] = (double)sv->dev_bytes;
    out[9] = (double)sv->graph_launches;
    if (reset) {
        sv->lat_ms.clear();
        sv->lat_n.clear();
        sv->ticks = sv->points_done = sv->fallbacks = sv->graph_launches = 0;
    }
    return BEM_OK;
}

int bem_server_latencies(bem_server* sv, int64_t cap, double* ms, int64_t* points, int64_t* count) {
    if (!sv || !count || cap < 0 || (cap > 0 && (!ms || !points))) {
        set_error("bem_server_latencies: bad arguments");
        return BEM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    const int64_t n = (int64_t)sv->lat_ms.size();
    const int64_t k = std::min(n, cap);
    for (int64_t i = 0; i < k; ++i) {
        ms[i] = sv->lat_ms[i];
        points[i] = sv->lat_n[i];
    }
    *count = n;
    return BEM_OK;
}

}  // extern "C"
