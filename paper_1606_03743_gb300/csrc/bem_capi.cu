// bem_capi.cu -- the extern "C" entry points declared in include/bem.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>
#include <string>

#include "bem_internal.cuh"
#include "bem_test.h"

namespace bem {

namespace {
thread_local std::string g_err;
std::atomic<int64_t> g_launches{0};
// DR band limits (Sec. 4) for phi and E together: per type the smallest DR from which the
// next rule's mean relative errors of phi and E stay at or below 2e-15, rounded up
const double kDefaultLimits[2][5] = {{4.5, 12.0, 30.0, 120.0, 2250.0}, {6.0, 18.0, 45.0, 160.0, 2800.0}};
constexpr double kEps0SI = 8.8541878128e-12;
constexpr int kMaxCellBits = 7;  // must match the key width of k_sort.cu
constexpr size_t kCells = size_t(1) << (3 * kMaxCellBits);
constexpr size_t kCounters = 24;
}  // namespace

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
std::atomic<int64_t> g_alloc_left{-1};  // allocations before injected failures (< 0: none injected)
std::atomic<int64_t> g_alloc_count{0};  // allocations attempted, process-wide

// true if this allocation is to fail (the test hook's budget is spent)
bool injected_failure() {
    g_alloc_count.fetch_add(1, std::memory_order_relaxed);
    int64_t left = g_alloc_left.load();
    while (left >= 0) {
        if (left == 0) return true;
        if (g_alloc_left.compare_exchange_weak(left, left - 1)) return false;
    }
    return false;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t pinned_malloc(void** p, size_t bytes) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocHost(p, bytes);
}

int check_flags(unsigned long long flags, const char* fn) {
    if (!flags) return BEM_OK;
    set_error("%s: the checked build skipped out-of-range accesses (flags 0x%llx:%s%s%s%s%s)", fn, flags,
              flags & kCheckPart ? " partial-sum slot" : "", flags & kCheckPoint ? " per-point array" : "",
              flags & kCheckRow ? " near-prefix row" : "", flags & kCheckElement ? " near-pair run" : "",
              flags & kCheckMatrix ? " matrix entry" : "");
    return BEM_ERR_CUDA;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    return e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA;
}

PtrLoc ptr_location(const void* p, int dev) {
    if (!p) return kPtrHost;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown host pointer
        return kPtrHost;
    }
    if (a.type == cudaMemoryTypeManaged) return kPtrDevice;
    if (a.type == cudaMemoryTypeDevice) return a.device == dev ? kPtrDevice : kPtrOtherDevice;
    return kPtrHost;
}

int reject_other_device(const char* fn, int dev, const void* const* ptrs, const char* const* names, int n) {
    for (int i = 0; i < n; ++i) {
        if (ptrs[i] && ptr_location(ptrs[i], dev) == kPtrOtherDevice) {
            set_error("%s: %s is in the memory of another GPU than the mesh's device %d", fn, names[i], dev);
            return BEM_ERR_INVALID;
        }
    }
    return BEM_OK;
}

namespace {

// the array is device memory the mesh's kernels can use directly (callers have
// already rejected arrays on another device)
bool is_device_ptr(const void* p, int dev) { return p && ptr_location(p, dev) == kPtrDevice; }

template <typename T>
int dalloc(bem_mesh* m, T** p, size_t count) {
    const size_t bytes = count * sizeof(T);
    if (m->w.bytes + bytes > m->budget) {
        set_error("device memory budget exceeded: need %zu more bytes, budget %zu, in use %zu", bytes, m->budget,
                  m->w.bytes);
        return BEM_ERR_OOM;
    }
    cudaError_t e = dev_malloc((void**)p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return BEM_ERR_OOM;
    }
    m->w.bytes += bytes;
    return BEM_OK;
}

template <typename T>
void dfree(bem_mesh* m, T** p, size_t count) {
    if (*p) {
        cudaFree(*p);
        m->w.bytes -= count * sizeof(T);
        *p = nullptr;
    }
}

void free_points(bem_mesh* m) {
    Work& w = m->w;
    const size_t c = w.cap_pts, cs = c * (size_t)m->n_chunks;
    dfree(m, &w.pts, 3 * c);
    dfree(m, &w.out, 4 * c);
    dfree(m, &w.perm, c);
    dfree(m, &w.key, c);
    dfree(m, &w.part, cs);
    dfree(m, &w.near_cnt, cs);
    dfree(m, &w.far, c);
    dfree(m, &w.near_tot, c);
    dfree(m, &w.near_row, c);
    dfree(m, &w.near_rows, cs);
    dfree(m, &w.near_off, c);
    dfree(m, &w.tile_done, tile_done_ints(c));
    dfree(m, &w.scan_tmp, scan_tmp_ints((int)std::max(c, kCells)));
    w.cap_pts = 0;
}

void free_near(bem_mesh* m) {
    Work& w = m->w;
    dfree(m, &w.near_rec, w.cap_near);
    dfree(m, &w.near_val, w.cap_near);
    w.cap_near = 0;
}

int ensure_points(bem_mesh* m, size_t n) {
    Work& w = m->w;
    if (n <= w.cap_pts) return BEM_OK;
    free_points(m);
    size_t c = 1024;
    while (c < n) c *= 2;
    const size_t cs = c * (size_t)m->n_chunks;
    if (cs >= (size_t(1) << 31)) {
        set_error("too many field points for one call (%zu x %d element chunks)", n, m->n_chunks);
        return BEM_ERR_INVALID;
    }
    int rc;
    if ((rc = dalloc(m, &w.pts, 3 * c)) || (rc = dalloc(m, &w.out, 4 * c)) || (rc = dalloc(m, &w.perm, c)) ||
        (rc = dalloc(m, &w.key, c)) || (rc = dalloc(m, &w.part, cs)) || (rc = dalloc(m, &w.near_cnt, cs)) ||
        (rc = dalloc(m, &w.far, c)) || (rc = dalloc(m, &w.near_tot, c)) || (rc = dalloc(m, &w.near_row, c)) ||
        (rc = dalloc(m, &w.near_rows, cs)) || (rc = dalloc(m, &w.near_off, c)) ||
        (rc = dalloc(m, &w.tile_done, tile_done_ints(c))) ||
        (rc = dalloc(m, &w.scan_tmp, scan_tmp_ints((int)std::max(c, kCells))))) {
        w.cap_pts = c;
        free_points(m);
        return rc;
    }
    w.cap_pts = c;
    return BEM_OK;
}

int ensure_near(bem_mesh* m, size_t n) {
    Work& w = m->w;
    if (n <= w.cap_near) return BEM_OK;
    free_near(m);
    size_t c = size_t(1) << 16;
    while (c < n) c *= 2;
    int rc;
    if ((rc = dalloc(m, &w.near_rec, c)) || (rc = dalloc(m, &w.near_val, c))) {
        w.cap_near = c;
        free_near(m);
        return rc;
    }
    w.cap_near = c;
    return BEM_OK;
}

void free_mesh(bem_mesh* m) {
    if (!m) return;
    free_points(m);
    free_near(m);
    MeshDev& d = m->d;
    cudaFree(d.chi);
    cudaFree(d.clo);
    cudaFree(d.e0);
    cudaFree(d.e1);
    cudaFree(d.nodes);
    cudaFree(d.cen);
    cudaFree(d.fr);
    cudaFree(d.geo);
    cudaFree(d.verts);
    cudaFree(d.egeo);
    cudaFree(d.type);
    cudaFree(d.sigma);
    cudaFree(d.slope);
    cudaFree(d.curv);
    cudaFree(m->w.cell_cnt);
    cudaFree(m->w.cell_off);
    cudaFree(m->w.counters);
    cudaFree(m->w.bbox);
    for (auto& e : m->ev)
        if (e) cudaEventDestroy(e);
    delete m;
}

// Stage an input array of `bytes` onto the device if it is a host array.
int stage_in(const void* src, size_t bytes, void* dev_buf, const void** out, cudaStream_t s, int dev) {
    if (is_device_ptr(src, dev)) {
        *out = src;
        return BEM_OK;
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(dev_buf, src, bytes, cudaMemcpyHostToDevice, s));
    *out = dev_buf;
    return BEM_OK;
}

// After launch_sort_points: fail on non-finite field points.
int check_points(bem_mesh* m, const char* fn, cudaStream_t s) {
    unsigned long long bad = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&bad, m->w.counters + 15, sizeof bad, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) {
        set_error("%s: a field point has a non-finite (or |x| >= 1e30) coordinate", fn);
        return BEM_ERR_INVALID;
    }
    return BEM_OK;
}

int check_mesh(const bem_mesh* m, const char* fn) {
    if (!m) {
        set_error("%s: mesh is NULL", fn);
        return BEM_ERR_INVALID;
    }
    return BEM_OK;
}

// Far pass + near pass + finalisation for n sorted points (m->w.perm filled).
// Retries once with a larger near list if the first pass overflowed it.
int run_eval(bem_mesh* m, const double* dpts, int n, const double* dsigma, double* dphi, double* dE, int stride4,
             bool want_e, cudaStream_t s) {
    Work& w = m->w;
    for (int attempt = 0; attempt < 3; ++attempt) {
        BEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, kCounters * sizeof(unsigned long long), s));
        FarArgs a{};
        a.pts = dpts;
        a.perm = w.perm;
        a.n_pts = n;
        a.sigma = dsigma;
        a.slope = eval_slope(m, dsigma);
        far_args_from_work(a, w, m->n_chunks);
        a.work = reinterpret_cast<int*>(w.counters + 14);
        a.near_rec = w.near_rec;
        a.counters = w.counters;
        a.near_cap = w.cap_near;
        a.kc = m->kc;
        a.want_e = want_e;
        a.bbox = reinterpret_cast<const unsigned*>(w.bbox);
        a.stats = m->stats;
        if (m->timing) BEM_CUDA_TRY(cudaEventRecord(m->ev[1], s));
        int rc;
        {
            NvtxRange r("bem.far");
            if ((rc = launch_far(m, a, s))) return rc;
        }
        if (m->timing) BEM_CUDA_TRY(cudaEventRecord(m->ev[2], s));
        {
            NvtxRange r("bem.near");
            if ((rc = launch_exclusive_scan(w.near_tot, w.near_off, n, w.scan_tmp, s))) return rc;
            if ((rc = launch_near_eval(m, dpts, w.perm, n, dsigma, 0, s, eval_slope(m, dsigma)))) return rc;
        }
        if (m->timing) BEM_CUDA_TRY(cudaEventRecord(m->ev[3], s));
        {
            NvtxRange r("bem.finalize");
            if ((rc = launch_finalize(m, w.perm, n, dphi, dE, stride4, s))) return rc;
        }
        if (m->timing) BEM_CUDA_TRY(cudaEventRecord(m->ev[4], s));
        unsigned long long cnt[kCounters];
        BEM_CUDA_TRY(cudaMemcpyAsync(cnt, w.counters, sizeof cnt, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (m->timing) {
            float t;
            for (int k = 0; k < 4; ++k) {
                BEM_CUDA_TRY(cudaEventElapsedTime(&t, m->ev[k], m->ev[k + 1]));
                m->last_times[k] = t;
            }
        }
        if ((rc = check_flags(cnt[kCheckCounter], "bem_eval"))) return rc;
        const unsigned long long pairs = cnt[kPairCounter];  // values; the run records are fewer
        if (pairs <= w.cap_near) {
            m->last_stats[12] = (int64_t)pairs;
            if (m->stats) {
                for (int k = 0; k < 12; ++k) m->last_stats[k] = (int64_t)cnt[2 + k];
                for (int k = 0; k < 3; ++k) m->last_stats[13 + k] = (int64_t)cnt[16 + k];
            }
            return BEM_OK;
        }
        if ((rc = ensure_near(m, (size_t)pairs))) return rc;  // grow and run again
    }
    set_error("near-pair list did not converge");
    return BEM_ERR_CAPACITY;
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" {

const char* bem_last_error(void) { return g_err.c_str(); }

const char* bem_version(void) {
    return BEM_CHECKED ? "bem-cubature-gb300 0.1 (sm_103a, checked)" : "bem-cubature-gb300 0.1 (sm_103a)";
}

int64_t bem_num_elements(const bem_mesh* m) { return m ? m->d.n : 0; }

int bem_create(const int32_t* types, const double* verts, const double* sigma, int64_t n, const bem_options* opt,
               void* stream, bem_mesh** out) {
    if (!out) {
        set_error("bem_create: out is NULL");
        return BEM_ERR_INVALID;
    }
    *out = nullptr;
    if (!types || !verts || !sigma || n < 1 || n >= (int64_t(1) << 31)) {
        set_error("bem_create: bad arguments (n = %lld)", (long long)n);
        return BEM_ERR_INVALID;
    }
    bem_mesh* m = new (std::nothrow) bem_mesh();
    if (!m) {
        set_error("bem_create: out of host memory");
        return BEM_ERR_OOM;
    }
    cudaStream_t s = (cudaStream_t)stream;
    m->precision = opt ? opt->precision : BEM_FP64;
    if (m->precision != BEM_FP64 && m->precision != BEM_MIXED) {
        set_error("bem_create: unknown precision %d", (int)m->precision);
        delete m;
        return BEM_ERR_INVALID;
    }
    if (opt && (opt->flags & ~BEM_FLAG_NODE_TABLE)) {
        set_error("bem_create: unknown flags 0x%x", (unsigned)opt->flags);
        delete m;
        return BEM_ERR_INVALID;
    }
    m->eps0 = (opt && opt->eps0 > 0.0) ? opt->eps0 : kEps0SI;
    m->kc = 1.0 / (4.0 * M_PI * m->eps0);
    m->budget = (opt && opt->device_mem_budget) ? opt->device_mem_budget : (size_t(4) << 30);
    for (int t = 0; t < 2; ++t)
        for (int k = 0; k < 5; ++k) {
            m->limits[t][k] = (opt && opt->limits) ? opt->limits[5 * t + k] : kDefaultLimits[t][k];
            if (!(m->limits[t][k] >= 0.0) || !isfinite(m->limits[t][k]) || (k && m->limits[t][k] < m->limits[t][k - 1])) {
                set_error("bem_create: limits must be finite, non-negative and ascending");
                delete m;
                return BEM_ERR_INVALID;
            }
        }
    cudaError_t ce = cudaGetDevice(&m->device);
    if (ce != cudaSuccess) {
        delete m;
        return cuda_fail(ce, "cudaGetDevice");
    }
    m->d.n = (int)n;
    // the far-field pass splits the elements into chunks fixed by the mesh
    // (so a point's sum is always split the same way): enough work items to
    // fill the GPU even for a few thousand points
    m->n_chunks = (int)std::min<int64_t>(kMaxChunks, std::max<int64_t>(1, (n + kChunkMinElements - 1) / kChunkMinElements));
    m->chunk_len = (int)(((n + m->n_chunks - 1) / m->n_chunks + 31) / 32 * 32);
    m->n_chunks = (int)((n + m->chunk_len - 1) / m->chunk_len);
    MeshDev& d = m->d;
    int rc = BEM_OK;
    // element arrays are owned by the mesh, outside the scratch budget
    const size_t nn = (size_t)n;
#define BEM_ALLOC(ptr, count)                                                              \
    if (!rc) {                                                                             \
        cudaError_t e_ = dev_malloc((void**)&(ptr), sizeof(*(ptr)) * (count));             \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            set_error("bem_create: cudaMalloc failed: %s", cudaGetErrorString(e_));        \
            rc = BEM_ERR_OOM;                                                              \
        }                                                                                  \
    }
    BEM_ALLOC(d.chi, nn);
    BEM_ALLOC(d.clo, nn);
    BEM_ALLOC(d.e0, nn);
    BEM_ALLOC(d.e1, nn);
    BEM_ALLOC(d.cen, 3 * nn);
    BEM_ALLOC(d.fr, 6 * nn);
    BEM_ALLOC(d.geo, 2 * nn);
    BEM_ALLOC(d.verts, 12 * nn);
    BEM_ALLOC(d.egeo, kEgeo * nn);
    BEM_ALLOC(d.type, nn);
    BEM_ALLOC(d.sigma, nn);
    BEM_ALLOC(m->w.cell_cnt, kCells);
    BEM_ALLOC(m->w.cell_off, kCells);
    BEM_ALLOC(m->w.counters, kCounters);
    BEM_ALLOC(m->w.bbox, 2);
#undef BEM_ALLOC
    if (rc) {
        free_mesh(m);
        return rc;
    }
    // stage the raw input (host or device) into scratch, then preprocess
    int* dtypes = nullptr;
    double *dverts = nullptr, *dsig = nullptr;
    ce = dev_malloc((void**)&dtypes, sizeof(int) * nn);
    if (ce == cudaSuccess) ce = dev_malloc((void**)&dverts, sizeof(double) * 12 * nn);
    if (ce == cudaSuccess) ce = dev_malloc((void**)&dsig, sizeof(double) * nn);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dtypes, types, sizeof(int) * nn, cudaMemcpyDefault, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dverts, verts, sizeof(double) * 12 * nn, cudaMemcpyDefault, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(dsig, sigma, sizeof(double) * nn, cudaMemcpyDefault, s);
    if (ce != cudaSuccess) {
        rc = cuda_fail(ce, "bem_create staging");
    } else {
        int64_t bad = -1;
        int code = 0;
        rc = launch_prep(m, dtypes, dverts, dsig, s, &bad, &code, &m->coord_max);
    }
    cudaFree(dtypes);
    cudaFree(dverts);
    cudaFree(dsig);
    if (rc) {
        free_mesh(m);
        return rc;
    }
    if (opt && (opt->flags & BEM_FLAG_NODE_TABLE) && m->precision == kMixed) {
        cudaError_t e = dev_malloc((void**)&d.nodes, sizeof(float4) * kNodeRecs * kTableSlots * nn);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("bem_create: cudaMalloc of the node table (%zu bytes) failed: %s",
                      sizeof(float4) * kNodeRecs * kTableSlots * nn, cudaGetErrorString(e));
            rc = BEM_ERR_OOM;
        } else {
            rc = launch_fill_nodes(m, s);
        }
        if (rc) {
            free_mesh(m);
            return rc;
        }
    }
    if ((rc = ensure_near(m, std::max<size_t>(size_t(1) << 20, 4 * nn)))) {
        free_mesh(m);
        return rc;
    }
    *out = m;
    return BEM_OK;
}

void bem_destroy(bem_mesh* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    free_mesh(m);
}

int bem_set_sigma(bem_mesh* m, const double* sigma, void* stream) {
    int rc = check_mesh(m, "bem_set_sigma");
    if (rc) return rc;
    if (!sigma) {
        set_error("bem_set_sigma: sigma is NULL");
        return BEM_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    BEM_CUDA_TRY(cudaMemcpyAsync(m->d.sigma, sigma, sizeof(double) * m->d.n, cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    m->linear = false;
    m->quadratic = false;
    return BEM_OK;
}

int bem_set_sigma_linear(bem_mesh* m, const double* coef, void* stream) {
    int rc = check_mesh(m, "bem_set_sigma_linear");
    if (rc) return rc;
    if (!coef) {
        set_error("bem_set_sigma_linear: coef is NULL");
        return BEM_ERR_INVALID;
    }
    const size_t n = (size_t)m->d.n;
    if (n == 0) return BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    if (!m->d.slope) {
        const cudaError_t e = dev_malloc((void**)&m->d.slope, sizeof(double) * 2 * n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            m->d.slope = nullptr;
            set_error("bem_set_sigma_linear: cudaMalloc failed: %s", cudaGetErrorString(e));
            return BEM_ERR_OOM;
        }
    }
    // (n x 3) -> sigma (n) and slopes (n x 2): strided copies of the columns
    BEM_CUDA_TRY(cudaMemcpy2DAsync(m->d.sigma, sizeof(double), coef, 3 * sizeof(double), sizeof(double), n,
                                   cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaMemcpy2DAsync(m->d.slope, 2 * sizeof(double), coef + 1, 3 * sizeof(double),
                                   2 * sizeof(double), n, cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    m->linear = true;
    m->quadratic = false;
    return BEM_OK;
}

int bem_set_sigma_quadratic(bem_mesh* m, const double* coef, void* stream) {
    int rc = check_mesh(m, "bem_set_sigma_quadratic");
    if (rc) return rc;
    if (!coef) {
        set_error("bem_set_sigma_quadratic: coef is NULL");
        return BEM_ERR_INVALID;
    }
    const size_t n = (size_t)m->d.n;
    if (n == 0) return BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    double** bufs[2] = {&m->d.slope, &m->d.curv};
    const size_t cols[2] = {2, 3};
    for (int b = 0; b < 2; ++b) {
        if (*bufs[b]) continue;
        const cudaError_t e = dev_malloc((void**)bufs[b], sizeof(double) * cols[b] * n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            *bufs[b] = nullptr;
            set_error("bem_set_sigma_quadratic: cudaMalloc failed: %s", cudaGetErrorString(e));
            return BEM_ERR_OOM;
        }
    }
    // (n x 6) -> sigma (n), slopes (n x 2) and second-order coefficients (n x 3)
    BEM_CUDA_TRY(cudaMemcpy2DAsync(m->d.sigma, sizeof(double), coef, 6 * sizeof(double), sizeof(double), n,
                                   cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaMemcpy2DAsync(m->d.slope, 2 * sizeof(double), coef + 1, 6 * sizeof(double),
                                   2 * sizeof(double), n, cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaMemcpy2DAsync(m->d.curv, 3 * sizeof(double), coef + 3, 6 * sizeof(double),
                                   3 * sizeof(double), n, cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    m->linear = true;
    m->quadratic = true;
    return BEM_OK;
}

int bem_set_stats(bem_mesh* m, int32_t enable) {
    int rc = check_mesh(m, "bem_set_stats");
    if (rc) return rc;
    m->stats = enable != 0;
    return BEM_OK;
}

int bem_last_stats(const bem_mesh* m, int64_t* out) {
    int rc = check_mesh(m, "bem_last_stats");
    if (rc) return rc;
    if (!out) {
        set_error("bem_last_stats: out is NULL");
        return BEM_ERR_INVALID;
    }
    for (int k = 0; k < 16; ++k) out[k] = m->last_stats[k];
    return BEM_OK;
}

int bem_set_timing(bem_mesh* m, int32_t enable) {
    int rc = check_mesh(m, "bem_set_timing");
    if (rc) return rc;
    if (enable && !m->ev[0]) {
        BEM_CUDA_TRY(cudaSetDevice(m->device));
        for (auto& e : m->ev) BEM_CUDA_TRY(cudaEventCreate(&e));
    }
    m->timing = enable != 0;
    return BEM_OK;
}

int bem_last_times(const bem_mesh* m, double* out) {
    int rc = check_mesh(m, "bem_last_times");
    if (rc) return rc;
    if (!out) {
        set_error("bem_last_times: out is NULL");
        return BEM_ERR_INVALID;
    }
    for (int k = 0; k < 4; ++k) out[k] = m->last_times[k];
    return BEM_OK;
}

int64_t bem_kernel_launches(void) { return g_launches.load(); }

int bem_test_fail_alloc_after(int64_t n) {
    g_alloc_left.store(n < 0 ? -1 : n);
    return BEM_OK;
}

int64_t bem_test_alloc_count(void) { return g_alloc_count.load(); }

int32_t bem_test_ptr_location(const void* p, int32_t dev) { return (int32_t)ptr_location(p, dev); }

int bem_default_limits(double* out) {
    if (!out) {
        set_error("bem_default_limits: out is NULL");
        return BEM_ERR_INVALID;
    }
    for (int t = 0; t < 2; ++t)
        for (int k = 0; k < 5; ++k) out[5 * t + k] = kDefaultLimits[t][k];
    return BEM_OK;
}

int bem_linear_coef_from_corners(const int32_t* types, const double* values, int64_t n, double* coef) {
    if (n < 0 || (n > 0 && (!types || !values || !coef))) {
        set_error("bem_linear_coef_from_corners: bad arguments (n = %lld)", (long long)n);
        return BEM_ERR_INVALID;
    }
    for (int64_t j = 0; j < n; ++j) {
        const double* v = values + 4 * j;
        double* c = coef + 3 * j;
        if (types[j] == BEM_TRIANGLE) {
            // sigma = m + (sA - m) alpha + (sB - m) beta: at A (alpha, beta) = (1, 0), at B (0, 1),
            // at C (-1, -1), which gives 3 m - sA - sB = sC
            const double mean = (v[0] + v[1] + v[2]) / 3.0;
            c[0] = mean;
            c[1] = v[0] - mean;
            c[2] = v[1] - mean;
        } else if (types[j] == BEM_RECTANGLE) {
            // corners P0..P3 at natural coordinates (-1,-1), (1,-1), (1,1), (-1,1):
            // the least-squares plane through the four values (exact if they are planar)
            c[0] = (v[0] + v[1] + v[2] + v[3]) / 4.0;
            c[1] = (v[1] + v[2] - v[0] - v[3]) / 4.0;
            c[2] = (v[2] + v[3] - v[0] - v[1]) / 4.0;
        } else {
            set_error("bem_linear_coef_from_corners: element %lld has unknown type %d", (long long)j, (int)types[j]);
            return BEM_ERR_INVALID;
        }
    }
    return BEM_OK;
}

int bem_centroids(bem_mesh* m, double* out, void* stream) {
    int rc = check_mesh(m, "bem_centroids");
    if (rc) return rc;
    if (!out) {
        set_error("bem_centroids: out is NULL");
        return BEM_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    BEM_CUDA_TRY(cudaMemcpyAsync(out, m->d.cen, sizeof(double) * 3 * m->d.n, cudaMemcpyDefault, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}

namespace {
// One slice of bem_eval (at most kEvalSlice points).
int eval_slice(bem_mesh* m, const double* points, int64_t n, double* phi, double* E, cudaStream_t s) {
    int rc;
    if ((rc = ensure_points(m, (size_t)n))) return rc;
    Work& w = m->w;
    const double* dpts;
    if ((rc = stage_in(points, sizeof(double) * 3 * n, w.pts, (const void**)&dpts, s, m->device))) return rc;
    const bool phi_dev = is_device_ptr(phi, m->device), E_dev = is_device_ptr(E, m->device);
    const bool phi_host = phi && !phi_dev, E_host = E && !E_dev;
    if ((phi_dev && E_host) || (phi_host && E_dev)) {
        set_error("bem_eval: phi and E must both be host or both be device arrays");
        return BEM_ERR_INVALID;
    }
    if (m->timing) BEM_CUDA_TRY(cudaEventRecord(m->ev[0], s));
    {
        NvtxRange r("bem.sort");
        if ((rc = launch_sort_points(m, dpts, (int)n, s))) return rc;
    }
    if ((rc = check_points(m, "bem_eval", s))) return rc;
    if (!phi_host && !E_host) return run_eval(m, dpts, (int)n, m->d.sigma, phi, E, 0, E != nullptr, s);
    // host outputs: finalise into the staging buffer (phi | E), then copy out
    double* sphi = w.out;
    double* sE = w.out + n;
    if ((rc = run_eval(m, dpts, (int)n, m->d.sigma, sphi, sE, 0, E != nullptr, s))) return rc;
    if (phi) BEM_CUDA_TRY(cudaMemcpyAsync(phi, sphi, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (E) BEM_CUDA_TRY(cudaMemcpyAsync(E, sE, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    return BEM_OK;
}
// Large calls run in slices: the scratch grows with the points of one
// slice, and results do not depend on how the points are grouped.
constexpr int64_t kEvalSlice = int64_t(1) << 21;
}  // namespace

int bem_eval(bem_mesh* m, const double* points, int64_t n, double* phi, double* E, void* stream) {
    NvtxRange range("bem_eval");
    int rc = check_mesh(m, "bem_eval");
    if (rc) return rc;
    if (n < 0 || n >= (int64_t(1) << 31) || (n > 0 && !points)) {
        set_error("bem_eval: bad arguments (n = %lld)", (long long)n);
        return BEM_ERR_INVALID;
    }
    if (n == 0) return BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    {
        const void* ptrs[3] = {points, phi, E};
        const char* names[3] = {"points", "phi", "E"};
        if ((rc = reject_other_device("bem_eval", m->device, ptrs, names, 3))) return rc;
    }
    for (int64_t off = 0; off < n; off += kEvalSlice) {
        const int64_t k = std::min(kEvalSlice, n - off);
        rc = eval_slice(m, points + 3 * off, k, phi ? phi + off : nullptr, E ? E + 3 * off : nullptr, s);
        if (rc) return rc;
    }
    return BEM_OK;
}


}  // extern "C"

namespace {
// Device buffer freed on scope exit.
template <typename T>
struct Scratch {
    T* p = nullptr;
    ~Scratch() {
        if (p) cudaFree(p);
    }
    int alloc(size_t count) {
        const cudaError_t e = dev_malloc((void**)&p, sizeof(T) * (count > 0 ? count : 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            set_error("bem_eval_grad: cudaMalloc of %zu bytes failed: %s", sizeof(T) * count, cudaGetErrorString(e));
            return BEM_ERR_OOM;
        }
        return BEM_OK;
    }
};

// One slice of bem_eval_grad: the far kernel in its gradient mode (the mesh's precision), the
// compacted near pairs' analytic gradients, the per-point sums.
int grad_slice(bem_mesh* m, const double* points, int64_t n, double* G, cudaStream_t s) {
    int rc;
    if ((rc = ensure_points(m, (size_t)n))) return rc;
    Work& w = m->w;
    const double* dpts;
    if ((rc = stage_in(points, sizeof(double) * 3 * n, w.pts, (const void**)&dpts, s, m->device))) return rc;
    if ((rc = launch_sort_points(m, dpts, (int)n, s))) return rc;
    if ((rc = check_points(m, "bem_eval_grad", s))) return rc;
    // tile-major partial slots for whole tiles (of at most 128 points) of every chunk
    const size_t np = ((size_t)n + 127) / 128 * 128 * (size_t)m->n_chunks;
    const bool g_dev = is_device_ptr(G, m->device);
    const size_t need = sizeof(double4) * 2 * (np + (size_t)n) + (g_dev ? 0 : sizeof(double) * 6 * (size_t)n);
    if (m->w.bytes + need > m->budget) {
        set_error("bem_eval_grad: needs %zu bytes beyond the %zu in use (budget %zu)", need, m->w.bytes, m->budget);
        return BEM_ERR_OOM;
    }
    Scratch<double4> part_g, far_g;
    Scratch<double> gout;
    if ((rc = part_g.alloc(2 * np)) || (rc = far_g.alloc(2 * (size_t)n))) return rc;
    if (!g_dev && (rc = gout.alloc(6 * (size_t)n))) return rc;
    double* dG = g_dev ? G : gout.p;
    for (int attempt = 0; attempt < 3; ++attempt) {
        BEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, kCounters * sizeof(unsigned long long), s));
        FarArgs a{};
        a.pts = dpts;
        a.perm = w.perm;
        a.n_pts = (int)n;
        a.sigma = m->d.sigma;
        a.slope = eval_slope(m, m->d.sigma);
        far_args_from_work(a, w, m->n_chunks);
        a.part_g = part_g.p;
        a.far_g = far_g.p;
        a.part_cap = std::min<unsigned long long>(a.part_cap, np);
        a.pts_cap = std::min<unsigned long long>(a.pts_cap, (unsigned long long)n);
        a.work = reinterpret_cast<int*>(w.counters + 14);
        a.near_rec = w.near_rec;
        a.counters = w.counters;
        a.near_cap = w.cap_near;
        a.kc = m->kc;
        a.want_e = 1;
        a.bbox = reinterpret_cast<const unsigned*>(w.bbox);
        if ((rc = launch_far(m, a, s))) return rc;
        if ((rc = launch_exclusive_scan(w.near_tot, w.near_off, (int)n, w.scan_tmp, s))) return rc;
        unsigned long long n_near = 0;  // near pairs (values)
        BEM_CUDA_TRY(cudaMemcpyAsync(&n_near, w.counters + kPairCounter, sizeof n_near, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
        if (n_near > w.cap_near) {
            if ((rc = ensure_near(m, (size_t)n_near))) return rc;  // grow and run again
            continue;
        }
        Scratch<double4> gval;
        if ((rc = gval.alloc(2 * (size_t)n_near))) return rc;
        if ((rc = launch_near_grad(m, dpts, w.perm, m->d.sigma, gval.p, n_near, s, eval_slope(m, m->d.sigma))))
            return rc;
        if ((rc = launch_finalize_grad(m, w.perm, (int)n, far_g.p, gval.p, n_near, dG, s))) return rc;
        if (!g_dev) BEM_CUDA_TRY(cudaMemcpyAsync(G, dG, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, s));
        unsigned long long flags = 0;
        BEM_CUDA_TRY(cudaMemcpyAsync(&flags, w.counters + kCheckCounter, sizeof flags, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
        if ((rc = check_flags(flags, "bem_eval_grad"))) return rc;
        m->last_stats[12] = (int64_t)n_near;
        return BEM_OK;
    }
    set_error("bem_eval_grad: near-pair list did not converge");
    return BEM_ERR_CAPACITY;
}
}  // namespace

extern "C" {

int bem_eval_grad(bem_mesh* m, const double* points, int64_t n, double* G, void* stream) {
    NvtxRange range("bem_eval_grad");
    int rc = check_mesh(m, "bem_eval_grad");
    if (rc) return rc;
    if (n < 0 || n >= (int64_t(1) << 31) || (n > 0 && (!points || !G))) {
        set_error("bem_eval_grad: bad arguments (n = %lld)", (long long)n);
        return BEM_ERR_INVALID;
    }
    if (n == 0) return BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    {
        const void* ptrs[2] = {points, G};
        const char* names[2] = {"points", "G"};
        if ((rc = reject_other_device("bem_eval_grad", m->device, ptrs, names, 2))) return rc;
    }
    for (int64_t off = 0; off < n; off += kEvalSlice) {
        const int64_t k = std::min(kEvalSlice, n - off);
        if ((rc = grad_slice(m, points + 3 * off, k, G + 6 * off, s))) return rc;
    }
    return BEM_OK;
}

int bem_matvec(bem_mesh* m, const double* x, double* y, void* stream) {
    NvtxRange range("bem_matvec");
    int rc = check_mesh(m, "bem_matvec");
    if (rc) return rc;
    if (!x || !y) {
        set_error("bem_matvec: x or y is NULL");
        return BEM_ERR_INVALID;
    }
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    {
        const void* ptrs[2] = {x, y};
        const char* names[2] = {"x", "y"};
        if ((rc = reject_other_device("bem_matvec", m->device, ptrs, names, 2))) return rc;
    }
    const int n = m->d.n;
    if ((rc = ensure_points(m, (size_t)n))) return rc;
    Work& w = m->w;
    // x is staged into the first n doubles of the (otherwise unused) points buffer
    const double* dx;
    if ((rc = stage_in(x, sizeof(double) * n, w.pts, (const void**)&dx, s, m->device))) return rc;
    if (m->timing) BEM_CUDA_TRY(cudaEventRecord(m->ev[0], s));
    if ((rc = launch_sort_points(m, m->d.cen, n, s))) return rc;
    const bool y_dev = is_device_ptr(y, m->device);
    double* dy = y_dev ? y : w.out;
    if ((rc = run_eval(m, m->d.cen, n, dx, dy, nullptr, 0, false, s))) return rc;
    if (!y_dev) {
        BEM_CUDA_TRY(cudaMemcpyAsync(y, dy, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return BEM_OK;
}

int bem_assemble(bem_mesh* m, const double* colloc, int64_t mrows, double* A, void* stream) {
    NvtxRange range("bem_assemble");
    int rc = check_mesh(m, "bem_assemble");
    if (rc) return rc;
    if (mrows < 0 || mrows >= (int64_t(1) << 31) || (mrows > 0 && (!colloc || !A))) {
        set_error("bem_assemble: bad arguments (m = %lld)", (long long)mrows);
        return BEM_ERR_INVALID;
    }
    if (mrows == 0) return BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    {
        const void* ptrs[2] = {colloc, A};
        const char* names[2] = {"colloc", "A"};
        if ((rc = reject_other_device("bem_assemble", m->device, ptrs, names, 2))) return rc;
    }
    if ((rc = ensure_points(m, (size_t)mrows))) return rc;
    Work& w = m->w;
    const double* dpts;
    if ((rc = stage_in(colloc, sizeof(double) * 3 * mrows, w.pts, (const void**)&dpts, s, m->device))) return rc;
    const size_t abytes = sizeof(double) * (size_t)mrows * (size_t)m->d.n;
    const bool a_dev = is_device_ptr(A, m->device);
    double* dA = A;
    if (!a_dev) {
        if ((rc = dalloc(m, &dA, (size_t)mrows * (size_t)m->d.n))) return rc;
    }
    rc = launch_sort_points(m, dpts, (int)mrows, s);
    if (!rc) rc = check_points(m, "bem_assemble", s);
    for (int attempt = 0; !rc && attempt < 3; ++attempt) {
        cudaError_t e = cudaMemsetAsync(w.counters, 0, kCounters * sizeof(unsigned long long), s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "bem_assemble");
            break;
        }
        FarArgs a{};
        a.pts = dpts;
        a.perm = w.perm;
        a.n_pts = (int)mrows;
        a.sigma = nullptr;  // assembly: unit charge density
        a.work = reinterpret_cast<int*>(w.counters + 14);
        a.near_rec = w.near_rec;
        a.counters = w.counters;
        a.near_cap = w.cap_near;
        a.bbox = reinterpret_cast<const unsigned*>(w.bbox);
        a.A = dA;
        a.kc = m->kc;
        a.stats = m->stats;
        if ((rc = launch_far(m, a, s))) break;
        if ((rc = launch_near_assemble(m, dpts, w.perm, dA, 0, s))) break;
        unsigned long long cnt[kCounters];
        e = cudaMemcpyAsync(cnt, w.counters, sizeof cnt, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "bem_assemble");
            break;
        }
        if ((rc = check_flags(cnt[kCheckCounter], "bem_assemble"))) break;
        const unsigned long long pairs = cnt[kPairCounter];  // at least the run records
        if (pairs <= w.cap_near) {
            m->last_stats[12] = (int64_t)pairs;
            if (m->stats) {
                for (int k = 0; k < 12; ++k) m->last_stats[k] = (int64_t)cnt[2 + k];
                for (int k = 0; k < 3; ++k) m->last_stats[13 + k] = (int64_t)cnt[16 + k];
            }
            break;
        }
        rc = ensure_near(m, (size_t)pairs);
        if (!rc && attempt == 2) {
            set_error("near-pair list did not converge");
            rc = BEM_ERR_CAPACITY;
        }
    }
    if (!rc && !a_dev) {
        cudaError_t e = cudaMemcpyAsync(A, dA, abytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e, "bem_assemble readback");
    }
    if (!a_dev) dfree(m, &dA, (size_t)mrows * (size_t)m->d.n);
    return rc;
}

}  // extern "C"
