// noalloc.cu -- bem_eval_noalloc: bem_eval for callers that must not have
// the library allocate device memory.
//
// bem_eval keeps its scratch (point order, per-point sums, the near-pair
// list, ...) in buffers that the mesh grows with cudaMalloc when a call
// needs more.  Some callers cannot allow that: an application that reserves
// all device memory for its own pool up front, or a latency-critical loop
// (a particle tracker asking for fields step after step) that must never
// wait on the allocator.  bem_eval_noalloc runs the same kernels with all
// scratch carved out of one fixed array in device memory that this file
// declares, so a call allocates nothing; in exchange one call is limited to
// BEM_NOALLOC_MAX_POINTS field points and BEM_NOALLOC_MAX_NEAR near-field
// pairs.
#include <string.h>

#include <mutex>

#include "bem_internal.cuh"

namespace bem {
namespace {

constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

constexpr size_t kMaxPts = BEM_NOALLOC_MAX_POINTS;
constexpr size_t kMaxNear = BEM_NOALLOC_MAX_NEAR;
constexpr size_t kChunksCap = kMaxChunks;  // element chunks of the far-field pass (at most kMaxChunks per mesh)
// cells of the spatial sort for at most kMaxPts points (the sort's own rule)
constexpr size_t kCellsMax = size_t(1) << (3 * sort_cell_bits(kMaxPts));
constexpr size_t kScanInts = 16384;    // block sums of every scan level, with room to spare

// byte offsets of the scratch areas inside the array
constexpr size_t kOffPerm = 0;
constexpr size_t kOffKey = kOffPerm + align_up(4 * kMaxPts);
constexpr size_t kOffCellCnt = kOffKey + align_up(4 * kMaxPts);
constexpr size_t kOffCellOff = kOffCellCnt + align_up(4 * kCellsMax);
constexpr size_t kOffPart = kOffCellOff + align_up(4 * kCellsMax);
constexpr size_t kOffNearCnt = kOffPart + align_up(32 * kMaxPts * kChunksCap);
constexpr size_t kOffNearRows = kOffNearCnt + align_up(4 * kMaxPts * kChunksCap);
constexpr size_t kOffFar = kOffNearRows + align_up(4 * kMaxPts * kChunksCap);
constexpr size_t kOffNearTot = kOffFar + align_up(32 * kMaxPts);
constexpr size_t kOffNearRow = kOffNearTot + align_up(4 * kMaxPts);
constexpr size_t kOffNearOff = kOffNearRow + align_up(4 * kMaxPts);
constexpr size_t kOffTileDone = kOffNearOff + align_up(4 * kMaxPts);
constexpr size_t kOffScan = kOffTileDone + align_up(4 * tile_done_ints(kMaxPts));
constexpr size_t kOffRec = kOffScan + align_up(4 * kScanInts);
constexpr size_t kOffVal = kOffRec + align_up(16 * kMaxNear);
constexpr size_t kOffCounters = kOffVal + align_up(32 * kMaxNear);
constexpr size_t kOffBbox = kOffCounters + align_up(24 * 8);
constexpr size_t kBytes = kOffBbox + align_up(32);
static_assert(kBytes <= BEM_NOALLOC_BYTES, "scratch layout outgrew the stated size");

// The scratch of every bem_eval_noalloc call on a device (one copy per GPU
// that loads the library, held until the process exits).
__device__ __align__(256) unsigned char g_noalloc_scratch[BEM_NOALLOC_BYTES];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void* g_base[kMaxDevices] = {};

// Device address of the scratch array on the current device `dev`, looked
// up once per device.  (In host code the array's name only stands for the
// symbol; the address must come from cudaGetSymbolAddress.)
int scratch_base(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("bem_eval_noalloc: device index %d out of range", dev);
        return BEM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_base[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_base[dev]);
    return BEM_OK;
}


}  // namespace
}  // namespace bem

using namespace bem;

extern "C" int bem_eval_noalloc(bem_mesh* m, const double* points, int64_t n, double* phi, double* E,
                                void* stream) {
    if (!m) {
        set_error("bem_eval_noalloc: mesh is NULL");
        return BEM_ERR_INVALID;
    }
    if (n < 0 || n > (int64_t)kMaxPts) {
        set_error("bem_eval_noalloc: %lld field points; one call takes at most %d (BEM_NOALLOC_MAX_POINTS)",
                  (long long)n, (int)kMaxPts);
        return BEM_ERR_INVALID;
    }
    if (n == 0) return BEM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));
    {
        const void* ptrs[3] = {points, phi, E};
        const char* names[3] = {"points", "phi", "E"};
        int rc0 = reject_other_device("bem_eval_noalloc", m->device, ptrs, names, 3);
        if (rc0) return rc0;
    }
    const int dev = m->device;
    if (!points || ptr_location(points, dev) != kPtrDevice || (phi && ptr_location(phi, dev) != kPtrDevice) ||
        (E && ptr_location(E, dev) != kPtrDevice)) {
        set_error("bem_eval_noalloc: points, phi and E must be device arrays (no staging buffers are used)");
        return BEM_ERR_INVALID;
    }
    unsigned char* base = nullptr;
    int rc = scratch_base(m->device, &base);
    if (rc) return rc;

    // the same kernels as bem_eval, pointed at the fixed scratch
    bem_mesh view = *m;
    memset(&view.w, 0, sizeof view.w);
    Work& w = view.w;
    w.cap_pts = kMaxPts;
    w.perm = reinterpret_cast<int*>(base + kOffPerm);
    w.key = reinterpret_cast<unsigned*>(base + kOffKey);
    w.cell_cnt = reinterpret_cast<int*>(base + kOffCellCnt);
    w.cell_off = reinterpret_cast<int*>(base + kOffCellOff);
    w.part = reinterpret_cast<double4*>(base + kOffPart);
    w.near_cnt = reinterpret_cast<int*>(base + kOffNearCnt);
    w.near_rows = reinterpret_cast<int*>(base + kOffNearRows);
    w.far = reinterpret_cast<double4*>(base + kOffFar);
    w.near_tot = reinterpret_cast<int*>(base + kOffNearTot);
    w.near_row = reinterpret_cast<int*>(base + kOffNearRow);
    w.near_off = reinterpret_cast<int*>(base + kOffNearOff);
    w.tile_done = reinterpret_cast<int*>(base + kOffTileDone);
    w.scan_tmp = reinterpret_cast<int*>(base + kOffScan);
    w.cap_near = kMaxNear;
    w.near_rec = reinterpret_cast<int4*>(base + kOffRec);
    w.near_val = reinterpret_cast<double4*>(base + kOffVal);
    w.counters = reinterpret_cast<unsigned long long*>(base + kOffCounters);
    w.bbox = reinterpret_cast<float4*>(base + kOffBbox);
    view.stats = false;
    view.timing = false;
    if (m->n_chunks > (int)kChunksCap || scan_tmp_ints((int)kMaxPts) > kScanInts ||
        scan_tmp_ints((int)kCellsMax) > kScanInts) {
        set_error("bem_eval_noalloc: internal scan scratch too small");
        return BEM_ERR_CAPACITY;
    }

    // the array keeps the previous call's contents: reset what must start at zero
    // (the sort clears its own cell histogram and flag)
    if ((rc = launch_sort_points(&view, points, (int)n, s))) return rc;
    unsigned long long bad = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&bad, w.counters + 15, sizeof bad, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (bad) {
        set_error("bem_eval_noalloc: a field point has a non-finite (or |x| >= 1e30) coordinate");
        return BEM_ERR_INVALID;
    }
    BEM_CUDA_TRY(cudaMemsetAsync(w.counters, 0, 24 * sizeof(unsigned long long), s));
    FarArgs a{};
    a.pts = points;
    a.perm = w.perm;
    a.n_pts = (int)n;
    a.sigma = m->d.sigma;
    a.slope = eval_slope(m, m->d.sigma);
    far_args_from_work(a, w, m->n_chunks);
    a.work = reinterpret_cast<int*>(w.counters + 14);
    a.near_rec = w.near_rec;
    a.counters = w.counters;
    a.near_cap = w.cap_near;
    a.kc = m->kc;
    a.want_e = E != nullptr;
    a.stats = 0;
    a.bbox = reinterpret_cast<const unsigned*>(w.bbox);
    if ((rc = launch_far(&view, a, s))) return rc;
    if ((rc = launch_exclusive_scan(w.near_tot, w.near_off, (int)n, w.scan_tmp, s))) return rc;
    if ((rc = launch_near_eval(&view, points, w.perm, (int)n, m->d.sigma, 0, s, eval_slope(m, m->d.sigma)))) return rc;
    if ((rc = launch_finalize(&view, w.perm, (int)n, phi, E, 0, s))) return rc;
    // the pair counter and, two further on, the checked build's flags
    static_assert(kCheckCounter == kPairCounter + 2, "counter layout");
    unsigned long long c[3] = {0, 0, 0};
    BEM_CUDA_TRY(cudaMemcpyAsync(c, w.counters + kPairCounter, sizeof c, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if ((rc = check_flags(c[2], "bem_eval_noalloc"))) return rc;
    const unsigned long long n_near = c[0];  // near pairs (values; the run records are fewer)
    if (n_near > kMaxNear) {
        set_error("bem_eval_noalloc: %llu near-field pairs; one call takes at most %d (BEM_NOALLOC_MAX_NEAR); "
                  "phi and E are incomplete -- split the points or use bem_eval",
                  n_near, (int)kMaxNear);
        return BEM_ERR_CAPACITY;
    }
    return BEM_OK;
}
