// bem_internal.cuh -- internal types shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "bem.h"

namespace bem {

// ---------------------------------------------------------------- rules
// Node slots of the five rules of one element type, concatenated in rule
// order r = 0..4 (N = 4, 7, 12, 19|17, 33; App. A / App. B).
constexpr int kMaxSlots = 80;  // 75 triangle slots, 73 rectangle slots, padded

struct RuleSet {
    int n[2][5];      // nodes per rule [type][r]
    int start[2][5];  // first slot of rule r
    double alpha[2][kMaxSlots], beta[2][kMaxSlots], w[2][kMaxSlots];
};
const RuleSet& rules();  // expanded once on the host (rules.cu)

// ---------------------------------------------------------------- bands
// Band of a pair: 0 = analytic near field, 1..5 = cubature with rule
// r = 5 - band (band 1 = 33 points ... band 5 = 4 points).
__host__ __device__ inline int band_rule(int band) { return 5 - band; }

// ---------------------------------------------------------------- mesh data in HBM
// Structure of arrays, one entry per element, element order as given.
constexpr int kTableSlots = 75;  // nodes per element in the node table (4 + 7 + 12 + 19 + 33)
// float4 records per node of the mixed path: (-alpha, -alpha, -beta, -beta),
// (|o|^2, |o|^2, w, w) and (-w alpha / 2, -w alpha / 2, -w beta / 2, -w beta / 2):
// the third record lets each node's four sums take one FMA each (9 packed
// operations per node and point pair instead of 10); it is halved because the
// kernel's frame records hold 2 e0 and 2 e1 (so that 2 d.e0 and 2 d.e1 need no
// doubling) and the field rebuild multiplies these sums by them
constexpr int kNodeRecs = 3;

// Element chunks of the far-field pass (fixed per mesh, so that a point's
// sum is always split the same way): at least kChunkMinElements elements
// each, at most kMaxChunks; more chunks give small point batches more work
// items to fill the GPU with.
#ifndef BEM_MAX_CHUNKS
#define BEM_MAX_CHUNKS 32
#endif
#ifndef BEM_CHUNK_MIN
#define BEM_CHUNK_MIN 625
#endif
constexpr int kMaxChunks = BEM_MAX_CHUNKS;
constexpr int kChunkMinElements = BEM_CHUNK_MIN;

// Element geometry of the analytic near field (FP64, per element): the unit
// normal n of the corners' plane, for each edge k (corner k to k + 1) its unit
// tangent t_k and in-plane outward normal m_k = t_k x n, and the mean side.
constexpr int kEgeo = 28;  // 3 + 4 x 6 + 1 (triangles leave the fourth edge zero)

struct MeshDev {
    int n = 0;
    // mixed path records (float4, 64 B per element)
    float4* chi = nullptr;  // centroid hi part xyz, w = type (0/1) as int bits
    float4* clo = nullptr;  // centroid lo part xyz, w = L
    float4* e0 = nullptr;   // frame vector e0 xyz, w = area
    float4* e1 = nullptr;   // frame vector e1 xyz, w = 0
    float4* nodes = nullptr;  // BEM_FLAG_NODE_TABLE: [n][kTableSlots][2] node records of every rule
    // FP64 path / near field / assembly
    double* cen = nullptr;    // [n][3] centroid
    double* fr = nullptr;     // [n][6] e0, e1 (FP64)
    double* geo = nullptr;    // [n][2] L, area
    double* verts = nullptr;  // [n][12] corners as given
    double* egeo = nullptr;   // [n][kEgeo] near field: unit normal, per edge unit tangent and outward normal, mean side
    int* type = nullptr;      // [n]
    double* sigma = nullptr;  // [n] (linear density: the value at the centroid)
    double* slope = nullptr;  // [n][2] linear density: d sigma / d alpha, d sigma / d beta (bem_set_sigma_linear)
    double* curv = nullptr;   // [n][3] quadratic density: the alpha^2, alpha beta, beta^2 coefficients
};

// Per-call scratch (grown on demand, owned by the mesh).
struct Work {
    size_t cap_pts = 0;
    double* pts = nullptr;        // staged points [cap][3] (host inputs)
    double* out = nullptr;        // staged outputs [cap][4]
    int* perm = nullptr;          // sorted -> original point index
    unsigned* key = nullptr;      // spatial cell key per point
    int* cell_cnt = nullptr;      // histogram of cells
    int* cell_off = nullptr;      // exclusive scan of cell_cnt
    // Far-field sums and near-pair counts of one work item (a tile of points x
    // an element chunk), laid out tile by tile: [tile][chunk][point of the tile].
    // They are transient: the tile's last item sums them into far / near_tot
    // and drops them from L2 without a write-back.
    double4* part = nullptr;
    int* near_cnt = nullptr;
    double4* far = nullptr;       // far-field sums per sorted point (the chunks summed in chunk order)
    int* near_tot = nullptr;      // near pairs per sorted point
    int* near_row = nullptr;      // per sorted point with near pairs: its row of near_rows
    int* near_rows = nullptr;     // [row][chunk]: near pairs of the point in the chunks before
    int* near_off = nullptr;      // exclusive scan of near_tot: first near value of each point
    int* tile_done = nullptr;     // work items finished per tile, then the near_rows row counter
    int* scan_tmp = nullptr;      // block sums of the scans
    size_t cap_near = 0;
    int4* near_rec = nullptr;     // runs: (sorted point, first element, first ordinal, pairs)
    double4* near_val = nullptr;  // analytic contributions in (point, ordinal) order
    unsigned long long* counters = nullptr;  // [0] near-pair runs (records), [1] bad element, [2..13] band
                                             // stats, [14] far work-item counter, [15] bad field point,
                                             // [16..18] far-kernel efficiency counts (statistics runs),
                                             // [19] near pairs (values)
    float4* bbox = nullptr;       // [2] points bbox (min, max)
    size_t bytes = 0;
};

enum Precision { kFP64 = 0, kMixed = 1 };
constexpr int kPairCounter = 19;  // counters[kPairCounter]: near pairs of a call

// Checked build (-DBEM_CHECKED=1): the kernels compare the global indices they
// compute with the capacities of the buffers they index, skip an access that
// would fall outside, and record which check failed in counters[kCheckCounter]
// (a bit per kind); the host turns a non-zero value into BEM_ERR_CUDA.  There
// are no device asserts or traps: a failed check leaves the context usable.
#ifndef BEM_CHECKED
#define BEM_CHECKED 0
#endif
constexpr int kCheckCounter = 21;
enum CheckBit : unsigned long long {
    kCheckPart = 1,       // a work item's slot of the tile-major partial areas
    kCheckPoint = 2,      // a per-point array (far sums, near totals, rows)
    kCheckRow = 4,        // a row of the near-pair prefix table
    kCheckElement = 8,    // an element index of a near-pair run
    kCheckMatrix = 16,    // an entry of the assembled matrix
};
__device__ __forceinline__ bool check_ok(bool ok, unsigned long long* counters, unsigned long long bit) {
    if (BEM_CHECKED && !ok) atomicOr(counters + kCheckCounter, bit);
    return !BEM_CHECKED || ok;
}
// Host side of the checked build: BEM_ERR_CUDA with a message if a kernel recorded a failed check.
int check_flags(unsigned long long flags, const char* fn);

}  // namespace bem

struct bem_mesh {
    int device = 0;
    int precision = bem::kFP64;
    double eps0 = 8.8541878128e-12;
    double kc = 0.0;          // 1 / (4 pi eps0)
    double limits[2][5];      // DR band limits per type
    double coord_max = 0.0;   // largest |coordinate| of any element corner
    double grid = 1.0;        // mixed path: spacing (a power of two) of the hi parts of points and centroids
    bool linear = false;      // densities are linear over the elements (d.slope holds the slopes)
    bool quadratic = false;   // ... and quadratic (d.curv holds the second-order coefficients)
    int n_chunks = 1;         // element chunks of the far-field pass (fixed by the mesh)
    int chunk_len = 0;        // elements per chunk (a multiple of 32)
    size_t budget = 0;
    bool stats = false;
    int64_t last_stats[16] = {0};
    bool timing = false;
    double last_times[4] = {0, 0, 0, 0};
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bem::MeshDev d;
    bem::Work w;
};

namespace bem {

// ---------------------------------------------------------------- helpers
// Where a caller's array lives relative to the mesh's device `dev`: host
// memory (staged by the library), memory the kernels on `dev` can use
// directly (that device's memory or managed memory), or another GPU's memory
// (rejected: a kernel on `dev` must not dereference it).
enum PtrLoc { kPtrHost = 0, kPtrDevice = 1, kPtrOtherDevice = 2 };
PtrLoc ptr_location(const void* p, int dev);
// BEM_ERR_INVALID (with a message naming fn and the argument) if any of the
// n arrays lives on another device; NULL entries are skipped.
int reject_other_device(const char* fn, int dev, const void* const* ptrs, const char* const* names, int n);

// Every device (and pinned host) allocation of the library goes through
// these: cudaMalloc / cudaMallocHost, except that the test hook
// bem_test_fail_alloc_after (include/bem_test.h) can make them fail with
// cudaErrorMemoryAllocation without calling the runtime.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t pinned_malloc(void** p, size_t bytes);

// A named NVTX range over a phase of host-side work (the launches of one
// step of the path), visible to Nsight tools; no cost without a tool.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const char* fmt, ...);
void count_launches(int n);  // adds n to the process-wide kernel launch counter
int cuda_fail(cudaError_t e, const char* what);

#define BEM_CUDA_TRY(call)                                   \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return ::bem::cuda_fail(_e, #call); \
    } while (0)

// ---------------------------------------------------------------- launchers
// Element preprocessing (k_prep.cu). Returns the index of the first invalid
// element through *bad (-1 if none) after synchronising.
int launch_prep(bem_mesh* m, const int* types, const double* verts, const double* sigma, cudaStream_t s,
                int64_t* bad, int* bad_code, double* coord_max);

// Bits per axis of the spatial sort's cells for n points: about one point per
// cell (1..7 bits per axis), so the Z-order curve orders the points finely and
// 32 x PT consecutive points are compact.  The sort uses 2^(3 b) cells.
constexpr int sort_cell_bits(size_t n) {
    int b = 1;
    while (b < 7 && (size_t(1) << (3 * b)) < n) ++b;
    return b;
}
// Spatial sort of field points (k_sort.cu): perm = points in cell order.
int launch_sort_points(bem_mesh* m, const double* pts, int n, cudaStream_t s, const int* n_dev = nullptr);
// Exclusive scan of n ints (k_sort.cu); tmp needs scan_tmp_ints(n) ints.
int launch_exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s);
size_t scan_tmp_ints(int n);

struct FarArgs {
    const double* pts;   // original field points [n][3]
    const int* perm;     // sorted -> original
    int n_pts;
    const double* sigma; // per element charge density (eval) or the x of a matvec
    const double* slope; // linear densities: [n][2] slopes, or nullptr (constant densities)
    double4* part;       // transient: far sums per (tile, chunk, point of the tile)
    double4* part_g;     // gradient pass: the same, 6 sums as two double4
    int* near_cnt;       // transient: near pairs per (tile, chunk, point of the tile)
    double4* far;        // out: far sums per sorted point (gradient pass: two double4, far_g)
    double4* far_g;
    int* near_tot;       // out: near pairs per sorted point
    int* near_row;       // out: row of near_rows per sorted point with near pairs
    int* near_rows;      // out: per row, the point's near pairs in the chunks before each chunk
    int* tile_done;      // finished items per tile (zeroed by launch_far), then the row counter
    unsigned long long part_cap;  // entries of part / near_cnt (part_g: of its double4 pairs)
    unsigned long long pts_cap;   // entries of far (far_g: pairs) / near_tot / near_row / near_rows rows
    int* work;           // work-item counter, zero at launch
    int4* near_rec;      // out: near pair list
    unsigned long long* counters;
    unsigned long long near_cap;
    double* A;           // assembly output (row-major m x n_el) or nullptr
    double kc;           // 1/(4 pi eps0) (assembly writes scaled entries)
    int want_e;          // 0: potential only
    const unsigned* bbox;  // field-point bounding box written by launch_sort_points
    int stats;           // count pairs per band into counters[2..13]
    const int* n_dev;    // if set: the point count is read on the device (n_pts is the capacity)
};
// The per-call buffers of the far pass (everything but part_g / far_g) from a workspace.
inline void far_args_from_work(FarArgs& a, Work& w, int n_chunks) {
    a.part = w.part;
    a.near_cnt = w.near_cnt;
    a.far = w.far;
    a.near_tot = w.near_tot;
    a.near_row = w.near_row;
    a.near_rows = w.near_rows;
    a.tile_done = w.tile_done;
    a.part_cap = (unsigned long long)w.cap_pts * (unsigned long long)n_chunks;
    a.pts_cap = w.cap_pts;
}
// Ints of Work::tile_done for cap points: one per tile of at least 32 points, plus the row counter.
constexpr size_t tile_done_ints(size_t cap) { return cap / 32 + 2; }
// Far-field cubature + near-pair compaction (k_far.cu).  Zeroes a.tile_done itself.
int launch_far(bem_mesh* m, const FarArgs& a, cudaStream_t s);
// Analytic near field over the compacted list and the per-point finalisation (k_near.cu).
int launch_near_eval(bem_mesh* m, const double* pts, const int* perm, int n_pts, const double* sigma,
                     unsigned long long n_near, cudaStream_t s, const double* slope = nullptr);
// slopes of the mesh's densities for an evaluation with the mesh's own sigma (nullptr if constant)
inline const double* eval_slope(const bem_mesh* m, const double* sigma) {
    return (m->linear && sigma == m->d.sigma) ? m->d.slope : nullptr;
}
// second-order coefficients that go with the slopes of an evaluation (nullptr unless quadratic)
inline const double* eval_curv(const bem_mesh* m, const double* slope) {
    return (slope && m->quadratic) ? m->d.curv : nullptr;
}
int launch_finalize(bem_mesh* m, const int* perm, int n_pts, double* phi, double* E, int out_stride4,
                    cudaStream_t s, const int* n_dev = nullptr);
// fill MeshDev::nodes from the element records (k_far.cu)
int launch_fill_nodes(bem_mesh* m, cudaStream_t s);
// field gradient over the compacted near list and its per-point finalisation (k_near.cu)
int launch_near_grad(bem_mesh* m, const double* pts, const int* perm, const double* sigma, double4* gval,
                     unsigned long long gcap, cudaStream_t s, const double* slope = nullptr);
int launch_finalize_grad(bem_mesh* m, const int* perm, int n_pts, const double4* far_g, const double4* gval,
                         unsigned long long gcap, double* G, cudaStream_t s);
// kc x potential of each element at its own centroid (sigma = 1): the diagonal of the
// collocation matrix at the centroids (k_near.cu)
int launch_self_potential(bem_mesh* m, double* out, cudaStream_t s);
int launch_near_assemble(bem_mesh* m, const double* pts, const int* perm, double* A, unsigned long long n_near,
                         cudaStream_t s);

}  // namespace bem
