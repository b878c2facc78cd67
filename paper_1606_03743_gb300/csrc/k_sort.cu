// k_sort.cu -- spatial ordering of field points and an exclusive scan.
//
// Field points are ordered by a Morton (Z-order) cell key over their bounding
// box (about one point per cell) so that the 32 * PT points of a warp are
// neighbours: the far-field
// kernel then usually finds every point of a warp in the same distance-ratio
// band of an element and runs one rule for the whole warp.  The order within
// a cell is whatever the atomics give; results do not depend on it because
// every point's arithmetic depends only on the point itself.
#include "bem_internal.cuh"

namespace bem {

namespace {

// order-preserving map of floats onto unsigned ints (for atomicMin / atomicMax)
__device__ __forceinline__ unsigned f2ord(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_bbox_init(unsigned* bb) {
    if (threadIdx.x < 3) bb[threadIdx.x] = 0xffffffffu;      // min
    else if (threadIdx.x < 6) bb[threadIdx.x] = 0u;          // max
}

__global__ void k_bbox(const double* __restrict__ pts, int n, const int* n_dev, unsigned* bb,
                       unsigned long long* bad) {
    if (n_dev) n = min(n, *n_dev);
    float mn[3] = {3.0e38f, 3.0e38f, 3.0e38f}, mx[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    bool finite = true;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double x = pts[3 * (size_t)i + k];
            finite = finite && isfinite(x) && fabs(x) < 1e30;
            const float v = (float)x;
            mn[k] = fminf(mn[k], v);
            mx[k] = fmaxf(mx[k], v);
        }
    }
    if (!finite) atomicOr(bad, 1ull);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o; o >>= 1) {
            mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
            mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(bb + k, f2ord(mn[k]));
            atomicMax(bb + 3 + k, f2ord(mx[k]));
        }
    }
}

__device__ __forceinline__ unsigned spread3(unsigned x) {  // 10 bits -> every third bit
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

// 1: cells are visited along a Hilbert curve (no jumps between distant
// octants, so runs of consecutive points -- the far-field kernel's tiles --
// are more compact than on the Z-order curve: on the coaxial 1 000 000-point
// workload 11.6 % instead of 13.0 % of (tile, element) pairs straddle a band
// limit); 0: Z order
#ifndef BEM_HILBERT
#define BEM_HILBERT 1
#endif

// Position of cell (x, y, z) (bits per axis) on the 3-D Hilbert curve:
// Skilling's transform of the axes into the curve's transposed index
// (J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004),
// then the transposed bits interleaved, most significant first.
__device__ __forceinline__ unsigned hilbert3(unsigned x, unsigned y, unsigned z, int bits) {
    unsigned X[3] = {x, y, z};
    const unsigned M = 1u << (bits - 1);
    for (unsigned Q = M; Q > 1; Q >>= 1) {  // undo the excess work of the inverse transform
        const unsigned P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;  // invert the low bits of the first axis
            } else {
                const unsigned t = (X[0] ^ X[i]) & P;  // exchange the low bits with the first axis
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];  // Gray encode
    X[2] ^= X[1];
    unsigned t = 0;
    for (unsigned Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    unsigned h = 0;
    for (int b = bits - 1; b >= 0; --b) h = (h << 3) | (((X[0] >> b) & 1u) << 2) | (((X[1] >> b) & 1u) << 1) | ((X[2] >> b) & 1u);
    return h;
}

__global__ void k_keys(const double* __restrict__ pts, int n, const int* n_dev, const unsigned* bb, int bits,
                       unsigned* key, int* cell_cnt) {
    if (n_dev) n = min(n, *n_dev);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float lim = (float)((1 << bits) - 1);
    unsigned c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = ord2f(bb[k]), hi = ord2f(bb[3 + k]);
        const float ext = hi - lo;
        const float t = ext > 0.0f ? ((float)pts[3 * (size_t)i + k] - lo) / ext * (lim + 1.0f) : 0.0f;
        c[k] = (unsigned)fminf(fmaxf(t, 0.0f), lim);
    }
    const unsigned kk = BEM_HILBERT ? hilbert3(c[0], c[1], c[2], bits)
                                    : (spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2));
    key[i] = kk;
    atomicAdd(cell_cnt + kk, 1);
}

__global__ void k_scatter(const unsigned* __restrict__ key, int n, const int* n_dev, int* cursor, int* perm) {
    if (n_dev) n = min(n, *n_dev);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int pos = atomicAdd(cursor + key[i], 1);
    perm[pos] = i;
}

// ---------------------------------------------------------------- scan
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

// Exclusive scan of one tile per block; the tile total goes to sums[block].
__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const int* __restrict__ in, int* __restrict__ out, int n,
                                                            int* __restrict__ sums) {
    __shared__ int s_warp[32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems], tot = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        tot += v[k];
    }
    // inclusive scan of the per-thread totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int run = x - tot + (warp ? s_warp[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = run;
}

__global__ void k_scan_add(int* __restrict__ out, int n, const int* __restrict__ offs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += offs[i / kScanTile];
}


}  // namespace

size_t scan_tmp_ints(int n) {
    size_t tot = 0;
    while (n > 1) {
        const int nb = (n + kScanTile - 1) / kScanTile;
        tot += 2 * (size_t)nb + 1;
        n = nb;
    }
    return tot + 2;
}

int launch_exclusive_scan(const int* in, int* out, int n, int* tmp, cudaStream_t s) {
    if (n <= 0) return BEM_OK;
    const int nb = (n + kScanTile - 1) / kScanTile;
    int* sums = tmp;
    int* sums_scanned = tmp + nb;
    k_scan_tile<<<nb, kScanThreads, 0, s>>>(in, out, n, sums);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    if (nb > 1) {
        int rc = launch_exclusive_scan(sums, sums_scanned, nb, tmp + 2 * nb + 1, s);
        if (rc) return rc;
        k_scan_add<<<(n + 255) / 256, 256, 0, s>>>(out, n, sums_scanned);
        BEM_CUDA_TRY(cudaGetLastError());
        count_launches(1);
    }
    return BEM_OK;
}

// Sort the first n points of pts into m->w.perm (cell order).  Non-finite
// (or absurdly large) coordinates set counters[15].  With n_dev the actual
// count is read on the device (n is then the capacity; the launch sequence
// can be captured once in a CUDA graph).
int launch_sort_points(bem_mesh* m, const double* pts, int n, cudaStream_t s, const int* n_dev) {
    Work& w = m->w;
    BEM_CUDA_TRY(cudaMemsetAsync(w.counters + 15, 0, sizeof(unsigned long long), s));
    const int bits = sort_cell_bits((size_t)n);
    const int ncell = 1 << (3 * bits);
    unsigned* bb = reinterpret_cast<unsigned*>(w.bbox);
    k_bbox_init<<<1, 32, 0, s>>>(bb);
    BEM_CUDA_TRY(cudaGetLastError());
    const int grid = min((n + 255) / 256, 152 * 4);
    k_bbox<<<grid, 256, 0, s>>>(pts, n, n_dev, bb, w.counters + 15);
    BEM_CUDA_TRY(cudaGetLastError());
    BEM_CUDA_TRY(cudaMemsetAsync(w.cell_cnt, 0, sizeof(int) * ncell, s));
    k_keys<<<(n + 255) / 256, 256, 0, s>>>(pts, n, n_dev, bb, bits, w.key, w.cell_cnt);
    BEM_CUDA_TRY(cudaGetLastError());
    int rc = launch_exclusive_scan(w.cell_cnt, w.cell_off, ncell, w.scan_tmp, s);
    if (rc) return rc;
    k_scatter<<<(n + 255) / 256, 256, 0, s>>>(w.key, n, n_dev, w.cell_off, w.perm);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(4);  // bbox_init, bbox, keys, scatter
    return BEM_OK;
}

}  // namespace bem
