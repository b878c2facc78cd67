// peaks.cu -- throughput of the arithmetic pipes that bound the far-field
// kernel: scalar FFMA, packed FFMA2, the MUFU reciprocal square root and
// DFMA.  The far-field cubature (Eq. 4.1) is bound by FP32 fused
// multiply-adds and one rsqrt per node (mixed path) or by FP64 arithmetic
// (FP64 path); these kernels measure what those pipes deliver on this GPU,
// so that the kernel's roofline fraction has a measured denominator.
//
// Each thread runs kChains independent dependency chains of one
// instruction kind (enough independent work to cover the pipe latency with
// a full SM), unrolled, for `iters` iterations.  The grid fills every SM
// with 2048 resident threads.  Block 0 also records clock64() and
// %globaltimer around its loop: their ratio is the SM clock during the run.
#include <math.h>

#include "bem_internal.cuh"

namespace bem {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 512;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// out: per-block sink (keeps the chains live); clk: block 0's (cycles, ns)
template <int KIND>
__global__ void __launch_bounds__(kThreads, 2048 / kThreads) k_peak(int iters, float seed, float* out, unsigned long long* clk) {
    unsigned long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        t0 = global_ns();
        c0 = clock64();
    }
    const float s = seed + 1e-7f * (float)(threadIdx.x & 31);
    float res = 0.0f;
    if constexpr (KIND == BEM_PEAK_FFMA) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = s + (float)k;
        const float b = 0.9999999f, c = 1e-7f;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) res += a[k];
    } else if constexpr (KIND == BEM_PEAK_FFMA2) {
        float2 a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = make_float2(s + (float)k, s - (float)k);
        const float2 b = make_float2(0.9999999f, 0.9999998f), c = make_float2(1e-7f, 2e-7f);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) res += a[k].x + a[k].y;
    } else if constexpr (KIND == BEM_PEAK_RSQRT) {
        // x <- rsqrt(x) converges to 1 and stays finite; this file is built
        // with denormals flushed, so rsqrtf is the bare MUFU instruction
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = s + 0.5f * (float)k;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = rsqrtf(a[k]);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) res += a[k];
    } else {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = (double)s + (double)k;
        const double b = 0.99999999999, c = 1e-11;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) res += (float)a[k];
    }
    if (res == 12345.678f) out[blockIdx.x] = res;  // practically never taken; keeps the chains
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long c1 = clock64(), t1 = global_ns();
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
}

template <int KIND>
int run_peak(int iters, int grid, float* sink, unsigned long long* clk, cudaStream_t s) {
    k_peak<KIND><<<grid, kThreads, 0, s>>>(iters, 1.0f, sink, clk);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

int launch_peak(int kind, int iters, int grid, float* sink, unsigned long long* clk, cudaStream_t s) {
    switch (kind) {
        case BEM_PEAK_FFMA: return run_peak<BEM_PEAK_FFMA>(iters, grid, sink, clk, s);
        case BEM_PEAK_FFMA2: return run_peak<BEM_PEAK_FFMA2>(iters, grid, sink, clk, s);
        case BEM_PEAK_RSQRT: return run_peak<BEM_PEAK_RSQRT>(iters, grid, sink, clk, s);
        default: return run_peak<BEM_PEAK_DFMA>(iters, grid, sink, clk, s);
    }
}

// lane operations of one kernel instruction of each kind (an FMA counts once)
double lane_ops_per_inst(int kind) { return kind == BEM_PEAK_FFMA2 ? 2.0 : 1.0; }

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" int bem_peak_rate(int32_t kind, double* out) {
    if (kind < BEM_PEAK_FFMA || kind > BEM_PEAK_DFMA || !out) {
        set_error("bem_peak_rate: unknown kind %d or out is NULL", (int)kind);
        return BEM_ERR_INVALID;
    }
    int dev = 0, sms = 0;
    BEM_CUDA_TRY(cudaGetDevice(&dev));
    BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * (2048 / kThreads);
    float* sink = nullptr;
    unsigned long long* clk = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t s = nullptr;
    int rc = BEM_OK;
    cudaError_t ce = dev_malloc((void**)&sink, sizeof(float) * grid);
    if (ce == cudaSuccess) ce = dev_malloc((void**)&clk, 2 * sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "bem_peak_rate setup");
    // a short run to load the kernel and size the real one (about 50 ms)
    int iters = 64;
    float ms = 0.0f;
    for (int pass = 0; !rc && pass < 2; ++pass) {
        if ((rc = launch_peak(kind, iters, grid, sink, clk, s))) break;  // warm-up of this size
        float best = 1e30f;
        for (int rep = 0; rep < 3 && !rc; ++rep) {
            ce = cudaEventRecord(e0, s);
            if (ce == cudaSuccess && (rc = launch_peak(kind, iters, grid, sink, clk, s))) break;
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
            if (ce != cudaSuccess) {
                rc = cuda_fail(ce, "bem_peak_rate timing");
                break;
            }
            best = fminf(best, t);
        }
        ms = best;
        if (pass == 0) {
            const double scale = 50.0 / fmax((double)ms, 1e-3);
            iters = (int)fmin(fmax(iters * scale, 64.0), 1 << 22);
        }
    }
    unsigned long long hclk[2] = {0, 0};
    if (!rc) {
        ce = cudaMemcpy(hclk, clk, sizeof hclk, cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) rc = cuda_fail(ce, "bem_peak_rate readback");
    }
    if (!rc) {
        const double inst = (double)grid * kThreads * (double)iters * kUnroll * kChains;
        out[0] = inst * lane_ops_per_inst(kind) / (ms * 1e-3);
        out[1] = ms;
        out[2] = hclk[1] ? 1e3 * (double)hclk[0] / (double)hclk[1] : 0.0;  // cycles per ns x 1000 = MHz
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    cudaFree(clk);
    return rc;
}
