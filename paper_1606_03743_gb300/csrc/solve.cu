// solve.cu -- bem_solve: the charge densities of the BEM collocation system
// A sigma = rhs at the element centroids (Sec. 1: the linear system for the
// charge densities; Sec. 5: matrices kept unstored, solved iteratively).
//
// Restarted GMRES with a Jacobi right preconditioner D = diag(A) (the self
// potentials of the elements): A D^-1 z = rhs, sigma = D^-1 z.  Every
// product is a bem_matvec; the Krylov basis lives on the device and the
// Gram-Schmidt steps (classical, applied twice), norms and updates are the
// kernels below, with fixed-order reductions so that a solve is bit-for-bit
// repeatable.  Only the small Hessenberg least-squares problem (at most
// restart x restart, Givens rotations) runs on the host, fed by one
// device-to-host copy of the new column per step.
#include <math.h>
#include <string.h>

#include <vector>

#include "bem_internal.cuh"

namespace bem {
namespace {

constexpr int kThreads = 256;
constexpr int kDotBlocks = 128;  // fixed, so that the summation order does not depend on the GPU
constexpr int kMaxRestart = 200;

// partial[j * kDotBlocks + b]: block b's share of sum_i V[j][i] w[i]
__global__ void k_dot_partial(int n, const double* __restrict__ V, size_t ldv, const double* __restrict__ w,
                              double* __restrict__ partial) {
    const double* v = V + (size_t)blockIdx.y * ldv;
    double acc = 0.0;
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += kDotBlocks * kThreads) acc = fma(v[i], w[i], acc);
    __shared__ double sh[kThreads];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[(size_t)blockIdx.y * kDotBlocks + blockIdx.x] = sh[0];
}

// out[j] = sum of vector j's kDotBlocks partials, in a fixed order
__global__ void k_dot_final(const double* __restrict__ partial, double* __restrict__ out) {
    __shared__ double sh[kDotBlocks];
    sh[threadIdx.x] = partial[(size_t)blockIdx.x * kDotBlocks + threadIdx.x];
    __syncthreads();
    for (int s = kDotBlocks / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

// w -= sum_{j < k} h[j] V[j]
__global__ void k_orth(int n, int k, const double* __restrict__ V, size_t ldv, const double* __restrict__ h,
                       double* __restrict__ w) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        double s = w[i];
        for (int j = 0; j < k; ++j) s = fma(-h[j], V[(size_t)j * ldv + i], s);
        w[i] = s;
    }
}

// out = a * in
__global__ void k_scale(int n, double a, const double* __restrict__ in, double* __restrict__ out) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) out[i] = a * in[i];
}

// out = in / d
__global__ void k_div(int n, const double* __restrict__ in, const double* __restrict__ d, double* __restrict__ out) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) out[i] = in[i] / d[i];
}

// r = b - r (r holds A x on entry)
__global__ void k_resid(int n, const double* __restrict__ b, double* __restrict__ r) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) r[i] = b[i] - r[i];
}

// x += d
__global__ void k_add(int n, const double* __restrict__ d, double* __restrict__ x) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) x[i] += d[i];
}

// x += D^-1 sum_{j < k} y[j] V[j]
__global__ void k_update(int n, int k, const double* __restrict__ V, size_t ldv, const double* __restrict__ y,
                         const double* __restrict__ d, double* __restrict__ x) {
    for (int i = blockIdx.x * kThreads + threadIdx.x; i < n; i += gridDim.x * kThreads) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s = fma(y[j], V[(size_t)j * ldv + i], s);
        x[i] += s / d[i];
    }
}

int grid_for(int n) {
    const int g = (n + kThreads - 1) / kThreads;
    return g < 1 ? 1 : (g > 4096 ? 4096 : g);
}

// Device buffers of one solve, released on every return path.
struct Buffers {
    std::vector<void*> ptrs;
    ~Buffers() {
        for (void* p : ptrs) cudaFree(p);
    }
    int get(double** p, size_t count) {
        const cudaError_t e = dev_malloc((void**)p, (count > 0 ? count : 1) * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            set_error("bem_solve: cudaMalloc of %zu bytes failed: %s", count * sizeof(double), cudaGetErrorString(e));
            return BEM_ERR_OOM;
        }
        ptrs.push_back(*p);
        return BEM_OK;
    }
};

// rhs and sigma are only copied (never read by a kernel), so any array the
// runtime can copy is accepted: host memory or any GPU's memory
bool on_device(const void* p, int dev) { return ptr_location(p, dev) != kPtrHost; }

struct Ctx {
    bem_mesh* m;
    cudaStream_t s;
    int n;
    double* partial;
};

// out[0 .. k-1] = V[0 .. k-1] . w  (device results)
int dots(const Ctx& c, const double* V, size_t ldv, int k, const double* w, double* out) {
    k_dot_partial<<<dim3(kDotBlocks, k), kThreads, 0, c.s>>>(c.n, V, ldv, w, c.partial);
    k_dot_final<<<k, kDotBlocks, 0, c.s>>>(c.partial, out);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(2);
    return BEM_OK;
}

// Workspace and state of one solve.
struct Solver {
    bem_mesh* m;
    cudaStream_t s;
    int n, restart, g;
    size_t ldv;
    double *V, *diag, *t, *partial, *hdev, *ydev, *r, *d;
    std::vector<double> H, cs, sn, gv, y, col;
    Ctx c() const { return Ctx{m, s, n, partial}; }
    double* vec(int j) const { return V + (size_t)j * ldv; }

    int host_dot(const double* a, const double* b, double* out) {
        int rc = dots(c(), a, ldv, 1, b, hdev);
        if (rc) return rc;
        BEM_CUDA_TRY(cudaMemcpyAsync(out, hdev, sizeof(double), cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(cudaStreamSynchronize(s));
        return BEM_OK;
    }

    // out = b - A x (one product); *rel2 = |out|^2
    int residual(const double* b, const double* x, double* out, double* norm2) {
        int rc = bem_matvec(m, x, out, s);
        if (rc) return rc;
        k_resid<<<g, kThreads, 0, s>>>(n, b, out);
        BEM_CUDA_TRY(cudaGetLastError());
        count_launches(1);
        return host_dot(out, out, norm2);
    }

    // Restarted GMRES for A x = b from the x given, until |b - A x| <= tol * bnorm
    // or `budget` products are spent; *products counts them, *rel is the last
    // relative residual |b - A x| / bnorm that was computed (a true residual).
    // x_zero: x is known to be zero, so the first residual is b itself (no product).
    int gmres(const double* b, double* x, double bnorm, double tol, long budget, long* products, double* rel,
              bool* converged, bool x_zero = false) {
        *converged = false;
        const long start = *products;
        auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * restart + j]; };
        int rc;
        for (;;) {
            double beta2 = 0.0;
            if (x_zero) {
                BEM_CUDA_TRY(cudaMemcpyAsync(vec(0), b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
                beta2 = bnorm * bnorm;
                x_zero = false;
            } else {
                if ((rc = residual(b, x, vec(0), &beta2))) return rc;
                ++*products;
            }
            const double beta = sqrt(beta2);
            *rel = beta / bnorm;
            if (*rel <= tol) {
                *converged = true;
                return BEM_OK;
            }
            if (*products - start >= budget) return BEM_OK;
            k_scale<<<g, kThreads, 0, s>>>(n, 1.0 / beta, vec(0), vec(0));
            BEM_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            std::fill(H.begin(), H.end(), 0.0);
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            int k = 0;  // basis vectors used in this cycle's update
            for (int j = 0; j < restart && *products - start < budget; ++j) {
                // w = A D^-1 v_j into slot j + 1
                k_div<<<g, kThreads, 0, s>>>(n, vec(j), diag, t);
                BEM_CUDA_TRY(cudaGetLastError());
                count_launches(1);
                if ((rc = bem_matvec(m, t, vec(j + 1), s))) return rc;
                ++*products;
                // classical Gram-Schmidt against v_0 .. v_j, twice
                if ((rc = dots(c(), V, ldv, j + 1, vec(j + 1), hdev))) return rc;
                k_orth<<<g, kThreads, 0, s>>>(n, j + 1, V, ldv, hdev, vec(j + 1));
                if ((rc = dots(c(), V, ldv, j + 1, vec(j + 1), hdev + (j + 1)))) return rc;
                k_orth<<<g, kThreads, 0, s>>>(n, j + 1, V, ldv, hdev + (j + 1), vec(j + 1));
                BEM_CUDA_TRY(cudaGetLastError());
                count_launches(2);
                if ((rc = dots(c(), vec(j + 1), ldv, 1, vec(j + 1), hdev + 2 * (j + 1)))) return rc;
                BEM_CUDA_TRY(cudaMemcpyAsync(col.data(), hdev, sizeof(double) * (2 * (j + 1) + 1),
                                             cudaMemcpyDeviceToHost, s));
                BEM_CUDA_TRY(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i) Hat(i, j) = col[i] + col[j + 1 + i];
                const double hnext = sqrt(col[2 * (j + 1)]);
                Hat(j + 1, j) = hnext;
                if (hnext > 0.0) {
                    k_scale<<<g, kThreads, 0, s>>>(n, 1.0 / hnext, vec(j + 1), vec(j + 1));
                    BEM_CUDA_TRY(cudaGetLastError());
                    count_launches(1);
                }
                // Givens rotations: earlier ones on the new column, then a new one
                for (int i = 0; i < j; ++i) {
                    const double a = Hat(i, j), bb = Hat(i + 1, j);
                    Hat(i, j) = cs[i] * a + sn[i] * bb;
                    Hat(i + 1, j) = -sn[i] * a + cs[i] * bb;
                }
                const double a = Hat(j, j), bb = Hat(j + 1, j);
                const double rr = hypot(a, bb);
                cs[j] = rr > 0.0 ? a / rr : 1.0;
                sn[j] = rr > 0.0 ? bb / rr : 0.0;
                Hat(j, j) = rr;
                Hat(j + 1, j) = 0.0;
                gv[j + 1] = -sn[j] * gv[j];
                gv[j] = cs[j] * gv[j];
                k = j + 1;
                if (fabs(gv[j + 1]) <= tol * bnorm || hnext == 0.0) break;
            }
            // y = R^-1 g (upper triangular), x += D^-1 V y
            for (int i = k - 1; i >= 0; --i) {
                double acc = gv[i];
                for (int l = i + 1; l < k; ++l) acc -= Hat(i, l) * y[l];
                y[i] = Hat(i, i) != 0.0 ? acc / Hat(i, i) : 0.0;
            }
            BEM_CUDA_TRY(cudaMemcpyAsync(ydev, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
            k_update<<<g, kThreads, 0, s>>>(n, k, V, ldv, ydev, diag, x);
            BEM_CUDA_TRY(cudaGetLastError());
            count_launches(1);
            if (*products - start >= budget) {  // the residual of the final iterate (one more product)
                double r2 = 0.0;
                if ((rc = residual(b, x, vec(0), &r2))) return rc;
                ++*products;
                *rel = sqrt(r2) / bnorm;
                *converged = *rel <= tol;
                return BEM_OK;
            }
        }
    }
};

// The mesh's precision for the products inside one scope.
struct PrecisionScope {
    bem_mesh* m;
    int saved;
    PrecisionScope(bem_mesh* mm, int p) : m(mm), saved(mm->precision) { m->precision = p; }
    ~PrecisionScope() { m->precision = saved; }
};

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" int bem_solve(bem_mesh* m, const double* rhs, double* sigma, const bem_solve_options* opt, double* info,
                         void* stream) {
    NvtxRange range("bem_solve");
    if (info) info[0] = info[1] = info[2] = 0.0;
    if (!m) {
        set_error("bem_solve: mesh is NULL");
        return BEM_ERR_INVALID;
    }
    const int n = m->d.n;
    if (n == 0) {
        if (info) info[2] = 1.0;
        return BEM_OK;
    }
    if (!rhs || !sigma) {
        set_error("bem_solve: rhs or sigma is NULL");
        return BEM_ERR_INVALID;
    }
    int restart = 50, max_iter = 1000, flags = 0;
    double tol = m->precision == kFP64 ? 1e-12 : 1e-6;
    if (opt) {
        if (opt->restart) restart = opt->restart;
        if (opt->max_iter) max_iter = opt->max_iter;
        if (opt->tol != 0.0) tol = opt->tol;
        flags = opt->flags;
    }
    if (restart < 1 || restart > kMaxRestart || max_iter < 1 || !(tol > 0.0) || !isfinite(tol)) {
        set_error("bem_solve: bad options (restart %d, max_iter %d, tol %g)", restart, max_iter, tol);
        return BEM_ERR_INVALID;
    }
    const bool refine = (flags & BEM_SOLVE_REFINE) && m->precision == kFP64;
    cudaStream_t s = (cudaStream_t)stream;
    BEM_CUDA_TRY(cudaSetDevice(m->device));

    const size_t ldv = ((size_t)n + 31) / 32 * 32;  // basis vectors start on 256-byte boundaries
    const size_t need = sizeof(double) * (ldv * (restart + 1) + 6 * (size_t)n + (size_t)kDotBlocks * (restart + 1) +
                                          3 * (size_t)(restart + 2));
    if (m->w.bytes + need > m->budget) {
        set_error("bem_solve: needs %zu bytes of device memory beyond the %zu in use (budget %zu)", need, m->w.bytes,
                  m->budget);
        return BEM_ERR_OOM;
    }
    Buffers buf;
    Solver sv;
    double *x, *b;
    int rc;
    if ((rc = buf.get(&sv.V, ldv * (restart + 1))) || (rc = buf.get(&sv.diag, n)) || (rc = buf.get(&x, n)) ||
        (rc = buf.get(&b, n)) || (rc = buf.get(&sv.t, n)) || (rc = buf.get(&sv.r, n)) || (rc = buf.get(&sv.d, n)) ||
        (rc = buf.get(&sv.partial, (size_t)kDotBlocks * (restart + 1))) ||
        (rc = buf.get(&sv.hdev, 2 * (size_t)(restart + 2))) || (rc = buf.get(&sv.ydev, restart + 1)))
        return rc;
    sv.m = m;
    sv.s = s;
    sv.n = n;
    sv.restart = restart;
    sv.g = grid_for(n);
    sv.ldv = ldv;
    sv.H.assign((size_t)(restart + 1) * restart, 0.0);
    sv.cs.assign(restart, 0.0);
    sv.sn.assign(restart, 0.0);
    sv.gv.assign(restart + 1, 0.0);
    sv.y.assign(restart, 0.0);
    sv.col.assign(2 * (restart + 2), 0.0);

    const bool rhs_dev = on_device(rhs, m->device), sig_dev = on_device(sigma, m->device);
    BEM_CUDA_TRY(cudaMemcpyAsync(b, rhs, sizeof(double) * n, rhs_dev ? cudaMemcpyDefault : cudaMemcpyHostToDevice, s));
    if (flags & BEM_SOLVE_X0)
        BEM_CUDA_TRY(cudaMemcpyAsync(x, sigma, sizeof(double) * n,
                                     sig_dev ? cudaMemcpyDefault : cudaMemcpyHostToDevice, s));
    else
        BEM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    if ((rc = launch_self_potential(m, sv.diag, s))) return rc;

    double bnorm2 = 0.0;
    if ((rc = sv.host_dot(b, b, &bnorm2))) return rc;
    const double bnorm = sqrt(bnorm2);
    long products = 0;
    double rel = 0.0;
    bool converged = false;
    if (bnorm == 0.0) {  // zero potentials: zero charge
        BEM_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
        converged = true;
    } else if (!refine) {
        if ((rc = sv.gmres(b, x, bnorm, tol, max_iter, &products, &rel, &converged))) return rc;
    } else {
        // Iterative refinement: FP64 residuals r = b - A x, corrections from
        // GMRES on the mixed-precision products (A d = r to 1e-6), x += d.
        // Each step gains about the mixed solve's six digits, at a fraction
        // of the FP64 products' cost.
        constexpr double kInnerTol = 1e-6;
        for (;;) {
            double r2 = 0.0;
            if ((rc = sv.residual(b, x, sv.r, &r2))) return rc;
            ++products;
            rel = sqrt(r2) / bnorm;
            if (rel <= tol) {
                converged = true;
                break;
            }
            if (products >= max_iter) break;
            BEM_CUDA_TRY(cudaMemsetAsync(sv.d, 0, sizeof(double) * n, s));
            long inner = 0;
            double irel = 0.0;
            bool iconv = false;
            {
                PrecisionScope mixed(m, kMixed);
                if ((rc = sv.gmres(sv.r, sv.d, sqrt(r2), kInnerTol, max_iter - products, &inner, &irel, &iconv,
                                   true)))
                    return rc;
            }
            products += inner;
            k_add<<<sv.g, kThreads, 0, s>>>(n, sv.d, x);
            BEM_CUDA_TRY(cudaGetLastError());
            count_launches(1);
        }
    }
    BEM_CUDA_TRY(cudaMemcpyAsync(sigma, x, sizeof(double) * n, sig_dev ? cudaMemcpyDefault : cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    if (info) {
        info[0] = (double)products;
        info[1] = rel;
        info[2] = converged ? 1.0 : 0.0;
    }
    if (!converged) {
        set_error("bem_solve: relative residual %.3e above tol %.3e after %ld products", rel, tol, products);
        return BEM_ERR_NOT_CONVERGED;
    }
    return BEM_OK;
}
