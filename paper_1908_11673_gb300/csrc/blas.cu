// Vector kernels of the solvers: axpy-type updates, precision conversions and
// deterministic reductions (block partial sums, then one block sums the
// partials in a fixed order; every sum is accumulated in FP64).
//
// A field is handled here as a flat array of n complex numbers: the
// structure-of-arrays chunks of the internal layout store (re, im) pairs
// contiguously in every precision (double2, two float2 per float4, two
// bfloat16 per 32-bit word).
#include "qxd_internal.h"
#include "blas.h"

namespace qxd {

template <int P> struct Elem;
template <> struct Elem<0> {
    using R = double;
    static QXD_HD cplx<double> ld(const void* p, size_t i) {
        double2 v = QXD_LDG(static_cast<const double2*>(p) + i);
        return {v.x, v.y};
    }
    static QXD_HD void st(void* p, size_t i, cplx<double> v) { static_cast<double2*>(p)[i] = make_double2(v.re, v.im); }
};
template <> struct Elem<1> {
    using R = float;
    static QXD_HD cplx<float> ld(const void* p, size_t i) {
        float2 v = QXD_LDG(static_cast<const float2*>(p) + i);
        return {v.x, v.y};
    }
    static QXD_HD void st(void* p, size_t i, cplx<float> v) { static_cast<float2*>(p)[i] = make_float2(v.re, v.im); }
};
template <> struct Elem<2> {
    using R = float;
    static QXD_HD cplx<float> ld(const void* p, size_t i) {
        uint32_t v = QXD_LDG(static_cast<const uint32_t*>(p) + i);
        return {bf16_lo(v), bf16_hi(v)};
    }
    static QXD_HD void st(void* p, size_t i, cplx<float> v) { static_cast<uint32_t*>(p)[i] = pack_bf16x2(v.re, v.im); }
};

constexpr int kRedThreads = 256;
constexpr int kMaxRedBlocks = 1024;

static int red_blocks(size_t n) {
    size_t b = (n + kRedThreads - 1) / kRedThreads;
    return (int)(b < (size_t)kMaxRedBlocks ? (b > 0 ? b : 1) : kMaxRedBlocks);
}

// sum of NC doubles over the block, written to partials[c * gridDim.x + blockIdx.x]
template <int NC>
__device__ void block_reduce_store(double v[NC], double* __restrict__ partials) {
    __shared__ double sh[NC][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        double x = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[c][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            double x = lane < kRedThreads / 32 ? sh[c][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) partials[(size_t)c * gridDim.x + blockIdx.x] = x;
        }
    }
}

// one block: result[c] = sum_b partials[c * nb + b], fixed order
__global__ void k_final(const double* __restrict__ partials, int nb, int ncomp, double* __restrict__ result) {
    __shared__ double sh[kRedThreads / 32];
    for (int c = 0; c < ncomp; ++c) {
        double x = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) x += partials[(size_t)c * nb + b];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) sh[warp] = x;
        __syncthreads();
        if (warp == 0) {
            x = lane < kRedThreads / 32 ? sh[lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) result[c] = x;
        }
        __syncthreads();
    }
}

static double eb(int P) { return P == 0 ? 16.0 : (P == 1 ? 8.0 : 4.0); }

static int finish(qxd_ctx* ctx, int nb, int ncomp, int slot, cudaStream_t st) {
    QXD_CUDA(ctx, cudaGetLastError());
    ProfScope prof(ctx, "reduce_final", 8.0 * nb * ncomp, st);
    k_final<<<1, kRedThreads, 0, st>>>(ctx->red_partials, nb, ncomp, ctx->red_result + slot);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// ---- reductions ---------------------------------------------------------------
template <int PA, int PB>
__global__ void __launch_bounds__(kRedThreads) k_dot(size_t n, const void* __restrict__ a, const void* __restrict__ b,
                                                     double* __restrict__ partials) {
    double v[2] = {0.0, 0.0};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        auto x = Elem<PA>::ld(a, i);
        auto y = Elem<PB>::ld(b, i);
        const double xr = x.re, xi = x.im, yr = y.re, yi = y.im;
        v[0] += xr * yr + xi * yi;
        v[1] += xr * yi - xi * yr;
    }
    block_reduce_store<2>(v, partials);
}

template <int P>
__global__ void __launch_bounds__(kRedThreads) k_norm2(size_t n, const void* __restrict__ a,
                                                       double* __restrict__ partials) {
    double v[2] = {0.0, 0.0};  // |a|^2 and a count of non-finite entries
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        auto x = Elem<P>::ld(a, i);
        const double xr = x.re, xi = x.im;
        const double s = xr * xr + xi * xi;
        if (isfinite(s)) v[0] += s;
        else v[1] += 1.0;
    }
    block_reduce_store<2>(v, partials);
}

// k dot products <W_j, v>, j < k (k <= kMultiMax)
template <int P, int K>
__global__ void __launch_bounds__(kRedThreads) k_multi_dot(size_t n, MultiPtr W, const void* __restrict__ v,
                                                           double* __restrict__ partials) {
    double acc[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) acc[c] = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        auto y = Elem<P>::ld(v, i);
        const double yr = y.re, yi = y.im;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            auto x = Elem<P>::ld(W.p[j], i);
            const double xr = x.re, xi = x.im;
            acc[2 * j] += xr * yr + xi * yi;
            acc[2 * j + 1] += xr * yi - xi * yr;
        }
    }
    block_reduce_store<2 * K>(acc, partials);
}

int blas_dot(qxd_ctx* ctx, int pa, int pb, size_t n, const void* a, const void* b, int slot, cudaStream_t st) {
    const int nb = red_blocks(n);
    {
    ProfScope prof(ctx, "dot", (double)n * (eb(pa) + eb(pb)), st);
#define QXD_DOT(A, B) k_dot<A, B><<<nb, kRedThreads, 0, st>>>(n, a, b, ctx->red_partials)
    // the flat complex order is the same only within one precision
    if (pa == 0 && pb == 0) QXD_DOT(0, 0);
    else if (pa == 1 && pb == 1) QXD_DOT(1, 1);
    else if (pa == 2 && pb == 2) QXD_DOT(2, 2);
    else return qxd_fail(ctx, QXD_EARG, "blas_dot: precisions must match");
#undef QXD_DOT
    }
    return finish(ctx, nb, 2, slot, st);
}

int blas_norm2(qxd_ctx* ctx, int p, size_t n, const void* a, int slot, cudaStream_t st) {
    const int nb = red_blocks(n);
    ProfScope prof(ctx, "norm2", (double)n * eb(p), st);
    if (p == 0) k_norm2<0><<<nb, kRedThreads, 0, st>>>(n, a, ctx->red_partials);
    else if (p == 1) k_norm2<1><<<nb, kRedThreads, 0, st>>>(n, a, ctx->red_partials);
    else k_norm2<2><<<nb, kRedThreads, 0, st>>>(n, a, ctx->red_partials);
    return finish(ctx, nb, 2, slot, st);
}

template <int P>
static void multi_dot_k(int k, int nb, size_t n, const MultiPtr& W, const void* v, double* partials, cudaStream_t st) {
    switch (k) {
        case 1: k_multi_dot<P, 1><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        case 2: k_multi_dot<P, 2><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        case 3: k_multi_dot<P, 3><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        case 4: k_multi_dot<P, 4><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        case 5: k_multi_dot<P, 5><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        case 6: k_multi_dot<P, 6><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        case 7: k_multi_dot<P, 7><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
        default: k_multi_dot<P, 8><<<nb, kRedThreads, 0, st>>>(n, W, v, partials); break;
    }
}

int blas_multi_dot(qxd_ctx* ctx, int p, size_t n, int k, const void* const* W, const void* v, int slot,
                   cudaStream_t st) {
    for (int j0 = 0; j0 < k; j0 += kMultiMax) {
        const int kk = (k - j0) < kMultiMax ? (k - j0) : kMultiMax;
        MultiPtr mp;
        for (int j = 0; j < kMultiMax; ++j) mp.p[j] = W[j0 + (j < kk ? j : 0)];
        const int nb = red_blocks(n);
        {
        ProfScope prof(ctx, "multi_dot", (double)n * eb(p) * (kk + 1), st);
        if (p == 0) multi_dot_k<0>(kk, nb, n, mp, v, ctx->red_partials, st);
        else if (p == 1) multi_dot_k<1>(kk, nb, n, mp, v, ctx->red_partials, st);
        else multi_dot_k<2>(kk, nb, n, mp, v, ctx->red_partials, st);
        }
        QXD_TRY(finish(ctx, nb, 2 * kk, slot + 2 * j0, st));
    }
    return QXD_OK;
}

// ---- updates -------------------------------------------------------------------
// y = a*x + b*y  (x may be a different precision than y)
template <int PX, int PY>
__global__ void k_axpby(size_t n, double ar, double ai, const void* __restrict__ x, double br, double bi,
                        void* __restrict__ y) {
    using R = typename Elem<PY>::R;
    const cplx<R> a = {(R)ar, (R)ai}, b = {(R)br, (R)bi};
    const bool useb = !(br == 0.0 && bi == 0.0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        auto xv = Elem<PX>::ld(x, i);
        cplx<R> xx = {(R)xv.re, (R)xv.im};
        cplx<R> r = a * xx;
        if (useb) {
            auto yv = Elem<PY>::ld(y, i);
            r = r + b * cplx<R>{(R)yv.re, (R)yv.im};
        }
        Elem<PY>::st(y, i, r);
    }
}

// Mixed-precision y = a*x + b*y.  The flat complex order differs between the
// precisions (one, two or four complex numbers per 16-byte chunk), so these
// kernels walk over sites and use the layout-aware spinor load and store.
template <int PX, int PY>
__global__ void k_axpby_site(int Vh, int nfields, double ar, double ai, const void* __restrict__ x, double br,
                             double bi, void* __restrict__ y) {
    using RX = typename Prec<PX>::real;
    using RY = typename Prec<PY>::real;
    using CX = typename Prec<PX>::chunk;
    using CY = typename Prec<PY>::chunk;
    const bool useb = !(br == 0.0 && bi == 0.0);
    const long long total = (long long)Vh * nfields;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int f = (int)(t / Vh), h = (int)(t % Vh);
        const CX* xb = static_cast<const CX*>(x) + (size_t)f * Prec<PX>::nchunk * Vh;
        CY* yb = static_cast<CY*>(y) + (size_t)f * Prec<PY>::nchunk * Vh;
        cplx<RX> xs[12];
        load_spinor<PX>(xb, Vh, h, xs);
        cplx<RY> ys[12];
        if (useb) load_spinor<PY>(yb, Vh, h, ys);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double xr = xs[k].re, xi = xs[k].im;
            double r = ar * xr - ai * xi, i = ar * xi + ai * xr;
            if (useb) {
                const double yr = ys[k].re, yi = ys[k].im;
                r += br * yr - bi * yi;
                i += br * yi + bi * yr;
            }
            ys[k] = {(RY)r, (RY)i};
        }
        store_spinor<PY>(yb, Vh, h, ys);
    }
}

// y += sum_j c_j X_j  (k <= kMultiMax)
template <int PX, int PY, int K>
__global__ void k_multi_axpy(size_t n, MultiPtr X, MultiCoef c, void* __restrict__ y) {
    using R = typename Elem<PY>::R;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        auto yv = Elem<PY>::ld(y, i);
        double ar = yv.re, ai = yv.im;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            auto xv = Elem<PX>::ld(X.p[j], i);
            const double xr = xv.re, xi = xv.im;
            ar += c.re[j] * xr - c.im[j] * xi;
            ai += c.re[j] * xi + c.im[j] * xr;
        }
        Elem<PY>::st(y, i, cplx<R>{(R)ar, (R)ai});
    }
}

static int upd_blocks(qxd_ctx* ctx, size_t n) {
    size_t b = (n + 255) / 256;
    size_t cap = (size_t)ctx->nsm * 16;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

int blas_axpby(qxd_ctx* ctx, int px, int py, size_t n, double ar, double ai, const void* x, double br, double bi,
               void* y, cudaStream_t st) {
    const bool rb = !(br == 0.0 && bi == 0.0);
    ProfScope prof(ctx, px == py ? "axpby" : "axpby_convert", (double)n * (eb(px) + eb(py) * (rb ? 2 : 1)), st);
    if (px == py) {
        const int nb = upd_blocks(ctx, n);
        if (px == 0) k_axpby<0, 0><<<nb, 256, 0, st>>>(n, ar, ai, x, br, bi, y);
        else if (px == 1) k_axpby<1, 1><<<nb, 256, 0, st>>>(n, ar, ai, x, br, bi, y);
        else k_axpby<2, 2><<<nb, 256, 0, st>>>(n, ar, ai, x, br, bi, y);
    } else {
        const int Vh = ctx->g.Vh;
        if (n % (12ull * Vh) != 0) return qxd_fail(ctx, QXD_EARG, "blas_axpby: mixed precision needs whole fields");
        const int nf = (int)(n / (12ull * Vh));
        const int nb = upd_blocks(ctx, (size_t)Vh * nf);
#define QXD_AXPBY(A, B) k_axpby_site<A, B><<<nb, 256, 0, st>>>(Vh, nf, ar, ai, x, br, bi, y)
        if (px == 0 && py == 1) QXD_AXPBY(0, 1);
        else if (px == 1 && py == 0) QXD_AXPBY(1, 0);
        else if (px == 0 && py == 2) QXD_AXPBY(0, 2);
        else if (px == 2 && py == 0) QXD_AXPBY(2, 0);
        else if (px == 1 && py == 2) QXD_AXPBY(1, 2);
        else QXD_AXPBY(2, 1);
#undef QXD_AXPBY
    }
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

template <int PX, int PY>
static void multi_axpy_k(int k, int nb, size_t n, const MultiPtr& X, const MultiCoef& c, void* y, cudaStream_t st) {
    switch (k) {
        case 1: k_multi_axpy<PX, PY, 1><<<nb, 256, 0, st>>>(n, X, c, y); break;
        case 2: k_multi_axpy<PX, PY, 2><<<nb, 256, 0, st>>>(n, X, c, y); break;
        case 3: k_multi_axpy<PX, PY, 3><<<nb, 256, 0, st>>>(n, X, c, y); break;
        case 4: k_multi_axpy<PX, PY, 4><<<nb, 256, 0, st>>>(n, X, c, y); break;
        case 5: k_multi_axpy<PX, PY, 5><<<nb, 256, 0, st>>>(n, X, c, y); break;
        case 6: k_multi_axpy<PX, PY, 6><<<nb, 256, 0, st>>>(n, X, c, y); break;
        case 7: k_multi_axpy<PX, PY, 7><<<nb, 256, 0, st>>>(n, X, c, y); break;
        default: k_multi_axpy<PX, PY, 8><<<nb, 256, 0, st>>>(n, X, c, y); break;
    }
}

int blas_multi_axpy(qxd_ctx* ctx, int px, int py, size_t n, int k, const double* cre, const double* cim,
                    const void* const* X, void* y, cudaStream_t st) {
    const int nb = upd_blocks(ctx, n);
    for (int j0 = 0; j0 < k; j0 += kMultiMax) {
        const int kk = (k - j0) < kMultiMax ? (k - j0) : kMultiMax;
        MultiPtr mp;
        MultiCoef mc;
        for (int j = 0; j < kMultiMax; ++j) {
            const int jj = j < kk ? j0 + j : j0;
            mp.p[j] = X[jj];
            mc.re[j] = j < kk ? cre[jj] : 0.0;
            mc.im[j] = j < kk ? cim[jj] : 0.0;
        }
        ProfScope prof(ctx, "multi_axpy", (double)n * (eb(px) * kk + 2 * eb(py)), st);
        // the flat complex order is the same only within one precision
        if (px == 0 && py == 0) multi_axpy_k<0, 0>(kk, nb, n, mp, mc, y, st);
        else if (px == 1 && py == 1) multi_axpy_k<1, 1>(kk, nb, n, mp, mc, y, st);
        else if (px == 2 && py == 2) multi_axpy_k<2, 2>(kk, nb, n, mp, mc, y, st);
        else return qxd_fail(ctx, QXD_EARG, "blas_multi_axpy: precisions must match");
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

int blas_fetch(qxd_ctx* ctx, int nslots, cudaStream_t st) {
    QXD_CUDA(ctx, cudaMemcpyAsync(ctx->red_host, ctx->red_result, sizeof(double) * nslots, cudaMemcpyDeviceToHost, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

}  // namespace qxd
