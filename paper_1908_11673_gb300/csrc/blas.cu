// Vector kernels of the solvers: axpy-type updates, precision conversions and
// deterministic reductions (block partial sums, then one block sums the
// partials in a fixed order; every sum is accumulated in FP64).
//
// Within one precision a field is handled as a flat array of n complex numbers
// (the structure-of-arrays chunks store (re, im) pairs contiguously); operations
// between two precisions go site by site through the layout-aware spinor access.
#include "qxd_internal.h"
#include "blas.h"

namespace qxd {

// Flat access in 16-byte chunks: one complex (FP64), two (FP32) or four (BF16)
// per chunk.  Arithmetic runs in the storage precision's real type (FP32 for
// FP32 and BF16 data: the FP64 pipe of this GPU is 1/64 of the FP32 one);
// reductions add FP32 partial sums of at most kFlush chunks into FP64 accumulators.
template <int P> struct Chunk;
template <> struct Chunk<0> {
    using R = double;
    static constexpr int NC = 1;
    static QXD_HD void ld(const void* p, size_t i, cplx<double> c[1]) {
        double2 v = QXD_LDG(static_cast<const double2*>(p) + i);
        c[0] = {v.x, v.y};
    }
    static QXD_HD void st(void* p, size_t i, const cplx<double> c[1]) {
        static_cast<double2*>(p)[i] = make_double2(c[0].re, c[0].im);
    }
};
template <> struct Chunk<1> {
    using R = float;
    static constexpr int NC = 2;
    static QXD_HD void ld(const void* p, size_t i, cplx<float> c[2]) {
        float4 v = QXD_LDG(static_cast<const float4*>(p) + i);
        c[0] = {v.x, v.y};
        c[1] = {v.z, v.w};
    }
    static QXD_HD void st(void* p, size_t i, const cplx<float> c[2]) {
        static_cast<float4*>(p)[i] = make_float4(c[0].re, c[0].im, c[1].re, c[1].im);
    }
};
template <> struct Chunk<2> {
    using R = float;
    static constexpr int NC = 4;
    static QXD_HD void ld(const void* p, size_t i, cplx<float> c[4]) {
        uint4 v = QXD_LDG(static_cast<const uint4*>(p) + i);
        c[0] = {bf16_lo(v.x), bf16_hi(v.x)};
        c[1] = {bf16_lo(v.y), bf16_hi(v.y)};
        c[2] = {bf16_lo(v.z), bf16_hi(v.z)};
        c[3] = {bf16_lo(v.w), bf16_hi(v.w)};
    }
    static QXD_HD void st(void* p, size_t i, const cplx<float> c[4]) {
        uint4 v;
        v.x = pack_bf16x2(c[0].re, c[0].im);
        v.y = pack_bf16x2(c[1].re, c[1].im);
        v.z = pack_bf16x2(c[2].re, c[2].im);
        v.w = pack_bf16x2(c[3].re, c[3].im);
        static_cast<uint4*>(p)[i] = v;
    }
};

constexpr int kFlush = 8;

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
// n counts complex numbers; every kernel walks over n / NC chunks.
template <int P>
__global__ void __launch_bounds__(kRedThreads) k_dot(size_t nch, const void* __restrict__ a,
                                                     const void* __restrict__ b, double* __restrict__ partials) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    double v[2] = {0.0, 0.0};
    R f[2] = {R(0), R(0)};
    int cnt = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> x[NC], y[NC];
        Chunk<P>::ld(a, i, x);
        Chunk<P>::ld(b, i, y);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            f[0] = fma(x[c].re, y[c].re, fma(x[c].im, y[c].im, f[0]));
            f[1] = fma(x[c].re, y[c].im, fma(-x[c].im, y[c].re, f[1]));
        }
        if (++cnt == kFlush) {
            v[0] += f[0]; v[1] += f[1];
            f[0] = f[1] = R(0);
            cnt = 0;
        }
    }
    v[0] += f[0];
    v[1] += f[1];
    block_reduce_store<2>(v, partials);
}

template <int P>
__global__ void __launch_bounds__(kRedThreads) k_norm2(size_t nch, const void* __restrict__ a,
                                                       double* __restrict__ partials) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    double v[2] = {0.0, 0.0};  // |a|^2 and a count of non-finite entries
    R f = R(0);
    int cnt = 0, bad = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> x[NC];
        Chunk<P>::ld(a, i, x);
        R s = R(0);
#pragma unroll
        for (int c = 0; c < NC; ++c) s = fma(x[c].re, x[c].re, fma(x[c].im, x[c].im, s));
        if (isfinite(s)) f += s;
        else ++bad;
        if (++cnt == kFlush) {
            v[0] += f;
            f = R(0);
            cnt = 0;
        }
    }
    v[0] += f;
    v[1] = bad;
    block_reduce_store<2>(v, partials);
}

// k dot products <W_j, v>, j < k (k <= kMultiMax)
template <int P, int K>
__global__ void __launch_bounds__(kRedThreads) k_multi_dot(size_t nch, MultiPtr W, const void* __restrict__ v,
                                                           double* __restrict__ partials) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    double acc[2 * K];
    R f[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        acc[c] = 0.0;
        f[c] = R(0);
    }
    int cnt = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> y[NC];
        Chunk<P>::ld(v, i, y);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            cplx<R> x[NC];
            Chunk<P>::ld(W.p[j], i, x);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                f[2 * j] = fma(x[c].re, y[c].re, fma(x[c].im, y[c].im, f[2 * j]));
                f[2 * j + 1] = fma(x[c].re, y[c].im, fma(-x[c].im, y[c].re, f[2 * j + 1]));
            }
        }
        if (++cnt == kFlush) {
#pragma unroll
            for (int c = 0; c < 2 * K; ++c) {
                acc[c] += f[c];
                f[c] = R(0);
            }
            cnt = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) acc[c] += f[c];
    block_reduce_store<2 * K>(acc, partials);
}

static size_t nchunks(int P, size_t n) { return n / (P == 0 ? 1 : (P == 1 ? 2 : 4)); }

int blas_dot(qxd_ctx* ctx, int pa, int pb, size_t n, const void* a, const void* b, int slot, cudaStream_t st) {
    // the flat complex order is the same only within one precision
    if (pa != pb) return qxd_fail(ctx, QXD_EARG, "blas_dot: precisions must match");
    const size_t nc = nchunks(pa, n);
    const int nb = red_blocks(nc);
    {
        ProfScope prof(ctx, "dot", (double)n * (eb(pa) + eb(pb)), st);
        if (pa == 0) k_dot<0><<<nb, kRedThreads, 0, st>>>(nc, a, b, ctx->red_partials);
        else if (pa == 1) k_dot<1><<<nb, kRedThreads, 0, st>>>(nc, a, b, ctx->red_partials);
        else k_dot<2><<<nb, kRedThreads, 0, st>>>(nc, a, b, ctx->red_partials);
    }
    return finish(ctx, nb, 2, slot, st);
}

int blas_norm2(qxd_ctx* ctx, int p, size_t n, const void* a, int slot, cudaStream_t st) {
    const size_t nc = nchunks(p, n);
    const int nb = red_blocks(nc);
    {
        ProfScope prof(ctx, "norm2", (double)n * eb(p), st);
        if (p == 0) k_norm2<0><<<nb, kRedThreads, 0, st>>>(nc, a, ctx->red_partials);
        else if (p == 1) k_norm2<1><<<nb, kRedThreads, 0, st>>>(nc, a, ctx->red_partials);
        else k_norm2<2><<<nb, kRedThreads, 0, st>>>(nc, a, ctx->red_partials);
    }
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
        const size_t nc = nchunks(p, n);
        const int nb = red_blocks(nc);
        {
        ProfScope prof(ctx, "multi_dot", (double)n * eb(p) * (kk + 1), st);
        if (p == 0) multi_dot_k<0>(kk, nb, nc, mp, v, ctx->red_partials, st);
        else if (p == 1) multi_dot_k<1>(kk, nb, nc, mp, v, ctx->red_partials, st);
        else multi_dot_k<2>(kk, nb, nc, mp, v, ctx->red_partials, st);
        }
        QXD_TRY(finish(ctx, nb, 2 * kk, slot + 2 * j0, st));
    }
    return QXD_OK;
}

// ---- updates -------------------------------------------------------------------
// y = a*x + b*y (same precision, arithmetic in its real type)
template <int P>
__global__ void k_axpby(size_t nch, double ar, double ai, const void* __restrict__ x, double br, double bi,
                        void* __restrict__ y) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    const cplx<R> a = {(R)ar, (R)ai}, b = {(R)br, (R)bi};
    const bool useb = !(br == 0.0 && bi == 0.0);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> xv[NC], yv[NC];
        Chunk<P>::ld(x, i, xv);
        if (useb) Chunk<P>::ld(y, i, yv);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            cplx<R> r = a * xv[c];
            if (useb) cmac(r, b, yv[c]);
            yv[c] = r;
        }
        Chunk<P>::st(y, i, yv);
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

// y += sum_j c_j X_j  (k <= kMultiMax; same precision, arithmetic in its real type)
template <int P, int K>
__global__ void k_multi_axpy(size_t nch, MultiPtr X, MultiCoef c, void* __restrict__ y) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    cplx<R> cf[K];
#pragma unroll
    for (int j = 0; j < K; ++j) cf[j] = {(R)c.re[j], (R)c.im[j]};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> yv[NC];
        Chunk<P>::ld(y, i, yv);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            cplx<R> xv[NC];
            Chunk<P>::ld(X.p[j], i, xv);
#pragma unroll
            for (int q = 0; q < NC; ++q) cmac(yv[q], cf[j], xv[q]);
        }
        Chunk<P>::st(y, i, yv);
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
        const size_t nc = nchunks(px, n);
        const int nb = upd_blocks(ctx, nc);
        if (px == 0) k_axpby<0><<<nb, 256, 0, st>>>(nc, ar, ai, x, br, bi, y);
        else if (px == 1) k_axpby<1><<<nb, 256, 0, st>>>(nc, ar, ai, x, br, bi, y);
        else k_axpby<2><<<nb, 256, 0, st>>>(nc, ar, ai, x, br, bi, y);
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

template <int P>
static void multi_axpy_k(int k, int nb, size_t nch, const MultiPtr& X, const MultiCoef& c, void* y, cudaStream_t st) {
    switch (k) {
        case 1: k_multi_axpy<P, 1><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        case 2: k_multi_axpy<P, 2><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        case 3: k_multi_axpy<P, 3><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        case 4: k_multi_axpy<P, 4><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        case 5: k_multi_axpy<P, 5><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        case 6: k_multi_axpy<P, 6><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        case 7: k_multi_axpy<P, 7><<<nb, 256, 0, st>>>(nch, X, c, y); break;
        default: k_multi_axpy<P, 8><<<nb, 256, 0, st>>>(nch, X, c, y); break;
    }
}

int blas_multi_axpy(qxd_ctx* ctx, int px, int py, size_t n, int k, const double* cre, const double* cim,
                    const void* const* X, void* y, cudaStream_t st) {
    // the flat complex order is the same only within one precision
    if (px != py) return qxd_fail(ctx, QXD_EARG, "blas_multi_axpy: precisions must match");
    const size_t nc = nchunks(px, n);
    const int nb = upd_blocks(ctx, nc);
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
        if (px == 0) multi_axpy_k<0>(kk, nb, nc, mp, mc, y, st);
        else if (px == 1) multi_axpy_k<1>(kk, nb, nc, mp, mc, y, st);
        else multi_axpy_k<2>(kk, nb, nc, mp, mc, y, st);
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
