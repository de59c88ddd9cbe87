// Vector kernels of the solvers: axpy-type updates, precision conversions and
// deterministic reductions.
//
// Within one precision a field is handled as a flat array of n complex numbers
// (the structure-of-arrays chunks store (re, im) pairs contiguously) and moved
// in 16-byte chunks: one complex (FP64), two (FP32) or four (BF16) per chunk.
// Arithmetic runs in the storage precision's real type (FP32 for FP32 and BF16
// data; the FP64 pipe of this GPU runs at 1/64 of the FP32 rate); reductions
// add FP32 partial sums of a few chunks into FP64 accumulators, and every sum
// across threads and blocks is FP64.  Operations between two precisions go
// site by site through the layout-aware spinor access, because the flat
// complex order of the internal layout depends on the precision.
//
// A reduction is one launch: every block writes its partial sums, and the last
// block to finish (a ticket counter) adds all partials in block order, so the
// result is the same on every run.
#include <map>
#include <mutex>
#include <type_traits>

#include "blas.h"
#include "qxd_internal.h"
#include "reduce.cuh"

namespace qxd {

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

constexpr int kFlush = 8;        // chunks summed in FP32 before an FP64 flush
constexpr int kUnroll = 4;       // independent chunk loads in flight per thread

static size_t nchunks(int P, size_t n) { return n / (P == 0 ? 1 : (P == 1 ? 2 : 4)); }
static double eb(int P) { return P == 0 ? 16.0 : (P == 1 ? 8.0 : 4.0); }

static int upd_blocks(qxd_ctx* ctx, size_t n) {
    size_t b = (n + 255) / 256;
    size_t cap = (size_t)ctx->nsm * 16;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}


// ---- reductions -------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kRedThreads) k_dot(size_t nch, const void* __restrict__ a,
                                                     const void* __restrict__ b, RedOut o) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    double v[2] = {0.0, 0.0};
    const size_t S = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < nch; i0 += S * kUnroll) {
        cplx<R> x[kUnroll][NC], y[kUnroll][NC];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < nch) {
                Chunk<P>::ld(a, i0 + u * S, x[u]);
                Chunk<P>::ld(b, i0 + u * S, y[u]);
            }
        R f[2] = {R(0), R(0)};
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < nch) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    f[0] = fma(x[u][c].re, y[u][c].re, fma(x[u][c].im, y[u][c].im, f[0]));
                    f[1] = fma(x[u][c].re, y[u][c].im, fma(-x[u][c].im, y[u][c].re, f[1]));
                }
            }
        v[0] += f[0];
        v[1] += f[1];
    }
    block_reduce_finish<2>(v, o);
}

template <int P>
__global__ void __launch_bounds__(kRedThreads) k_norm2(size_t nch, const void* __restrict__ a, RedOut o) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    double v[2] = {0.0, 0.0};  // |a|^2 over finite chunks, count of non-finite chunks
    const size_t S = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < nch; i0 += S * kUnroll) {
        cplx<R> x[kUnroll][NC];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < nch) Chunk<P>::ld(a, i0 + u * S, x[u]);
        R f = R(0);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < nch) {
                R s = R(0);
#pragma unroll
                for (int c = 0; c < NC; ++c) s = fma(x[u][c].re, x[u][c].re, fma(x[u][c].im, x[u][c].im, s));
                if (isfinite(s)) f += s;
                else v[1] += 1.0;
            }
        v[0] += f;
    }
    block_reduce_finish<2>(v, o);
}

// <W_j, v> for j < K.  With few vectors each thread takes U chunks per pass, so
// that about four loads are in flight per thread whatever K is.
template <int P, int K>
__global__ void __launch_bounds__(kRedThreads) k_multi_dot(size_t nch, MultiPtr W, const void* __restrict__ v,
                                                           RedOut o) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    constexpr int U = (K + 1 >= 4) ? 1 : ((K + 1 >= 2) ? 2 : 4);
    double acc[2 * K];
    R f[2 * K];
#pragma unroll
    for (int c = 0; c < 2 * K; ++c) {
        acc[c] = 0.0;
        f[c] = R(0);
    }
    int cnt = 0;
    const size_t S = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < nch; i0 += S * U) {
        cplx<R> y[U][NC];
        cplx<R> x[U][K][NC];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * S < nch) {
                Chunk<P>::ld(v, i0 + u * S, y[u]);
#pragma unroll
                for (int j = 0; j < K; ++j) Chunk<P>::ld(W.p[j], i0 + u * S, x[u][j]);
            }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * S < nch) {
#pragma unroll
                for (int j = 0; j < K; ++j)
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        f[2 * j] = fma(x[u][j][c].re, y[u][c].re, fma(x[u][j][c].im, y[u][c].im, f[2 * j]));
                        f[2 * j + 1] = fma(x[u][j][c].re, y[u][c].im, fma(-x[u][j][c].im, y[u][c].re, f[2 * j + 1]));
                    }
            }
        cnt += U;
        if (cnt >= kFlush) {
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
    block_reduce_finish<2 * K>(acc, o);
}

// <a, b> between two precisions, site by site over whole half-lattice fields
template <int PA, int PB>
__global__ void __launch_bounds__(kRedThreads) k_dot_site(int Vh, int nf, const void* __restrict__ a,
                                                          const void* __restrict__ b, RedOut o) {
    using CA = typename Prec<PA>::chunk;
    using CB = typename Prec<PB>::chunk;
    double v[2] = {0.0, 0.0};
    float f[2] = {0.f, 0.f};
    int cnt = 0;
    const long long total = (long long)Vh * nf;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int fi = (int)(t / Vh), h = (int)(t % Vh);
        cplx<typename Prec<PA>::real> x[12];
        cplx<typename Prec<PB>::real> y[12];
        load_spinor<PA>(static_cast<const CA*>(a) + (size_t)fi * Prec<PA>::nchunk * Vh, Vh, h, x);
        load_spinor<PB>(static_cast<const CB*>(b) + (size_t)fi * Prec<PB>::nchunk * Vh, Vh, h, y);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float xr = (float)x[k].re, xi = (float)x[k].im, yr = (float)y[k].re, yi = (float)y[k].im;
            f[0] = fmaf(xr, yr, fmaf(xi, yi, f[0]));
            f[1] = fmaf(xr, yi, fmaf(-xi, yr, f[1]));
        }
        if (++cnt == 2) {
            v[0] += f[0];
            v[1] += f[1];
            f[0] = f[1] = 0.f;
            cnt = 0;
        }
    }
    v[0] += f[0];
    v[1] += f[1];
    block_reduce_finish<2>(v, o);
}

int blas_dot(qxd_ctx* ctx, int pa, int pb, size_t n, const void* a, const void* b, int slot, cudaStream_t st) {
    if (pa != pb) {
        const int Vh = ctx->g.Vh;
        if (pa == 0 || pb == 0 || n % (12ull * Vh) != 0)
            return qxd_fail(ctx, QXD_EARG, "blas_dot: mixed precision only between FP32 and BF16 whole fields");
        const int nf = (int)(n / (12ull * Vh));
        ProfScope prof(ctx, "dot_mixed", (double)n * (eb(pa) + eb(pb)), st);
        const RedOut o = red_out(ctx, slot);
        const size_t wpb = kRedThreads;
        if (pa == 1) k_dot_site<1, 2><<<wave_blocks(ctx, k_dot_site<1, 2>, kRedThreads, wpb, (size_t)Vh * nf),
                                        kRedThreads, 0, st>>>(Vh, nf, a, b, o);
        else k_dot_site<2, 1><<<wave_blocks(ctx, k_dot_site<2, 1>, kRedThreads, wpb, (size_t)Vh * nf), kRedThreads,
                                0, st>>>(Vh, nf, a, b, o);
        QXD_CUDA(ctx, cudaGetLastError());
        return QXD_OK;
    }
    const size_t nc = nchunks(pa, n);
    ProfScope prof(ctx, "dot", (double)n * 2 * eb(pa), st);
    const RedOut o = red_out(ctx, slot);
    const size_t wpb = (size_t)kRedThreads * kUnroll;
#define QXD_LAUNCH(P) k_dot<P><<<wave_blocks(ctx, k_dot<P>, kRedThreads, wpb, nc), kRedThreads, 0, st>>>(nc, a, b, o)
    if (pa == 0) QXD_LAUNCH(0);
    else if (pa == 1) QXD_LAUNCH(1);
    else QXD_LAUNCH(2);
#undef QXD_LAUNCH
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// ---- double-float conversions (FP64 layout <-> double-float layout, same 16-byte chunks) ----
// elementwise; in and out may be the same array
// The conversions go through the integer forms of df64.cuh (df_split, df_widen): the
// FP64 <-> FP32 conversion instructions would load the FP64 pipe.  Each thread keeps
// kUnroll independent 16-byte loads in flight (in == out allowed: every entry is read
// and written by the same thread).
__global__ void k_split_df64(const double2* in, float4* out, size_t n) {
    const size_t S = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < n; i0 += S * kUnroll) {
        double2 d[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < n) d[u] = in[i0 + u * S];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < n) {
                const dfl a = df_split(d[u].x), b = df_split(d[u].y);
                out[i0 + u * S] = make_float4(a.hi, a.lo, b.hi, b.lo);
            }
    }
}
__global__ void k_join_df64(const float4* in, double2* out, size_t n) {
    const size_t S = (size_t)gridDim.x * blockDim.x;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i0 < n; i0 += S * kUnroll) {
        float4 f[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < n) f[u] = in[i0 + u * S];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (i0 + u * S < n)
                out[i0 + u * S] = make_double2(df_widen(f[u].x) + df_widen(f[u].y), df_widen(f[u].z) + df_widen(f[u].w));
    }
}
int blas_split_df64(qxd_ctx* ctx, const void* in, void* out, size_t n, cudaStream_t st) {
    ProfScope prof(ctx, "split_df64", (double)n * 32, st);
    k_split_df64<<<upd_blocks(ctx, n), 256, 0, st>>>(static_cast<const double2*>(in), static_cast<float4*>(out), n);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}
int blas_join_df64(qxd_ctx* ctx, const void* in, void* out, size_t n, cudaStream_t st) {
    ProfScope prof(ctx, "join_df64", (double)n * 32, st);
    k_join_df64<<<upd_blocks(ctx, n), 256, 0, st>>>(static_cast<const float4*>(in), static_cast<double2*>(out), n);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// ---- the mixed solver's outer loop in double-float (site by site, FP32 pipe only) ----
// r = eta - dx (eta an FP64 half-lattice field, split into double-float on the fly by
// integer operations; dx double-float): r32 = r rounded to the FP32 layout,
// result[slot] = |r|^2 (leading parts, FP32 per site, FP64 sums), result[slot+1] =
// count of non-finite sites
__global__ void __launch_bounds__(kRedThreads) k_df_residual(int Vh, const double2* __restrict__ eta,
                                                             const float4* __restrict__ dx,
                                                             float4* __restrict__ r32, RedOut o) {
    double v[2] = {0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<dfl> e[12], d[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 x = QXD_LDG(eta + (size_t)k * Vh + h);
            e[k] = {df_split(x.x), df_split(x.y)};
        }
        load_spinor<3>(dx, Vh, h, d);
        cplx<float> r[12];
        float f = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dfl re = df_norm(e[k].re - d[k].re), im = df_norm(e[k].im - d[k].im);
            r[k] = {re.hi, im.hi};
            f = fmaf(re.hi, re.hi, fmaf(im.hi, im.hi, f));
        }
        if (isfinite(f)) v[0] += f;
        else v[1] += 1.0;
        store_spinor<1>(r32, Vh, h, r);
    }
    block_reduce_finish<2>(v, o);
}

// r32 = FP32(b - y - sigma x) for double-float b, y = Q2 x and x (one half-lattice
// field); result[slot] = |r|^2, result[slot+1] = count of non-finite sites
__global__ void __launch_bounds__(kRedThreads) k_df_shift_residual(int Vh, const float4* __restrict__ b,
                                                                   const float4* __restrict__ y,
                                                                   const float4* __restrict__ x, float sig_hi,
                                                                   float sig_lo, float4* __restrict__ r32, RedOut o) {
    double v[2] = {0.0, 0.0};
    const dfl sig(sig_hi, sig_lo);
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        cplx<dfl> bs[12], ys[12], xs[12];
        load_spinor<3>(b, Vh, h, bs);
        load_spinor<3>(y, Vh, h, ys);
        load_spinor<3>(x, Vh, h, xs);
        cplx<float> r[12];
        float f = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dfl re = df_norm(bs[k].re - (ys[k].re + sig * xs[k].re));
            const dfl im = df_norm(bs[k].im - (ys[k].im + sig * xs[k].im));
            r[k] = {re.hi, im.hi};
            f = fmaf(re.hi, re.hi, fmaf(im.hi, im.hi, f));
        }
        if (isfinite(f)) v[0] += f;
        else v[1] += 1.0;
        store_spinor<1>(r32, Vh, h, r);
    }
    block_reduce_finish<2>(v, o);
}

int blas_df_shift_residual(qxd_ctx* ctx, const void* b, const void* y, const void* x, double sigma, void* r32,
                           int slot, cudaStream_t st) {
    const int Vh = ctx->g.Vh;
    ProfScope prof(ctx, "df_shift_residual", (double)Vh * (3 * 192 + 96), st);
    const RedOut o = red_out(ctx, slot);
    const dfl sg(sigma);
    k_df_shift_residual<<<wave_blocks(ctx, k_df_shift_residual, kRedThreads, (size_t)kRedThreads, (size_t)Vh),
                          kRedThreads, 0, st>>>(Vh, static_cast<const float4*>(b), static_cast<const float4*>(y),
                                                static_cast<const float4*>(x), sg.hi, sg.lo,
                                                static_cast<float4*>(r32), o);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// x += e (x double-float, e FP32), one half-lattice field
__global__ void k_df_add_f32(int Vh, const float4* __restrict__ e32, float4* __restrict__ x) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cplx<float> e[12];
    load_spinor<1>(e32, Vh, h, e);
    cplx<dfl> xs[12];
    load_spinor<3>(x, Vh, h, xs);
#pragma unroll
    for (int k = 0; k < 12; ++k) xs[k] = {xs[k].re + dfl(e[k].re, 0.f), xs[k].im + dfl(e[k].im, 0.f)};
    store_spinor<3>(x, Vh, h, xs);
}

// r32 = FP32 rounding of an FP64 half-lattice field (integer conversion), result[slot] =
// its |.|^2 over the finite sites and result[slot+1] = count of the others; a site's
// |x|^2 is sum hi (hi + 2 lo) in FP32 (about 2^-23 relative) where that lies in
// [1e-30, 1e30], else FP64
__global__ void __launch_bounds__(kRedThreads) k_f64_to_f32_norm(int Vh, const double2* __restrict__ x,
                                                                 float4* __restrict__ r32, RedOut o) {
    double v[2] = {0.0, 0.0};
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < Vh; h += gridDim.x * blockDim.x) {
        double2 xs[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) xs[k] = QXD_LDG(x + (size_t)k * Vh + h);
        cplx<float> r[12];
        float f = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const dfl a = df_split(xs[k].x), b = df_split(xs[k].y);
            r[k] = {a.hi, b.hi};
            f = fmaf(a.hi, fmaf(2.f, a.lo, a.hi), fmaf(b.hi, fmaf(2.f, b.lo, b.hi), f));
        }
        if (f >= 1e-30f && f <= 1e30f) {
            v[0] += f;
        } else {
            double dd = 0.0;
#pragma unroll
            for (int k = 0; k < 12; ++k) dd += xs[k].x * xs[k].x + xs[k].y * xs[k].y;
            if (isfinite(dd)) v[0] += dd;
            else v[1] += 1.0;
        }
        store_spinor<1>(r32, Vh, h, r);
    }
    block_reduce_finish<2>(v, o);
}

// r32 = leading parts of a double-float field, one half-lattice field
__global__ void k_df_to_f32(int Vh, const float4* __restrict__ x, float4* __restrict__ r32) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    cplx<dfl> xs[12];
    load_spinor<3>(x, Vh, h, xs);
    cplx<float> r[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) r[k] = {df_norm(xs[k].re).hi, df_norm(xs[k].im).hi};
    store_spinor<1>(r32, Vh, h, r);
}

int blas_df_residual(qxd_ctx* ctx, const void* eta, const void* dx, void* r32, int slot, cudaStream_t st) {
    const int Vh = ctx->g.Vh;
    ProfScope prof(ctx, "df_residual", (double)Vh * (192 + 192 + 96), st);
    const RedOut o = red_out(ctx, slot);
    k_df_residual<<<wave_blocks(ctx, k_df_residual, kRedThreads, (size_t)kRedThreads, (size_t)Vh), kRedThreads, 0,
                    st>>>(Vh, static_cast<const double2*>(eta), static_cast<const float4*>(dx),
                          static_cast<float4*>(r32), o);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}
int blas_df_add_f32(qxd_ctx* ctx, const void* e32, void* x, cudaStream_t st) {
    const int Vh = ctx->g.Vh;
    ProfScope prof(ctx, "df_add_f32", (double)Vh * (96 + 192 + 192), st);
    k_df_add_f32<<<nblocks(Vh, 128), 128, 0, st>>>(Vh, static_cast<const float4*>(e32), static_cast<float4*>(x));
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}
int blas_f64_to_f32_norm(qxd_ctx* ctx, const void* x, void* r32, int slot, cudaStream_t st) {
    const int Vh = ctx->g.Vh;
    ProfScope prof(ctx, "f64_to_f32_norm", (double)Vh * (192 + 96), st);
    const RedOut o = red_out(ctx, slot);
    k_f64_to_f32_norm<<<wave_blocks(ctx, k_f64_to_f32_norm, kRedThreads, (size_t)kRedThreads, (size_t)Vh),
                        kRedThreads, 0, st>>>(Vh, static_cast<const double2*>(x), static_cast<float4*>(r32), o);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}
int blas_df_to_f32(qxd_ctx* ctx, const void* x, void* r32, cudaStream_t st) {
    const int Vh = ctx->g.Vh;
    ProfScope prof(ctx, "df_to_f32", (double)Vh * (192 + 96), st);
    k_df_to_f32<<<nblocks(Vh, 128), 128, 0, st>>>(Vh, static_cast<const float4*>(x), static_cast<float4*>(r32));
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// sum of a real FP64 array over its finite entries, and the count of the others
__global__ void __launch_bounds__(kRedThreads) k_sum_real(size_t n, const double* __restrict__ a, RedOut o) {
    double v[2] = {0.0, 0.0};
    const size_t S = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += S) {
        const double x = __ldg(a + i);
        if (isfinite(x)) v[0] += x;
        else v[1] += 1.0;
    }
    block_reduce_finish<2>(v, o);
}

int blas_sum_real(qxd_ctx* ctx, const double* a, size_t n, int slot, cudaStream_t st) {
    ProfScope prof(ctx, "sum_real", (double)n * 8, st);
    const RedOut o = red_out(ctx, slot);
    k_sum_real<<<wave_blocks(ctx, k_sum_real, kRedThreads, (size_t)kRedThreads, n), kRedThreads, 0, st>>>(n, a, o);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int blas_norm2(qxd_ctx* ctx, int p, size_t n, const void* a, int slot, cudaStream_t st) {
    const size_t nc = nchunks(p, n);
    ProfScope prof(ctx, "norm2", (double)n * eb(p), st);
    const RedOut o = red_out(ctx, slot);
    const size_t wpb = (size_t)kRedThreads * kUnroll;
#define QXD_LAUNCH(P) k_norm2<P><<<wave_blocks(ctx, k_norm2<P>, kRedThreads, wpb, nc), kRedThreads, 0, st>>>(nc, a, o)
    if (p == 0) QXD_LAUNCH(0);
    else if (p == 1) QXD_LAUNCH(1);
    else QXD_LAUNCH(2);
#undef QXD_LAUNCH
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

template <int P, int K>
static void multi_dot_launch(qxd_ctx* ctx, size_t nch, const MultiPtr& W, const void* v, const RedOut& o,
                             cudaStream_t st) {
    const int nb = wave_blocks(ctx, k_multi_dot<P, K>, kRedThreads, (size_t)kRedThreads * 2, nch);
    k_multi_dot<P, K><<<nb, kRedThreads, 0, st>>>(nch, W, v, o);
}

template <int P>
static void multi_dot_k(qxd_ctx* ctx, int k, size_t nch, const MultiPtr& W, const void* v, const RedOut& o,
                        cudaStream_t st) {
    switch (k) {
        case 1: multi_dot_launch<P, 1>(ctx, nch, W, v, o, st); break;
        case 2: multi_dot_launch<P, 2>(ctx, nch, W, v, o, st); break;
        case 3: multi_dot_launch<P, 3>(ctx, nch, W, v, o, st); break;
        case 4: multi_dot_launch<P, 4>(ctx, nch, W, v, o, st); break;
        case 5: multi_dot_launch<P, 5>(ctx, nch, W, v, o, st); break;
        case 6: multi_dot_launch<P, 6>(ctx, nch, W, v, o, st); break;
        case 7: multi_dot_launch<P, 7>(ctx, nch, W, v, o, st); break;
        default: multi_dot_launch<P, 8>(ctx, nch, W, v, o, st); break;
    }
}

int blas_multi_dot(qxd_ctx* ctx, int p, size_t n, int k, const void* const* W, const void* v, int slot,
                   cudaStream_t st) {
    const size_t nc = nchunks(p, n);
    for (int j0 = 0; j0 < k; j0 += kMultiMax) {
        const int kk = (k - j0) < kMultiMax ? (k - j0) : kMultiMax;
        MultiPtr mp;
        for (int j = 0; j < kMultiMax; ++j) mp.p[j] = W[j0 + (j < kk ? j : 0)];
        ProfScope prof(ctx, "multi_dot", (double)n * eb(p) * (kk + 1), st);
        const RedOut o = red_out(ctx, slot + 2 * j0);
        if (p == 0) multi_dot_k<0>(ctx, kk, nc, mp, v, o, st);
        else if (p == 1) multi_dot_k<1>(ctx, kk, nc, mp, v, o, st);
        else multi_dot_k<2>(ctx, kk, nc, mp, v, o, st);
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

// ---- updates --------------------------------------------------------------------
// y = a*x + b*y (same precision)
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

// z = x + a*w (same precision, z distinct from x and w)
template <int P>
__global__ void k_axpy3(size_t nch, double ar, double ai, const void* __restrict__ w, const void* __restrict__ x,
                        void* __restrict__ z) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    const cplx<R> a = {(R)ar, (R)ai};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> xv[NC], wv[NC];
        Chunk<P>::ld(x, i, xv);
        Chunk<P>::ld(w, i, wv);
#pragma unroll
        for (int c = 0; c < NC; ++c) cmac(xv[c], a, wv[c]);
        Chunk<P>::st(z, i, xv);
    }
}

// y = a*x + b*y between two precisions, site by site (grid: sites x fields)
template <int PX, int PY>
__global__ void k_axpby_site(int Vh, double ar, double ai, const void* __restrict__ x, double br, double bi,
                             void* __restrict__ y) {
    using RX = typename Prec<PX>::real;
    using RY = typename Prec<PY>::real;
    using CX = typename Prec<PX>::chunk;
    using CY = typename Prec<PY>::chunk;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= Vh) return;
    const int f = blockIdx.y;
    const CX* xb = static_cast<const CX*>(x) + (size_t)f * Prec<PX>::nchunk * Vh;
    CY* yb = static_cast<CY*>(y) + (size_t)f * Prec<PY>::nchunk * Vh;
    cplx<RX> xs[12];
    load_spinor<PX>(xb, Vh, h, xs);
    cplx<RY> ys[12];
    const bool copy = ar == 1.0 && ai == 0.0 && br == 0.0 && bi == 0.0;
    if (copy) {
#pragma unroll
        for (int k = 0; k < 12; ++k) ys[k] = {(RY)xs[k].re, (RY)xs[k].im};
    } else {
        const bool useb = !(br == 0.0 && bi == 0.0);
        if (useb) load_spinor<PY>(yb, Vh, h, ys);
        // the wider of the two precisions carries the arithmetic
        using RW = typename std::conditional<(sizeof(RX) > sizeof(RY)), RX, RY>::type;
        const RW a_r = (RW)ar, a_i = (RW)ai, b_r = (RW)br, b_i = (RW)bi;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const RW xr = xs[k].re, xi = xs[k].im;
            RW r = a_r * xr - a_i * xi, i = a_r * xi + a_i * xr;
            if (useb) {
                const RW yr = ys[k].re, yi = ys[k].im;
                r += b_r * yr - b_i * yi;
                i += b_r * yi + b_i * yr;
            }
            ys[k] = {(RY)r, (RY)i};
        }
    }
    store_spinor<PY>(yb, Vh, h, ys);
}

// y += sum_j c_j X_j (same precision); with NORM also |y|^2 of the result
template <int P, int K, bool NORM>
__global__ void __launch_bounds__(kRedThreads) k_multi_axpy(size_t nch, MultiPtr X, MultiCoef c,
                                                            void* __restrict__ y, RedOut o) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    cplx<R> cf[K];
#pragma unroll
    for (int j = 0; j < K; ++j) cf[j] = {(R)c.re[j], (R)c.im[j]};
    double v[2] = {0.0, 0.0};
    R f = R(0);
    int cnt = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> yv[NC];
        Chunk<P>::ld(y, i, yv);
        cplx<R> xv[K][NC];
#pragma unroll
        for (int j = 0; j < K; ++j) Chunk<P>::ld(X.p[j], i, xv[j]);
#pragma unroll
        for (int j = 0; j < K; ++j)
#pragma unroll
            for (int q = 0; q < NC; ++q) cmac(yv[q], cf[j], xv[j][q]);
        Chunk<P>::st(y, i, yv);
        if (NORM) {
            R s = R(0);
#pragma unroll
            for (int q = 0; q < NC; ++q) s = fma(yv[q].re, yv[q].re, fma(yv[q].im, yv[q].im, s));
            if (isfinite(s)) f += s;
            else v[1] += 1.0;
            if (++cnt == kFlush) {
                v[0] += f;
                f = R(0);
                cnt = 0;
            }
        }
    }
    if (NORM) {
        v[0] += f;
        block_reduce_finish<2>(v, o);
    }
}

// One GCR step's update in one pass (same precision): w += sum_j c_j X_j, then
// z = x + a w with the updated w (the residual update r_{k+1} = r_k - alpha w_k').
template <int P, int K>
__global__ void k_gcr_update(size_t nch, MultiPtr X, MultiCoef c, void* __restrict__ w, double ar, double ai,
                             const void* __restrict__ x, void* __restrict__ z) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    cplx<R> cf[K > 0 ? K : 1];
#pragma unroll
    for (int j = 0; j < K; ++j) cf[j] = {(R)c.re[j], (R)c.im[j]};
    const cplx<R> a = {(R)ar, (R)ai};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> wv[NC], xv[NC];
        Chunk<P>::ld(w, i, wv);
        Chunk<P>::ld(x, i, xv);
        if constexpr (K > 0) {
            cplx<R> yv[K][NC];
#pragma unroll
            for (int j = 0; j < K; ++j) Chunk<P>::ld(X.p[j], i, yv[j]);
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int q = 0; q < NC; ++q) cmac(wv[q], cf[j], yv[j][q]);
            Chunk<P>::st(w, i, wv);
        }
#pragma unroll
        for (int q = 0; q < NC; ++q) cmac(xv[q], a, wv[q]);
        Chunk<P>::st(z, i, xv);
    }
}

template <int P>
static void gcr_update_k(qxd_ctx* ctx, int k, size_t nch, const MultiPtr& X, const MultiCoef& c, void* w, double ar,
                         double ai, const void* x, void* z, cudaStream_t st) {
    const int nb = upd_blocks(ctx, nch);
#define QXD_GU(K) k_gcr_update<P, K><<<nb, 256, 0, st>>>(nch, X, c, w, ar, ai, x, z)
    switch (k) {
        case 0: QXD_GU(0); break;
        case 1: QXD_GU(1); break;
        case 2: QXD_GU(2); break;
        case 3: QXD_GU(3); break;
        case 4: QXD_GU(4); break;
        case 5: QXD_GU(5); break;
        case 6: QXD_GU(6); break;
        case 7: QXD_GU(7); break;
        default: QXD_GU(8); break;
    }
#undef QXD_GU
}

int blas_gcr_update(qxd_ctx* ctx, int p, size_t n, int k, const double* cre, const double* cim,
                    const void* const* X, void* w, double ar, double ai, const void* x, void* z, cudaStream_t st) {
    if (k > kMultiMax) {
        // all but the last eight basis vectors in a separate pass
        const int k0 = k - kMultiMax;
        QXD_TRY(blas_multi_axpy(ctx, p, p, n, k0, cre, cim, X, w, st));
        return blas_gcr_update(ctx, p, n, kMultiMax, cre + k0, cim + k0, X + k0, w, ar, ai, x, z, st);
    }
    MultiPtr mp;
    MultiCoef mc;
    for (int j = 0; j < kMultiMax; ++j) {
        mp.p[j] = j < k ? X[j] : w;
        mc.re[j] = j < k ? cre[j] : 0.0;
        mc.im[j] = j < k ? cim[j] : 0.0;
    }
    ProfScope prof(ctx, "gcr_update", (double)n * eb(p) * (k + (k > 0 ? 4 : 3)), st);
    const size_t nc = nchunks(p, n);
    if (p == 0) gcr_update_k<0>(ctx, k, nc, mp, mc, w, ar, ai, x, z, st);
    else if (p == 1) gcr_update_k<1>(ctx, k, nc, mp, mc, w, ar, ai, x, z, st);
    else gcr_update_k<2>(ctx, k, nc, mp, mc, w, ar, ai, x, z, st);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
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
        const dim3 grid(nblocks(Vh, 128), nf);
#define QXD_AXPBY(A, B) k_axpby_site<A, B><<<grid, 128, 0, st>>>(Vh, ar, ai, x, br, bi, y)
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

int blas_axpy3(qxd_ctx* ctx, int p, size_t n, double ar, double ai, const void* w, const void* x, void* z,
               cudaStream_t st) {
    ProfScope prof(ctx, "axpy3", (double)n * eb(p) * 3, st);
    const size_t nc = nchunks(p, n);
    const int nb = upd_blocks(ctx, nc);
    if (p == 0) k_axpy3<0><<<nb, 256, 0, st>>>(nc, ar, ai, w, x, z);
    else if (p == 1) k_axpy3<1><<<nb, 256, 0, st>>>(nc, ar, ai, w, x, z);
    else k_axpy3<2><<<nb, 256, 0, st>>>(nc, ar, ai, w, x, z);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

template <int P, int K, bool NORM>
static void multi_axpy_launch(qxd_ctx* ctx, size_t nch, const MultiPtr& X, const MultiCoef& c, void* y,
                              const RedOut& o, cudaStream_t st) {
    const int nb = NORM ? wave_blocks(ctx, k_multi_axpy<P, K, NORM>, kRedThreads, (size_t)kRedThreads * 2, nch)
                        : upd_blocks(ctx, nch);
    k_multi_axpy<P, K, NORM><<<nb, kRedThreads, 0, st>>>(nch, X, c, y, o);
}

template <int P, bool NORM>
static void multi_axpy_k(qxd_ctx* ctx, int k, size_t nch, const MultiPtr& X, const MultiCoef& c, void* y,
                         const RedOut& o, cudaStream_t st) {
    switch (k) {
        case 1: multi_axpy_launch<P, 1, NORM>(ctx, nch, X, c, y, o, st); break;
        case 2: multi_axpy_launch<P, 2, NORM>(ctx, nch, X, c, y, o, st); break;
        case 3: multi_axpy_launch<P, 3, NORM>(ctx, nch, X, c, y, o, st); break;
        case 4: multi_axpy_launch<P, 4, NORM>(ctx, nch, X, c, y, o, st); break;
        case 5: multi_axpy_launch<P, 5, NORM>(ctx, nch, X, c, y, o, st); break;
        case 6: multi_axpy_launch<P, 6, NORM>(ctx, nch, X, c, y, o, st); break;
        case 7: multi_axpy_launch<P, 7, NORM>(ctx, nch, X, c, y, o, st); break;
        default: multi_axpy_launch<P, 8, NORM>(ctx, nch, X, c, y, o, st); break;
    }
}

static int multi_axpy_impl(qxd_ctx* ctx, int px, int py, size_t n, int k, const double* cre, const double* cim,
                           const void* const* X, void* y, int norm_slot, cudaStream_t st) {
    if (px != py) return qxd_fail(ctx, QXD_EARG, "blas_multi_axpy: precisions must match");
    const size_t nc = nchunks(px, n);
    for (int j0 = 0; j0 < k; j0 += kMultiMax) {
        const int kk = (k - j0) < kMultiMax ? (k - j0) : kMultiMax;
        const bool norm = norm_slot >= 0 && j0 + kk == k;  // the norm is taken after the last chunk
        MultiPtr mp;
        MultiCoef mc;
        for (int j = 0; j < kMultiMax; ++j) {
            const int jj = j < kk ? j0 + j : j0;
            mp.p[j] = X[jj];
            mc.re[j] = j < kk ? cre[jj] : 0.0;
            mc.im[j] = j < kk ? cim[jj] : 0.0;
        }
        ProfScope prof(ctx, norm ? "multi_axpy_norm" : "multi_axpy", (double)n * (eb(px) * kk + 2 * eb(py)), st);
        const RedOut o = red_out(ctx, norm ? norm_slot : 0);
        if (norm) {
            if (px == 0) multi_axpy_k<0, true>(ctx, kk, nc, mp, mc, y, o, st);
            else if (px == 1) multi_axpy_k<1, true>(ctx, kk, nc, mp, mc, y, o, st);
            else multi_axpy_k<2, true>(ctx, kk, nc, mp, mc, y, o, st);
        } else {
            if (px == 0) multi_axpy_k<0, false>(ctx, kk, nc, mp, mc, y, o, st);
            else if (px == 1) multi_axpy_k<1, false>(ctx, kk, nc, mp, mc, y, o, st);
            else multi_axpy_k<2, false>(ctx, kk, nc, mp, mc, y, o, st);
        }
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

int blas_multi_axpy(qxd_ctx* ctx, int px, int py, size_t n, int k, const double* cre, const double* cim,
                    const void* const* X, void* y, cudaStream_t st) {
    return multi_axpy_impl(ctx, px, py, n, k, cre, cim, X, y, -1, st);
}

int blas_multi_axpy_norm(qxd_ctx* ctx, int p, size_t n, int k, const double* cre, const double* cim,
                         const void* const* X, void* y, int slot, cudaStream_t st) {
    if (k < 1) return blas_norm2(ctx, p, n, y, slot, st);
    return multi_axpy_impl(ctx, p, p, n, k, cre, cim, X, y, slot, st);
}

// ---- multi-shift CG update ---------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(256) k_msg_update(size_t nch, int ns, ShiftPtrs ptr, ShiftCoef c,
                                                    const void* __restrict__ r) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> rv[NC];
        Chunk<P>::ld(r, i, rv);
        for (int j = 0; j < ns; ++j) {
            cplx<R> xv[NC], pv[NC];
            Chunk<P>::ld(ptr.x[j], i, xv);
            Chunk<P>::ld(ptr.p[j], i, pv);
            const R a = (R)c.alpha[j], z = (R)c.zeta[j], b = (R)c.beta[j];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                xv[q].re = fma(a, pv[q].re, xv[q].re);
                xv[q].im = fma(a, pv[q].im, xv[q].im);
                pv[q].re = fma(z, rv[q].re, b * pv[q].re);
                pv[q].im = fma(z, rv[q].im, b * pv[q].im);
            }
            Chunk<P>::st(ptr.x[j], i, xv);
            Chunk<P>::st(ptr.p[j], i, pv);
        }
    }
}

int blas_msg_update(qxd_ctx* ctx, int P, size_t n, int ns, const ShiftPtrs& ptr, const ShiftCoef& c, const void* r,
                    cudaStream_t st) {
    if (ns < 1) return QXD_OK;
    if (ns > kMaxShifts) return qxd_fail(ctx, QXD_EARG, "msg_update: too many shifts");
    const size_t nc = nchunks(P, n);
    const int nb = upd_blocks(ctx, nc);
    ProfScope prof(ctx, "msg_update", (double)n * eb(P) * (1 + 4 * ns), st);
    if (P == 0) k_msg_update<0><<<nb, 256, 0, st>>>(nc, ns, ptr, c, r);
    else if (P == 1) k_msg_update<1><<<nb, 256, 0, st>>>(nc, ns, ptr, c, r);
    else k_msg_update<2><<<nb, 256, 0, st>>>(nc, ns, ptr, c, r);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// ---- device-scalar variants ----------------------------------------------------------
template <int P>
__global__ void k_axpby_dev(size_t nch, const double* __restrict__ c, const void* __restrict__ x,
                            void* __restrict__ y) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    const R a = (R)c[0], b = (R)c[1];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> xv[NC], yv[NC];
        Chunk<P>::ld(x, i, xv);
        Chunk<P>::ld(y, i, yv);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            yv[q].re = fma(a, xv[q].re, b * yv[q].re);
            yv[q].im = fma(a, xv[q].im, b * yv[q].im);
        }
        Chunk<P>::st(y, i, yv);
    }
}

template <int P>
__global__ void __launch_bounds__(kRedThreads) k_axpy_norm_dev(size_t nch, const double* __restrict__ c,
                                                               const void* __restrict__ x, void* __restrict__ y,
                                                               RedOut o) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    const R a = (R)c[0];
    double v[2] = {0.0, 0.0};
    R f = R(0);
    int cnt = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> xv[NC], yv[NC];
        Chunk<P>::ld(x, i, xv);
        Chunk<P>::ld(y, i, yv);
        R s = R(0);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            yv[q].re = fma(a, xv[q].re, yv[q].re);
            yv[q].im = fma(a, xv[q].im, yv[q].im);
            s = fma(yv[q].re, yv[q].re, fma(yv[q].im, yv[q].im, s));
        }
        Chunk<P>::st(y, i, yv);
        if (isfinite(s)) f += s;
        else v[1] += 1.0;
        if (++cnt == kFlush) {
            v[0] += f;
            f = R(0);
            cnt = 0;
        }
    }
    v[0] += f;
    block_reduce_finish<2>(v, o);
}

template <int P>
__global__ void __launch_bounds__(256) k_msg_update_dev(size_t nch, int ns, ShiftPtrs ptr, ShiftCoefDev c,
                                                        const void* __restrict__ r) {
    using R = typename Chunk<P>::R;
    constexpr int NC = Chunk<P>::NC;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nch; i += (size_t)gridDim.x * blockDim.x) {
        cplx<R> rv[NC];
        Chunk<P>::ld(r, i, rv);
        for (int j = 0; j < ns; ++j) {
            if (!c.upd[j]) continue;
            cplx<R> xv[NC], pv[NC];
            Chunk<P>::ld(ptr.x[j], i, xv);
            Chunk<P>::ld(ptr.p[j], i, pv);
            const R a = (R)c.alpha[j], z = (R)c.zeta[j], bb = (R)c.beta[j];
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                xv[q].re = fma(a, pv[q].re, xv[q].re);
                xv[q].im = fma(a, pv[q].im, xv[q].im);
                pv[q].re = fma(z, rv[q].re, bb * pv[q].re);
                pv[q].im = fma(z, rv[q].im, bb * pv[q].im);
            }
            Chunk<P>::st(ptr.x[j], i, xv);
            Chunk<P>::st(ptr.p[j], i, pv);
        }
    }
}

int blas_axpby_dev(qxd_ctx* ctx, int P, size_t n, const double* c, const void* x, void* y, cudaStream_t st) {
    const size_t nc = nchunks(P, n);
    const int nb = upd_blocks(ctx, nc);
    ProfScope prof(ctx, "axpby", (double)n * 3 * eb(P), st);
    if (P == 0) k_axpby_dev<0><<<nb, 256, 0, st>>>(nc, c, x, y);
    else if (P == 1) k_axpby_dev<1><<<nb, 256, 0, st>>>(nc, c, x, y);
    else k_axpby_dev<2><<<nb, 256, 0, st>>>(nc, c, x, y);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int blas_axpy_norm_dev(qxd_ctx* ctx, int P, size_t n, const double* c, const void* x, void* y, int slot,
                       cudaStream_t st) {
    const size_t nc = nchunks(P, n);
    ProfScope prof(ctx, "multi_axpy_norm", (double)n * 3 * eb(P), st);
    const RedOut o = red_out(ctx, slot);
    const size_t wpb = (size_t)kRedThreads * 2;
#define QXD_LAUNCH(Q) \
    k_axpy_norm_dev<Q><<<wave_blocks(ctx, k_axpy_norm_dev<Q>, kRedThreads, wpb, nc), kRedThreads, 0, st>>>(nc, c, x, y, o)
    if (P == 0) QXD_LAUNCH(0);
    else if (P == 1) QXD_LAUNCH(1);
    else QXD_LAUNCH(2);
#undef QXD_LAUNCH
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int blas_msg_update_dev(qxd_ctx* ctx, int P, size_t n, int ns, const ShiftPtrs& ptr, const ShiftCoefDev& c,
                        const void* r, cudaStream_t st) {
    if (ns < 1 || ns > kMaxShifts) return qxd_fail(ctx, QXD_EARG, "msg_update: shift count out of range");
    const size_t nc = nchunks(P, n);
    const int nb = upd_blocks(ctx, nc);
    ProfScope prof(ctx, "msg_update", (double)n * eb(P) * (1 + 4 * ns), st);
    if (P == 0) k_msg_update_dev<0><<<nb, 256, 0, st>>>(nc, ns, ptr, c, r);
    else if (P == 1) k_msg_update_dev<1><<<nb, 256, 0, st>>>(nc, ns, ptr, c, r);
    else k_msg_update_dev<2><<<nb, 256, 0, st>>>(nc, ns, ptr, c, r);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int blas_fetch(qxd_ctx* ctx, int nslots, cudaStream_t st) {
    QXD_CUDA(ctx, cudaMemcpyAsync(ctx->red_host, ctx->red_result, sizeof(double) * nslots, cudaMemcpyDeviceToHost, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

}  // namespace qxd
