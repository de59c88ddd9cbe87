// Hopping kernels of the Wilson-Dirac operator (Sec. 2.3):
//   (H psi)(x) = -1/2 sum_mu [(1 - gamma_mu) V(x,mu) psi(x+mu) + (1 + gamma_mu) V(x-mu,mu)^+ psi(x-mu)]
// with V = U z^qhat, evaluated for all sites of one parity from a field on the
// other parity (even-odd preconditioning, Sec. 2.3).  One thread per output
// site; the neighbour indices are computed on the fly from the coordinates
// (C* shifted boundaries included); (1 -+ gamma_mu) are applied as spin
// projections onto two-spinors before the colour multiplication.
#include <cstdio>
#include <tuple>

#include "hop.cuh"
#include "qxd_internal.h"

namespace qxd {

static const char* prec_name(int P) { return P == 0 ? "fp64" : (P == 1 ? "fp32" : (P == 2 ? "bf16" : "df64")); }
static double spinor_bytes(int P) { return (P == 0 || P == 3) ? 192.0 : (P == 1 ? 96.0 : 48.0); }
static double link_bytes(int P) { return (P == 0 || P == 3) ? 144.0 : 56.0; }   // V (FP64) or 2 rows of U + z (FP32)
static double diag_bytes(int P) { return (P == 0 || P == 3) ? 576.0 : 288.0; }

// MINB: resident blocks per SM the register allocation must allow (launch bound);
// the double-float kernel is compiled for several and the fastest is picked per lattice
template <int P, int SELF, int POST, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_hop(Geo g, HopDev a) {
    using R = typename Prec<P>::real;
    using CH = typename Prec<P>::chunk;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const size_t rhs_off = (size_t)blockIdx.y * Prec<P>::nchunk * g.Vh;
    const CH* in = static_cast<const CH*>(a.in_nb) + rhs_off;
    int x[4];
    site_coords(g, a.pout, h, x);
    cplx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    hop_dir<P, 0>(g, a, in, x, h, acc);
    hop_dir<P, 1>(g, a, in, x, h, acc);
    hop_dir<P, 2>(g, a, in, x, h, acc);
    hop_dir<P, 3>(g, a, in, x, h, acc);
    const R c = R(-0.5 * a.c_hop);
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = c * acc[k];
    if constexpr (SELF != 0) {
        cplx<R> s[12];
        load_spinor<P>(static_cast<const CH*>(a.in_self) + rhs_off, g.Vh, h, s);
        if (a.g5_self) {
#pragma unroll
            for (int k = 6; k < 12; ++k) s[k] = -s[k];
        }
        if constexpr (SELF == 1) {
            R d[72];
            load_diag<P == 0 ? 0 : (P == 3 ? 3 : 1)>(a.diag, g.Vh, h, d);
            apply_diag(d, s);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = acc[k] + s[k];
    }
    if constexpr (POST == 1) {
        if constexpr (P == 3) {
            // the lazy double-float sums are renormalised before they become factors
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = {df_norm(acc[k].re), df_norm(acc[k].im)};
        }
        R d[72];
        load_diag<P == 0 ? 0 : (P == 3 ? 3 : 1)>(a.diaginv, g.Vh, h, d);
        apply_diag(d, acc);
    }
    if (a.g5_out) {
#pragma unroll
        for (int k = 6; k < 12; ++k) acc[k] = -acc[k];
    }
    store_spinor<P>(static_cast<CH*>(a.out) + rhs_off, g.Vh, h, acc);
}

template <int P>
__global__ void __launch_bounds__(kThreads) k_diag(Geo g, const void* __restrict__ diag, const void* __restrict__ in,
                                                   void* __restrict__ out, int g5) {
    using R = typename Prec<P>::real;
    using CH = typename Prec<P>::chunk;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const size_t rhs_off = (size_t)blockIdx.y * Prec<P>::nchunk * g.Vh;
    cplx<R> s[12];
    load_spinor<P>(static_cast<const CH*>(in) + rhs_off, g.Vh, h, s);
    R d[72];
    load_diag<P == 0 ? 0 : 1>(diag, g.Vh, h, d);
    apply_diag(d, s);
    if (g5) {
#pragma unroll
        for (int k = 6; k < 12; ++k) s[k] = -s[k];
    }
    store_spinor<P>(static_cast<CH*>(out) + rhs_off, g.Vh, h, s);
}

// ---- double-float hop with two threads per site --------------------------------------
// The pair of adjacent lanes (2k, 2k+1) shares one output site; lane `half` forms the
// half-spinor component half of every spin projection (spins half and its partner),
// multiplies it by the link and adds it into the output spin half (accO) and into the
// lower spins it feeds: accP (spin 2 + half: directions 0 and 3) or accQ (spin
// 3 - half: directions 1 and 2).  Every lane runs the same instruction stream (the
// half only selects addresses and signs), so the pair does not diverge.  At the end
// the lanes exchange their partial sums: lane 0 owns the upper chiral block (spins 0,
// 1), lane 1 the lower one (spins 2, 3), each applying its 6 x 6 site-diagonal block.
// Per lane this halves the arithmetic and the live registers of the one-thread kernel.
using cdf = cplx<dfl>;

__device__ __forceinline__ void load3_df(const float4* __restrict__ base, int Vh, int h, int sp, cdf v[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 f = QXD_LDG(base + (size_t)(3 * sp + c) * Vh + h);
        v[c] = {dfl(f.x, f.y), dfl(f.z, f.w)};
    }
}
__device__ __forceinline__ cdf mul_i(cdf a) { return {-a.im, a.re}; }
__device__ __forceinline__ cdf scale_sign(cdf a, bool neg) { return neg ? cdf{-a.re, -a.im} : a; }

// one hop direction (MU, FWD) for this lane: its half-spinor component, times the link
template <int MU, bool FWD>
__device__ __forceinline__ void hop_half_df(const Geo& g, const HopDev& a, const float4* __restrict__ in,
                                            const int x[4], int h, int half, bool g5nb, cdf accO[3], cdf accP[3],
                                            cdf accQ[3]) {
    const int Vh = g.Vh;
    const int n = neighbour_lex(g, x, MU, FWD ? +1 : -1) >> 1;
    // spins of this lane's projection: (half, partner)
    const int partner = (MU == 0 || MU == 3) ? 2 + half : 3 - half;
    cdf sa[3], sb[3];
    load3_df(in, Vh, n, half, sa);
    load3_df(in, Vh, n, partner, sb);
    if (g5nb) {
#pragma unroll
        for (int c = 0; c < 3; ++c) sb[c] = {-sb[c].re, -sb[c].im};  // the partner is a lower spin
    }
    // projection: hp = s_half + f s_partner with f = +-1 or +-i (the one-thread kernel's
    // project<MU, FWD> for component `half`)
    cdf hp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (MU == 0) hp[c] = FWD ? sa[c] + sb[c] : sa[c] - sb[c];
        else if (MU == 1) hp[c] = FWD ? sa[c] + mul_i(sb[c]) : sa[c] - mul_i(sb[c]);
        else if (MU == 2) hp[c] = sa[c] + scale_sign(sb[c], FWD == (half == 1));
        else hp[c] = sa[c] + scale_sign(mul_i(sb[c]), FWD == (half == 1));
    }
    // colour: r = V hp (forward, link of x) or V^+ hp (backward, link of the neighbour)
    const float4* V = FWD ? a.Vdf_out : a.Vdf_in;
    const int hl = FWD ? h : n;
    cdf r[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) r[i] = {dfl(0.0), dfl(0.0)};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int e = FWD ? i * 3 + j : j * 3 + i;
            const float4 f = QXD_LDG(V + (size_t)(MU * 9 + e) * Vh + hl);
            const cdf m = {dfl(f.x, f.y), dfl(f.z, f.w)};
            if (FWD) cmac(r[i], m, hp[j]);
            else cmac_conj(r[i], m, hp[j]);
        }
    // reconstruction (the one-thread kernel's reconstruct<MU, FWD> for component `half`)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        accO[c] = accO[c] + r[c];
        if (MU == 0) accP[c] = FWD ? accP[c] + r[c] : accP[c] - r[c];
        else if (MU == 1) accQ[c] = FWD ? accQ[c] - mul_i(r[c]) : accQ[c] + mul_i(r[c]);
        else if (MU == 2) accQ[c] = accQ[c] + scale_sign(r[c], FWD == (half == 1));
        else accP[c] = accP[c] + scale_sign(mul_i(r[c]), FWD == (half == 0));
    }
}

template <int SELF, int POST, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_hop_df2(Geo g, HopDev a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int h = t >> 1;
    const int half = t & 1;
    const bool live = h < g.Vh;
    const int hh = live ? h : g.Vh - 1;  // the pair's lanes stay together for the exchange
    const size_t rhs_off = (size_t)blockIdx.y * 12 * g.Vh;
    const float4* in = static_cast<const float4*>(a.in_nb) + rhs_off;
    int x[4];
    site_coords(g, a.pout, hh, x);
    cdf accO[3], accP[3], accQ[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) accO[c] = accP[c] = accQ[c] = {dfl(0.0), dfl(0.0)};
    const bool g5nb = a.g5_nb != 0;
    hop_half_df<0, true>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<0, false>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<1, true>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<1, false>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<2, true>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<2, false>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<3, true>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    hop_half_df<3, false>(g, a, in, x, hh, half, g5nb, accO, accP, accQ);
    // exchange: lane 0 takes spins 0 (own accO) and 1 (partner's accO); lane 1 takes
    // spin 2 = lane0.accP + lane1.accQ and spin 3 = lane0.accQ + lane1.accP
    cdf pO[3], pP[3], pQ[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        auto sh = [](dfl v) {
            return dfl(__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1));
        };
        pO[c] = {sh(accO[c].re), sh(accO[c].im)};
        pP[c] = {sh(accP[c].re), sh(accP[c].im)};
        pQ[c] = {sh(accQ[c].re), sh(accQ[c].im)};
    }
    if (!live) return;
    const dfl ch(-0.5 * a.c_hop);
    cdf v[6];  // this lane's chiral block: spins (2 half, 2 half + 1) x colours
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cdf s0 = half == 0 ? accO[c] : pP[c] + accQ[c];
        const cdf s1 = half == 0 ? pO[c] : pQ[c] + accP[c];
        v[c] = {ch * s0.re, ch * s0.im};
        v[3 + c] = {ch * s1.re, ch * s1.im};
    }
    const size_t dstride = (size_t)g.Vh;
    if constexpr (SELF != 0) {
        cdf s[6];
        const float4* self = static_cast<const float4*>(a.in_self) + rhs_off;
        load3_df(self, g.Vh, h, 2 * half, s);
        load3_df(self, g.Vh, h, 2 * half + 1, s + 3);
        if (a.g5_self && half == 1) {
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k] = {-s[k].re, -s[k].im};
        }
        if constexpr (SELF == 1) {
            dfl d[36];
            const float4* D = static_cast<const float4*>(a.diag) + (size_t)half * 18 * dstride;
#pragma unroll
            for (int k = 0; k < 18; ++k) {
                const float4 f = QXD_LDG(D + (size_t)k * dstride + h);
                d[2 * k] = dfl(f.x, f.y);
                d[2 * k + 1] = dfl(f.z, f.w);
            }
            cdf o[6];
            herm6_mul(d, s, o);
#pragma unroll
            for (int k = 0; k < 6; ++k) s[k] = o[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = v[k] + s[k];
    }
    if constexpr (POST == 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = {df_norm(v[k].re), df_norm(v[k].im)};
        dfl d[36];
        const float4* D = static_cast<const float4*>(a.diaginv) + (size_t)half * 18 * dstride;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const float4 f = QXD_LDG(D + (size_t)k * dstride + h);
            d[2 * k] = dfl(f.x, f.y);
            d[2 * k + 1] = dfl(f.z, f.w);
        }
        cdf o[6];
        herm6_mul(d, v, o);
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = o[k];
    }
    if (a.g5_out && half == 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = {-v[k].re, -v[k].im};
    }
    float4* out = static_cast<float4*>(a.out) + rhs_off;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const int comp = 6 * half + k;  // complex index 3 spin + colour
        const dfl re = df_norm(v[k].re), im = df_norm(v[k].im);
        out[(size_t)comp * g.Vh + h] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

// --- host dispatch ---------------------------------------------------------------
template <int P, int SELF, int POST>
static void launch_hop_t(const Geo& g, const HopDev& d, int nrhs, cudaStream_t st, int minb) {
    dim3 grid(nblocks(g.Vh), nrhs);
    if constexpr (P == 3) {
        if (minb == 2) k_hop<P, SELF, POST, 2><<<grid, kThreads, 0, st>>>(g, d);
        else if (minb == 3) k_hop<P, SELF, POST, 3><<<grid, kThreads, 0, st>>>(g, d);
        else k_hop<P, SELF, POST, 4><<<grid, kThreads, 0, st>>>(g, d);
    } else {
        k_hop<P, SELF, POST, 1><<<grid, kThreads, 0, st>>>(g, d);
    }
}

template <int SELF, int POST>
static void launch_hop_df2_t(const Geo& g, const HopDev& d, int nrhs, cudaStream_t st, int minb) {
    dim3 grid(nblocks(2ll * g.Vh), nrhs);
    if (minb == 5) k_hop_df2<SELF, POST, 5><<<grid, kThreads, 0, st>>>(g, d);
    else k_hop_df2<SELF, POST, 4><<<grid, kThreads, 0, st>>>(g, d);
}

// the double-float operators use two modes: D_w (self 1, post 0) and the first half
// of Dhat (self 0, post 1); only these are compiled
static void launch_hop_df(const Geo& g, const HopDev& d, int self, int post, int nrhs, cudaStream_t st, int minb) {
    if (minb < 0) {  // two threads per site, launch bound -minb CTAs per SM
        if (self == 1) launch_hop_df2_t<1, 0>(g, d, nrhs, st, -minb);
        else launch_hop_df2_t<0, 1>(g, d, nrhs, st, -minb);
    } else {
        if (self == 1) launch_hop_t<3, 1, 0>(g, d, nrhs, st, minb);
        else launch_hop_t<3, 0, 1>(g, d, nrhs, st, minb);
    }
}

template <int P>
static void launch_hop_p(const Geo& g, const HopDev& d, int self, int post, int nrhs, cudaStream_t st,
                         int minb = 1) {
    if (self == 0 && post == 0) launch_hop_t<P, 0, 0>(g, d, nrhs, st, minb);
    else if (self == 0 && post == 1) launch_hop_t<P, 0, 1>(g, d, nrhs, st, minb);
    else if (self == 1 && post == 0) launch_hop_t<P, 1, 0>(g, d, nrhs, st, minb);
    else if (self == 1 && post == 1) launch_hop_t<P, 1, 1>(g, d, nrhs, st, minb);
    else if (self == 2 && post == 0) launch_hop_t<P, 2, 0>(g, d, nrhs, st, minb);
    else launch_hop_t<P, 2, 1>(g, d, nrhs, st, minb);
}

// Double-float hop: one thread per site with the launch bound 2, 3 or 4 resident
// blocks per SM (up to 255, 168 or 128 registers per thread; codes 2, 3, 4), or two
// threads per site (k_hop_df2) with 4 or 5 (128 or 96 registers; codes -4, -5);
// chosen per (mode, nrhs, lattice) by timing the five on the caller's data on first use (the kernel reads its
// inputs and writes a distinct output, so repeating it is harmless); the choice
// is cached in the context like the multi-right-hand-side shapes.
static int launch_hop_df64(qxd_ctx* ctx, const HopDev& d, const HopArgs& a, cudaStream_t st) {
    const Geo& g = ctx->g;
    if (!((a.self_mode == 1 && a.post_mode == 0) || (a.self_mode == 0 && a.post_mode == 1)))
        return qxd_fail(ctx, QXD_EARG, "double-float hop: only D_w and the first half of Dhat are compiled");
    const auto key = std::make_tuple((int)QXD_DF64, a.self_mode, a.post_mode, a.nrhs, (long long)g.Vh);
    auto it = ctx->tune_hop.find(key);
    int minb = 4;
    if (it != ctx->tune_hop.end()) {
        minb = it->second.first;
    } else if (!t_no_autotune) {
        cudaEvent_t e0, e1;
        QXD_CUDA(ctx, cudaEventCreate(&e0));
        QXD_CUDA(ctx, cudaEventCreate(&e1));
        float best = 1e30f;
        for (int mb : {-4, -5, 2, 3, 4}) {
            launch_hop_df(g, d, a.self_mode, a.post_mode, a.nrhs, st, mb);
            QXD_CUDA(ctx, cudaEventRecord(e0, st));
            for (int rep = 0; rep < 3; ++rep) launch_hop_df(g, d, a.self_mode, a.post_mode, a.nrhs, st, mb);
            QXD_CUDA(ctx, cudaEventRecord(e1, st));
            QXD_CUDA(ctx, cudaEventSynchronize(e1));
            float ms = 0.f;
            QXD_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                minb = mb;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->tune_hop.emplace(key, std::make_pair(minb, kThreads));
    }
    launch_hop_df(g, d, a.self_mode, a.post_mode, a.nrhs, st, minb);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int launch_hop(qxd_ctx* ctx, int fl, int prec, const HopArgs& a, cudaStream_t st) {
    const Geo& g = ctx->g;
    const QxdFlavour& F = ctx->fl[fl];
    const size_t Vh = g.Vh;
    const int po = a.pout, pi = 1 - a.pout;
    HopDev d;
    d.pout = po;
    d.in_nb = a.in_nb;
    d.in_self = a.in_self;
    d.out = a.out;
    d.V64_out = F.V64 + (size_t)po * 36 * Vh;
    d.V64_in = F.V64 + (size_t)pi * 36 * Vh;
    d.Vdf_out = F.Vdf + (size_t)po * 36 * Vh;
    d.Vdf_in = F.Vdf + (size_t)pi * 36 * Vh;
    d.U32_out = ctx->U32 + (size_t)po * 12 * Vh;
    d.U32_in = ctx->U32 + (size_t)pi * 12 * Vh;
    d.Z32_out = F.Z32 + (size_t)po * 2 * Vh;
    d.Z32_in = F.Z32 + (size_t)pi * 2 * Vh;
    if (prec == QXD_FP64) {
        d.diag = F.C64[0] + (size_t)po * 36 * Vh;
        d.diaginv = F.C64[1] + (size_t)po * 36 * Vh;
    } else if (prec == QXD_DF64) {
        // the copies are built by ensure_df64 (the inverse only for operators that need it)
        if (!F.Vdf || !F.Cdf[0] || (a.post_mode == 1 && !F.Cdf[1]))
            return qxd_fail(ctx, QXD_ESTATE, "double-float hop: copies of the flavour not built");
        d.diag = F.Cdf[0] + (size_t)po * 36 * Vh;
        d.diaginv = F.Cdf[1] ? F.Cdf[1] + (size_t)po * 36 * Vh : nullptr;
    } else {
        d.diag = F.C32[0] + (size_t)po * 18 * Vh;
        d.diaginv = F.C32[1] + (size_t)po * 18 * Vh;
    }
    d.c_hop = a.c_hop;
    d.g5_nb = a.g5_nb;
    d.g5_self = a.g5_self;
    d.g5_out = a.g5_out;
    // algorithmic bytes: links of both parities touching the output sites and the
    // site-diagonal terms once, spinors (neighbour, self, output) once per right-hand side
    char name[48];
    // FP32 and BF16 go through the autotuned multi-right-hand-side kernel (also
    // for one right-hand side); FP64 and double-float keep the one-site-per-thread kernel
    const bool mr = prec == QXD_FP32 || prec == QXD_BF16;
    std::snprintf(name, sizeof name, "hop_%s_self%d_post%d%s", prec_name(prec), a.self_mode, a.post_mode,
                  a.nrhs > 1 ? "_mrhs" : "");
    const double per_rhs = spinor_bytes(prec) * (2 + (a.self_mode ? 1 : 0));
    const double once = 8 * link_bytes(prec) + diag_bytes(prec) * ((a.self_mode == 1) + (a.post_mode == 1));
    ProfScope prof(ctx, name, (double)Vh * (once + per_rhs * a.nrhs), st);
    if (mr) {
        int nr = 1;
        return launch_hop_mr(ctx, prec, d, a, st, &nr);
    }
    if (prec == QXD_FP64) launch_hop_p<0>(g, d, a.self_mode, a.post_mode, a.nrhs, st);
    else if (prec == QXD_DF64) return launch_hop_df64(ctx, d, a, st);
    else if (prec == QXD_FP32) launch_hop_p<1>(g, d, a.self_mode, a.post_mode, a.nrhs, st);
    else launch_hop_p<2>(g, d, a.self_mode, a.post_mode, a.nrhs, st);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int launch_diag(qxd_ctx* ctx, int fl, int prec, int p, int inv, const void* in, void* out, int nrhs,
                cudaStream_t st) {
    const Geo& g = ctx->g;
    const QxdFlavour& F = ctx->fl[fl];
    const size_t Vh = g.Vh;
    dim3 grid(nblocks(g.Vh), nrhs);
    char name[32];
    std::snprintf(name, sizeof name, "diag_%s", prec_name(prec));
    ProfScope prof(ctx, name, (double)Vh * (diag_bytes(prec) + 2 * spinor_bytes(prec) * nrhs), st);
    if (prec == QXD_FP64)
        k_diag<0><<<grid, kThreads, 0, st>>>(g, F.C64[inv] + (size_t)p * 36 * Vh, in, out, 0);
    else if (prec == QXD_FP32)
        k_diag<1><<<grid, kThreads, 0, st>>>(g, F.C32[inv] + (size_t)p * 18 * Vh, in, out, 0);
    else
        k_diag<2><<<grid, kThreads, 0, st>>>(g, F.C32[inv] + (size_t)p * 18 * Vh, in, out, 0);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

}  // namespace qxd
