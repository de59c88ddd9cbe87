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

// Double-float hop: the launch bound (2, 3 or 4 resident blocks per SM, i.e. up
// to 255, 168 or 128 registers per thread) is chosen per (mode, nrhs, lattice) by
// timing the three on the caller's data on first use (the kernel reads its
// inputs and writes a distinct output, so repeating it is harmless); the choice
// is cached in the context like the multi-right-hand-side shapes.
static int launch_hop_df64(qxd_ctx* ctx, const HopDev& d, const HopArgs& a, cudaStream_t st) {
    const Geo& g = ctx->g;
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
        for (int mb : {2, 3, 4}) {
            launch_hop_p<3>(g, d, a.self_mode, a.post_mode, a.nrhs, st, mb);
            QXD_CUDA(ctx, cudaEventRecord(e0, st));
            for (int rep = 0; rep < 3; ++rep) launch_hop_p<3>(g, d, a.self_mode, a.post_mode, a.nrhs, st, mb);
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
    launch_hop_p<3>(g, d, a.self_mode, a.post_mode, a.nrhs, st, minb);
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
