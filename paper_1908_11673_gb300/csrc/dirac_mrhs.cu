// Multi-right-hand-side hopping kernel: one thread applies the hopping term at
// one site to NR right-hand sides, loading each link (and the site-diagonal
// term) once for all of them.  The blocks of the NR-groups of a tile of sites
// are adjacent in launch order, so the groups after the first find the links
// in L2: every link crosses HBM once per launch.  (NR, threads per block) are
// chosen per (precision, mode, number of right-hand sides, volume) by timing
// the candidates on the first call (autotuner, cached in the context).
#include <algorithm>
#include <cstdio>
#include <map>
#include <tuple>

#include "hop.cuh"
#include "qxd_internal.h"

namespace qxd {

template <int P, int MU, int NR, typename R>
QXD_HD void hop_dir_mr(const Geo& g, const HopDev& a, const typename Prec<P>::chunk* __restrict__ in, size_t rstride,
                       int nv, const int x[4], int h, cplx<R> acc[NR][12]) {
    const int Vh = g.Vh;
    const int nf = neighbour_lex(g, x, MU, +1) >> 1;
    const int nb = neighbour_lex(g, x, MU, -1) >> 1;
    Mat3<R> m;
    cplx<float> z;
    // forward: (1 - gamma_mu) V(x,mu) psi(x+mu)
    if constexpr (P == 0) load_link64(a.V64_out, Vh, MU, h, m);
    else load_link32(a.U32_out, a.Z32_out, Vh, MU, h, m, z);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r >= nv) break;
        cplx<R> s[12];
        Half<R> hp, o;
        load_spinor<P>(in + r * rstride, Vh, nf, s);
        if (a.g5_nb) {
#pragma unroll
            for (int k = 6; k < 12; ++k) s[k] = -s[k];
        }
        project<MU, true>(s, hp);
        mul_half<false>(m, hp, o);
        if constexpr (P != 0) {
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.a[sp][c] = z * o.a[sp][c];
        }
        reconstruct<MU, true>(o, acc[r]);
    }
    // backward: (1 + gamma_mu) V(x-mu,mu)^+ psi(x-mu)
    if constexpr (P == 0) load_link64(a.V64_in, Vh, MU, nb, m);
    else load_link32(a.U32_in, a.Z32_in, Vh, MU, nb, m, z);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r >= nv) break;
        cplx<R> s[12];
        Half<R> hp, o;
        load_spinor<P>(in + r * rstride, Vh, nb, s);
        if (a.g5_nb) {
#pragma unroll
            for (int k = 6; k < 12; ++k) s[k] = -s[k];
        }
        project<MU, false>(s, hp);
        mul_half<true>(m, hp, o);
        if constexpr (P != 0) {
#pragma unroll
            for (int sp = 0; sp < 2; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.a[sp][c] = cmul_conj(z, o.a[sp][c]);
        }
        reconstruct<MU, false>(o, acc[r]);
    }
}

// 1-D grid: block b covers right-hand-side group b % ngroups of site tile b / ngroups
template <int P, int SELF, int POST, int NR>
__global__ void k_hop_mr(Geo g, HopDev a, int nrhs, int ngroups) {
    using R = typename Prec<P>::real;
    using CH = typename Prec<P>::chunk;
    const int grp = blockIdx.x % ngroups;
    const int tile = blockIdx.x / ngroups;
    const int h = tile * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const int r0 = grp * NR;
    const int nv = min(NR, nrhs - r0);
    const size_t rstride = (size_t)Prec<P>::nchunk * g.Vh;
    const CH* in = static_cast<const CH*>(a.in_nb) + r0 * rstride;
    int x[4];
    site_coords(g, a.pout, h, x);
    cplx<R> acc[NR][12];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = {R(0), R(0)};
    hop_dir_mr<P, 0, NR>(g, a, in, rstride, nv, x, h, acc);
    hop_dir_mr<P, 1, NR>(g, a, in, rstride, nv, x, h, acc);
    hop_dir_mr<P, 2, NR>(g, a, in, rstride, nv, x, h, acc);
    hop_dir_mr<P, 3, NR>(g, a, in, rstride, nv, x, h, acc);
    const R c = R(-0.5 * a.c_hop);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        if (r >= nv) break;
        const size_t off = (size_t)(r0 + r) * rstride;
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[r][k] = c * acc[r][k];
        if constexpr (SELF != 0) {
            cplx<R> s[12];
            load_spinor<P>(static_cast<const CH*>(a.in_self) + off, g.Vh, h, s);
            if (a.g5_self) {
#pragma unroll
                for (int k = 6; k < 12; ++k) s[k] = -s[k];
            }
            if constexpr (SELF == 1) {
                R d[72];
                load_diag<P == 0 ? 0 : 1>(a.diag, g.Vh, h, d);
                apply_diag(d, s);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[r][k] = acc[r][k] + s[k];
        }
        if constexpr (POST == 1) {
            R d[72];
            load_diag<P == 0 ? 0 : 1>(a.diaginv, g.Vh, h, d);
            apply_diag(d, acc[r]);
        }
        if (a.g5_out) {
#pragma unroll
            for (int k = 6; k < 12; ++k) acc[r][k] = -acc[r][k];
        }
        store_spinor<P>(static_cast<CH*>(a.out) + off, g.Vh, h, acc[r]);
    }
}

template <int P, int SELF, int POST>
static void launch_nr(int nr, int threads, const Geo& g, const HopDev& d, int nrhs, cudaStream_t st) {
    const int ngroups = (nrhs + nr - 1) / nr;
    const int tiles = nblocks(g.Vh, threads);
    const int grid = ngroups * tiles;
    switch (nr) {
        case 1: k_hop_mr<P, SELF, POST, 1><<<grid, threads, 0, st>>>(g, d, nrhs, ngroups); break;
        case 2: k_hop_mr<P, SELF, POST, 2><<<grid, threads, 0, st>>>(g, d, nrhs, ngroups); break;
        default: k_hop_mr<P, SELF, POST, 4><<<grid, threads, 0, st>>>(g, d, nrhs, ngroups); break;
    }
}

template <int P>
static void launch_mode(int self, int post, int nr, int threads, const Geo& g, const HopDev& d, int nrhs,
                        cudaStream_t st) {
    if (self == 0 && post == 0) launch_nr<P, 0, 0>(nr, threads, g, d, nrhs, st);
    else if (self == 0 && post == 1) launch_nr<P, 0, 1>(nr, threads, g, d, nrhs, st);
    else if (self == 1 && post == 0) launch_nr<P, 1, 0>(nr, threads, g, d, nrhs, st);
    else if (self == 1 && post == 1) launch_nr<P, 1, 1>(nr, threads, g, d, nrhs, st);
    else if (self == 2 && post == 0) launch_nr<P, 2, 0>(nr, threads, g, d, nrhs, st);
    else launch_nr<P, 2, 1>(nr, threads, g, d, nrhs, st);
}

static void launch_cfg(int prec, int self, int post, int nr, int threads, const Geo& g, const HopDev& d, int nrhs,
                       cudaStream_t st) {
    if (prec == QXD_FP32) launch_mode<1>(self, post, nr, threads, g, d, nrhs, st);
    else launch_mode<2>(self, post, nr, threads, g, d, nrhs, st);
}

// Autotuner: candidate (NR, threads) pairs timed on the caller's own data (the
// kernel reads in_nb/in_self and writes out, which do not overlap, so
// repeating it is harmless); the fastest is kept for this key.
thread_local bool t_no_autotune = false;

int launch_hop_mr(qxd_ctx* ctx, int prec, const HopDev& d, const HopArgs& a, cudaStream_t st, int* nr_used) {
    const Geo& g = ctx->g;
    const auto key = std::make_tuple(prec, a.self_mode, a.post_mode, a.nrhs, (long long)g.Vh);
    auto it = ctx->tune_hop.find(key);
    if (it == ctx->tune_hop.end() && t_no_autotune) {
        // untuned key while tuning is off: the default shape, nothing timed or cached
        *nr_used = 1;
        launch_cfg(prec, a.self_mode, a.post_mode, 1, 128, g, d, a.nrhs, st);
        QXD_CUDA(ctx, cudaGetLastError());
        return QXD_OK;
    }
    if (it == ctx->tune_hop.end()) {
        const int nrs[3] = {1, 2, 4};
        const int ths[3] = {64, 128, 256};
        cudaEvent_t e0, e1;
        QXD_CUDA(ctx, cudaEventCreate(&e0));
        QXD_CUDA(ctx, cudaEventCreate(&e1));
        float best = 1e30f;
        std::pair<int, int> pick{1, 128};
        for (int nr : nrs) {
            if (nr > 1 && nr > a.nrhs) continue;
            for (int th : ths) {
                if (nr == 4 && th == 256) continue;  // register file: 4 x 256 x ~200 registers per block
                launch_cfg(prec, a.self_mode, a.post_mode, nr, th, g, d, a.nrhs, st);
                QXD_CUDA(ctx, cudaEventRecord(e0, st));
                for (int rep = 0; rep < 3; ++rep) launch_cfg(prec, a.self_mode, a.post_mode, nr, th, g, d, a.nrhs, st);
                QXD_CUDA(ctx, cudaEventRecord(e1, st));
                QXD_CUDA(ctx, cudaEventSynchronize(e1));
                float ms = 0.f;
                QXD_CUDA(ctx, cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    pick = {nr, th};
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        it = ctx->tune_hop.emplace(key, pick).first;
    }
    *nr_used = it->second.first;
    launch_cfg(prec, a.self_mode, a.post_mode, it->second.first, it->second.second, g, d, a.nrhs, st);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

}  // namespace qxd
