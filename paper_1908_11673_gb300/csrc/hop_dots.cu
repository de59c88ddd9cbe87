// Second half of Dhat with the inner products of a GCR step fused into its epilogue
// (Sec. 2.3 operator; the solver of Sec. 4.4).
//
//   w = A_ee r - H_eo t,   t = A_oo^-1 H_oe r  (the first half, an ordinary launch)
//
// The GCR step that applies Dhat to its direction r (the current residual, when the
// solve has no preconditioner) next needs <W_j, w> for the K earlier basis fields,
// <r, w> and |w|^2.  Here the thread that has just formed w(x) reads W_j(x) and
// accumulates them, so the step saves the separate pass that would read w, r and
// every W_j once more.  FP32 fields, one right-hand side, no gamma5 flags.
//
// Sums: FP32 over the components of a site and over at most eight sites of a
// thread, FP64 beyond, and the grid's partial sums added by the last block in block
// order (reduce.cuh): the result is the same on every run.
//   result[slot + 2j], [slot + 2j + 1]  = <W_j, w>  (j < K)
//   result[slot + 2K], [slot + 2K + 1]  = <r, w>
//   result[slot + 2K + 2]               = |w|^2 over the sites where it is finite
//   result[slot + 2K + 3]               = the number of the other sites
#include "blas.h"
#include "hop.cuh"
#include "ops.h"
#include "reduce.cuh"

namespace qxd {

namespace {

__device__ __forceinline__ void dot_site(const cplx<float> x[12], const cplx<float> w[12], float& re, float& im) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        re = fmaf(x[i].re, w[i].re, fmaf(x[i].im, w[i].im, re));
        im = fmaf(x[i].re, w[i].im, fmaf(-x[i].im, w[i].re, im));
    }
}

// grid-stride over the output sites, one wave of resident blocks; each thread keeps
// FP32 sums over up to kDotsFlush sites in registers and adds them into FP64 sums in
// shared memory (the FP64 accumulators would not fit the registers of the hop)
constexpr int kDotsFlush = 8;

template <int K>
__global__ void __launch_bounds__(kRedThreads, 2) k_hop_dots(Geo g, HopDev a, MultiPtr W, RedOut o) {
    constexpr int NC = 2 * K + 4;
    __shared__ double vs[NC][kRedThreads];
    float fa[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        vs[c][threadIdx.x] = 0.0;
        fa[c] = 0.f;
    }
    const float4* in = static_cast<const float4*>(a.in_nb);
    const float4* rin = static_cast<const float4*>(a.in_self);
    float4* out = static_cast<float4*>(a.out);
    const int S = gridDim.x * blockDim.x;
    int cnt = 0;
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Vh; h += S) {
        int x[4];
        site_coords(g, a.pout, h, x);
        cplx<float> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
        hop_dir<1, 0>(g, a, in, x, h, acc);
        hop_dir<1, 1>(g, a, in, x, h, acc);
        hop_dir<1, 2>(g, a, in, x, h, acc);
        hop_dir<1, 3>(g, a, in, x, h, acc);
        const float c = (float)(-0.5 * a.c_hop);
        {
            cplx<float> s[12];
            load_spinor<1>(rin, g.Vh, h, s);
            float d[72];
            load_diag<1>(a.diag, g.Vh, h, d);
            apply_diag(d, s);
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = c * acc[k] + s[k];
        }
        store_spinor<1>(out, g.Vh, h, acc);
#pragma unroll
        for (int j = 0; j <= K; ++j) {  // the K basis fields, then r
            cplx<float> wj[12];
            load_spinor<1>(j < K ? static_cast<const float4*>(W.p[j]) : rin, g.Vh, h, wj);
            dot_site(wj, acc, fa[2 * j], fa[2 * j + 1]);
        }
        float ww = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) ww = fmaf(acc[k].re, acc[k].re, fmaf(acc[k].im, acc[k].im, ww));
        if (isfinite(ww)) fa[2 * K + 2] += ww;
        else fa[2 * K + 3] += 1.f;
        if (++cnt == kDotsFlush) {
            cnt = 0;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                vs[q][threadIdx.x] += fa[q];
                fa[q] = 0.f;
            }
        }
    }
    double v[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = vs[q][threadIdx.x] + fa[q];
    block_reduce_finish<NC>(v, o);
}

template <int K>
void launch_k(qxd_ctx* ctx, const HopDev& d, const MultiPtr& W, int slot, cudaStream_t st) {
    int nb = wave_blocks(ctx, k_hop_dots<K>, kRedThreads, (size_t)kRedThreads, (size_t)ctx->g.Vh);
    const int cap = kPartials / (2 * K + 4);  // partial sums of every block fit the buffer
    if (nb > cap) nb = cap;
    k_hop_dots<K><<<nb, kRedThreads, 0, st>>>(ctx->g, d, W, red_out(ctx, slot));
}

}  // namespace

int launch_hop_dots(qxd_ctx* ctx, int fl, const HopArgs& a, int k, const void* const* W, int slot, cudaStream_t st) {
    if (k < 0 || k > kMultiMax) return qxd_fail(ctx, QXD_EARG, "fused hop: at most 8 basis fields");
    if (a.self_mode != 1 || a.post_mode != 0 || a.nrhs != 1 || a.g5_nb || a.g5_self || a.g5_out)
        return qxd_fail(ctx, QXD_EARG, "fused hop: only the second half of Dhat, one right-hand side");
    const Geo& g = ctx->g;
    const QxdFlavour& F = ctx->fl[fl];
    const size_t Vh = g.Vh;
    const int po = a.pout, pi = 1 - a.pout;
    HopDev d{};
    d.pout = po;
    d.in_nb = a.in_nb;
    d.in_self = a.in_self;
    d.out = a.out;
    d.U32_out = ctx->U32 + (size_t)po * 12 * Vh;
    d.U32_in = ctx->U32 + (size_t)pi * 12 * Vh;
    d.Z32_out = F.Z32 + (size_t)po * 2 * Vh;
    d.Z32_in = F.Z32 + (size_t)pi * 2 * Vh;
    d.diag = F.C32[0] + (size_t)po * 18 * Vh;
    d.diaginv = F.C32[1] + (size_t)po * 18 * Vh;
    d.c_hop = a.c_hop;
    MultiPtr mp{};
    for (int j = 0; j < kMultiMax; ++j) mp.p[j] = W[j < k ? j : 0];
    // algorithmic bytes: the hop with its self term (links 8 x 56, A_ee 288, spinors
    // neighbours + self + output 3 x 96) and the K basis fields
    ProfScope prof(ctx, "hop_fp32_self1_post0_dots", (double)Vh * (8 * 56.0 + 288.0 + 96.0 * (3 + k)), st);
    switch (k) {
        case 0: launch_k<0>(ctx, d, mp, slot, st); break;
        case 1: launch_k<1>(ctx, d, mp, slot, st); break;
        case 2: launch_k<2>(ctx, d, mp, slot, st); break;
        case 3: launch_k<3>(ctx, d, mp, slot, st); break;
        case 4: launch_k<4>(ctx, d, mp, slot, st); break;
        case 5: launch_k<5>(ctx, d, mp, slot, st); break;
        case 6: launch_k<6>(ctx, d, mp, slot, st); break;
        case 7: launch_k<7>(ctx, d, mp, slot, st); break;
        default: launch_k<8>(ctx, d, mp, slot, st); break;
    }
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

}  // namespace qxd
