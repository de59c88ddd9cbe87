// Conversions between the canonical spinor layout of the C ABI
// ([site][4][3] complex, lexicographic over the simulated lattice, or over the
// sites of one parity) and the internal parity-split structure-of-arrays fields.
#include <type_traits>

#include "df64.cuh"
#include "qxd_internal.h"

namespace qxd {

// canonical precision: 0 = complex128, 1 = complex64
template <int CIN, int PINT>
__global__ void k_pack(Geo g, const void* __restrict__ canon, int cfull, int p, void* __restrict__ internal) {
    using R = typename Prec<PINT>::real;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    const int rhs = blockIdx.y;
    long long site = h;
    if (cfull) {
        int x[4];
        site_coords(g, p, h, x);
        site = lex_index(g, x);
    }
    const long long nsites = cfull ? g.V : g.Vh;
    cplx<R> s[12];
    if (CIN == 0) {
        const double2* c = static_cast<const double2*>(canon) + ((long long)rhs * nsites + site) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = c[k];
            s[k] = {(R)v.x, (R)v.y};
        }
    } else {
        const float2* c = static_cast<const float2*>(canon) + ((long long)rhs * nsites + site) * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            float2 v = c[k];
            s[k] = {(R)v.x, (R)v.y};
        }
    }
    using CH = typename Prec<PINT>::chunk;
    store_spinor<PINT>(static_cast<CH*>(internal) + (size_t)rhs * Prec<PINT>::nchunk * g.Vh, g.Vh, h, s);
}

// The canonical layout keeps a site's 12 complex numbers together, and the sites of one
// parity are every other site: a thread writing its own site would write 16-byte pieces
// 384 bytes apart across the warp (half sectors).  So each warp stages its 32 sites in
// shared memory and then writes them as consecutive pieces, lane by lane.
template <int PINT, int COUT>
__global__ void __launch_bounds__(kThreads) k_unpack(Geo g, const void* __restrict__ internal, int p,
                                                     void* __restrict__ canon, int cfull) {
    using R = typename Prec<PINT>::real;
    using CH = typename Prec<PINT>::chunk;
    using OT = typename std::conditional<COUT == 0, double2, float2>::type;
    constexpr int kPad = 13;  // staging row of one site (12 values and one pad against bank conflicts)
    __shared__ OT stage[kThreads / 32][32 * kPad];
    __shared__ long long dst[kThreads / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int rhs = blockIdx.y;
    const long long nsites = cfull ? g.V : g.Vh;
    if (h < g.Vh) {
        long long site = h;
        if (cfull) {
            int x[4];
            site_coords(g, p, h, x);
            site = lex_index(g, x);
        }
        cplx<R> s[12];
        load_spinor<PINT>(static_cast<const CH*>(internal) + (size_t)rhs * Prec<PINT>::nchunk * g.Vh, g.Vh, h, s);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            OT v;
            if constexpr (COUT == 0 && PINT != 0) {  // FP32 to FP64 by integer operations
                v.x = df_widen(s[k].re);
                v.y = df_widen(s[k].im);
            } else {
                v.x = s[k].re;
                v.y = s[k].im;
            }
            stage[warp][lane * kPad + k] = v;
        }
        dst[warp][lane] = ((long long)rhs * nsites + site) * 12;
    } else {
        dst[warp][lane] = -1;
    }
    __syncwarp();
    OT* c = static_cast<OT*>(canon);
#pragma unroll
    for (int j0 = 0; j0 < 12; ++j0) {
        const int j = j0 * 32 + lane;  // value j of the warp: site j / 12, component j % 12
        const int sl = j / 12, k = j - sl * 12;
        const long long d = dst[warp][sl];
        if (d >= 0) c[d + k] = stage[warp][sl * kPad + k];
    }
}

int launch_pack(qxd_ctx* ctx, int cin, const void* canon, int cfull, int p, int pint, void* internal, int nrhs,
                cudaStream_t st) {
    const Geo& g = ctx->g;
    dim3 grid(nblocks(g.Vh), nrhs);
    const double ib = pint == 0 ? 192.0 : (pint == 1 ? 96.0 : 48.0);
    ProfScope prof(ctx, "pack", (double)g.Vh * nrhs * ((cin == 0 ? 192.0 : 96.0) + ib), st);
    if (cin == 0) {
        if (pint == 0) k_pack<0, 0><<<grid, kThreads, 0, st>>>(g, canon, cfull, p, internal);
        else if (pint == 1) k_pack<0, 1><<<grid, kThreads, 0, st>>>(g, canon, cfull, p, internal);
        else k_pack<0, 2><<<grid, kThreads, 0, st>>>(g, canon, cfull, p, internal);
    } else {
        if (pint == 0) k_pack<1, 0><<<grid, kThreads, 0, st>>>(g, canon, cfull, p, internal);
        else if (pint == 1) k_pack<1, 1><<<grid, kThreads, 0, st>>>(g, canon, cfull, p, internal);
        else k_pack<1, 2><<<grid, kThreads, 0, st>>>(g, canon, cfull, p, internal);
    }
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int launch_unpack(qxd_ctx* ctx, int pint, const void* internal, int p, int cout, void* canon, int cfull, int nrhs,
                  cudaStream_t st) {
    const Geo& g = ctx->g;
    dim3 grid(nblocks(g.Vh), nrhs);
    const double ib = pint == 0 ? 192.0 : (pint == 1 ? 96.0 : 48.0);
    ProfScope prof(ctx, "unpack", (double)g.Vh * nrhs * ((cout == 0 ? 192.0 : 96.0) + ib), st);
    if (cout == 0) {
        if (pint == 0) k_unpack<0, 0><<<grid, kThreads, 0, st>>>(g, internal, p, canon, cfull);
        else if (pint == 1) k_unpack<1, 0><<<grid, kThreads, 0, st>>>(g, internal, p, canon, cfull);
        else k_unpack<2, 0><<<grid, kThreads, 0, st>>>(g, internal, p, canon, cfull);
    } else {
        if (pint == 0) k_unpack<0, 1><<<grid, kThreads, 0, st>>>(g, internal, p, canon, cfull);
        else if (pint == 1) k_unpack<1, 1><<<grid, kThreads, 0, st>>>(g, internal, p, canon, cfull);
        else k_unpack<2, 1><<<grid, kThreads, 0, st>>>(g, internal, p, canon, cfull);
    }
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

}  // namespace qxd
