// Learned preconditioner: a gauge-covariant network of parallel-transport
// layers (not part of the paper), with its training kernels.
//
// Layer l:  b_c(x) = sum_{c'} sum_{d=0..8} W[c][c'][d] (T_d a_{c'})(x)
//   T_0 a(x) = a(x),  T_{1+mu} a(x) = V(x,mu) a(x+mu),  T_{5+mu} a(x) = V(x-mu,mu)^+ a(x-mu)
// with V = U z^qhat and the boundary conditions of the Dirac operator (the
// FP32 links and phases the hopping kernels use), W[c][c'][d] a complex 4x4
// spin matrix.  Channels 1 -> nch -> ... -> nch -> 1.  As a preconditioner of
// Dhat the network acts on an even-site field embedded in the full lattice and
// its output is restricted to the even sites.
//
// Layout: a channel is a full-lattice FP32 field, the even then the odd
// half-lattice field (6 float4 chunks x V/2 each); weights are complex (float2)
// [cout][cin][9][4][4] per layer, layers one after the other.
//
// Training: loss L = sum_i |(M r_i)_e - e_i|^2 / |e_i|^2 over a batch of pairs;
// gradient G = dL/dW^* = sum_x delta_c(x) (T_d a_{c'}(x))^+ (colour summed),
// delta propagated backwards through the adjoint layers (W^+ and T_d^+ =
// T_{opposite d}); Adam on the real and imaginary parts (gradient 2 Re G, 2 Im G).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "blas.h"
#include "hop.cuh"
#include "ops.h"
#include "qxd_internal.h"

namespace qxd {

constexpr int kPtcMaxCh = 16;

struct PtcLinks {
    const float4* U32;  // [p][12][Vh]
    const float4* Z32;  // [p][2][Vh]
};

static size_t layer_weights(int cin, int cout) { return (size_t)cout * cin * 9 * 16; }  // complex entries

static void layer_shape(int l, int nlayers, int nch, int* cin, int* cout) {
    *cin = l == 0 ? 1 : nch;
    *cout = l == nlayers - 1 ? 1 : nch;
}

size_t ptc_weight_count(int nlayers, int nch) {
    size_t n = 0;
    for (int l = 0; l < nlayers; ++l) {
        int ci, co;
        layer_shape(l, nlayers, nch, &ci, &co);
        n += layer_weights(ci, co);
    }
    return n;
}

// ---- transports --------------------------------------------------------------
// Colour row I of (T_d a)(x), all four spins: t[s] = (T_d a)(x)[s][I].  The link
// of direction d (and its phase) is loaded once per d by the caller (link_for);
// `src` is the neighbour's half index (d > 0) on parity 1 - p.
struct PtcLink {
    Mat3<float> m;
    cplx<float> z;
    int src;
};

QXD_HD void link_for(const Geo& g, const PtcLinks& L, int d, int p, int h, const int x[4], PtcLink& lk) {
    const int Vh = g.Vh;
    const int mu = (d - 1) & 3;
    const bool fwd = d <= 4;
    lk.src = neighbour_lex(g, x, mu, fwd ? +1 : -1) >> 1;
    const int ps = 1 - p;
    if (fwd) load_link32(L.U32 + (size_t)p * 12 * Vh, L.Z32 + (size_t)p * 2 * Vh, Vh, mu, h, lk.m, lk.z);
    else load_link32(L.U32 + (size_t)ps * 12 * Vh, L.Z32 + (size_t)ps * 2 * Vh, Vh, mu, lk.src, lk.m, lk.z);
}

template <int I>
QXD_HD void transport_row(const Geo& g, int d, int p, int h, const PtcLink& lk, const float4* __restrict__ a_ch,
                          cplx<float> t[4]) {
    const int Vh = g.Vh;
    if (d == 0) {
        const float4* b = a_ch + (size_t)p * 6 * Vh;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const int q = 3 * sp + I;
            const float4 v = QXD_LDG(b + (size_t)(q >> 1) * Vh + h);
            t[sp] = (q & 1) ? cplx<float>{v.z, v.w} : cplx<float>{v.x, v.y};
        }
        return;
    }
    cplx<float> s[12];
    load_spinor<1>(a_ch + (size_t)(1 - p) * 6 * Vh, Vh, lk.src, s);
    const bool fwd = d <= 4;
#pragma unroll
    for (int sp = 0; sp < 4; ++sp) {
        cplx<float> acc = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            if (fwd) cmac(acc, lk.m.a[I][j], s[3 * sp + j]);
            else cmac_conj(acc, lk.m.a[j][I], s[3 * sp + j]);
        }
        t[sp] = fwd ? lk.z * acc : cmul_conj(lk.z, acc);
    }
}

// ---- forward layer ------------------------------------------------------------------
// Thread (site, colour I): a tile of kPtcSites sites of one parity, the three
// colour rows in three groups of kPtcSites threads (warp-uniform colour).  Each
// thread forms T_d a_{c'} once per (d, c') and accumulates all COUT output
// channels of its group from it; the group's weights [9][cin][COUT][4][4] sit in
// shared memory (read as broadcasts).  Persistent: a block loops over tiles.
constexpr int kPtcSites = 64;
constexpr int kPtcFwdThreads = 3 * kPtcSites;
constexpr int kPtcGroup = 8;  // output channels per block (grid.z splits larger layers)

template <int I, int COUT>
__device__ void ptc_fwd_site(const Geo& g, const PtcLinks& L, const float4* __restrict__ a, int cin, int ng,
                             const float2* __restrict__ wsh, float4* __restrict__ out, int c0, int p, int h) {
    const size_t chs = (size_t)12 * g.Vh;  // float4 per channel
    int x[4];
    site_coords(g, p, h, x);
    cplx<float> acc[COUT][4];
#pragma unroll
    for (int c = 0; c < COUT; ++c)
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) acc[c][sp] = {0.f, 0.f};
    for (int d = 0; d < 9; ++d) {
        PtcLink lk;
        if (d > 0) link_for(g, L, d, p, h, x, lk);
        for (int cp = 0; cp < cin; ++cp) {
            cplx<float> t[4];
            transport_row<I>(g, d, p, h, lk, a + cp * chs, t);
            const float4* w = reinterpret_cast<const float4*>(wsh + (size_t)(d * cin + cp) * COUT * 16);
#pragma unroll
            for (int c = 0; c < COUT; ++c) {
                if (c >= ng) break;
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    const float4 w01 = w[c * 8 + sp * 2], w23 = w[c * 8 + sp * 2 + 1];
                    cmac(acc[c][sp], cplx<float>{w01.x, w01.y}, t[0]);
                    cmac(acc[c][sp], cplx<float>{w01.z, w01.w}, t[1]);
                    cmac(acc[c][sp], cplx<float>{w23.x, w23.y}, t[2]);
                    cmac(acc[c][sp], cplx<float>{w23.z, w23.w}, t[3]);
                }
            }
        }
    }
    // complex (spin sp, colour I) is component (q & 1) of chunk q >> 1, q = 3 sp + I
#pragma unroll
    for (int c = 0; c < COUT; ++c) {
        if (c >= ng) break;
        float2* o = reinterpret_cast<float2*>(out + (c0 + c) * chs + (size_t)p * 6 * g.Vh);
#pragma unroll
        for (int sp = 0; sp < 4; ++sp) {
            const int q = 3 * sp + I;
            o[2 * ((size_t)(q >> 1) * g.Vh + h) + (q & 1)] = make_float2(acc[c][sp].re, acc[c][sp].im);
        }
    }
}

template <int COUT>
__global__ void __launch_bounds__(kPtcFwdThreads) k_ptc_fwd(Geo g, PtcLinks L, const float4* __restrict__ a, int cin,
                                                           int cout, const float2* __restrict__ W,
                                                           float4* __restrict__ out) {
    extern __shared__ float4 wsh4[];
    float2* wsh = reinterpret_cast<float2*>(wsh4);
    const int c0 = blockIdx.z * kPtcGroup;
    const int ng = min(kPtcGroup, cout - c0);
    // W[c][c'][d][s][s'] (global) -> wsh[d][c'][c - c0][s][s'] (zero for c >= ng)
    const int nw = 9 * cin * COUT * 16;
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
        const int e = i % 16, c = (i / 16) % COUT, cp = (i / (16 * COUT)) % cin, d = i / (16 * COUT * cin);
        wsh[i] = c < ng ? W[((size_t)((c0 + c) * cin + cp) * 9 + d) * 16 + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const int colour = threadIdx.x / kPtcSites;
    const int lane_site = threadIdx.x % kPtcSites;
    const int tiles = (g.Vh + kPtcSites - 1) / kPtcSites;
    for (int t = blockIdx.x; t < 2 * tiles; t += gridDim.x) {
        const int p = t / tiles;
        const int h = (t % tiles) * kPtcSites + lane_site;
        if (h >= g.Vh) continue;
        if (colour == 0) ptc_fwd_site<0, COUT>(g, L, a, cin, ng, wsh, out, c0, p, h);
        else if (colour == 1) ptc_fwd_site<1, COUT>(g, L, a, cin, ng, wsh, out, c0, p, h);
        else ptc_fwd_site<2, COUT>(g, L, a, cin, ng, wsh, out, c0, p, h);
    }
}

// W'[c'][c][d'] = W[c][c'][opposite(d')]^+ (the adjoint layer as a forward layer)
__global__ void k_ptc_adjoint_weights(const float2* __restrict__ W, int cin, int cout, float2* __restrict__ Wa) {
    const int n = cout * cin * 9;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const int d = q % 9, cp = (q / 9) % cin, c = q / (9 * cin);
        const int dop = d == 0 ? 0 : (d <= 4 ? d + 4 : d - 4);
        const float2* src = W + ((size_t)(c * cin + cp) * 9 + d) * 16;
        float2* dst = Wa + ((size_t)(cp * cout + c) * 9 + dop) * 16;
        for (int s = 0; s < 4; ++s)
            for (int t = 0; t < 4; ++t) dst[4 * t + s] = make_float2(src[4 * s + t].x, -src[4 * s + t].y);
    }
}

// ---- weight gradient ----------------------------------------------------------------
// G[c][c'][d][s][s'] = sum_{x,i} delta_c(x)[s][i] conj((T_d a_{c'})(x)[s'][i]): for each d
// the product of the (c,s) x (x,i) matrix of delta with the (x,i) x (c',s') matrix of
// conjugated transports, summed over K = 3V rows in tiles of 3 kPtcSites rows.  A block
// owns one chunk (blockIdx.z) of at most 32 (c,s) x 32 (c',s') entries for all nine d;
// each of its 256 threads a 2 x 2 sub-block of the chunk for every d (36 complex
// accumulators).  Per tile the delta rows are staged once and the transports once per
// d, both in shared memory; T_d a_{c'} is formed once per site, colour, d and c'.
// Sums run in FP32 within a block; the blocks' partials are added in FP64 in a fixed
// order by k_ptc_wgrad_final.
constexpr int kWgThreads = 256;
constexpr int kWgRows = 3 * kPtcSites;
constexpr size_t kWgSmem = 2ull * kWgRows * 32 * sizeof(float2);  // delta and transport tiles

template <int I>
__device__ void wgrad_stage(const Geo& g, const PtcLinks& L, const float4* __restrict__ delta,
                            const float4* __restrict__ a, int d, int p, int h, bool live, int r_c0, int nr_c,
                            int c_c0, int nc_c, float2 (*dsh)[32], float2 (*tsh)[32], int row) {
    const size_t chs = (size_t)12 * g.Vh;
    int x[4];
    if (live) site_coords(g, p, h, x);
    if (d < 0) {
        // delta_c(x)[s][I] for the chunk's output channels
        for (int c = 0; c < 8; ++c) {
            cplx<float> t[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            if (live && c < nr_c) {
                PtcLink none;
                transport_row<I>(g, 0, p, h, none, delta + (r_c0 + c) * chs, t);
            }
            for (int sp = 0; sp < 4; ++sp) dsh[row][c * 4 + sp] = make_float2(t[sp].re, t[sp].im);
        }
        return;
    }
    PtcLink lk;
    if (live && d > 0) link_for(g, L, d, p, h, x, lk);
    for (int c = 0; c < 8; ++c) {
        cplx<float> t[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        if (live && c < nc_c) transport_row<I>(g, d, p, h, lk, a + (c_c0 + c) * chs, t);
        for (int sp = 0; sp < 4; ++sp) tsh[row][c * 4 + sp] = make_float2(t[sp].re, t[sp].im);
    }
}

__global__ void __launch_bounds__(kWgThreads) k_ptc_wgrad(Geo g, PtcLinks L, const float4* __restrict__ delta,
                                                         const float4* __restrict__ a, int cin, int cout,
                                                         float2* __restrict__ partials) {
    extern __shared__ float4 wg_sh[];
    float2 (*dsh)[32] = reinterpret_cast<float2 (*)[32]>(wg_sh);
    float2 (*tsh)[32] = dsh + kWgRows;
    const int nzc = (cin + 7) / 8;
    const int zr = blockIdx.z / nzc, zc = blockIdx.z % nzc;
    const int r_c0 = 8 * zr, nr_c = min(8, cout - r_c0);  // output channels of the chunk
    const int c_c0 = 8 * zc, nc_c = min(8, cin - c_c0);   // input channels of the chunk
    const int tid = threadIdx.x;
    const int r0 = 2 * (tid / 16), q0 = 2 * (tid % 16);  // this thread's 2 x 2 sub-block
    cplx<float> acc[9][2][2];
#pragma unroll
    for (int d = 0; d < 9; ++d)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc[d][i][j] = {0.f, 0.f};
    const int colour = tid / kPtcSites;  // staging threads: tid < kWgRows
    const int lane_site = tid % kPtcSites;
    const int tiles = (g.Vh + kPtcSites - 1) / kPtcSites;
    for (int t = blockIdx.x; t < 2 * tiles; t += gridDim.x) {
        const int p = t / tiles;
        const int h = (t % tiles) * kPtcSites + lane_site;
        const bool live = h < g.Vh;
        __syncthreads();  // the previous tile's rows are no longer read
        if (tid < kWgRows) {
            if (colour == 0) wgrad_stage<0>(g, L, delta, a, -1, p, h, live, r_c0, nr_c, c_c0, nc_c, dsh, tsh, tid);
            else if (colour == 1) wgrad_stage<1>(g, L, delta, a, -1, p, h, live, r_c0, nr_c, c_c0, nc_c, dsh, tsh, tid);
            else wgrad_stage<2>(g, L, delta, a, -1, p, h, live, r_c0, nr_c, c_c0, nc_c, dsh, tsh, tid);
        }
#pragma unroll
        for (int d = 0; d < 9; ++d) {
            __syncthreads();
            if (tid < kWgRows) {
                if (colour == 0) wgrad_stage<0>(g, L, delta, a, d, p, h, live, r_c0, nr_c, c_c0, nc_c, dsh, tsh, tid);
                else if (colour == 1) wgrad_stage<1>(g, L, delta, a, d, p, h, live, r_c0, nr_c, c_c0, nc_c, dsh, tsh, tid);
                else wgrad_stage<2>(g, L, delta, a, d, p, h, live, r_c0, nr_c, c_c0, nc_c, dsh, tsh, tid);
            }
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < kWgRows; ++k) {
                const float4 dv = *reinterpret_cast<const float4*>(&dsh[k][r0]);
                const float4 tv = *reinterpret_cast<const float4*>(&tsh[k][q0]);
                const cplx<float> dd[2] = {{dv.x, dv.y}, {dv.z, dv.w}};
                const cplx<float> tt[2] = {{tv.x, tv.y}, {tv.z, tv.w}};
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) cmac_conj(acc[d][i][j], tt[j], dd[i]);
            }
        }
    }
    float2* out = partials + ((size_t)blockIdx.z * gridDim.x + blockIdx.x) * 9 * 1024;
#pragma unroll
    for (int d = 0; d < 9; ++d)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                out[d * 1024 + (r0 + i) * 32 + (q0 + j)] = make_float2(acc[d][i][j].re, acc[d][i][j].im);
}

// G (+)= sum over the blocks' partials in FP64, blocks in a fixed order
__global__ void k_ptc_wgrad_final(const float2* __restrict__ partials, int nblk, int cin, int cout,
                                  float2* __restrict__ G, int accumulate) {
    const int nzc = (cin + 7) / 8, nz = ((cout + 7) / 8) * nzc;
    const int n = nz * 9 * 1024;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int e = t % 1024, d = (t / 1024) % 9, z = t / (9 * 1024);
        const int r = e / 32, q = e % 32;
        const int c = 8 * (z / nzc) + r / 4, cp = 8 * (z % nzc) + q / 4;
        if (c >= cout || cp >= cin) continue;
        double re = 0.0, im = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const float2 v = partials[((size_t)z * nblk + b) * 9 * 1024 + d * 1024 + e];
            re += v.x;
            im += v.y;
        }
        const size_t o = ((size_t)(c * cin + cp) * 9 + d) * 16 + (r % 4) * 4 + (q % 4);
        const float2 g0 = accumulate ? G[o] : make_float2(0.f, 0.f);
        G[o] = make_float2(g0.x + (float)re, g0.y + (float)im);
    }
}

// ---- forward layer on the tensor cores (tcgen05) ------------------------------------
// The channel mixing of a layer is, per colour row i, the dense product
//   out_i[site][(c,s)] = sum_d sum_{(c',s')} W[c][c'][d][s][s'] (T_d a_{c'})_i[site][s'],
// written over the reals ([Re, Im] of the transports times the 2 x 2 real form of
// each complex weight): M = 128 sites of a tile, N = 2*4*COUTP, K = 2*4*CINP per
// direction d.  A CTA of 512 threads forms the transports of one direction for its
// tile (thread = site and a pair of input channels), rounds them to bfloat16 into
// shared memory in the canonical K-major layout (8-row x 16-byte core matrices),
// and one thread issues the tcgen05.mma instructions for the three colour rows,
// accumulating in FP32 in tensor memory (three N-column accumulators), while the
// other threads form the next direction's transports into a second buffer (an
// mbarrier signalled by tcgen05.commit says when a buffer is free again).  After
// the nine directions the accumulators are read back with tcgen05.ld and stored as
// the output channels.  The weights, as bfloat16 real matrices, stay in shared memory
// for all tiles of the persistent CTA.  Every wait on an mbarrier is bounded: on a
// time-out the CTA flags the error, writes NaN to its tile, releases its tensor
// memory and returns.
constexpr int kTcThreads = 512;
constexpr int kTcRows = 128;      // sites per tile (MMA M)
constexpr int kTcTmemCols = 256;  // three accumulators of up to 64 columns
constexpr unsigned kTcSpin = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a K-major bfloat16 tile with K columns in the
// canonical no-swizzle layout: core matrices of 8 rows x 8 elements (16 bytes per
// row, 128 bytes each), adjacent along K 128 bytes apart, along rows 16 K bytes apart
__host__ __device__ constexpr uint32_t tc_off(int row, int k, int K) {
    return (uint32_t)((row >> 3) * (K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading (K) and stride (row-group) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, int K) {
    const uint64_t lbo = 128, sbo = (uint64_t)K * 16;
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, bfloat16 A and B, both
// K-major, N and M
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bounded wait for the completion of the phase with the given parity; false on time-out
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    for (unsigned it = 0; it < kTcSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi) { return pack_bf16x2(lo, hi); }

template <int CINP, int COUTP>
struct TcShape {
    static constexpr int K = 8 * CINP;                  // K per direction
    static constexpr int N = 8 * COUTP;                 // output columns per colour
    static constexpr int A_BYTES = kTcRows * K * 2;     // one colour's A tile
    static constexpr int B_BYTES = N * K * 2;           // one direction's B tile
    static constexpr size_t SMEM = 2ull * 3 * A_BYTES + 9ull * B_BYTES + 64;
};

// transports of direction d for this thread's site and input channels c0, c0 + 1
// (zero beyond cin or past the lattice), rounded to bfloat16 into A[colour]
template <int CINP>
__device__ __forceinline__ void tc_produce_pair(const Geo& g, int d, int p, int h, bool live, const PtcLink& lk,
                                                const float4* __restrict__ a, int cin, int c0, int row,
                                                unsigned char* Abuf) {
    constexpr int K = 8 * CINP;
    const size_t chs = (size_t)12 * g.Vh;
    cplx<float> t[2][12];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int c = c0 + q;
#pragma unroll
        for (int k = 0; k < 12; ++k) t[q][k] = {0.f, 0.f};
        if (!live || c >= cin) continue;
        const float4* ach = a + c * chs;
        if (d == 0) {
            load_spinor<1>(ach + (size_t)p * 6 * g.Vh, g.Vh, h, t[q]);
            continue;
        }
        cplx<float> s[12];
        load_spinor<1>(ach + (size_t)(1 - p) * 6 * g.Vh, g.Vh, lk.src, s);
        const bool fwd = d <= 4;
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                cplx<float> acc = {0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    if (fwd) cmac(acc, lk.m.a[i][j], s[3 * sp + j]);
                    else cmac_conj(acc, lk.m.a[j][i], s[3 * sp + j]);
                }
                t[q][3 * sp + i] = fwd ? lk.z * acc : cmul_conj(lk.z, acc);
            }
    }
    // K index (ri, c', s') -> ri * 4 CINP + 4 c' + s': channels c0, c0 + 1 fill one
    // 16-byte chunk of real parts and one of imaginary parts per colour row
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        unsigned char* A = Abuf + i * (kTcRows * K * 2);
        uint4 re, im;
        re.x = bf2(t[0][i].re, t[0][3 + i].re);
        re.y = bf2(t[0][6 + i].re, t[0][9 + i].re);
        re.z = bf2(t[1][i].re, t[1][3 + i].re);
        re.w = bf2(t[1][6 + i].re, t[1][9 + i].re);
        im.x = bf2(t[0][i].im, t[0][3 + i].im);
        im.y = bf2(t[0][6 + i].im, t[0][9 + i].im);
        im.z = bf2(t[1][i].im, t[1][3 + i].im);
        im.w = bf2(t[1][6 + i].im, t[1][9 + i].im);
        *reinterpret_cast<uint4*>(A + tc_off(row, 4 * c0, K)) = re;
        *reinterpret_cast<uint4*>(A + tc_off(row, 4 * CINP + 4 * c0, K)) = im;
    }
}

template <int CINP, int COUTP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_ptc_fwd_tc(Geo g, PtcLinks L, const float4* __restrict__ a, int cin, int cout, const float2* __restrict__ W,
                 float4* __restrict__ out, int* __restrict__ err) {
    using S = TcShape<CINP, COUTP>;
    constexpr int K = S::K, N = S::N;
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char* Abuf[2] = {tc_smem, tc_smem + 3 * S::A_BYTES};
    unsigned char* Bsm = tc_smem + 6 * S::A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Bsm + 9 * S::B_BYTES);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(mbar + 2);
    int* bad = reinterpret_cast<int*>(tmem_holder + 1);
    const int tid = threadIdx.x;
    const int c_out0 = blockIdx.z * COUTP;
    const int ng = min(COUTP, cout - c_out0);
    // weights: B_d[n][k], n = (ro, c, s), k = (ri, c', s'), the real form of W[c][c'][d][s][s']
    for (int e = tid; e < 9 * N * K; e += kTcThreads) {
        const int k = e % K, n = (e / K) % N, d = e / (K * N);
        const int ri = k / (4 * CINP), cp = (k / 4) % CINP, sp = k % 4;
        const int ro = n / (4 * COUTP), c = (n / 4) % COUTP, so = n % 4;
        float v = 0.f;
        if (c < ng && cp < cin) {
            const float2 w = W[((size_t)((c_out0 + c) * cin + cp) * 9 + d) * 16 + so * 4 + sp];
            v = (ro == ri) ? w.x : (ro == 0 ? -w.y : w.y);
        }
        *reinterpret_cast<__nv_bfloat16*>(Bsm + d * S::B_BYTES + tc_off(n, k, K)) = __float2bfloat16_rn(v);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *bad = 0;
    }
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;
    constexpr uint32_t idesc = tc_idesc(kTcRows, N);
    uint32_t phase[2] = {0u, 0u};
    const int row = tid % kTcRows;
    const int quarter = tid / kTcRows;  // input channels 2 quarter, 2 quarter + 1
    const int tiles = (g.Vh + kTcRows - 1) / kTcRows;
    bool failed = false;
    for (int tile = blockIdx.x; tile < 2 * tiles && !failed; tile += gridDim.x) {
        const int p = tile / tiles;
        const int h = (tile % tiles) * kTcRows + row;
        const bool live = h < g.Vh;
        int x[4] = {0, 0, 0, 0};
        if (live) site_coords(g, p, h, x);
        for (int d = 0; d < 9; ++d) {
            const int b = d & 1;
            if (d >= 2) {
                // the MMAs of direction d - 2 read this buffer
                const bool ok = tc_wait(smem_u32(&mbar[b]), phase[b]);
                phase[b] ^= 1u;
                if (__syncthreads_or(!ok)) {
                    failed = true;
                    break;
                }
            }
            PtcLink lk;
            if (live && d > 0) link_for(g, L, d, p, h, x, lk);
            if (CINP == 8 || quarter == 0)
                tc_produce_pair<CINP>(g, d, p, h, live, lk, a, cin, 2 * quarter, row, Abuf[b]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const uint32_t a_base = smem_u32(Abuf[b] + i * S::A_BYTES);
                    const uint32_t b_base = smem_u32(Bsm + d * S::B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < K / 16; ++kk)
                        tc_mma(tmem + (uint32_t)(i * 64), tc_desc(a_base + kk * 256, K), tc_desc(b_base + kk * 256, K),
                               idesc, (d > 0 || kk > 0) ? 1 : 0);
                }
                tc_commit(smem_u32(&mbar[b]));
            }
        }
        if (failed) break;
        // all MMAs of the tile: the commits of directions 7 and 8
        bool ok = tc_wait(smem_u32(&mbar[1]), phase[1]);
        phase[1] ^= 1u;
        ok = tc_wait(smem_u32(&mbar[0]), phase[0]) && ok;
        phase[0] ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: warp w reads lanes 32 (w % 4) ..; warps 4i .. 4i + 3 colour row i
        const int warp = tid >> 5, lane = tid & 31;
        const int q = warp & 3;
        const int site = 32 * q + lane;
        const int hs = (tile % tiles) * kTcRows + site;
        const size_t chs = (size_t)12 * g.Vh;
        const int i = warp >> 2;  // warps 12-15 have no colour row to read
        if (i < 3) {
            float v[N];
#pragma unroll
            for (int c16 = 0; c16 < N / 16; ++c16)
                tc_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(i * 64 + 16 * c16), v + 16 * c16);
            if (hs < g.Vh) {
#pragma unroll
                for (int c = 0; c < COUTP; ++c) {
                    if (c >= ng) break;
                    float2* o = reinterpret_cast<float2*>(out + (c_out0 + c) * chs + (size_t)p * 6 * g.Vh);
#pragma unroll
                    for (int sp = 0; sp < 4; ++sp) {
                        const int qq = 3 * sp + i;
                        o[2 * ((size_t)(qq >> 1) * g.Vh + hs) + (qq & 1)] =
                            make_float2(v[4 * c + sp], v[4 * COUTP + 4 * c + sp]);
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    if (failed) {
        // a wait timed out: flag it, give the tensor cores a bounded time to finish, and
        // leave NaN in this CTA's first tile so that a solver using the output stops
        if (tid == 0) {
            atomicExch(err, 1);
            tc_wait(smem_u32(&mbar[0]), phase[0]);
            tc_wait(smem_u32(&mbar[1]), phase[1]);
        }
        const int tiles_ = (g.Vh + kTcRows - 1) / kTcRows;
        const int p = blockIdx.x / tiles_;
        const int hs = (blockIdx.x % tiles_) * kTcRows + row;
        if (quarter == 0 && p < 2 && hs < g.Vh) {
            const size_t chs = (size_t)12 * g.Vh;
            for (int c = 0; c < ng; ++c)
                for (int k = 0; k < 6; ++k)
                    out[(c_out0 + c) * chs + (size_t)p * 6 * g.Vh + (size_t)k * g.Vh + hs] =
                        make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        }
        __syncthreads();
    }
    if (tid < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
    (void)bad;
}

// Adam on the real view of W: gradient = scale * 2 (Re G, Im G)
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ G, float* __restrict__ m, float* __restrict__ v,
                       size_t n, float scale, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gr = 2.f * scale * G[i];
        const float mi = b1 * m[i] + (1.f - b1) * gr;
        const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---- host side -------------------------------------------------------------------
static PtcLinks links_of(qxd_ctx* ctx, int fl) { return PtcLinks{ctx->U32, ctx->fl[fl].Z32}; }

static size_t chan_bytes(const qxd_ctx* ctx) { return (size_t)ctx->g.Vh * 2 * 96; }

// one forward layer: COUT = output channels per block (the smallest of 1, 2, 4, 8 that
// holds min(cout, 8)), grid.z = groups of 8 output channels, a persistent grid of
// resident blocks over the tiles of both parities
template <int COUT>
static int launch_fwd(qxd_ctx* ctx, int fl, const float4* a, int cin, const float2* W, float4* out, int cout,
                      cudaStream_t st) {
    const Geo& g = ctx->g;
    const size_t smem = 9ull * cin * COUT * 16 * sizeof(float2);
    QXD_CUDA(ctx, cudaFuncSetAttribute(k_ptc_fwd<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    QXD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ptc_fwd<COUT>, kPtcFwdThreads, smem));
    const int groups = (cout + kPtcGroup - 1) / kPtcGroup;
    const int tiles = 2 * ((g.Vh + kPtcSites - 1) / kPtcSites);
    const int nx = std::max(1, std::min(tiles, std::max(1, per_sm) * ctx->nsm / groups));
    k_ptc_fwd<COUT><<<dim3(nx, 1, groups), kPtcFwdThreads, smem, st>>>(g, links_of(ctx, fl), a, cin, cout, W, out);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// algorithmic bytes of a layer: every input and output channel once, the links once
static double layer_bytes(const qxd_ctx* ctx, int cin, int cout) {
    return (double)chan_bytes(ctx) * (cin + cout) + (double)ctx->g.V * 4 * 56;
}

static int launch_layer(qxd_ctx* ctx, int fl, const float4* a, int cin, const float2* W, float4* out, int cout,
                        cudaStream_t st) {
    ProfScope prof(ctx, "ptc_layer", layer_bytes(ctx, cin, cout), st);
    const int cg = std::min(cout, kPtcGroup);
    if (cg <= 1) return launch_fwd<1>(ctx, fl, a, cin, W, out, cout, st);
    if (cg <= 2) return launch_fwd<2>(ctx, fl, a, cin, W, out, cout, st);
    if (cg <= 4) return launch_fwd<4>(ctx, fl, a, cin, W, out, cout, st);
    return launch_fwd<8>(ctx, fl, a, cin, W, out, cout, st);
}

// one forward layer on the tensor cores (bfloat16 operands, FP32 accumulation): input
// channels padded to 2 or 8, output channels in groups of 2 or 8 (grid.z); at most
// two CTAs per SM (each holds 256 of the SM's 512 tensor-memory columns)
template <int CINP, int COUTP>
static int launch_fwd_tc(qxd_ctx* ctx, int fl, const float4* a, int cin, const float2* W, float4* out, int cout,
                         cudaStream_t st) {
    const Geo& g = ctx->g;
    const size_t smem = std::max<size_t>(TcShape<CINP, COUTP>::SMEM, 100 * 1024);
    QXD_CUDA(ctx, cudaFuncSetAttribute(k_ptc_fwd_tc<CINP, COUTP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    const int groups = (cout + COUTP - 1) / COUTP;
    const int tiles = 2 * ((g.Vh + kTcRows - 1) / kTcRows);
    int per_sm = 0;
    QXD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ptc_fwd_tc<CINP, COUTP>, kTcThreads, smem));
    per_sm = std::max(1, std::min(per_sm, 2));
    const int nx = std::max(1, std::min(tiles, per_sm * ctx->nsm / groups));
    k_ptc_fwd_tc<CINP, COUTP><<<dim3(nx, 1, groups), kTcThreads, smem, st>>>(g, links_of(ctx, fl), a, cin, cout, W,
                                                                             out, ctx->dev_flag);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

static int launch_layer_tc(qxd_ctx* ctx, int fl, const float4* a, int cin, const float2* W, float4* out, int cout,
                           cudaStream_t st) {
    if (cin > 8 || cout > 8) return launch_layer(ctx, fl, a, cin, W, out, cout, st);
    ProfScope prof(ctx, "ptc_layer_tc", layer_bytes(ctx, cin, cout), st);
    if (cin <= 2 && cout <= 2) return launch_fwd_tc<2, 2>(ctx, fl, a, cin, W, out, cout, st);
    if (cin <= 2) return launch_fwd_tc<2, 8>(ctx, fl, a, cin, W, out, cout, st);
    if (cout <= 2) return launch_fwd_tc<8, 2>(ctx, fl, a, cin, W, out, cout, st);
    return launch_fwd_tc<8, 8>(ctx, fl, a, cin, W, out, cout, st);
}

// weight gradient of one layer into G (accumulated): grid (blocks, 1, chunks)
static int wgrad_blocks(const qxd_ctx* ctx) {
    const int tiles = 2 * ((ctx->g.Vh + kPtcSites - 1) / kPtcSites);
    return std::max(1, std::min(tiles, 2 * ctx->nsm));
}

static size_t wgrad_partial_bytes(const qxd_ctx* ctx, int cin, int cout) {
    const size_t nz = (size_t)((cout + 7) / 8) * ((cin + 7) / 8);
    return nz * wgrad_blocks(ctx) * 9 * 1024 * sizeof(float2);
}

static int launch_wgrad(qxd_ctx* ctx, int fl, const float4* delta, const float4* a, int cin, int cout, float2* part,
                        float2* G, cudaStream_t st) {
    const Geo& g = ctx->g;
    ProfScope prof(ctx, "ptc_wgrad", layer_bytes(ctx, cin, cout), st);
    QXD_CUDA(ctx, cudaFuncSetAttribute(k_ptc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem));
    const int nblk = wgrad_blocks(ctx);
    const int nz = ((cout + 7) / 8) * ((cin + 7) / 8);
    k_ptc_wgrad<<<dim3(nblk, 1, nz), kWgThreads, kWgSmem, st>>>(g, links_of(ctx, fl), delta, a, cin, cout, part);
    QXD_CUDA(ctx, cudaGetLastError());
    k_ptc_wgrad_final<<<nblocks((long long)nz * 9 * 1024, 256), 256, 0, st>>>(part, nblk, cin, cout, G, 1);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// Forward pass: acts[0] = embedded input (1 channel); acts[l+1] = layer l (acts[l]).
// prec QXD_FP32: CUDA-core FP32 layers; QXD_BF16: the channel mixing on the tensor cores
static int ptc_forward(qxd_ctx* ctx, int fl, const float2* W, int nlayers, int nch, float4* const* acts,
                       cudaStream_t st, int prec = QXD_FP32) {
    const float2* w = W;
    for (int l = 0; l < nlayers; ++l) {
        int ci, co;
        layer_shape(l, nlayers, nch, &ci, &co);
        if (prec == QXD_BF16) QXD_TRY(launch_layer_tc(ctx, fl, acts[l], ci, w, acts[l + 1], co, st));
        else QXD_TRY(launch_layer(ctx, fl, acts[l], ci, w, acts[l + 1], co, st));
        w += layer_weights(ci, co);
    }
    return QXD_OK;
}

static int check_shape(qxd_ctx* ctx, int nlayers, int nch) {
    if (nlayers < 1 || nlayers > 8 || nch < 1 || nch > kPtcMaxCh)
        return qxd_fail(ctx, QXD_EARG, "learned preconditioner: 1..8 layers of 1..16 channels");
    return QXD_OK;
}

// Activation buffers of one pass: acts[0..nlayers] (channel counts 1, nch.., 1)
static int ptc_buffers(qxd_ctx* ctx, int nlayers, int nch, int slot0, std::vector<float4*>& acts) {
    acts.resize(nlayers + 1);
    for (int l = 0; l <= nlayers; ++l) {
        const int ch = (l == 0 || l == nlayers) ? 1 : nch;
        void* p;
        QXD_TRY(qxd_ws(ctx, slot0 + l, chan_bytes(ctx) * ch, &p));
        acts[l] = static_cast<float4*>(p);
    }
    return QXD_OK;
}

// z_e = (M r_e)_e for FP32 internal even fields (prec: QXD_FP32 or QXD_BF16 mixing)
int ptc_apply_internal(qxd_ctx* ctx, int fl, const float2* W, int nlayers, int nch, const void* r_e, void* z_e,
                       cudaStream_t st, int prec) {
    std::vector<float4*> acts;
    QXD_TRY(ptc_buffers(ctx, nlayers, nch, WS_PTC, acts));
    const size_t hb = half_bytes(ctx, QXD_FP32);
    QXD_CUDA(ctx, cudaMemcpyAsync(acts[0], r_e, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemsetAsync(reinterpret_cast<char*>(acts[0]) + hb, 0, hb, st));
    if (prec == QXD_BF16) QXD_CUDA(ctx, cudaMemsetAsync(ctx->dev_flag, 0, sizeof(int), st));
    QXD_TRY(ptc_forward(ctx, fl, W, nlayers, nch, acts.data(), st, prec));
    QXD_CUDA(ctx, cudaMemcpyAsync(z_e, acts[nlayers], hb, cudaMemcpyDeviceToDevice, st));
    return QXD_OK;
}

// Loss and gradient over pairs (internal FP32 even fields r[i], e[i]); G accumulated
// (complex, layout of W).  Returns the summed loss in *loss.
static int ptc_loss_grad_internal(qxd_ctx* ctx, int fl, const float2* W, int nlayers, int nch, const char* r,
                                  const char* e, const double* ee, const double* rr, int kind, const int* idx, int nb,
                                  float2* G, double* loss, cudaStream_t st) {
    const Geo& g = ctx->g;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const size_t n = 12ull * g.Vh;
    std::vector<float4*> acts;
    QXD_TRY(ptc_buffers(ctx, nlayers, nch, WS_PTC, acts));
    void *dA, *dB, *Wa, *part;
    QXD_TRY(qxd_ws(ctx, WS_PTC + 10, chan_bytes(ctx) * nch, &dA));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 11, chan_bytes(ctx) * nch, &dB));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 12, layer_weights(nch, nch) * sizeof(float2), &Wa));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 13, wgrad_partial_bytes(ctx, nch, nch), &part));
    // offsets of each layer's weights
    std::vector<size_t> off(nlayers + 1, 0);
    for (int l = 0; l < nlayers; ++l) {
        int ci, co;
        layer_shape(l, nlayers, nch, &ci, &co);
        off[l + 1] = off[l] + layer_weights(ci, co);
    }
    double tot = 0.0;
    for (int k = 0; k < nb; ++k) {
        const int i = idx[k];
        QXD_CUDA(ctx, cudaMemcpyAsync(acts[0], r + (size_t)i * hb, hb, cudaMemcpyDeviceToDevice, st));
        QXD_CUDA(ctx, cudaMemsetAsync(reinterpret_cast<char*>(acts[0]) + hb, 0, hb, st));
        QXD_TRY(ptc_forward(ctx, fl, W, nlayers, nch, acts.data(), st));
        float4* delta = static_cast<float4*>(dA);
        if (kind == 1) {
            // residual norm: res = Dhat (M r)_e - r; delta = Dhat^+ res / |r|^2 on even sites
            void *res, *to;
            QXD_TRY(qxd_ws(ctx, WS_PTC + 14, hb, &res));
            QXD_TRY(qxd_ws(ctx, WS_PTC + 15, hb, &to));
            QXD_TRY(op_Dhat(ctx, fl, QXD_FP32, 0, acts[nlayers], res, to, st));
            QXD_TRY(blas_axpby(ctx, 1, 1, n, -1.0, 0.0, r + (size_t)i * hb, 1.0, 0.0, res, st));
            QXD_TRY(blas_norm2(ctx, 1, n, res, 0, st));
            QXD_TRY(blas_fetch(ctx, 2, st));
            if (ctx->red_host[1] != 0.0) return qxd_fail(ctx, QXD_ENAN, "learned preconditioner: non-finite output");
            tot += ctx->red_host[0] / rr[i];
            QXD_TRY(op_Dhat(ctx, fl, QXD_FP32, 1, res, delta, to, st));
            QXD_CUDA(ctx, cudaMemsetAsync(reinterpret_cast<char*>(delta) + hb, 0, hb, st));
            QXD_TRY(blas_axpby(ctx, 1, 1, n, 0.0, 0.0, delta, 1.0 / rr[i], 0.0, delta, st));
        } else {
            // Euclidean error: delta = ((M r)_e - e) / |e|^2 on even sites, 0 on odd sites
            QXD_CUDA(ctx, cudaMemcpyAsync(delta, acts[nlayers], hb, cudaMemcpyDeviceToDevice, st));
            QXD_CUDA(ctx, cudaMemsetAsync(reinterpret_cast<char*>(delta) + hb, 0, hb, st));
            QXD_TRY(blas_axpby(ctx, 1, 1, n, -1.0, 0.0, e + (size_t)i * hb, 1.0, 0.0, delta, st));
            QXD_TRY(blas_norm2(ctx, 1, n, delta, 0, st));
            QXD_TRY(blas_fetch(ctx, 2, st));
            if (ctx->red_host[1] != 0.0) return qxd_fail(ctx, QXD_ENAN, "learned preconditioner: non-finite output");
            tot += ctx->red_host[0] / ee[i];
            QXD_TRY(blas_axpby(ctx, 1, 1, n, 0.0, 0.0, delta, 1.0 / ee[i], 0.0, delta, st));
        }
        if (!G) continue;
        float4* dcur = delta;
        float4* dnext = static_cast<float4*>(dB);
        for (int l = nlayers - 1; l >= 0; --l) {
            int ci, co;
            layer_shape(l, nlayers, nch, &ci, &co);
            const int nq = co * ci * 9;
            QXD_TRY(launch_wgrad(ctx, fl, dcur, acts[l], ci, co, static_cast<float2*>(part), G + off[l], st));
            if (l > 0) {
                k_ptc_adjoint_weights<<<nblocks(nq, 128), 128, 0, st>>>(W + off[l], ci, co,
                                                                        static_cast<float2*>(Wa));
                QXD_CUDA(ctx, cudaGetLastError());
                QXD_TRY(launch_layer(ctx, fl, dcur, co, static_cast<float2*>(Wa), dnext, ci, st));
                std::swap(dcur, dnext);
            }
        }
    }
    *loss = tot;
    return QXD_OK;
}

// pack canonical complex64 even fields into internal FP32 fields and their norms
static int pack_pairs(qxd_ctx* ctx, const void* r, const void* e, int npairs, char** R, char** E,
                      std::vector<double>& ee, std::vector<double>& rr, cudaStream_t st) {
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const size_t cb = (size_t)ctx->g.Vh * 12 * 8;
    void *dr, *de, *pr, *pe;
    QXD_TRY(qxd_ws(ctx, WS_PTC + 20, cb * npairs, &dr));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 21, cb * npairs, &de));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 22, hb * npairs, &pr));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 23, hb * npairs, &pe));
    QXD_CUDA(ctx, cudaMemcpyAsync(dr, r, cb * npairs, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(de, e, cb * npairs, cudaMemcpyDefault, st));
    QXD_TRY(launch_pack(ctx, 1, dr, 0, 0, QXD_FP32, pr, npairs, st));
    QXD_TRY(launch_pack(ctx, 1, de, 0, 0, QXD_FP32, pe, npairs, st));
    *R = static_cast<char*>(pr);
    *E = static_cast<char*>(pe);
    ee.resize(npairs);
    rr.resize(npairs);
    const size_t n = 12ull * ctx->g.Vh;
    for (int i = 0; i < npairs; ++i) {
        QXD_TRY(blas_norm2(ctx, 1, n, *E + (size_t)i * hb, 0, st));
        QXD_TRY(blas_norm2(ctx, 1, n, *R + (size_t)i * hb, 2, st));
        QXD_TRY(blas_fetch(ctx, 4, st));
        if (!(ctx->red_host[0] > 0.0) || !(ctx->red_host[2] > 0.0) || ctx->red_host[1] != 0.0 || ctx->red_host[3] != 0.0)
            return qxd_fail(ctx, QXD_EARG, "learned preconditioner: pair vectors must be finite and non-zero");
        ee[i] = ctx->red_host[0];
        rr[i] = ctx->red_host[2];
    }
    return QXD_OK;
}

static int weights_on_device(qxd_ctx* ctx, const float* W, size_t nw, int slot, float2** out, cudaStream_t st) {
    void* d;
    QXD_TRY(qxd_ws(ctx, slot, nw * sizeof(float2), &d));
    QXD_CUDA(ctx, cudaMemcpyAsync(d, W, nw * sizeof(float2), cudaMemcpyDefault, st));
    *out = static_cast<float2*>(d);
    return QXD_OK;
}

}  // namespace qxd

using namespace qxd;

static int ptc_check(qxd_ctx* ctx, int fl) {
    if (!ctx) return QXD_EARG;
    if (fl < 0 || fl >= QXD_MAX_FLAVOURS) return qxd_fail(ctx, QXD_EARG, "flavour id out of range 0..7");
    if (!ctx->links_set || !ctx->fl[fl].set)
        return qxd_fail(ctx, QXD_ESTATE, "learned preconditioner: links and SW term must be set first");
    cudaSetDevice(ctx->device);
    return QXD_OK;
}

extern "C" {

int qxd_set_precond_weights(qxd_ctx* ctx, int fl, const float* W, int nlayers, int nch, int prec) {
    QXD_TRY(ptc_check(ctx, fl));
    QXD_TRY(check_shape(ctx, nlayers, nch));
    if (prec != QXD_FP32 && prec != QXD_BF16)
        return qxd_fail(ctx, QXD_EARG, "set_precond_weights: precision must be QXD_FP32 or QXD_BF16");
    if (!W) return qxd_fail(ctx, QXD_EARG, "set_precond_weights: NULL weights");
    QxdFlavour& F = ctx->fl[fl];
    const size_t nw = ptc_weight_count(nlayers, nch);
    cudaFree(F.W);
    F.W = nullptr;
    if (cudaMalloc(&F.W, nw * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        return qxd_fail(ctx, QXD_ENOMEM, "set_precond_weights: allocation failed");
    }
    QXD_CUDA(ctx, cudaMemcpy(F.W, W, nw * sizeof(float2), cudaMemcpyDefault));
    F.nlayers = nlayers;
    F.nch = nch;
    F.wprec = prec;
    return QXD_OK;
}

int qxd_ptc_apply(qxd_ctx* ctx, int fl, int prec, const float* W, int nlayers, int nch, const void* in_e,
                  void* out_e, void* stream) {
    QXD_TRY(ptc_check(ctx, fl));
    QXD_TRY(check_shape(ctx, nlayers, nch));
    if (!W || !in_e || !out_e) return qxd_fail(ctx, QXD_EARG, "ptc_apply: NULL argument");
    if (prec != QXD_FP32 && prec != QXD_BF16)
        return qxd_fail(ctx, QXD_EARG, "ptc_apply: precision must be QXD_FP32 or QXD_BF16");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.Vh * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    float2* Wd;
    QXD_TRY(weights_on_device(ctx, W, ptc_weight_count(nlayers, nch), WS_PTC + 30, &Wd, st));
    void *ci, *ri, *zi, *co;
    QXD_TRY(qxd_ws(ctx, WS_PTC + 31, cb, &ci));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 32, hb, &ri));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 33, hb, &zi));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 34, cb, &co));
    QXD_CUDA(ctx, cudaMemcpyAsync(ci, in_e, cb, cudaMemcpyDefault, st));
    QXD_TRY(launch_pack(ctx, 1, ci, 0, 0, QXD_FP32, ri, 1, st));
    QXD_TRY(ptc_apply_internal(ctx, fl, Wd, nlayers, nch, ri, zi, st, prec));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, zi, 0, 1, co, 0, 1, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(out_e, co, cb, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    if (prec == QXD_BF16) {
        int flag = 0;
        QXD_CUDA(ctx, cudaMemcpy(&flag, ctx->dev_flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) return qxd_fail(ctx, QXD_ECUDA, "ptc_apply: a tensor-core completion wait timed out");
    }
    return QXD_OK;
}

int qxd_ptc_loss_grad(qxd_ctx* ctx, int fl, const float* W, int nlayers, int nch, const void* r, const void* e,
                      int npairs, int kind, double* loss, float* grad, void* stream) {
    QXD_TRY(ptc_check(ctx, fl));
    QXD_TRY(check_shape(ctx, nlayers, nch));
    if (!W || !r || !e || npairs < 1 || !loss || (kind != 0 && kind != 1))
        return qxd_fail(ctx, QXD_EARG, "ptc_loss_grad: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nw = ptc_weight_count(nlayers, nch);
    float2* Wd;
    QXD_TRY(weights_on_device(ctx, W, nw, WS_PTC + 30, &Wd, st));
    char *R, *E;
    std::vector<double> ee, rr;
    QXD_TRY(pack_pairs(ctx, r, e, npairs, &R, &E, ee, rr, st));
    void* G = nullptr;
    if (grad) {
        QXD_TRY(qxd_ws(ctx, WS_PTC + 35, nw * sizeof(float2), &G));
        QXD_CUDA(ctx, cudaMemsetAsync(G, 0, nw * sizeof(float2), st));
    }
    std::vector<int> idx(npairs);
    for (int i = 0; i < npairs; ++i) idx[i] = i;
    QXD_TRY(ptc_loss_grad_internal(ctx, fl, Wd, nlayers, nch, R, E, ee.data(), rr.data(), kind, idx.data(), npairs,
                                   static_cast<float2*>(G), loss, st));
    if (grad) QXD_CUDA(ctx, cudaMemcpyAsync(grad, G, nw * sizeof(float2), cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_ptc_train(qxd_ctx* ctx, int fl, float* W, float* m, float* v, int nlayers, int nch, const void* r,
                  const void* e, int npairs, int batch, int nsteps, double lr, int kind, int* t, double* losses,
                  void* stream) {
    QXD_TRY(ptc_check(ctx, fl));
    QXD_TRY(check_shape(ctx, nlayers, nch));
    if (!W || !m || !v || !r || !e || !t || npairs < 1 || batch < 1 || nsteps < 0 || !(lr > 0.0) ||
        (kind != 0 && kind != 1))
        return qxd_fail(ctx, QXD_EARG, "ptc_train: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nw = ptc_weight_count(nlayers, nch);
    float2 *Wd, *md, *vd;
    QXD_TRY(weights_on_device(ctx, W, nw, WS_PTC + 30, &Wd, st));
    QXD_TRY(weights_on_device(ctx, m, nw, WS_PTC + 36, &md, st));
    QXD_TRY(weights_on_device(ctx, v, nw, WS_PTC + 37, &vd, st));
    char *R, *E;
    std::vector<double> ee, rr;
    QXD_TRY(pack_pairs(ctx, r, e, npairs, &R, &E, ee, rr, st));
    void* G;
    QXD_TRY(qxd_ws(ctx, WS_PTC + 35, nw * sizeof(float2), &G));
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    std::vector<int> idx(batch);
    for (int s = 0; s < nsteps; ++s) {
        for (int k = 0; k < batch; ++k) idx[k] = (s * batch + k) % npairs;
        QXD_CUDA(ctx, cudaMemsetAsync(G, 0, nw * sizeof(float2), st));
        double L = 0.0;
        QXD_TRY(ptc_loss_grad_internal(ctx, fl, Wd, nlayers, nch, R, E, ee.data(), rr.data(), kind, idx.data(), batch,
                                       static_cast<float2*>(G), &L, st));
        if (losses) losses[s] = L / batch;
        *t += 1;
        const float c1 = 1.f - std::pow(b1, (float)*t), c2 = 1.f - std::pow(b2, (float)*t);
        ProfScope prof(ctx, "ptc_adam", 4.0 * 2 * nw * 4, st);
        k_adam<<<nblocks(2 * nw, 256), 256, 0, st>>>(reinterpret_cast<float*>(Wd), static_cast<const float*>(G),
                                                     reinterpret_cast<float*>(md), reinterpret_cast<float*>(vd),
                                                     2 * nw, 1.f / batch, (float)lr, b1, b2, eps, c1, c2);
        QXD_CUDA(ctx, cudaGetLastError());
    }
    QXD_CUDA(ctx, cudaMemcpyAsync(W, Wd, nw * sizeof(float2), cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(m, md, nw * sizeof(float2), cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(v, vd, nw * sizeof(float2), cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_ptc_record_pairs(qxd_ctx* ctx, int fl, const void* b, int npairs, int stride, void* r_out, void* e_out,
                         void* stream) {
    QXD_TRY(ptc_check(ctx, fl));
    if (!b || !r_out || !e_out || npairs < 1 || stride < 1) return qxd_fail(ctx, QXD_EARG, "ptc_record_pairs: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    const size_t cb64 = (size_t)ctx->g.Vh * 12 * 16, cb32 = (size_t)ctx->g.Vh * 12 * 8;
    void *cbuf, *bb, *y, *s, *z, *p, *w, *to, *ys, *c32;
    QXD_TRY(qxd_ws(ctx, WS_PTC + 40, cb64, &cbuf));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 41, hb, &bb));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 42, hb, &y));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 43, hb, &s));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 44, hb, &z));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 45, hb, &p));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 46, hb, &w));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 47, hb, &to));
    QXD_TRY(qxd_ws(ctx, WS_PTC + 48, hb * npairs, &ys));      // iterates x_k (FP64)
    QXD_TRY(qxd_ws(ctx, WS_PTC + 49, 2 * cb32 * npairs, &c32));  // canonical r, e (complex64)
    QXD_CUDA(ctx, cudaMemcpyAsync(cbuf, b, cb64, cudaMemcpyDefault, st));
    QXD_TRY(launch_pack(ctx, 0, cbuf, 0, 0, QXD_FP64, bb, 1, st));
    // CGNR on Dhat y = b (y = 0), recording (s_k, y_k) every `stride` iterations
    QXD_CUDA(ctx, cudaMemsetAsync(y, 0, hb, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(s, bb, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(op_Dhat(ctx, fl, 0, 1, s, z, to, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(p, z, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, 0, n, bb, 0, st));
    QXD_TRY(blas_norm2(ctx, 0, n, z, 2, st));
    QXD_TRY(blas_fetch(ctx, 4, st));
    const double bn = std::sqrt(ctx->red_host[0]);
    double zz = ctx->red_host[2];
    if (!(bn > 0.0) || ctx->red_host[1] != 0.0) return qxd_fail(ctx, QXD_EARG, "ptc_record_pairs: bad source");
    char* R32 = static_cast<char*>(c32);
    char* E32 = R32 + cb32 * npairs;
    int rec = 0;
    const int nmx = 100000;
    bool conv = false;
    for (int k = 1; k <= nmx; ++k) {
        QXD_TRY(op_Dhat(ctx, fl, 0, 0, p, w, to, st));
        QXD_TRY(blas_norm2(ctx, 0, n, w, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        const double alpha = zz / ctx->red_host[0];
        QXD_TRY(blas_axpby(ctx, 0, 0, n, alpha, 0.0, p, 1.0, 0.0, y, st));
        QXD_TRY(blas_axpby(ctx, 0, 0, n, -alpha, 0.0, w, 1.0, 0.0, s, st));
        if (rec < npairs && k % stride == 0) {
            // r_k = s_k (the residual b - Dhat y_k), keep y_k for e_k = x* - y_k
            QXD_TRY(launch_unpack(ctx, QXD_FP64, s, 0, 1, R32 + (size_t)rec * cb32, 0, 1, st));
            QXD_CUDA(ctx, cudaMemcpyAsync(static_cast<char*>(ys) + (size_t)rec * hb, y, hb, cudaMemcpyDeviceToDevice,
                                          st));
            ++rec;
        }
        QXD_TRY(op_Dhat(ctx, fl, 0, 1, s, z, to, st));
        QXD_TRY(blas_norm2(ctx, 0, n, s, 0, st));
        QXD_TRY(blas_norm2(ctx, 0, n, z, 2, st));
        QXD_TRY(blas_fetch(ctx, 4, st));
        if (std::sqrt(ctx->red_host[0]) <= 1e-10 * bn) {
            conv = true;
            break;
        }
        const double beta = ctx->red_host[2] / zz;
        zz = ctx->red_host[2];
        QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, z, beta, 0.0, p, st));
    }
    if (!conv) return qxd_fail(ctx, QXD_ENOCONV, "ptc_record_pairs: CGNR did not converge");
    if (rec < npairs) return qxd_fail(ctx, QXD_EARG, "ptc_record_pairs: fewer iterations than npairs * stride");
    // e_i = x* - y_i
    for (int i = 0; i < npairs; ++i) {
        char* yi = static_cast<char*>(ys) + (size_t)i * hb;
        QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, y, -1.0, 0.0, yi, st));
        QXD_TRY(launch_unpack(ctx, QXD_FP64, yi, 0, 1, E32 + (size_t)i * cb32, 0, 1, st));
    }
    QXD_CUDA(ctx, cudaMemcpyAsync(r_out, R32, cb32 * npairs, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(e_out, E32, cb32 * npairs, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

}  // extern "C"
