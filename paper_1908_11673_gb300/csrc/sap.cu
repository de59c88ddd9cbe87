// Schwarz alternating procedure (SAP) preconditioner (Sec. 4.1 and 4.4: SAP+GCR,
// blocks of 4^4 sites, ncy cycles, nmr minimal-residual steps per block).
//
// Blocks of 4^4 sites tile the simulated lattice and are coloured like a
// checkerboard by the parity of the block coordinates.  The block operator is
// D with Dirichlet block boundaries (hops leaving the block dropped).  One
// application M eta: psi = 0, rho = eta; ncy times, for each colour: every block
// of that colour solves its block system approximately (even-odd system of the
// block, nmr minimal-residual steps from zero) for the current residual
// rho = eta - D psi restricted to the block, and psi += d on the block.  As a
// preconditioner of Dhat: z_e = (M (r_e, 0))_e.  Every extent must hold an even
// number of blocks, so that blocks of one colour never touch, across the
// periodic boundary included.
//
// GPU layout: one launch per colour sweep, one CTA per block, 128 threads; thread
// t owns the t-th even and the t-th odd site of the block.  The block's links are
// staged in shared memory once per sweep, so the 2 nmr + 2 block hops of the
// minimal-residual steps read links and neighbour spinors from shared memory only.
// The sweep also computes the block residual rho = eta - D psi itself (the
// other colour's psi on the one-site halo comes from global memory), so no
// full-lattice residual is formed between colours.  Site-diagonal terms are
// streamed from global memory.  FP32 throughout, block sums in FP32.
#include <cmath>

#include "blas.h"
#include "block.cuh"
#include "hop.cuh"
#include "ops.h"
#include "qxd_internal.h"

namespace qxd {

constexpr int kSapB = kBlk;
constexpr int kSapThreads = kBlkThreads;
constexpr int kSapSites = kBlkSites;

struct SapDev {
    int nb[4];              // blocks per direction
    const float4* U32[2];   // links per parity
    const float4* Z32[2];   // phases per parity
    const float4* A[2];     // site-diagonal term per parity
    const float4* Aoo_inv;  // its inverse, odd sites
    const float4* eta;      // source, full field (even half, odd half)
    float4* psi;            // solution, full field
    int nmr;
};

// shared memory of one block: its links, two half-block spinor buffers and the
// odd residual, all structure-of-arrays over the block's sites
struct SapShared {
    float2 lk[4][7][kSapSites];      // U rows 0, 1 (6 complex) and z^qhat, per direction and local site
    float2 sp[2][12][kSapThreads];   // spinor buffers by parity
    float2 rho_o[12][kSapThreads];   // residual on the odd sites
    float red[3 * kSapThreads / 32];
};

__device__ __forceinline__ void load_sm(const float2 (*sm)[kSapThreads], int t, cplx<float> s[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float2 v = sm[k][t];
        s[k] = {v.x, v.y};
    }
}
__device__ __forceinline__ void store_sm(float2 (*sm)[kSapThreads], int t, const cplx<float> s[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) sm[k][t] = make_float2(s[k].re, s[k].im);
}

// link of direction mu at the block's local site sid (= parity * 128 + thread) from shared memory
__device__ __forceinline__ void link_sm(const SapShared& S, int mu, int sid, Mat3<float>& m, cplx<float>& z) {
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float2 v = S.lk[mu][3 * i + j][sid];
            m.a[i][j] = {v.x, v.y};
        }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        m.a[2][j] = conj(m.a[0][j1] * m.a[1][j2] - m.a[0][j2] * m.a[1][j1]);
    }
    const float2 zz = S.lk[mu][6][sid];
    z = {zz.x, zz.y};
}

__device__ __forceinline__ void phase_mul(cplx<float> z, bool dag, Half<float>& o) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.a[sp][c] = dag ? cmul_conj(z, o.a[sp][c]) : z * o.a[sp][c];
}

// acc += hop terms of direction MU at site s (parity p) from the opposite-parity
// spinor buffer nb.  HALO = false: hops leaving the block are dropped (block
// operator).  HALO = true: they take the spinor of the neighbouring site from the
// global field nb_glob (opposite parity) and, backwards, its link from global memory.
// spin projection / reconstruction for the hop d = 2 mu + (0 forward, 1 backward),
// chosen at run time
__device__ __forceinline__ void project_rt(int d, const cplx<float> v[12], Half<float>& hp) {
    switch (d) {
        case 0: project<0, true>(v, hp); break;
        case 1: project<0, false>(v, hp); break;
        case 2: project<1, true>(v, hp); break;
        case 3: project<1, false>(v, hp); break;
        case 4: project<2, true>(v, hp); break;
        case 5: project<2, false>(v, hp); break;
        case 6: project<3, true>(v, hp); break;
        default: project<3, false>(v, hp); break;
    }
}
__device__ __forceinline__ void reconstruct_rt(int d, const Half<float>& o, cplx<float> acc[12]) {
    switch (d) {
        case 0: reconstruct<0, true>(o, acc); break;
        case 1: reconstruct<0, false>(o, acc); break;
        case 2: reconstruct<1, true>(o, acc); break;
        case 3: reconstruct<1, false>(o, acc); break;
        case 4: reconstruct<2, true>(o, acc); break;
        case 5: reconstruct<2, false>(o, acc); break;
        case 6: reconstruct<3, true>(o, acc); break;
        default: reconstruct<3, false>(o, acc); break;
    }
}

// out = -1/2 sum_mu [(1 - gamma_mu) V(x,mu) f(x+mu) + (1 + gamma_mu) V(x-mu,mu)^+ f(x-mu)]
// at site s of parity p, f the opposite-parity spinors in the buffer nb.
// HALO = false: hops leaving the block are dropped (block operator).  HALO = true:
// they take the spinor of the neighbouring site from the global field nb_glob
// (opposite parity) and, backwards, its link from global memory.
// The eight hops run as one loop with the direction chosen at run time, so the
// colour multiplication exists once in the code: the sweep calls this six times,
// and fully unrolled copies overflow the instruction cache.
template <bool HALO>
__device__ __forceinline__ void hop_sap(const Geo& g, const SapDev& a, const SapShared& S, const SiteRef& s, int p,
                                        const float2 (*nb)[kSapThreads], const float4* nb_glob, cplx<float> out[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = {0.f, 0.f};
    const int t = block_thread(s.l);
    const int sid = p * kSapThreads + t;
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int lmu = mu == 0 ? s.l[0] : mu == 1 ? s.l[1] : mu == 2 ? s.l[2] : s.l[3];
        const bool inside = fwd ? lmu + 1 < kSapB : lmu > 0;
        if (!inside && !HALO) continue;
        cplx<float> v[12];
        Mat3<float> m;
        cplx<float> z;
        if (inside) {
            // thread index of the neighbour within its parity
            const int l3 = s.l[3];
            const int step = mu == 0 ? 32 : mu == 1 ? 8 : mu == 2 ? 2 : 0;
            const int tn = mu < 3 ? (fwd ? t + step : t - step) : (fwd ? t + (l3 & 1) : t - ((l3 & 1) ^ 1));
            load_sm(nb, tn, v);
            link_sm(S, mu, fwd ? sid : (1 - p) * kSapThreads + tn, m, z);
        } else {
            const int hn = neighbour_lex(g, s.x, mu, fwd ? +1 : -1) >> 1;
            load_spinor<1>(nb_glob, g.Vh, hn, v);
            if (fwd) link_sm(S, mu, sid, m, z);
            else load_link32(a.U32[1 - p], a.Z32[1 - p], g.Vh, mu, hn, m, z);
        }
        Half<float> hp, o;
        project_rt(d, v, hp);
        if (fwd) mul_half<false>(m, hp, o);
        else mul_half<true>(m, hp, o);
        phase_mul(z, !fwd, o);
        reconstruct_rt(d, o, out);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = -0.5f * out[k];
}

// s = D s for a packed site-diagonal term (two Hermitian 6x6 blocks), streamed
// from global memory one block at a time
__device__ __forceinline__ void diag_mul(const float4* __restrict__ D, int Vh, int h, cplx<float> s[12]) {
#pragma unroll
    for (int blk = 0; blk < 2; ++blk) {
        float d[36];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 v = QXD_LDG(D + (size_t)(blk * 9 + k) * Vh + h);
            d[4 * k] = v.x;
            d[4 * k + 1] = v.y;
            d[4 * k + 2] = v.z;
            d[4 * k + 3] = v.w;
        }
        cplx<float> o[6];
        herm6_mul(d, s + 6 * blk, o);
#pragma unroll
        for (int i = 0; i < 6; ++i) s[6 * blk + i] = o[i];
    }
}

// sum over the CTA of three floats
__device__ __forceinline__ void cta_sum3(float v[3], float* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < 3; ++k) sh[warp * 3 + k] = v[k];
    __syncthreads();
    for (int k = 0; k < 3; ++k) {
        float s = 0.f;
        for (int w = 0; w < kSapThreads / 32; ++w) s += sh[w * 3 + k];
        v[k] = s;
    }
    __syncthreads();
}

// One colour sweep of SAP: every block of colour `colour` (one CTA each) takes
// its residual rho = eta - D psi (FIRST: psi = 0, so rho = eta), solves its
// Dirichlet block system approximately by nmr minimal-residual steps on the
// block's even-odd system, and adds the block solution to psi.  Blocks of one
// colour never touch, so every CTA reads the other colour's psi on its halo
// and writes its own sites only.
template <bool FIRST>
__global__ void __launch_bounds__(kSapThreads) k_sap_sweep(Geo g, SapDev a, int colour) {
    extern __shared__ __align__(16) unsigned char sap_smem[];
    SapShared& S = *reinterpret_cast<SapShared*>(sap_smem);
    int bc[4];
    block_coords(blockIdx.x, a.nb, bc);
    if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) return;
    const int t = threadIdx.x;
    const int Vh = g.Vh;
    SiteRef se, so;
    block_site(g, bc, 0, t, se);
    block_site(g, bc, 1, t, so);
    // the block's links into shared memory (this thread: its even and its odd site)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int h = p == 0 ? se.h : so.h;
        const int sid = p * kSapThreads + t;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            const float4 c0 = QXD_LDG(a.U32[p] + (size_t)(mu * 3 + 0) * Vh + h);
            const float4 c1 = QXD_LDG(a.U32[p] + (size_t)(mu * 3 + 1) * Vh + h);
            const float4 c2 = QXD_LDG(a.U32[p] + (size_t)(mu * 3 + 2) * Vh + h);
            S.lk[mu][0][sid] = make_float2(c0.x, c0.y);
            S.lk[mu][1][sid] = make_float2(c0.z, c0.w);
            S.lk[mu][2][sid] = make_float2(c1.x, c1.y);
            S.lk[mu][3][sid] = make_float2(c1.z, c1.w);
            S.lk[mu][4][sid] = make_float2(c2.x, c2.y);
            S.lk[mu][5][sid] = make_float2(c2.z, c2.w);
        }
        const float4 z01 = QXD_LDG(a.Z32[p] + h);
        const float4 z23 = QXD_LDG(a.Z32[p] + (size_t)Vh + h);
        S.lk[0][6][sid] = make_float2(z01.x, z01.y);
        S.lk[1][6][sid] = make_float2(z01.z, z01.w);
        S.lk[2][6][sid] = make_float2(z23.x, z23.y);
        S.lk[3][6][sid] = make_float2(z23.z, z23.w);
    }
    const float4* psi_e = a.psi;
    const float4* psi_o = a.psi + 6 * (size_t)Vh;
    cplx<float> v[12], r[12], y[12], p[12];
    // residual rho = eta - D psi on the block's sites: r (even), rho_o (odd, shared)
    load_spinor<1>(a.eta, Vh, se.h, r);
    load_spinor<1>(a.eta + 6 * (size_t)Vh, Vh, so.h, y);
    if (!FIRST) {
        load_spinor<1>(psi_e, Vh, se.h, v);
        store_sm(S.sp[0], t, v);
        load_spinor<1>(psi_o, Vh, so.h, p);
        store_sm(S.sp[1], t, p);
        __syncthreads();
        // even site: A_ee psi_e + H_eo psi_o
        diag_mul(a.A[0], Vh, se.h, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) r[k] = r[k] - v[k];
        hop_sap<true>(g, a, S, se, 0, S.sp[1], psi_o, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) r[k] = r[k] - v[k];
        // odd site: A_oo psi_o + H_oe psi_e
        diag_mul(a.A[1], Vh, so.h, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = y[k] - p[k];
        hop_sap<true>(g, a, S, so, 1, S.sp[0], psi_e, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = y[k] - v[k];
    }
    store_sm(S.rho_o, t, y);
    // t_o = A_oo^-1 rho_o;  b_e = rho_e - H^B_eo t_o
    diag_mul(a.Aoo_inv, Vh, so.h, y);
    __syncthreads();  // every thread is done with the psi buffers
    store_sm(S.sp[1], t, y);
    __syncthreads();
    hop_sap<false>(g, a, S, se, 0, S.sp[1], nullptr, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        r[k] = r[k] - v[k];
        y[k] = {0.f, 0.f};
    }
    store_sm(S.sp[0], t, r);
    __syncthreads();
    for (int it = 0; it < a.nmr; ++it) {
        // t_o = A_oo^-1 H^B_oe r_e
        hop_sap<false>(g, a, S, so, 1, S.sp[0], nullptr, v);
        diag_mul(a.Aoo_inv, Vh, so.h, v);
        store_sm(S.sp[1], t, v);
        __syncthreads();
        // p = Dhat_B r = A_ee r - H^B_eo t_o
        hop_sap<false>(g, a, S, se, 0, S.sp[1], nullptr, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = r[k];
        diag_mul(a.A[0], Vh, se.h, p);
        float s3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k] = p[k] - v[k];
            s3[0] += p[k].re * r[k].re + p[k].im * r[k].im;  // <p, r> = sum conj(p) r
            s3[1] += p[k].re * r[k].im - p[k].im * r[k].re;
            s3[2] += p[k].re * p[k].re + p[k].im * p[k].im;
        }
        cta_sum3(s3, S.red);
        const cplx<float> alpha = s3[2] > 0.f ? cplx<float>{s3[0] / s3[2], s3[1] / s3[2]} : cplx<float>{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            cmac(y[k], alpha, r[k]);
            r[k] = r[k] - alpha * p[k];
        }
        store_sm(S.sp[0], t, r);
        __syncthreads();
    }
    // d_o = A_oo^-1 (rho_o - H^B_oe y);  psi += d
    store_sm(S.sp[0], t, y);
    __syncthreads();
    hop_sap<false>(g, a, S, so, 1, S.sp[0], nullptr, v);
    load_sm(S.rho_o, t, p);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = p[k] - v[k];
    diag_mul(a.Aoo_inv, Vh, so.h, v);
    if (!FIRST) {
        load_spinor<1>(psi_e, Vh, se.h, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) y[k] = y[k] + p[k];
        load_spinor<1>(psi_o, Vh, so.h, p);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = v[k] + p[k];
    }
    store_spinor<1>(a.psi, Vh, se.h, y);
    store_spinor<1>(a.psi + 6 * (size_t)Vh, Vh, so.h, v);
}

int sap_check(qxd_ctx* ctx) {
    for (int mu = 0; mu < 4; ++mu)
        if (ctx->g.N[mu] % (2 * kSapB))
            return qxd_fail(ctx, QXD_EARG, "SAP: every simulated extent must be a multiple of 8 (an even number of 4^4 blocks)");
    return QXD_OK;
}

// psi = M eta on full FP32 fields (even half then odd half); psi must not alias eta
int sap_apply_full(qxd_ctx* ctx, int fl, const float4* eta, float4* psi, cudaStream_t st) {
    QXD_TRY(sap_check(ctx));
    const Geo& g = ctx->g;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const QxdFlavour& F = ctx->fl[fl];
    SapDev a;
    int nblk = 1;
    for (int mu = 0; mu < 4; ++mu) {
        a.nb[mu] = g.N[mu] / kSapB;
        nblk *= a.nb[mu];
    }
    for (int p = 0; p < 2; ++p) {
        a.U32[p] = ctx->U32 + (size_t)p * 12 * g.Vh;
        a.Z32[p] = F.Z32 + (size_t)p * 2 * g.Vh;
        a.A[p] = F.C32[0] + (size_t)p * 18 * g.Vh;
    }
    a.Aoo_inv = F.C32[1] + (size_t)18 * g.Vh;
    a.eta = eta;
    a.psi = psi;
    a.nmr = ctx->sap_nmr;
    const int smem = (int)sizeof(SapShared);
    QXD_CUDA(ctx, cudaFuncSetAttribute(k_sap_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    QXD_CUDA(ctx, cudaFuncSetAttribute(k_sap_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    QXD_CUDA(ctx, cudaMemsetAsync(psi, 0, 2 * hb, st));
    // algorithmic bytes per site of a sweep's colour: own links 224, eta 96, psi of the
    // block and its halo 192, psi written 96, A 288, A_oo^-1 on odd sites 144, halo links 56
    const double site_bytes = 224 + 96 + 192 + 96 + 288 + 144 + 56;
    for (int cy = 0; cy < ctx->sap_ncy; ++cy) {
        for (int colour = 0; colour < 2; ++colour) {
            ProfScope prof(ctx, "sap_sweep", (double)g.Vh * site_bytes, st);
            if (cy == 0 && colour == 0)
                k_sap_sweep<true><<<nblk, kSapThreads, smem, st>>>(g, a, colour);
            else
                k_sap_sweep<false><<<nblk, kSapThreads, smem, st>>>(g, a, colour);
            QXD_CUDA(ctx, cudaGetLastError());
        }
    }
    return QXD_OK;
}

// z_e = (M (r_e, 0))_e on FP32 even fields
int sap_apply_even(qxd_ctx* ctx, int fl, const void* r_e, void* z_e, cudaStream_t st) {
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void *eta, *psi;
    QXD_TRY(qxd_ws(ctx, WS_SAP + 2, 2 * hb, &eta));
    QXD_TRY(qxd_ws(ctx, WS_SAP + 3, 2 * hb, &psi));
    QXD_CUDA(ctx, cudaMemcpyAsync(eta, r_e, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemsetAsync(static_cast<char*>(eta) + hb, 0, hb, st));
    QXD_TRY(sap_apply_full(ctx, fl, static_cast<const float4*>(eta), static_cast<float4*>(psi), st));
    QXD_CUDA(ctx, cudaMemcpyAsync(z_e, psi, hb, cudaMemcpyDeviceToDevice, st));
    return QXD_OK;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_set_sap(qxd_ctx* ctx, int ncy, int nmr) {
    if (!ctx) return QXD_EARG;
    if (ncy < 1 || ncy > 64 || nmr < 1 || nmr > 64) return qxd_fail(ctx, QXD_EARG, "set_sap: ncy and nmr in 1..64");
    ctx->sap_ncy = ncy;
    ctx->sap_nmr = nmr;
    return QXD_OK;
}

int qxd_sap_apply(qxd_ctx* ctx, int fl, const void* in, void* out, void* stream) {
    if (!ctx) return QXD_EARG;
    if (fl < 0 || fl >= QXD_MAX_FLAVOURS) return qxd_fail(ctx, QXD_EARG, "flavour id out of range 0..7");
    if (!ctx->links_set || !ctx->fl[fl].set) return qxd_fail(ctx, QXD_ESTATE, "sap_apply: links and SW term first");
    if (!in || !out) return qxd_fail(ctx, QXD_EARG, "sap_apply: NULL argument");
    QXD_TRY(sap_check(ctx));
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void *cin, *cout, *fin, *fout;
    QXD_TRY(qxd_ws(ctx, WS_SAP + 4, cb, &cin));
    QXD_TRY(qxd_ws(ctx, WS_SAP + 5, cb, &cout));
    QXD_TRY(qxd_ws(ctx, WS_SAP + 6, 2 * hb, &fin));
    QXD_TRY(qxd_ws(ctx, WS_SAP + 7, 2 * hb, &fout));
    QXD_CUDA(ctx, cudaMemcpyAsync(cin, in, cb, cudaMemcpyDefault, st));
    char* fi = static_cast<char*>(fin);
    char* fo = static_cast<char*>(fout);
    QXD_TRY(launch_pack(ctx, 1, cin, 1, 0, QXD_FP32, fi, 1, st));
    QXD_TRY(launch_pack(ctx, 1, cin, 1, 1, QXD_FP32, fi + hb, 1, st));
    QXD_TRY(sap_apply_full(ctx, fl, reinterpret_cast<const float4*>(fi), reinterpret_cast<float4*>(fo), st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, fo, 0, 1, cout, 1, 1, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, fo + hb, 1, 1, cout, 1, 1, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(out, cout, cb, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

}  // extern "C"
