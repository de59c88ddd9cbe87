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
// GPU layout: one launch per colour sweep, one CTA per block, 256 threads; the lane
// pair (2u, 2u + 1) owns the u-th even and the u-th odd site of the block, lane h
// the chiral block (spins 2h, 2h + 1) of every field, so that a lane keeps half a
// spinor per field and applies one 6 x 6 block of the site-diagonal terms (128
// registers, two CTAs and 16 warps per SM).  The block's links are
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
constexpr int kSapLanes = 2 * kSapThreads;  // threads of a sweep CTA: two lanes per (even, odd) site pair

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
    float red[3 * kSapLanes / 32];
};

// A pair of adjacent lanes (2u, 2u + 1) owns the u-th even and the u-th odd site
// of the block; lane `half` holds the spins 2 half, 2 half + 1 (its chiral block,
// complex components 6 half .. 6 half + 5) of every field it keeps.
__device__ __forceinline__ void load6_sm(const float2 (*sm)[kSapThreads], int u, int half, cplx<float> v[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 x = sm[6 * half + k][u];
        v[k] = {x.x, x.y};
    }
}
__device__ __forceinline__ void store6_sm(float2 (*sm)[kSapThreads], int u, int half, const cplx<float> v[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) sm[6 * half + k][u] = make_float2(v[k].re, v[k].im);
}
// the chiral block of a global FP32 field: complex 6 half + k is in chunk 3 half + k / 2
__device__ __forceinline__ void load6_glob(const float4* __restrict__ b, int Vh, int h, int half, cplx<float> v[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 f = QXD_LDG(b + (size_t)(3 * half + c) * Vh + h);
        v[2 * c] = {f.x, f.y};
        v[2 * c + 1] = {f.z, f.w};
    }
}
__device__ __forceinline__ void store6_glob(float4* __restrict__ b, int Vh, int h, int half, const cplx<float> v[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
        b[(size_t)(3 * half + c) * Vh + h] = make_float4(v[2 * c].re, v[2 * c].im, v[2 * c + 1].re, v[2 * c + 1].im);
}
// spin sp (three colours) of a site
__device__ __forceinline__ void load_spin_sm(const float2 (*sm)[kSapThreads], int u, int sp, cplx<float> v[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float2 x = sm[3 * sp + c][u];
        v[c] = {x.x, x.y};
    }
}
__device__ __forceinline__ void load_spin_glob(const float4* __restrict__ b, int Vh, int h, int sp, cplx<float> v[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int k = 3 * sp + c;
        const float4 f = QXD_LDG(b + (size_t)(k >> 1) * Vh + h);
        v[c] = (k & 1) ? cplx<float>{f.z, f.w} : cplx<float>{f.x, f.y};
    }
}

// link of direction mu at the block's local site sid (= parity * 128 + slot) from shared memory
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

// This lane's chiral block of
//   out = -1/2 sum_mu [(1 - gamma_mu) V(x,mu) f(x+mu) + (1 + gamma_mu) V(x-mu,mu)^+ f(x-mu)]
// at site s of parity p, f the opposite-parity spinors in the buffer nb.  HALO = false:
// hops leaving the block are dropped (block operator); HALO = true: they take the
// spinor of the neighbouring site from the global field nb_glob and, backwards, its
// link from global memory.  Lane `half` forms the half-spinor component `half` of
// each projection (spins half and its partner), multiplies it by the link and adds it
// into spin half (accO) and into the lower spin it feeds (accP = spin 2 + half for
// directions 0, 3; accQ = spin 3 - half for directions 1, 2); the two lanes then
// exchange their partial sums.  The eight hops run as one loop with run-time signs,
// so the colour multiplication exists once in the code.
template <bool HALO>
__device__ __forceinline__ void hop_pair(const Geo& g, const SapDev& a, const SapShared& S, const SiteRef& s, int p,
                                         const float2 (*nb)[kSapThreads], const float4* nb_glob, int half,
                                         cplx<float> out[6]) {
    cplx<float> accO[3], accP[3], accQ[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) accO[c] = accP[c] = accQ[c] = {0.f, 0.f};
    const int t = block_thread(s.l);
    const int sid = p * kSapThreads + t;
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const int lmu = mu == 0 ? s.l[0] : mu == 1 ? s.l[1] : mu == 2 ? s.l[2] : s.l[3];
        const bool inside = fwd ? lmu + 1 < kSapB : lmu > 0;
        if (!inside && !HALO) continue;
        const int partner = (mu == 0 || mu == 3) ? 2 + half : 3 - half;
        cplx<float> sa[3], sb[3];
        Mat3<float> m;
        cplx<float> z;
        if (inside) {
            const int l3 = s.l[3];
            const int step = mu == 0 ? 32 : mu == 1 ? 8 : mu == 2 ? 2 : 0;
            const int tn = mu < 3 ? (fwd ? t + step : t - step) : (fwd ? t + (l3 & 1) : t - ((l3 & 1) ^ 1));
            load_spin_sm(nb, tn, half, sa);
            load_spin_sm(nb, tn, partner, sb);
            link_sm(S, mu, fwd ? sid : (1 - p) * kSapThreads + tn, m, z);
        } else {
            const int hn = neighbour_lex(g, s.x, mu, fwd ? +1 : -1) >> 1;
            load_spin_glob(nb_glob, g.Vh, hn, half, sa);
            load_spin_glob(nb_glob, g.Vh, hn, partner, sb);
            if (fwd) link_sm(S, mu, sid, m, z);
            else load_link32(a.U32[1 - p], a.Z32[1 - p], g.Vh, mu, hn, m, z);
        }
        // projection (1 -+ gamma_mu), component `half`: s_half + f s_partner, f = +-1 or +-i
        const bool imag = (mu & 1) != 0;
        const bool negp = mu < 2 ? !fwd : (fwd == (half == 1));
        cplx<float> hp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cplx<float> tb = imag ? times_i(sb[c]) : sb[c];
            hp[c] = negp ? sa[c] - tb : sa[c] + tb;
        }
        // colour: V hp forwards, V^+ hp backwards; then the U(1) phase
        cplx<float> r[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cplx<float> acc = {0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (fwd) cmac(acc, m.a[i][j], hp[j]);
                else cmac_conj(acc, m.a[j][i], hp[j]);
            }
            r[i] = fwd ? z * acc : cmul_conj(z, acc);
        }
        // reconstruction: spin half gets r, the lower spin it feeds +-r or +-i r
        const bool negr = mu == 0 ? !fwd : mu == 1 ? fwd : mu == 2 ? (fwd == (half == 1)) : (fwd == (half == 0));
        const bool to_p = mu == 0 || mu == 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            accO[c] = accO[c] + r[c];
            cplx<float> dl = imag ? times_i(r[c]) : r[c];
            if (negr) dl = -dl;
            if (to_p) accP[c] = accP[c] + dl;
            else accQ[c] = accQ[c] + dl;
        }
    }
    // lane 0 takes spins 0 (own accO) and 1 (partner's accO); lane 1 spin 2 (lane 0's
    // accP + own accQ) and spin 3 (lane 0's accQ + own accP)
    cplx<float> pO[3], pP[3], pQ[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        pO[c] = {__shfl_xor_sync(0xffffffffu, accO[c].re, 1), __shfl_xor_sync(0xffffffffu, accO[c].im, 1)};
        pP[c] = {__shfl_xor_sync(0xffffffffu, accP[c].re, 1), __shfl_xor_sync(0xffffffffu, accP[c].im, 1)};
        pQ[c] = {__shfl_xor_sync(0xffffffffu, accQ[c].re, 1), __shfl_xor_sync(0xffffffffu, accQ[c].im, 1)};
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<float> s0 = half == 0 ? accO[c] : pP[c] + accQ[c];
        const cplx<float> s1 = half == 0 ? pO[c] : pQ[c] + accP[c];
        out[c] = -0.5f * s0;
        out[3 + c] = -0.5f * s1;
    }
}

// v = D v for this lane's chiral block of a packed site-diagonal term (one
// Hermitian 6x6 block, 9 float4), streamed from global memory
__device__ __forceinline__ void diag6(const float4* __restrict__ D, int Vh, int h, int half, cplx<float> v[6]) {
    float d[36];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float4 f = QXD_LDG(D + (size_t)(half * 9 + k) * Vh + h);
        d[4 * k] = f.x;
        d[4 * k + 1] = f.y;
        d[4 * k + 2] = f.z;
        d[4 * k + 3] = f.w;
    }
    cplx<float> o[6];
    herm6_mul(d, v, o);
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = o[i];
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
        for (int w = 0; w < kSapLanes / 32; ++w) s += sh[w * 3 + k];
        v[k] = s;
    }
    __syncthreads();
}

// One colour sweep of SAP: every block of colour `colour` (one CTA each) takes
// its residual rho = eta - D psi (FIRST: psi = 0, so rho = eta), solves its
// Dirichlet block system approximately by nmr minimal-residual steps on the
// block's even-odd system, and adds the block solution to psi.  Blocks of one
// colour never touch, so every CTA reads the other colour's psi on its halo
// and writes its own sites only.  Two lanes per site pair (one chiral block each).
template <bool FIRST>
__global__ void __launch_bounds__(kSapLanes, 2) k_sap_sweep(Geo g, SapDev a, int colour) {
    extern __shared__ __align__(16) unsigned char sap_smem[];
    SapShared& S = *reinterpret_cast<SapShared*>(sap_smem);
    int bc[4];
    block_coords(blockIdx.x, a.nb, bc);
    if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) return;
    const int u = threadIdx.x >> 1;
    const int half = threadIdx.x & 1;
    const int Vh = g.Vh;
    SiteRef se, so;
    block_site(g, bc, 0, u, se);
    block_site(g, bc, 1, u, so);
    // the block's links into shared memory: lane `half` stages directions 2 half, 2 half + 1
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const int h = p == 0 ? se.h : so.h;
        const int sid = p * kSapThreads + u;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int mu = 2 * half + q;
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
        const float4 zz = QXD_LDG(a.Z32[p] + (size_t)half * Vh + h);
        S.lk[2 * half][6][sid] = make_float2(zz.x, zz.y);
        S.lk[2 * half + 1][6][sid] = make_float2(zz.z, zz.w);
    }
    const float4* psi_e = a.psi;
    const float4* psi_o = a.psi + 6 * (size_t)Vh;
    cplx<float> v[6], r[6], y[6], pv[6];
    // residual rho = eta - D psi on the block's sites: r (even), rho_o (odd, shared)
    load6_glob(a.eta, Vh, se.h, half, r);
    load6_glob(a.eta + 6 * (size_t)Vh, Vh, so.h, half, y);
    if (!FIRST) {
        load6_glob(psi_e, Vh, se.h, half, v);
        store6_sm(S.sp[0], u, half, v);
        load6_glob(psi_o, Vh, so.h, half, pv);
        store6_sm(S.sp[1], u, half, pv);
        __syncthreads();
        // even site: A_ee psi_e + H_eo psi_o
        diag6(a.A[0], Vh, se.h, half, v);
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = r[k] - v[k];
        hop_pair<true>(g, a, S, se, 0, S.sp[1], psi_o, half, v);
#pragma unroll
        for (int k = 0; k < 6; ++k) r[k] = r[k] - v[k];
        // odd site: A_oo psi_o + H_oe psi_e
        diag6(a.A[1], Vh, so.h, half, pv);
#pragma unroll
        for (int k = 0; k < 6; ++k) y[k] = y[k] - pv[k];
        hop_pair<true>(g, a, S, so, 1, S.sp[0], psi_e, half, v);
#pragma unroll
        for (int k = 0; k < 6; ++k) y[k] = y[k] - v[k];
    }
    store6_sm(S.rho_o, u, half, y);
    // t_o = A_oo^-1 rho_o;  b_e = rho_e - H^B_eo t_o
    diag6(a.Aoo_inv, Vh, so.h, half, y);
    __syncthreads();  // every lane is done with the psi buffers
    store6_sm(S.sp[1], u, half, y);
    __syncthreads();
    hop_pair<false>(g, a, S, se, 0, S.sp[1], nullptr, half, v);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        r[k] = r[k] - v[k];
        y[k] = {0.f, 0.f};
    }
    store6_sm(S.sp[0], u, half, r);
    __syncthreads();
    for (int it = 0; it < a.nmr; ++it) {
        // t_o = A_oo^-1 H^B_oe r_e
        hop_pair<false>(g, a, S, so, 1, S.sp[0], nullptr, half, v);
        diag6(a.Aoo_inv, Vh, so.h, half, v);
        store6_sm(S.sp[1], u, half, v);
        __syncthreads();
        // p = Dhat_B r = A_ee r - H^B_eo t_o
        hop_pair<false>(g, a, S, se, 0, S.sp[1], nullptr, half, v);
#pragma unroll
        for (int k = 0; k < 6; ++k) pv[k] = r[k];
        diag6(a.A[0], Vh, se.h, half, pv);
        float s3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            pv[k] = pv[k] - v[k];
            s3[0] += pv[k].re * r[k].re + pv[k].im * r[k].im;  // <p, r> = sum conj(p) r
            s3[1] += pv[k].re * r[k].im - pv[k].im * r[k].re;
            s3[2] += pv[k].re * pv[k].re + pv[k].im * pv[k].im;
        }
        cta_sum3(s3, S.red);
        const cplx<float> alpha = s3[2] > 0.f ? cplx<float>{s3[0] / s3[2], s3[1] / s3[2]} : cplx<float>{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            cmac(y[k], alpha, r[k]);
            r[k] = r[k] - alpha * pv[k];
        }
        store6_sm(S.sp[0], u, half, r);
        __syncthreads();
    }
    // d_o = A_oo^-1 (rho_o - H^B_oe y);  psi += d
    store6_sm(S.sp[0], u, half, y);
    __syncthreads();
    hop_pair<false>(g, a, S, so, 1, S.sp[0], nullptr, half, v);
    load6_sm(S.rho_o, u, half, pv);
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = pv[k] - v[k];
    diag6(a.Aoo_inv, Vh, so.h, half, v);
    if (!FIRST) {
        load6_glob(psi_e, Vh, se.h, half, pv);
#pragma unroll
        for (int k = 0; k < 6; ++k) y[k] = y[k] + pv[k];
        load6_glob(psi_o, Vh, so.h, half, pv);
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] = v[k] + pv[k];
    }
    store6_glob(a.psi, Vh, se.h, half, y);
    store6_glob(a.psi + 6 * (size_t)Vh, Vh, so.h, half, v);
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
                k_sap_sweep<true><<<nblk, kSapLanes, smem, st>>>(g, a, colour);
            else
                k_sap_sweep<false><<<nblk, kSapLanes, smem, st>>>(g, a, colour);
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
