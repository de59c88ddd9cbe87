// Schwarz alternating procedure (SAP) preconditioner (Sec. 4.1 and 4.4: SAP+GCR,
// blocks of 4^4 sites, ncy cycles, nmr minimal-residual steps per block).
//
// Blocks of 4^4 sites tile the simulated lattice and are coloured like a
// checkerboard by the parity of the block coordinates.  The block operator is
// D with Dirichlet block boundaries (hops leaving the block dropped).  One
// application M eta: psi = 0, rho = eta; ncy times, for each colour: every block
// of that colour solves its block system approximately (even-odd system of the
// block, nmr minimal-residual steps from zero), psi += d on the block, and then
// rho = eta - D psi.  As a preconditioner of Dhat: z_e = (M (r_e, 0))_e.
//
// GPU layout: one CTA per block, 128 threads; thread t owns the t-th even and the
// t-th odd site of the block.  The block's residual and odd intermediate live in
// shared memory; links and site-diagonal terms are read from global memory (the
// nmr steps re-read them from L1/L2).  FP32 throughout, block sums in FP32.
#include <cmath>

#include "blas.h"
#include "hop.cuh"
#include "ops.h"
#include "qxd_internal.h"

namespace qxd {

constexpr int kSapB = 4;       // block extent
constexpr int kSapThreads = 128;  // half of the 4^4 block sites

struct SapDev {
    int nb[4];              // blocks per direction
    const float4* U32[2];   // links per parity
    const float4* Z32[2];   // phases per parity
    const float4* Aee;      // diagonal term, even sites
    const float4* Aoo_inv;  // inverse diagonal term, odd sites
    const float4* rho;      // residual, full field (even half, odd half)
    float4* psi;            // solution, full field
    int nmr;
};

struct SiteRef {
    int l[4];  // local coordinates in the block
    int x[4];  // global coordinates
    int h;     // half index of the site
};

// the t-th site of parity p in block bc
__device__ __forceinline__ void block_site(const Geo& g, const int bc[4], int p, int t, SiteRef& s) {
    s.l[3] = 0;
    int r = t;
    const int x3h = r & 1;
    r >>= 1;
    s.l[2] = r & 3;
    r >>= 2;
    s.l[1] = r & 3;
    s.l[0] = r >> 2;
    s.l[3] = 2 * x3h + ((p + s.l[0] + s.l[1] + s.l[2]) & 1);
    for (int mu = 0; mu < 4; ++mu) s.x[mu] = kSapB * bc[mu] + s.l[mu];
    s.h = lex_index(g, s.x) >> 1;
}

// thread index of the local site l (any parity)
__device__ __forceinline__ int block_thread(const int l[4]) { return (((l[0] * 4 + l[1]) * 4 + l[2]) * 2) + (l[3] >> 1); }

__device__ __forceinline__ void load_sm(const float2* __restrict__ sm, int t, cplx<float> s[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        float2 v = sm[t * 12 + k];
        s[k] = {v.x, v.y};
    }
}
__device__ __forceinline__ void store_sm(float2* __restrict__ sm, int t, const cplx<float> s[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) sm[t * 12 + k] = make_float2(s[k].re, s[k].im);
}

// acc += hopping term at site s (parity p) from the opposite-parity field in
// shared memory, hops leaving the block dropped.  acc = -1/2 sum_mu [...].
template <int MU>
__device__ __forceinline__ void hop_dir_block(const Geo& g, const SapDev& a, const SiteRef& s, int p,
                                              const float2* __restrict__ sm, cplx<float> acc[12]) {
    const int Vh = g.Vh;
    Half<float> hp, o;
    Mat3<float> m;
    cplx<float> z;
    cplx<float> v[12];
    if (s.l[MU] + 1 < kSapB) {
        int ln[4] = {s.l[0], s.l[1], s.l[2], s.l[3]};
        ln[MU] += 1;
        load_sm(sm, block_thread(ln), v);
        project<MU, true>(v, hp);
        load_link32(a.U32[p], a.Z32[p], Vh, MU, s.h, m, z);
        mul_half<false>(m, hp, o);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.a[sp][c] = z * o.a[sp][c];
        reconstruct<MU, true>(o, acc);
    }
    if (s.l[MU] > 0) {
        int ln[4] = {s.l[0], s.l[1], s.l[2], s.l[3]};
        ln[MU] -= 1;
        load_sm(sm, block_thread(ln), v);
        project<MU, false>(v, hp);
        int xn[4] = {s.x[0], s.x[1], s.x[2], s.x[3]};
        xn[MU] -= 1;
        const int hn = lex_index(g, xn) >> 1;
        load_link32(a.U32[1 - p], a.Z32[1 - p], Vh, MU, hn, m, z);
        mul_half<true>(m, hp, o);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.a[sp][c] = cmul_conj(z, o.a[sp][c]);
        reconstruct<MU, false>(o, acc);
    }
}

// out = -1/2 sum_mu [...] (block hopping term) at site s of parity p
__device__ __forceinline__ void hop_block(const Geo& g, const SapDev& a, const SiteRef& s, int p,
                                          const float2* __restrict__ sm, cplx<float> out[12]) {
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = {0.f, 0.f};
    hop_dir_block<0>(g, a, s, p, sm, out);
    hop_dir_block<1>(g, a, s, p, sm, out);
    hop_dir_block<2>(g, a, s, p, sm, out);
    hop_dir_block<3>(g, a, s, p, sm, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = -0.5f * out[k];
}

__device__ __forceinline__ void diag_mul(const float4* __restrict__ D, int Vh, int h, cplx<float> s[12]) {
    float d[72];
    load_diag<1>(D, Vh, h, d);
    apply_diag(d, s);
}

// sum over the CTA of two complex numbers (re, im of <p, r>) and a real (|p|^2)
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

__global__ void __launch_bounds__(kSapThreads) k_sap_block(Geo g, SapDev a, int colour) {
    __shared__ float2 sm_e[kSapThreads * 12];  // block residual / solution on even sites
    __shared__ float2 sm_o[kSapThreads * 12];  // odd intermediate
    __shared__ float red[3 * kSapThreads / 32];
    int bc[4];
    {
        int b = blockIdx.x;
        bc[3] = b % a.nb[3];
        b /= a.nb[3];
        bc[2] = b % a.nb[2];
        b /= a.nb[2];
        bc[1] = b % a.nb[1];
        bc[0] = b / a.nb[1];
    }
    if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) return;
    const int t = threadIdx.x;
    const int Vh = g.Vh;
    SiteRef se, so;
    block_site(g, bc, 0, t, se);
    block_site(g, bc, 1, t, so);
    cplx<float> rho_e[12], v[12], r[12], y[12], p[12];
    load_spinor<1>(a.rho, Vh, se.h, rho_e);
    // t_o = A_oo^-1 rho_o
    load_spinor<1>(a.rho + 6 * (size_t)Vh, Vh, so.h, v);
    diag_mul(a.Aoo_inv, Vh, so.h, v);
    store_sm(sm_o, t, v);
    __syncthreads();
    // b_e = rho_e - H^B_eo t_o
    hop_block(g, a, se, 0, sm_o, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        r[k] = rho_e[k] - v[k];
        y[k] = {0.f, 0.f};
    }
    store_sm(sm_e, t, r);
    __syncthreads();
    for (int it = 0; it < a.nmr; ++it) {
        // t_o = A_oo^-1 H^B_oe r_e
        hop_block(g, a, so, 1, sm_e, v);
        diag_mul(a.Aoo_inv, Vh, so.h, v);
        store_sm(sm_o, t, v);
        __syncthreads();
        // p = A_ee r - H^B_eo t_o
        hop_block(g, a, se, 0, sm_o, v);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[k] = r[k];
        diag_mul(a.Aee, Vh, se.h, p);
        float s3[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k] = p[k] - v[k];
            s3[0] += p[k].re * r[k].re + p[k].im * r[k].im;  // <p, r> = sum conj(p) r
            s3[1] += p[k].re * r[k].im - p[k].im * r[k].re;
            s3[2] += p[k].re * p[k].re + p[k].im * p[k].im;
        }
        cta_sum3(s3, red);
        const cplx<float> alpha = s3[2] > 0.f ? cplx<float>{s3[0] / s3[2], s3[1] / s3[2]} : cplx<float>{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            cmac(y[k], alpha, r[k]);
            r[k] = r[k] - alpha * p[k];
        }
        store_sm(sm_e, t, r);
        __syncthreads();
    }
    // d_o = A_oo^-1 (rho_o - H^B_oe y);  psi += d
    store_sm(sm_e, t, y);
    __syncthreads();
    hop_block(g, a, so, 1, sm_e, v);
    cplx<float> rho_o[12];
    load_spinor<1>(a.rho + 6 * (size_t)Vh, Vh, so.h, rho_o);
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = rho_o[k] - v[k];
    diag_mul(a.Aoo_inv, Vh, so.h, v);
    cplx<float> ps[12];
    load_spinor<1>(a.psi, Vh, se.h, ps);
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k] = ps[k] + y[k];
    store_spinor<1>(a.psi, Vh, se.h, ps);
    load_spinor<1>(a.psi + 6 * (size_t)Vh, Vh, so.h, ps);
#pragma unroll
    for (int k = 0; k < 12; ++k) ps[k] = ps[k] + v[k];
    store_spinor<1>(a.psi + 6 * (size_t)Vh, Vh, so.h, ps);
}

int sap_check(qxd_ctx* ctx) {
    for (int mu = 0; mu < 4; ++mu)
        if (ctx->g.N[mu] % kSapB || ctx->g.N[mu] < 2 * kSapB)
            return qxd_fail(ctx, QXD_EARG, "SAP: every simulated extent must be a multiple of 4 and at least 8");
    return QXD_OK;
}

// psi = M eta on full FP32 fields (even half then odd half)
int sap_apply_full(qxd_ctx* ctx, int fl, const float4* eta, float4* psi, cudaStream_t st) {
    QXD_TRY(sap_check(ctx));
    const Geo& g = ctx->g;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const size_t n2 = 24ull * g.Vh;  // complex numbers of a full field
    void *rho, *dpsi;
    QXD_TRY(qxd_ws(ctx, WS_SAP + 0, 2 * hb, &rho));
    QXD_TRY(qxd_ws(ctx, WS_SAP + 1, 2 * hb, &dpsi));
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
    }
    a.Aee = F.C32[0];
    a.Aoo_inv = F.C32[1] + (size_t)18 * g.Vh;
    a.rho = static_cast<const float4*>(rho);
    a.psi = psi;
    a.nmr = ctx->sap_nmr;
    QXD_CUDA(ctx, cudaMemsetAsync(psi, 0, 2 * hb, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(rho, eta, 2 * hb, cudaMemcpyDeviceToDevice, st));
    char* pc = reinterpret_cast<char*>(psi);
    char* rc = static_cast<char*>(rho);
    char* dc = static_cast<char*>(dpsi);
    for (int cy = 0; cy < ctx->sap_ncy; ++cy) {
        for (int colour = 0; colour < 2; ++colour) {
            {
                ProfScope prof(ctx, "sap_block", (double)g.Vh * 2 * (96 * 3 + 4 * 56 + 288), st);
                k_sap_block<<<nblk, kSapThreads, 0, st>>>(g, a, colour);
                QXD_CUDA(ctx, cudaGetLastError());
            }
            if (cy == ctx->sap_ncy - 1 && colour == 1) break;
            // rho = eta - D psi
            QXD_TRY(op_Dw(ctx, fl, QXD_FP32, Full{pc, pc + hb}, Full{dc, dc + hb}, st));
            QXD_CUDA(ctx, cudaMemcpyAsync(rc, eta, 2 * hb, cudaMemcpyDeviceToDevice, st));
            QXD_TRY(blas_axpby(ctx, 1, 1, n2, -1.0, 0.0, dc, 1.0, 0.0, rc, st));
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
