// Inexact deflation with SAP (Sec. 4.4, DFL+SAP+GCR; one subspace per flavour
// slot, hence per charge).
//
//   subspace   Ns fields phi_k, started from given random fields; ninv times
//              phi_k <- M_sap phi_k, each time followed by block orthonormalisation
//              (Gram-Schmidt of the restrictions to every 4^4 block, in k order)
//   P, P^+     P c = sum_{B,k} c_{B,k} phi_k|_B,  (P^+ v)_{B,k} = <phi_k|_B, v>
//   A          little Dirac operator P^+ D P: per block B, nine Ns x Ns blocks
//              (B itself and the blocks across its eight faces)
//   M_dfl v  = P A^-1 P^+ v + M_sap (v - D P A^-1 P^+ v), with A^-1 from restarted
//              GCR on the block grid to a relative residual ctol
//
// Layout.  The basis is Ns full FP32 fields in the internal layout (even half,
// odd half).  Coarse vectors are complex FP32 arrays [Nb][Ns].  A is stored as
// A[B][s][l][k] = <phi_k|_B, D phi_l|_{B_s}> (s = 0 the block itself, 1 + 2 mu the
// block across the +mu face, 2 + 2 mu across the -mu face), so that lane k of a
// warp reads consecutive entries when it forms row k of A x.
#include <algorithm>
#include <cmath>
#include <vector>

#include "blas.h"
#include "block.cuh"
#include "hop.cuh"
#include "ops.h"
#include "qxd_internal.h"

namespace qxd {

namespace {

constexpr int kDflMaxNs = 32;

struct DflGrid {
    int nb[4];
    int Nb;
    int Vh;
};

// CTA-wide sums of n <= kDflMaxNs complex values per thread; thread 0 writes them
__device__ __forceinline__ void cta_sum_cplx(cplx<float>* v, int n, float2* __restrict__ out, float2* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < n; ++k) {
        float re = v[k].re, im = v[k].im;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) sh[warp * kDflMaxNs + k] = make_float2(re, im);
    }
    __syncthreads();
    if (threadIdx.x < n) {
        float2 s = make_float2(0.f, 0.f);
        for (int w = 0; w < kBlkThreads / 32; ++w) {
            const float2 t = sh[w * kDflMaxNs + threadIdx.x];
            s.x += t.x;
            s.y += t.y;
        }
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void dot_acc(const cplx<float> a[12], const cplx<float> b[12], cplx<float>& acc) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        acc.re += a[i].re * b[i].re + a[i].im * b[i].im;
        acc.im += a[i].re * b[i].im - a[i].im * b[i].re;
    }
}

// out[B][k] = <X_k|_B, v|_B> for k < nk; X_k = X + k * fstride (full FP32 fields)
__global__ void __launch_bounds__(kBlkThreads) k_dfl_dots(Geo g, DflGrid G, const float4* __restrict__ X,
                                                          size_t fstride, int nk, const float4* __restrict__ v,
                                                          float2* __restrict__ out) {
    __shared__ float2 sh[kBlkThreads / 32 * kDflMaxNs];
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    SiteRef se, so;
    block_site(g, bc, 0, threadIdx.x, se);
    block_site(g, bc, 1, threadIdx.x, so);
    const int Vh = g.Vh;
    cplx<float> ve[12], vo[12], x[12];
    load_spinor<1>(v, Vh, se.h, ve);
    load_spinor<1>(v + 6 * (size_t)Vh, Vh, so.h, vo);
    cplx<float> acc[kDflMaxNs];
    for (int k = 0; k < nk; ++k) {
        acc[k] = {0.f, 0.f};
        const float4* Xk = X + (size_t)k * fstride;
        load_spinor<1>(Xk, Vh, se.h, x);
        dot_acc(x, ve, acc[k]);
        load_spinor<1>(Xk + 6 * (size_t)Vh, Vh, so.h, x);
        dot_acc(x, vo, acc[k]);
    }
    cta_sum_cplx(acc, nk, out + (size_t)blockIdx.x * nk, sh);
}

// y = sign * sum_{k < nk} c[B][k] X_k (+ y if accumulate) on every block B
__global__ void __launch_bounds__(kBlkThreads) k_dfl_prolong(Geo g, DflGrid G, const float4* __restrict__ X,
                                                             size_t fstride, int nk, const float2* __restrict__ c,
                                                             float sign, int accumulate, float4* __restrict__ y) {
    __shared__ float2 cs[kDflMaxNs];
    if (threadIdx.x < nk) cs[threadIdx.x] = c[(size_t)blockIdx.x * nk + threadIdx.x];
    __syncthreads();
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    const int Vh = g.Vh;
    for (int p = 0; p < 2; ++p) {
        SiteRef s;
        block_site(g, bc, p, threadIdx.x, s);
        const size_t off = (size_t)p * 6 * Vh;
        cplx<float> acc[12], x[12];
        if (accumulate) load_spinor<1>(y + off, Vh, s.h, acc);
        else
            for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
        for (int k = 0; k < nk; ++k) {
            load_spinor<1>(X + (size_t)k * fstride + off, Vh, s.h, x);
            const cplx<float> ck = {sign * cs[k].x, sign * cs[k].y};
#pragma unroll
            for (int i = 0; i < 12; ++i) cmac(acc[i], ck, x[i]);
        }
        store_spinor<1>(y + off, Vh, s.h, acc);
    }
}

// x|_B <- x|_B / |x|_B| on every block
__global__ void __launch_bounds__(kBlkThreads) k_dfl_normalise(Geo g, DflGrid G, float4* __restrict__ x) {
    __shared__ float2 sh[kBlkThreads / 32 * kDflMaxNs];
    __shared__ float2 nrm;
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    SiteRef se, so;
    block_site(g, bc, 0, threadIdx.x, se);
    block_site(g, bc, 1, threadIdx.x, so);
    const int Vh = g.Vh;
    cplx<float> e[12], o[12];
    load_spinor<1>(x, Vh, se.h, e);
    load_spinor<1>(x + 6 * (size_t)Vh, Vh, so.h, o);
    cplx<float> acc[1] = {{0.f, 0.f}};
    dot_acc(e, e, acc[0]);
    dot_acc(o, o, acc[0]);
    cta_sum_cplx(acc, 1, &nrm, sh);
    const float f = nrm.x > 0.f ? rsqrtf(nrm.x) : 0.f;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
        e[i] = f * e[i];
        o[i] = f * o[i];
    }
    store_spinor<1>(x, Vh, se.h, e);
    store_spinor<1>(x + 6 * (size_t)Vh, Vh, so.h, o);
}

struct DflOpDev {
    const float4* U32[2];
    const float4* Z32[2];
    const float4* A[2];
};

// -1/2 (1 - gamma_mu) V(x,mu) f(x+mu) (FWD) or -1/2 (1 + gamma_mu) V(x-mu,mu)^+ f(x-mu),
// f an opposite-parity half field, neighbour half index hn; added to acc
template <int MU, bool FWD>
__device__ __forceinline__ void hop_term(const Geo& g, const DflOpDev& d, int p, int h, int hn,
                                         const float4* __restrict__ f, cplx<float> acc[12]) {
    cplx<float> v[12], t[12];
    Half<float> hp, o;
    Mat3<float> m;
    cplx<float> z;
    load_spinor<1>(f, g.Vh, hn, v);
    project<MU, FWD>(v, hp);
    if (FWD) {
        load_link32(d.U32[p], d.Z32[p], g.Vh, MU, h, m, z);
        mul_half<false>(m, hp, o);
    } else {
        load_link32(d.U32[1 - p], d.Z32[1 - p], g.Vh, MU, hn, m, z);
        mul_half<true>(m, hp, o);
    }
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.a[sp][c] = FWD ? z * o.a[sp][c] : cmul_conj(z, o.a[sp][c]);
#pragma unroll
    for (int i = 0; i < 12; ++i) t[i] = {0.f, 0.f};
    reconstruct<MU, FWD>(o, t);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = acc[i] + (-0.5f) * t[i];
}

// the part of (D phi_l)(x) coming from slot s: s = 0 the site term and the hops
// within the block; s = 1 + 2 mu (2 + 2 mu) the hop from x + mu (x - mu) if that
// site lies in another block, else nothing
__device__ __forceinline__ void slot_term(const Geo& g, const DflOpDev& d, const SiteRef& s, int p, int slot,
                                          const float4* __restrict__ phi, cplx<float> acc[12]) {
    const int Vh = g.Vh;
    const float4* fo = phi + (size_t)(1 - p) * 6 * Vh;  // opposite parity half
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = {0.f, 0.f};
    if (slot == 0) {
        cplx<float> v[12];
        load_spinor<1>(phi + (size_t)p * 6 * Vh, Vh, s.h, v);
        float a[72];
        load_diag<1>(d.A[p], Vh, s.h, a);
        apply_diag(a, v);
#pragma unroll
        for (int i = 0; i < 12; ++i) acc[i] = v[i];
#define QXD_INNER(MU)                                                                          \
    if (s.l[MU] + 1 < kBlk) hop_term<MU, true>(g, d, p, s.h, neighbour_lex(g, s.x, MU, +1) >> 1, fo, acc); \
    if (s.l[MU] > 0) hop_term<MU, false>(g, d, p, s.h, neighbour_lex(g, s.x, MU, -1) >> 1, fo, acc);
        QXD_INNER(0) QXD_INNER(1) QXD_INNER(2) QXD_INNER(3)
#undef QXD_INNER
        return;
    }
    const int mu = (slot - 1) >> 1;
    const bool fwd = ((slot - 1) & 1) == 0;
    if (fwd ? s.l[mu] != kBlk - 1 : s.l[mu] != 0) return;
    const int hn = neighbour_lex(g, s.x, mu, fwd ? +1 : -1) >> 1;
    switch (slot) {
        case 1: hop_term<0, true>(g, d, p, s.h, hn, fo, acc); break;
        case 2: hop_term<0, false>(g, d, p, s.h, hn, fo, acc); break;
        case 3: hop_term<1, true>(g, d, p, s.h, hn, fo, acc); break;
        case 4: hop_term<1, false>(g, d, p, s.h, hn, fo, acc); break;
        case 5: hop_term<2, true>(g, d, p, s.h, hn, fo, acc); break;
        case 6: hop_term<2, false>(g, d, p, s.h, hn, fo, acc); break;
        case 7: hop_term<3, true>(g, d, p, s.h, hn, fo, acc); break;
        default: hop_term<3, false>(g, d, p, s.h, hn, fo, acc); break;
    }
}

// A[B][s][l][k] = <phi_k|_B, (slot-s part of D phi_l)|_B> for one l, all blocks and slots
__global__ void __launch_bounds__(kBlkThreads) k_dfl_little(Geo g, DflGrid G, DflOpDev d, const float4* __restrict__ X,
                                                            size_t fstride, int Ns, int l, float2* __restrict__ A) {
    __shared__ float2 sh[kBlkThreads / 32 * kDflMaxNs];
    int bc[4];
    block_coords(blockIdx.x, G.nb, bc);
    SiteRef se, so;
    block_site(g, bc, 0, threadIdx.x, se);
    block_site(g, bc, 1, threadIdx.x, so);
    const int Vh = g.Vh;
    const float4* phi = X + (size_t)l * fstride;
    for (int slot = 0; slot < 9; ++slot) {
        cplx<float> te[12], to[12], x[12];
        slot_term(g, d, se, 0, slot, phi, te);
        slot_term(g, d, so, 1, slot, phi, to);
        cplx<float> acc[kDflMaxNs];
        for (int k = 0; k < Ns; ++k) {
            acc[k] = {0.f, 0.f};
            load_spinor<1>(X + (size_t)k * fstride, Vh, se.h, x);
            dot_acc(x, te, acc[k]);
            load_spinor<1>(X + (size_t)k * fstride + 6 * (size_t)Vh, Vh, so.h, x);
            dot_acc(x, to, acc[k]);
        }
        cta_sum_cplx(acc, Ns, A + (((size_t)blockIdx.x * 9 + slot) * Ns + l) * Ns, sh);
    }
}

// y = A x on the block grid: one warp per block, lane k forms row k
__global__ void k_dfl_coarse(DflGrid G, int Ns, const int* __restrict__ nbr, const float2* __restrict__ A,
                             const float2* __restrict__ x, float2* __restrict__ y) {
    const int B = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int k = threadIdx.x & 31;
    if (B >= G.Nb || k >= Ns) return;
    cplx<float> acc = {0.f, 0.f};
    for (int s = 0; s < 9; ++s) {
        const float2* As = A + ((size_t)B * 9 + s) * Ns * Ns;
        const float2* xs = x + (size_t)__ldg(nbr + B * 9 + s) * Ns;
        for (int l = 0; l < Ns; ++l) {
            const float2 a = __ldg(As + (size_t)l * Ns + k);
            const float2 xv = __ldg(xs + l);
            acc.re += a.x * xv.x - a.y * xv.y;
            acc.im += a.x * xv.y + a.y * xv.x;
        }
    }
    y[(size_t)B * Ns + k] = make_float2(acc.re, acc.im);
}

DflGrid dfl_grid(const Geo& g) {
    DflGrid G;
    G.Nb = 1;
    for (int mu = 0; mu < 4; ++mu) {
        G.nb[mu] = g.N[mu] / kBlk;
        G.Nb *= G.nb[mu];
    }
    G.Vh = g.Vh;
    return G;
}
DflGrid dfl_grid(const qxd_ctx* ctx) { return dfl_grid(ctx->g); }

size_t field_chunks(const qxd_ctx* ctx) { return (size_t)12 * ctx->g.Vh; }  // float4 per full FP32 field

int launch_dots(qxd_ctx* ctx, const float4* X, int nk, const float4* v, float2* out, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    ProfScope prof(ctx, "dfl_dots", (double)ctx->g.V * 96 * (nk + 1), st);
    k_dfl_dots<<<G.Nb, kBlkThreads, 0, st>>>(ctx->g, G, X, field_chunks(ctx), nk, v, out);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

int launch_prolong(qxd_ctx* ctx, const float4* X, int nk, const float2* c, float sign, int accumulate, float4* y,
                   cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    ProfScope prof(ctx, "dfl_prolong", (double)ctx->g.V * 96 * (nk + 1 + accumulate), st);
    k_dfl_prolong<<<G.Nb, kBlkThreads, 0, st>>>(ctx->g, G, X, field_chunks(ctx), nk, c, sign, accumulate, y);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// block Gram-Schmidt of the basis (classical, twice per vector, then normalised)
int orthonormalise(qxd_ctx* ctx, QxdFlavour& F, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    void* c;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 0, sizeof(float2) * (size_t)G.Nb * kDflMaxNs, &c));
    const size_t fs = field_chunks(ctx);
    for (int k = 0; k < F.dfl_Ns; ++k) {
        float4* xk = F.dfl_basis + (size_t)k * fs;
        for (int pass = 0; pass < 2 && k > 0; ++pass) {
            QXD_TRY(launch_dots(ctx, F.dfl_basis, k, xk, static_cast<float2*>(c), st));
            QXD_TRY(launch_prolong(ctx, F.dfl_basis, k, static_cast<const float2*>(c), -1.f, 1, xk, st));
        }
        ProfScope prof(ctx, "dfl_normalise", (double)ctx->g.V * 192, st);
        k_dfl_normalise<<<G.Nb, kBlkThreads, 0, st>>>(ctx->g, G, xk);
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

// block neighbour table [Nb][9] from the lattice neighbour map (C* shifts included)
void neighbour_table(const Geo& g, std::vector<int>& nbr) {
    const DflGrid G = dfl_grid(g);
    nbr.assign((size_t)G.Nb * 9, 0);
    auto block_of = [&](int lex) {
        int x[4];
        int r = lex;
        for (int mu = 3; mu >= 0; --mu) {
            x[mu] = r % g.N[mu];
            r /= g.N[mu];
        }
        int b = 0;
        for (int mu = 0; mu < 4; ++mu) b = b * G.nb[mu] + x[mu] / kBlk;
        return b;
    };
    for (int B = 0; B < G.Nb; ++B) {
        int bc[4], b = B;
        for (int mu = 3; mu >= 0; --mu) {
            bc[mu] = b % G.nb[mu];
            b /= G.nb[mu];
        }
        nbr[(size_t)B * 9] = B;
        for (int mu = 0; mu < 4; ++mu) {
            int x[4];
            for (int nu = 0; nu < 4; ++nu) x[nu] = kBlk * bc[nu];
            x[mu] = kBlk * bc[mu] + kBlk - 1;  // a site on the +mu face
            nbr[(size_t)B * 9 + 1 + 2 * mu] = block_of(neighbour_lex(g, x, mu, +1));
            x[mu] = kBlk * bc[mu];  // a site on the -mu face
            nbr[(size_t)B * 9 + 2 + 2 * mu] = block_of(neighbour_lex(g, x, mu, -1));
        }
    }
}

int assemble_little(qxd_ctx* ctx, int fl, QxdFlavour& F, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    const Geo& g = ctx->g;
    DflOpDev d;
    for (int p = 0; p < 2; ++p) {
        d.U32[p] = ctx->U32 + (size_t)p * 12 * g.Vh;
        d.Z32[p] = F.Z32 + (size_t)p * 2 * g.Vh;
        d.A[p] = F.C32[0] + (size_t)p * 18 * g.Vh;
    }
    (void)fl;
    for (int l = 0; l < F.dfl_Ns; ++l) {
        ProfScope prof(ctx, "dfl_little", (double)g.V * (96.0 * (9 * F.dfl_Ns + 3) + 224 + 288), st);
        k_dfl_little<<<G.Nb, kBlkThreads, 0, st>>>(g, G, d, F.dfl_basis, field_chunks(ctx), F.dfl_Ns, l, F.dfl_A);
        QXD_CUDA(ctx, cudaGetLastError());
    }
    return QXD_OK;
}

int coarse_apply(qxd_ctx* ctx, const QxdFlavour& F, const float2* x, float2* y, cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    const int wpb = 4;
    ProfScope prof(ctx, "dfl_coarse", (double)G.Nb * 9 * F.dfl_Ns * (F.dfl_Ns + 1) * 8.0, st);
    k_dfl_coarse<<<(G.Nb + wpb - 1) / wpb, 32 * wpb, 0, st>>>(G, F.dfl_Ns, F.dfl_nbr, F.dfl_A, x, y);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// GCR on A x = b (block grid, FP32 vectors, sums in FP64), restarted every nkv
// steps, x from zero, until |b - A x| <= tol |b| or nmx steps
int coarse_gcr(qxd_ctx* ctx, const QxdFlavour& F, const float2* b, float2* x, int* iters, double* relres,
               cudaStream_t st) {
    const DflGrid G = dfl_grid(ctx);
    const size_t n = (size_t)G.Nb * F.dfl_Ns;  // complex entries
    const int nkv = F.dfl_cnkv;
    const size_t vb = sizeof(float2) * n;
    void* slab;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 1, vb * (2 * nkv + 1), &slab));
    char* base = static_cast<char*>(slab);
    auto Pv = [&](int j) { return reinterpret_cast<float2*>(base + vb * j); };
    auto Wv = [&](int j) { return reinterpret_cast<float2*>(base + vb * (nkv + j)); };
    float2* r = reinterpret_cast<float2*>(base + vb * 2 * nkv);
    QXD_CUDA(ctx, cudaMemsetAsync(x, 0, vb, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r, b, vb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, 1, n, r, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    const double bb = ctx->red_host[0];
    *iters = 0;
    *relres = 0.0;
    if (!(bb > 0.0)) return QXD_OK;
    double rr = bb;
    int it = 0;
    while (it < F.dfl_cnmx) {
        for (int k = 0; k < nkv && it < F.dfl_cnmx; ++k) {
            QXD_CUDA(ctx, cudaMemcpyAsync(Pv(k), r, vb, cudaMemcpyDeviceToDevice, st));
            QXD_TRY(coarse_apply(ctx, F, Pv(k), Wv(k), st));
            // orthogonalise w_k (and p_k alike) against the orthonormal w_j, j < k
            for (int j0 = 0; j0 < k; j0 += kMultiMax) {
                const int kk = std::min(kMultiMax, k - j0);
                const void* Wp[kMultiMax];
                const void* Pp[kMultiMax];
                for (int i = 0; i < kk; ++i) {
                    Wp[i] = Wv(j0 + i);
                    Pp[i] = Pv(j0 + i);
                }
                QXD_TRY(blas_multi_dot(ctx, 1, n, kk, Wp, Wv(k), 0, st));
                QXD_TRY(blas_fetch(ctx, 2 * kk, st));
                double cre[kMultiMax], cim[kMultiMax];
                for (int i = 0; i < kk; ++i) {
                    cre[i] = -ctx->red_host[2 * i];
                    cim[i] = -ctx->red_host[2 * i + 1];
                }
                QXD_TRY(blas_multi_axpy(ctx, 1, 1, n, kk, cre, cim, Wp, Wv(k), st));
                QXD_TRY(blas_multi_axpy(ctx, 1, 1, n, kk, cre, cim, Pp, Pv(k), st));
            }
            // |w_k|^2 and <w_k, r>
            {
                const void* Wp[2] = {Wv(k), r};
                QXD_TRY(blas_multi_dot(ctx, 1, n, 2, Wp, Wv(k), 0, st));
                QXD_TRY(blas_fetch(ctx, 4, st));
            }
            const double ww = ctx->red_host[0];
            if (!(ww > 0.0) || !std::isfinite(ww)) {
                *iters = it;
                *relres = std::sqrt(rr / bb);
                return QXD_OK;  // breakdown: keep the current iterate (the outer solver is flexible)
            }
            // normalise w_k and p_k alike; <w_k, r> = conj(<r, w_k>)
            const double sc = 1.0 / std::sqrt(ww);
            const double ar = ctx->red_host[2] * sc, ai = -ctx->red_host[3] * sc;
            QXD_TRY(blas_axpby(ctx, 1, 1, n, 0.0, 0.0, Wv(k), sc, 0.0, Wv(k), st));
            QXD_TRY(blas_axpby(ctx, 1, 1, n, 0.0, 0.0, Pv(k), sc, 0.0, Pv(k), st));
            QXD_TRY(blas_axpby(ctx, 1, 1, n, ar, ai, Pv(k), 1.0, 0.0, x, st));
            {
                const void* Wp[1] = {Wv(k)};
                const double cre[1] = {-ar}, cim[1] = {-ai};
                QXD_TRY(blas_multi_axpy_norm(ctx, 1, n, 1, cre, cim, Wp, r, 0, st));
                QXD_TRY(blas_fetch(ctx, 2, st));
            }
            rr = ctx->red_host[0];
            ++it;
            if (rr <= F.dfl_ctol * F.dfl_ctol * bb) {
                *iters = it;
                *relres = std::sqrt(rr / bb);
                return QXD_OK;
            }
        }
    }
    *iters = it;
    *relres = std::sqrt(rr / bb);
    return QXD_OK;
}

}  // namespace

// out = M_dfl v on full FP32 fields (v, out distinct)
int dfl_apply_full(qxd_ctx* ctx, int fl, const float4* v, float4* out, int* citers, double* crel, cudaStream_t st) {
    QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    const DflGrid G = dfl_grid(ctx);
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const size_t cvb = sizeof(float2) * (size_t)G.Nb * F.dfl_Ns;
    void *c, *y, *u, *t;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 2, cvb, &c));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 3, cvb, &y));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 4, 2 * hb, &u));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 5, 2 * hb, &t));
    // u = P A^-1 P^+ v
    QXD_TRY(launch_dots(ctx, F.dfl_basis, F.dfl_Ns, v, static_cast<float2*>(c), st));
    int it = 0;
    double rel = 0.0;
    QXD_TRY(coarse_gcr(ctx, F, static_cast<const float2*>(c), static_cast<float2*>(y), &it, &rel, st));
    if (citers) *citers = it;
    if (crel) *crel = rel;
    float4* uf = static_cast<float4*>(u);
    float4* tf = static_cast<float4*>(t);
    QXD_TRY(launch_prolong(ctx, F.dfl_basis, F.dfl_Ns, static_cast<const float2*>(y), 1.f, 0, uf, st));
    // t = v - D u;  out = M_sap t + u
    char* uc = static_cast<char*>(u);
    char* tc = static_cast<char*>(t);
    QXD_TRY(op_Dw(ctx, fl, QXD_FP32, Full{uc, uc + hb}, Full{tc, tc + hb}, st));
    const size_t n2 = 24ull * ctx->g.Vh;
    QXD_TRY(blas_axpby(ctx, 1, 1, n2, 1.0, 0.0, v, -1.0, 0.0, tf, st));
    QXD_TRY(sap_apply_full(ctx, fl, tf, out, st));
    QXD_TRY(blas_axpby(ctx, 1, 1, n2, 1.0, 0.0, uf, 1.0, 0.0, out, st));
    return QXD_OK;
}

// z_e = (M_dfl (r_e, 0))_e on FP32 even fields
int dfl_apply_even(qxd_ctx* ctx, int fl, const void* r_e, void* z_e, cudaStream_t st) {
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void *eta, *psi;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 6, 2 * hb, &eta));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 7, 2 * hb, &psi));
    QXD_CUDA(ctx, cudaMemcpyAsync(eta, r_e, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemsetAsync(static_cast<char*>(eta) + hb, 0, hb, st));
    QXD_TRY(dfl_apply_full(ctx, fl, static_cast<const float4*>(eta), static_cast<float4*>(psi), nullptr, nullptr, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(z_e, psi, hb, cudaMemcpyDeviceToDevice, st));
    return QXD_OK;
}

void dfl_free(QxdFlavour& F) {
    cudaFree(F.dfl_basis);
    cudaFree(F.dfl_A);
    cudaFree(F.dfl_nbr);
    F.dfl_basis = nullptr;
    F.dfl_A = nullptr;
    F.dfl_nbr = nullptr;
    F.dfl_Ns = 0;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_dfl_setup(qxd_ctx* ctx, int fl, const qxd_dfl_params* prm, const void* seeds, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!prm || !seeds) return qxd_fail(ctx, QXD_EARG, "dfl_setup: NULL argument");
    if (prm->Ns < 1 || prm->Ns > kDflMaxNs) return qxd_fail(ctx, QXD_EARG, "dfl_setup: Ns must be 1..32");
    if (prm->ninv < 0 || prm->ninv > 64) return qxd_fail(ctx, QXD_EARG, "dfl_setup: ninv must be 0..64");
    if (!(prm->ctol > 0.0) || prm->cnmx < 1 || prm->cnkv < 1 || prm->cnkv > 32)
        return qxd_fail(ctx, QXD_EARG, "dfl_setup: need ctol > 0, cnmx >= 1, cnkv in 1..32");
    QXD_TRY(sap_check(ctx));
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    QxdFlavour& F = ctx->fl[fl];
    dfl_free(F);
    const DflGrid G = dfl_grid(ctx);
    const size_t fs = field_chunks(ctx);
    const int Ns = prm->Ns;
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_basis, sizeof(float4) * fs * Ns));
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_A, sizeof(float2) * (size_t)G.Nb * 9 * Ns * Ns));
    QXD_CUDA(ctx, cudaMalloc(&F.dfl_nbr, sizeof(int) * (size_t)G.Nb * 9));
    F.dfl_Ns = Ns;
    F.dfl_ctol = prm->ctol;
    F.dfl_cnmx = prm->cnmx;
    F.dfl_cnkv = prm->cnkv;
    std::vector<int> nbr;
    neighbour_table(ctx->g, nbr);
    QXD_CUDA(ctx, cudaMemcpyAsync(F.dfl_nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice, st));
    // seeds: complex64 [Ns][V][4][3] -> internal FP32 fields
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    const void* din;
    int rc = stage_in(ctx, WS_STAGE_IN, seeds, cb * Ns, &din, st);
    if (rc == QXD_OK) {
        for (int k = 0; k < Ns && rc == QXD_OK; ++k) {
            const char* src = static_cast<const char*>(din) + cb * k;
            char* dst = reinterpret_cast<char*>(F.dfl_basis + fs * k);
            rc = launch_pack(ctx, 1, src, 1, 0, QXD_FP32, dst, 1, st);
            if (rc == QXD_OK) rc = launch_pack(ctx, 1, src, 1, 1, QXD_FP32, dst + hb, 1, st);
        }
    }
    if (rc == QXD_OK) rc = orthonormalise(ctx, F, st);
    void* tmp = nullptr;
    if (rc == QXD_OK) rc = qxd_ws(ctx, WS_DFL + 8, 2 * hb, &tmp);
    for (int i = 0; i < prm->ninv && rc == QXD_OK; ++i) {
        for (int k = 0; k < Ns && rc == QXD_OK; ++k) {
            float4* xk = F.dfl_basis + fs * k;
            rc = sap_apply_full(ctx, fl, xk, static_cast<float4*>(tmp), st);
            if (rc == QXD_OK) {
                cudaError_t e = cudaMemcpyAsync(xk, tmp, 2 * hb, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) rc = qxd_fail(ctx, QXD_ECUDA, cudaGetErrorString(e));
            }
        }
        if (rc == QXD_OK) rc = orthonormalise(ctx, F, st);
    }
    if (rc == QXD_OK) rc = assemble_little(ctx, fl, F, st);
    if (rc == QXD_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = qxd_fail(ctx, QXD_ECUDA, cudaGetErrorString(e));
    }
    if (rc != QXD_OK) dfl_free(F);
    return rc;
}

int qxd_dfl_basis(qxd_ctx* ctx, int fl, int k, void* out, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    if (k < 0 || k >= F.dfl_Ns || !out) return qxd_fail(ctx, QXD_EARG, "dfl_basis: k out of range or NULL output");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void* dout;
    bool host_out;
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, out, cb, &dout, &host_out));
    const char* src = reinterpret_cast<const char*>(F.dfl_basis + field_chunks(ctx) * k);
    QXD_TRY(launch_unpack(ctx, QXD_FP32, src, 0, 1, dout, 1, 1, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, src + hb, 1, 1, dout, 1, 1, st));
    QXD_TRY(finish_out(ctx, out, dout, cb, host_out, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_dfl_little(qxd_ctx* ctx, int fl, void* A_out, int* nbr_out, int* nblocks, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QxdFlavour& F = ctx->fl[fl];
    if (!F.dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const DflGrid G = dfl_grid(ctx);
    if (nblocks) *nblocks = G.Nb;
    if (A_out)
        QXD_CUDA(ctx, cudaMemcpyAsync(A_out, F.dfl_A, sizeof(float2) * (size_t)G.Nb * 9 * F.dfl_Ns * F.dfl_Ns,
                                      cudaMemcpyDefault, st));
    if (nbr_out)
        QXD_CUDA(ctx, cudaMemcpyAsync(nbr_out, F.dfl_nbr, sizeof(int) * (size_t)G.Nb * 9, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_dfl_apply(qxd_ctx* ctx, int fl, const void* in, void* out, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!in || !out) return qxd_fail(ctx, QXD_EARG, "dfl_apply: NULL argument");
    if (!ctx->fl[fl].dfl_basis) return qxd_fail(ctx, QXD_ESTATE, "deflation subspace not set up (qxd_dfl_setup)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.V * 12 * 8;
    const size_t hb = half_bytes(ctx, QXD_FP32);
    void *cin, *cout, *fin, *fout;
    QXD_TRY(qxd_ws(ctx, WS_DFL + 9, cb, &cin));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 10, cb, &cout));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 11, 2 * hb, &fin));
    QXD_TRY(qxd_ws(ctx, WS_DFL + 12, 2 * hb, &fout));
    QXD_CUDA(ctx, cudaMemcpyAsync(cin, in, cb, cudaMemcpyDefault, st));
    char* fi = static_cast<char*>(fin);
    char* fo = static_cast<char*>(fout);
    QXD_TRY(launch_pack(ctx, 1, cin, 1, 0, QXD_FP32, fi, 1, st));
    QXD_TRY(launch_pack(ctx, 1, cin, 1, 1, QXD_FP32, fi + hb, 1, st));
    int it = 0;
    double rel = 0.0;
    QXD_TRY(dfl_apply_full(ctx, fl, reinterpret_cast<const float4*>(fi), reinterpret_cast<float4*>(fo), &it, &rel, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, fo, 0, 1, cout, 1, 1, st));
    QXD_TRY(launch_unpack(ctx, QXD_FP32, fo + hb, 1, 1, cout, 1, 1, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(out, cout, cb, cudaMemcpyDefault, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    if (info) {
        *info = qxd_info{};
        info->iters = it;
        info->true_relres = rel;
    }
    return QXD_OK;
}

int qxd_block_neighbours(const qxd_geom* geom, int* nbr_out, int* nblocks) {
    if (!geom) return QXD_EARG;
    Geo g;
    if (!make_geo(geom, &g)) return QXD_EARG;
    for (int mu = 0; mu < 4; ++mu)
        if (g.N[mu] % (2 * kBlk)) return QXD_EARG;
    const DflGrid G = dfl_grid(g);
    if (nblocks) *nblocks = G.Nb;
    if (nbr_out) {
        std::vector<int> nbr;
        neighbour_table(g, nbr);
        std::copy(nbr.begin(), nbr.end(), nbr_out);
    }
    return QXD_OK;
}

}  // extern "C"
