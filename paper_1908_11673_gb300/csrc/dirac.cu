// Hopping kernels of the Wilson-Dirac operator (Sec. 2.2):
//   (H psi)(x) = -1/2 sum_mu [(1 - gamma_mu) V(x,mu) psi(x+mu) + (1 + gamma_mu) V(x-mu,mu)^+ psi(x-mu)]
// with V = U z^qhat, evaluated for all sites of one parity from a field on the
// other parity (even-odd preconditioning, Sec. 2.2).  One thread per output
// site; the neighbour indices are computed on the fly from the coordinates
// (C* shifted boundaries included); (1 -+ gamma_mu) are applied as spin
// projections onto two-spinors before the colour multiplication.
#include <cstdio>

#include "qxd_internal.h"

namespace qxd {

static const char* prec_name(int P) { return P == 0 ? "fp64" : (P == 1 ? "fp32" : "bf16"); }
static double spinor_bytes(int P) { return P == 0 ? 192.0 : (P == 1 ? 96.0 : 48.0); }
static double link_bytes(int P) { return P == 0 ? 144.0 : 56.0; }   // V (FP64) or 2 rows of U + z (FP32)
static double diag_bytes(int P) { return P == 0 ? 576.0 : 288.0; }

template <typename R>
struct Half {
    cplx<R> a[2][3];
};

// --- spin projection and reconstruction in the chiral basis ------------------------
// forward hop uses (1 - gamma_mu), backward hop (1 + gamma_mu).
template <int MU, bool FWD, typename R>
QXD_HD void project(const cplx<R> s[12], Half<R>& hp) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> s0 = s[c], s1 = s[3 + c], s2 = s[6 + c], s3 = s[9 + c];
        if (MU == 0) {
            hp.a[0][c] = FWD ? s0 + s2 : s0 - s2;
            hp.a[1][c] = FWD ? s1 + s3 : s1 - s3;
        } else if (MU == 1) {
            hp.a[0][c] = FWD ? add_i(s0, s3) : sub_i(s0, s3);
            hp.a[1][c] = FWD ? add_i(s1, s2) : sub_i(s1, s2);
        } else if (MU == 2) {
            hp.a[0][c] = FWD ? s0 + s3 : s0 - s3;
            hp.a[1][c] = FWD ? s1 - s2 : s1 + s2;
        } else {
            hp.a[0][c] = FWD ? add_i(s0, s2) : sub_i(s0, s2);
            hp.a[1][c] = FWD ? sub_i(s1, s3) : add_i(s1, s3);
        }
    }
}

template <int MU, bool FWD, typename R>
QXD_HD void reconstruct(const Half<R>& r, cplx<R> acc[12]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cplx<R> r0 = r.a[0][c], r1 = r.a[1][c];
        acc[c] = acc[c] + r0;
        acc[3 + c] = acc[3 + c] + r1;
        if (MU == 0) {
            acc[6 + c] = FWD ? acc[6 + c] + r0 : acc[6 + c] - r0;
            acc[9 + c] = FWD ? acc[9 + c] + r1 : acc[9 + c] - r1;
        } else if (MU == 1) {
            acc[6 + c] = FWD ? sub_i(acc[6 + c], r1) : add_i(acc[6 + c], r1);
            acc[9 + c] = FWD ? sub_i(acc[9 + c], r0) : add_i(acc[9 + c], r0);
        } else if (MU == 2) {
            acc[6 + c] = FWD ? acc[6 + c] - r1 : acc[6 + c] + r1;
            acc[9 + c] = FWD ? acc[9 + c] + r0 : acc[9 + c] - r0;
        } else {
            acc[6 + c] = FWD ? sub_i(acc[6 + c], r0) : add_i(acc[6 + c], r0);
            acc[9 + c] = FWD ? add_i(acc[9 + c], r1) : sub_i(acc[9 + c], r1);
        }
    }
}

// --- links ------------------------------------------------------------------------
template <typename R>
struct Mat3 {
    cplx<R> a[3][3];
};

// FP64: full V = U z^qhat per flavour
QXD_HD void load_link64(const double2* __restrict__ V64, int Vh, int mu, int h, Mat3<double>& m) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double2 v = QXD_LDG(V64 + (size_t)(mu * 9 + i * 3 + j) * Vh + h);
            m.a[i][j] = {v.x, v.y};
        }
}

// FP32: two rows of U, third row = conj(row0 x row1), then the phase z
QXD_HD void load_link32(const float4* __restrict__ U32, const float4* __restrict__ Z32, int Vh, int mu, int h,
                        Mat3<float>& m, cplx<float>& z) {
    float4 c0 = QXD_LDG(U32 + (size_t)(mu * 3 + 0) * Vh + h);
    float4 c1 = QXD_LDG(U32 + (size_t)(mu * 3 + 1) * Vh + h);
    float4 c2 = QXD_LDG(U32 + (size_t)(mu * 3 + 2) * Vh + h);
    float4 zz = QXD_LDG(Z32 + (size_t)(mu >> 1) * Vh + h);
    m.a[0][0] = {c0.x, c0.y};
    m.a[0][1] = {c0.z, c0.w};
    m.a[0][2] = {c1.x, c1.y};
    m.a[1][0] = {c1.z, c1.w};
    m.a[1][1] = {c2.x, c2.y};
    m.a[1][2] = {c2.z, c2.w};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        cplx<float> t = m.a[0][j1] * m.a[1][j2] - m.a[0][j2] * m.a[1][j1];
        m.a[2][j] = conj(t);
    }
    z = (mu & 1) ? cplx<float>{zz.z, zz.w} : cplx<float>{zz.x, zz.y};
}

template <bool DAG, typename R>
QXD_HD void mul_half(const Mat3<R>& m, const Half<R>& in, Half<R>& out) {
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cplx<R> acc = {R(0), R(0)};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                if (DAG)
                    cmac_conj(acc, m.a[j][i], in.a[s][j]);
                else
                    cmac(acc, m.a[i][j], in.a[s][j]);
            }
            out.a[s][i] = acc;
        }
}

// --- kernel -----------------------------------------------------------------------
struct HopDev {
    int pout;
    const void* in_nb;
    const void* in_self;
    void* out;
    // links of the output parity (forward) and of the input parity (backward)
    const double2* V64_out;
    const double2* V64_in;
    const float4* U32_out;
    const float4* U32_in;
    const float4* Z32_out;
    const float4* Z32_in;
    const void* diag;     // diag term of the output parity (SELF == 1)
    const void* diaginv;  // inverse diag term of the output parity (POST == 1)
    double c_hop;
    int g5_nb, g5_self, g5_out;
};

template <int P, int MU, typename R>
QXD_HD void hop_dir(const Geo& g, const HopDev& a, const typename Prec<P>::chunk* __restrict__ in, const int x[4],
                    int h, cplx<R> acc[12]) {
    const int Vh = g.Vh;
    const int nf = neighbour_lex(g, x, MU, +1) >> 1;
    const int nb = neighbour_lex(g, x, MU, -1) >> 1;
    cplx<R> s[12];
    Half<R> hp, r;
    Mat3<R> m;
    // forward: (1 - gamma_mu) V(x,mu) psi(x+mu)
    load_spinor<P>(in, Vh, nf, s);
    if (a.g5_nb) {
#pragma unroll
        for (int k = 6; k < 12; ++k) s[k] = -s[k];
    }
    project<MU, true>(s, hp);
    if constexpr (P == 0) {
        load_link64(a.V64_out, Vh, MU, h, m);
        mul_half<false>(m, hp, r);
    } else {
        cplx<float> z;
        load_link32(a.U32_out, a.Z32_out, Vh, MU, h, m, z);
        mul_half<false>(m, hp, r);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) r.a[sp][c] = z * r.a[sp][c];
    }
    reconstruct<MU, true>(r, acc);
    // backward: (1 + gamma_mu) V(x-mu,mu)^+ psi(x-mu)
    load_spinor<P>(in, Vh, nb, s);
    if (a.g5_nb) {
#pragma unroll
        for (int k = 6; k < 12; ++k) s[k] = -s[k];
    }
    project<MU, false>(s, hp);
    if constexpr (P == 0) {
        load_link64(a.V64_in, Vh, MU, nb, m);
        mul_half<true>(m, hp, r);
    } else {
        cplx<float> z;
        load_link32(a.U32_in, a.Z32_in, Vh, MU, nb, m, z);
        mul_half<true>(m, hp, r);
#pragma unroll
        for (int sp = 0; sp < 2; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) r.a[sp][c] = cmul_conj(z, r.a[sp][c]);
    }
    reconstruct<MU, false>(r, acc);
}

template <int P, int SELF, int POST>
__global__ void __launch_bounds__(kThreads) k_hop(Geo g, HopDev a) {
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
            load_diag<P == 0 ? 0 : 1>(a.diag, g.Vh, h, d);
            apply_diag(d, s);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = acc[k] + s[k];
    }
    if constexpr (POST == 1) {
        R d[72];
        load_diag<P == 0 ? 0 : 1>(a.diaginv, g.Vh, h, d);
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
static void launch_hop_t(const Geo& g, const HopDev& d, int nrhs, cudaStream_t st) {
    dim3 grid(nblocks(g.Vh), nrhs);
    k_hop<P, SELF, POST><<<grid, kThreads, 0, st>>>(g, d);
}

template <int P>
static void launch_hop_p(const Geo& g, const HopDev& d, int self, int post, int nrhs, cudaStream_t st) {
    if (self == 0 && post == 0) launch_hop_t<P, 0, 0>(g, d, nrhs, st);
    else if (self == 0 && post == 1) launch_hop_t<P, 0, 1>(g, d, nrhs, st);
    else if (self == 1 && post == 0) launch_hop_t<P, 1, 0>(g, d, nrhs, st);
    else if (self == 1 && post == 1) launch_hop_t<P, 1, 1>(g, d, nrhs, st);
    else if (self == 2 && post == 0) launch_hop_t<P, 2, 0>(g, d, nrhs, st);
    else launch_hop_t<P, 2, 1>(g, d, nrhs, st);
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
    d.U32_out = ctx->U32 + (size_t)po * 12 * Vh;
    d.U32_in = ctx->U32 + (size_t)pi * 12 * Vh;
    d.Z32_out = F.Z32 + (size_t)po * 2 * Vh;
    d.Z32_in = F.Z32 + (size_t)pi * 2 * Vh;
    if (prec == QXD_FP64) {
        d.diag = F.C64[0] + (size_t)po * 36 * Vh;
        d.diaginv = F.C64[1] + (size_t)po * 36 * Vh;
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
    std::snprintf(name, sizeof name, "hop_%s_self%d_post%d", prec_name(prec), a.self_mode, a.post_mode);
    const double per_rhs = spinor_bytes(prec) * (2 + (a.self_mode ? 1 : 0));
    const double once = 8 * link_bytes(prec) + diag_bytes(prec) * ((a.self_mode == 1) + (a.post_mode == 1));
    ProfScope prof(ctx, name, (double)Vh * (once + per_rhs * a.nrhs), st);
    if (prec == QXD_FP64) launch_hop_p<0>(g, d, a.self_mode, a.post_mode, a.nrhs, st);
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
