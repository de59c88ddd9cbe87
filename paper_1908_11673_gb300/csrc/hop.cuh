// Device building blocks of the hopping term (Sec. 2.3):
//   (H psi)(x) = -1/2 sum_mu [(1 - gamma_mu) V(x,mu) psi(x+mu) + (1 + gamma_mu) V(x-mu,mu)^+ psi(x-mu)]
// in the chiral basis: spin projection onto two-spinors, colour multiplication
// by the link (FP64: stored V = U z^qhat; FP32: two rows of U rebuilt to three
// and the phase z^qhat), reconstruction into the four-spinor.
#pragma once

#include "qxd_internal.h"

namespace qxd {

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

// double-float copy of the FP64 links (one float4 per complex entry)
QXD_HD void load_link_df(const float4* __restrict__ Vdf, int Vh, int mu, int h, Mat3<dfl>& m) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float4 v = QXD_LDG(Vdf + (size_t)(mu * 9 + i * 3 + j) * Vh + h);
            m.a[i][j] = {dfl(v.x, v.y), dfl(v.z, v.w)};
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
    const float4* Vdf_out;  // double-float copies of V64 (precision 3)
    const float4* Vdf_in;
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
    } else if constexpr (P == 3) {
        load_link_df(a.Vdf_out, Vh, MU, h, m);
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
    } else if constexpr (P == 3) {
        load_link_df(a.Vdf_in, Vh, MU, nb, m);
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

// multi-right-hand-side launcher with autotuned tile shape (dirac_mrhs.cu)
int launch_hop_mr(qxd_ctx* ctx, int prec, const HopDev& d, const HopArgs& a, cudaStream_t st, int* nr_used);
// While true on the calling thread, launch_hop_mr does not tune a key it has not
// seen: it launches the default shape (one right-hand side per thread, 128
// threads) without timing, synchronising or caching anything.  Keys tuned
// earlier keep their cached shape.
extern thread_local bool t_no_autotune;

}  // namespace qxd
