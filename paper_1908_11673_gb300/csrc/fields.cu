// Field set-up kernels: gauge-field ingest with the C* mirror fill, per-flavour
// hopping phases, and the site-diagonal term 1/(2 kappa) + dD_sw with its
// inverse (Sec. 2.1 eq. cstar-bc-gauge; Sec. 2.3 eqs. frw-covder, sw-term).
#include "blas.h"
#include "qxd_internal.h"

namespace qxd {

using C64 = cplx<double>;

struct M3 {
    C64 a[9];
};

QXD_HD M3 m3_load(const double2* __restrict__ U, int stride, int mu, int h) {
    M3 m;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 v = QXD_LDG(U + (size_t)(mu * 9 + k) * stride + h);
        m.a[k] = {v.x, v.y};
    }
    return m;
}

// product a*b with a or b optionally daggered
template <bool DA, bool DB>
QXD_HD M3 m3_mul(const M3& a, const M3& b) {
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            C64 s = {0.0, 0.0};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                C64 x = DA ? conj(a.a[k * 3 + i]) : a.a[i * 3 + k];
                C64 y = DB ? conj(b.a[j * 3 + k]) : b.a[k * 3 + j];
                cmac(s, x, y);
            }
            c.a[i * 3 + j] = s;
        }
    return c;
}

QXD_HD void m3_acc(M3& q, const M3& l) {
#pragma unroll
    for (int k = 0; k < 9; ++k) q.a[k] = q.a[k] + l.a[k];
}

// link U(y, mu) of the simulated site with coordinates y
QXD_HD M3 link_at(const Geo& g, const double2* __restrict__ U64, const int y[4], int mu) {
    int lex = lex_index(g, y);
    int par = (y[0] + y[1] + y[2] + y[3]) & 1;
    return m3_load(U64 + (size_t)par * 36 * g.Vh, g.Vh, mu, lex >> 1);
}

QXD_HD void step(const Geo& g, const int x[4], int mu, int sign, int y[4]) {
    int lex = neighbour_lex(g, x, mu, sign);
    int n3 = g.N[3], n2 = g.N[2], n1 = g.N[1];
    y[3] = lex % n3;
    lex /= n3;
    y[2] = lex % n2;
    lex /= n2;
    y[1] = lex % n1;
    y[0] = lex / n1;
}

QXD_HD double A_at(const Geo& g, const double* __restrict__ A64, const int y[4], int mu) {
    int lex = lex_index(g, y);
    int par = (y[0] + y[1] + y[2] + y[3]) & 1;
    return QXD_LDG(A64 + (size_t)par * 4 * g.Vh + (size_t)mu * g.Vh + (lex >> 1));
}

// ------------------------------------------------------------------------------
// set_links: physical-lattice input -> internal extended-lattice fields.
__global__ void k_set_links(Geo g, int L1phys, int L2, int L3, const double2* __restrict__ Uin,
                            const double* __restrict__ Ain, double2* __restrict__ U64, double* __restrict__ A64,
                            float4* __restrict__ U32) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (h >= g.Vh) return;
    int x[4];
    site_coords(g, p, h, x);
    bool mirror = g.cstar >= 1 && x[1] >= L1phys;
    int x1 = mirror ? x[1] - L1phys : x[1];
    long long phys = (((long long)x[0] * L1phys + x1) * L2 + x[2]) * L3 + x[3];
    const size_t Vh = g.Vh;
    for (int mu = 0; mu < 4; ++mu) {
        // open time boundary: the time link leaving x0 = N0 - 1 would cross it; held
        // as zero, so that no hop and no clover leaf uses it
        const bool cut = g.open0 && mu == 0 && x[0] == g.N[0] - 1;
        double2 u[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            u[k] = cut ? make_double2(0.0, 0.0) : Uin[(phys * 4 + mu) * 9 + k];
            if (mirror) u[k].y = -u[k].y;  // U(x + L1 e1) = U(x)^*
            U64[(size_t)p * 36 * Vh + (size_t)(mu * 9 + k) * Vh + h] = u[k];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            U32[(size_t)p * 12 * Vh + (size_t)(mu * 3 + c) * Vh + h] =
                make_float4((float)u[2 * c].x, (float)u[2 * c].y, (float)u[2 * c + 1].x, (float)u[2 * c + 1].y);
        double a = Ain[phys * 4 + mu];
        A64[(size_t)p * 4 * Vh + (size_t)mu * Vh + h] = mirror ? -a : a;  // A(x + L1 e1) = -A(x)
    }
}

int launch_set_links(qxd_ctx* ctx, const double2* U, const double* A, cudaStream_t st) {
    const Geo& g = ctx->g;
    dim3 grid(nblocks(g.Vh), 2);
    ProfScope prof(ctx, "set_links", (double)g.V * 4 * (144 + 8 + 144 + 8 + 48), st);
    k_set_links<<<grid, kThreads, 0, st>>>(g, ctx->geom.L[1], ctx->geom.L[2], ctx->geom.L[3], U, A, ctx->U64,
                                           ctx->A64, ctx->U32);
    QXD_CUDA(ctx, cudaGetLastError());
    return QXD_OK;
}

// ------------------------------------------------------------------------------
// Hopping phases z(x,mu)^qhat exp(i theta_mu [x crosses the boundary forward]).
// The fermion phase of eq. periodic-bc-quark sits on the link leaving x at
// x_mu = N_mu - 1; the backward hop reads the same link daggered and so picks
// up exp(-i theta_mu).  C* directions carry no phase (theta = 0 there).
__global__ void k_phases(Geo g, int qhat, double th0, double th1, double th2, double th3,
                         const double2* __restrict__ U64, const double* __restrict__ A64,
                         double2* __restrict__ V64, float4* __restrict__ Z32) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (h >= g.Vh) return;
    int x[4];
    site_coords(g, p, h, x);
    const double th[4] = {th0, th1, th2, th3};
    const size_t Vh = g.Vh;
    double2 z[4];
    for (int mu = 0; mu < 4; ++mu) {
        double ang = (double)qhat * A64[(size_t)p * 4 * Vh + (size_t)mu * Vh + h];
        bool phase_dir = !(g.cstar >= 1 && mu >= 1 && mu <= g.cstar);
        if (phase_dir && x[mu] == g.N[mu] - 1) ang += th[mu];
        double s, c;
        sincos(ang, &s, &c);
        z[mu] = make_double2(c, s);
        for (int k = 0; k < 9; ++k) {
            double2 u = U64[(size_t)p * 36 * Vh + (size_t)(mu * 9 + k) * Vh + h];
            V64[(size_t)p * 36 * Vh + (size_t)(mu * 9 + k) * Vh + h] =
                make_double2(u.x * c - u.y * s, u.x * s + u.y * c);
        }
    }
    Z32[(size_t)p * 2 * Vh + h] = make_float4((float)z[0].x, (float)z[0].y, (float)z[1].x, (float)z[1].y);
    Z32[(size_t)p * 2 * Vh + Vh + h] = make_float4((float)z[2].x, (float)z[2].y, (float)z[3].x, (float)z[3].y);
}

// ------------------------------------------------------------------------------
// Site-diagonal term.  For each plane mu < nu:
//   Fhat = (Q - Q^+)/8, Q = sum of the four clover leaves at x;
//   G_{mu nu} = su3csw Fhat_{mu nu} + u1csw qhat (i/4) Im{sum of the four U(1)
//               plaquettes} 1   (q Ahat = qhat (i/4) Im{...}, qel cancels).
// In the chiral basis sum_{mu,nu} (i/4) sigma_{mu nu} (x) G_{mu nu} is block diagonal:
//   block(+-) = (i/2) [[E3, E1 - i E2], [E1 + i E2, -E3]],
//   E+_l = G_{0l} - B_l,  E-_l = -G_{0l} - B_l,  B_1 = G_23, B_2 = -G_13, B_3 = G_12.
// Each block gets 1/(2 kappa) on the diagonal and is inverted by Gauss-Jordan
// elimination with partial pivoting.

QXD_HD void leaf_sum(const Geo& g, const double2* __restrict__ U64, const int x[4], int mu, int nu, M3& Q) {
    int xpm[4], xpn[4], xmm[4], xmn[4], xmm_pn[4], xmm_mn[4], xmn_pm[4];
    step(g, x, mu, +1, xpm);
    step(g, x, nu, +1, xpn);
    step(g, x, mu, -1, xmm);
    step(g, x, nu, -1, xmn);
    step(g, xmm, nu, +1, xmm_pn);
    step(g, xmm, nu, -1, xmm_mn);
    step(g, xmn, mu, +1, xmn_pm);
    M3 Umu_x = link_at(g, U64, x, mu), Unu_x = link_at(g, U64, x, nu);
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    M3 t = m3_mul<false, false>(Umu_x, link_at(g, U64, xpm, nu));
    t = m3_mul<false, true>(t, link_at(g, U64, xpn, mu));
    Q = m3_mul<false, true>(t, Unu_x);
    // leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    M3 Umu_xmm = link_at(g, U64, xmm, mu);
    t = m3_mul<false, true>(Unu_x, link_at(g, U64, xmm_pn, mu));
    t = m3_mul<false, true>(t, link_at(g, U64, xmm, nu));
    m3_acc(Q, m3_mul<false, false>(t, Umu_xmm));
    // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    M3 Unu_xmn = link_at(g, U64, xmn, nu);
    t = m3_mul<true, true>(Umu_xmm, link_at(g, U64, xmm_mn, nu));
    t = m3_mul<false, false>(t, link_at(g, U64, xmm_mn, mu));
    m3_acc(Q, m3_mul<false, false>(t, Unu_xmn));
    // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    t = m3_mul<true, false>(Unu_xmn, link_at(g, U64, xmn, mu));
    t = m3_mul<false, false>(t, link_at(g, U64, xmn_pm, nu));
    m3_acc(Q, m3_mul<false, true>(t, Umu_x));
}

QXD_HD double u1_im_sum(const Geo& g, const double* __restrict__ A64, const int x[4], int mu, int nu) {
    // Im{z_mn(x) + z_mn(x-mu) + z_mn(x-nu) + z_mn(x-mu-nu)}, z_mn(y) = exp(i(A_mu(y)
    // + A_nu(y+mu) - A_mu(y+nu) - A_nu(y)))
    int ys[4][4];
    for (int k = 0; k < 4; ++k) ys[0][k] = x[k];
    step(g, x, mu, -1, ys[1]);
    step(g, x, nu, -1, ys[2]);
    step(g, ys[1], nu, -1, ys[3]);
    double s = 0.0;
    for (int i = 0; i < 4; ++i) {
        // open time boundary: a plaquette of a time plane with corner x0 = N0 - 1 is absent
        if (g.open0 && mu == 0 && ys[i][0] == g.N[0] - 1) continue;
        int ypm[4], ypn[4];
        step(g, ys[i], mu, +1, ypm);
        step(g, ys[i], nu, +1, ypn);
        double ang = A_at(g, A64, ys[i], mu) + A_at(g, A64, ypm, nu) - A_at(g, A64, ypn, mu) - A_at(g, A64, ys[i], nu);
        s += sin(ang);
    }
    return s;
}

// Invert a 6x6 complex matrix m (row-major) in place; returns false if singular.
QXD_HD bool invert6(C64 m[36]) {
    C64 inv[36];
    for (int i = 0; i < 36; ++i) inv[i] = {0.0, 0.0};
    for (int i = 0; i < 6; ++i) inv[i * 6 + i] = {1.0, 0.0};
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        double best = norm2(m[c * 6 + c]);
        for (int r = c + 1; r < 6; ++r) {
            double v = norm2(m[r * 6 + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 1e-280) || !isfinite(best)) return false;
        if (piv != c) {
            for (int k = 0; k < 6; ++k) {
                C64 t = m[c * 6 + k]; m[c * 6 + k] = m[piv * 6 + k]; m[piv * 6 + k] = t;
                t = inv[c * 6 + k]; inv[c * 6 + k] = inv[piv * 6 + k]; inv[piv * 6 + k] = t;
            }
        }
        C64 d = m[c * 6 + c];
        double dn = norm2(d);
        C64 r = {d.re / dn, -d.im / dn};  // 1/d
        for (int k = 0; k < 6; ++k) {
            m[c * 6 + k] = m[c * 6 + k] * r;
            inv[c * 6 + k] = inv[c * 6 + k] * r;
        }
        for (int rr = 0; rr < 6; ++rr) {
            if (rr == c) continue;
            C64 f = m[rr * 6 + c];
            for (int k = 0; k < 6; ++k) {
                m[rr * 6 + k] = m[rr * 6 + k] - f * m[c * 6 + k];
                inv[rr * 6 + k] = inv[rr * 6 + k] - f * inv[c * 6 + k];
            }
        }
    }
    for (int i = 0; i < 36; ++i) m[i] = inv[i];
    return true;
}

QXD_HD void pack_herm(const C64 m[36], double out[36]) {
    for (int i = 0; i < 6; ++i) out[i] = m[i * 6 + i].re;
    for (int i = 0; i < 6; ++i)
        for (int j = i + 1; j < 6; ++j) {
            // average the two triangles (Hermitian up to rounding)
            C64 a = m[i * 6 + j], b = conj(m[j * 6 + i]);
            int o = 6 + 2 * herm_off(i, j);
            out[o] = 0.5 * (a.re + b.re);
            out[o + 1] = 0.5 * (a.im + b.im);
        }
}

QXD_HD void store_packed(const double pk[36], int blk, int p, int h, size_t Vh, double2* __restrict__ D64,
                         float4* __restrict__ D32) {
    for (int k = 0; k < 18; ++k)
        D64[(size_t)p * 36 * Vh + (size_t)(blk * 18 + k) * Vh + h] = make_double2(pk[2 * k], pk[2 * k + 1]);
    for (int k = 0; k < 9; ++k)
        D32[(size_t)p * 18 * Vh + (size_t)(blk * 9 + k) * Vh + h] =
            make_float4((float)pk[4 * k], (float)pk[4 * k + 1], (float)pk[4 * k + 2], (float)pk[4 * k + 3]);
}

__global__ void k_clover(Geo g, int qhat, double kappa, double su3csw, double u1csw, double cF,
                         const double2* __restrict__ U64,
                         const double* __restrict__ A64, double2* __restrict__ A_64, float4* __restrict__ A_32,
                         double2* __restrict__ Ai_64, float4* __restrict__ Ai_32, int* __restrict__ flag) {
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    int p = blockIdx.y;
    if (h >= g.Vh) return;
    int x[4];
    site_coords(g, p, h, x);
    // E[chirality][l-1]
    M3 E[2][3];
    for (int c = 0; c < 2; ++c)
        for (int l = 0; l < 3; ++l)
            for (int k = 0; k < 9; ++k) E[c][l].a[k] = {0.0, 0.0};
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) {
            M3 Q;
            leaf_sum(g, U64, x, mu, nu, Q);
            double im = u1_im_sum(g, A64, x, mu, nu);
            M3 G;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    C64 q = Q.a[i * 3 + j], qd = conj(Q.a[j * 3 + i]);
                    G.a[i * 3 + j] = (su3csw / 8.0) * (q - qd);
                }
            for (int i = 0; i < 3; ++i) G.a[i * 4].im += u1csw * (double)qhat * 0.25 * im;
            if (mu == 0) {
                // G_{0l}: +G into E+, -G into E-
                for (int k = 0; k < 9; ++k) {
                    E[0][nu - 1].a[k] = E[0][nu - 1].a[k] + G.a[k];
                    E[1][nu - 1].a[k] = E[1][nu - 1].a[k] - G.a[k];
                }
            } else {
                // B_l with B_1 = G_23, B_2 = -G_13, B_3 = G_12; E-+_l -= B_l
                int l = 6 - mu - nu;  // (1,2)->3, (1,3)->2, (2,3)->1
                double sgn = (l == 2) ? -1.0 : 1.0;
                for (int k = 0; k < 9; ++k) {
                    C64 b = sgn * G.a[k];
                    E[0][l - 1].a[k] = E[0][l - 1].a[k] - b;
                    E[1][l - 1].a[k] = E[1][l - 1].a[k] - b;
                }
            }
        }
    // 1/(2 kappa), plus dD_b = cF - 1 on the slices x0 = 0 and x0 = N0 - 1 of an open lattice
    const double m0 = 0.5 / kappa + ((g.open0 && (x[0] == 0 || x[0] == g.N[0] - 1)) ? cF - 1.0 : 0.0);
    for (int c = 0; c < 2; ++c) {
        C64 m[36];
        const M3& E1 = E[c][0];
        const M3& E2 = E[c][1];
        const M3& E3 = E[c][2];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                C64 e1 = E1.a[i * 3 + j], e2 = E2.a[i * 3 + j], e3 = E3.a[i * 3 + j];
                // (i/2) * entry
                m[i * 6 + j] = 0.5 * times_i(e3);
                m[(i + 3) * 6 + (j + 3)] = 0.5 * times_i(-e3);
                m[i * 6 + (j + 3)] = 0.5 * times_i(e1 - times_i(e2));
                m[(i + 3) * 6 + j] = 0.5 * times_i(e1 + times_i(e2));
            }
        for (int i = 0; i < 6; ++i) m[i * 6 + i].re += m0;
        double pk[36];
        pack_herm(m, pk);
        store_packed(pk, c, p, h, g.Vh, A_64, A_32);
        if (!invert6(m)) {
            atomicExch(flag, 1);
            for (int i = 0; i < 36; ++i) m[i] = {0.0, 0.0};
        }
        pack_herm(m, pk);
        store_packed(pk, c, p, h, g.Vh, Ai_64, Ai_32);
    }
}

int launch_set_flavour(qxd_ctx* ctx, int fl, cudaStream_t st) {
    const Geo& g = ctx->g;
    QxdFlavour& F = ctx->fl[fl];
    dim3 grid(nblocks(g.Vh), 2);
    const double* th = ctx->geom.theta;
    {
    ProfScope prof(ctx, "set_phases", (double)g.V * 4 * (144 + 8 + 144 + 8), st);
    k_phases<<<grid, kThreads, 0, st>>>(g, F.f.qhat, th[0], th[1], th[2], th[3], ctx->U64, ctx->A64, F.V64, F.Z32);
    }
    QXD_CUDA(ctx, cudaGetLastError());
    QXD_CUDA(ctx, cudaMemsetAsync(ctx->dev_flag, 0, sizeof(int), st));
    dim3 grid64(nblocks(g.Vh, 64), 2);
    {
    ProfScope prof(ctx, "set_clover", (double)g.V * (4 * 144 + 4 * 8 + 2 * (576 + 288)), st);
    k_clover<<<grid64, 64, 0, st>>>(g, F.f.qhat, F.f.kappa, F.f.su3csw, F.f.u1csw, ctx->geom.cF, ctx->U64, ctx->A64,
                                  F.C64[0],
                                  F.C32[0], F.C64[1], F.C32[1], ctx->dev_flag);
    }
    QXD_CUDA(ctx, cudaGetLastError());
    int flag = 0;
    QXD_CUDA(ctx, cudaMemcpyAsync(&flag, ctx->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    if (flag) return qxd_fail(ctx, QXD_ENAN, "set_clover: singular site-diagonal block");
    return QXD_OK;
}

// Double-float copies of the FP64 links and of the site-diagonal term (and, when
// an operator needs it, of its inverse), built on the first double-float
// application of the flavour: each is as large as its FP64 original, so they
// exist only where the mixed solvers or QXD_DF64 are used.
int ensure_df64(qxd_ctx* ctx, int fl, cudaStream_t st, bool inverse) {
    QxdFlavour& F = ctx->fl[fl];
    const size_t n = 2ull * 36 * ctx->g.Vh;
    float4** made[3] = {nullptr, nullptr, nullptr};  // copies allocated by this call
    int nmade = 0;
    auto build = [&](float4** dst, const double2* src) -> int {
        if (*dst) return QXD_OK;
        if (cudaMalloc(dst, n * sizeof(float4)) != cudaSuccess) {
            cudaGetLastError();
            *dst = nullptr;
            // leave no partial set behind: a caller may go on without the copies
            for (int i = 0; i < nmade; ++i) {
                cudaFree(*made[i]);
                *made[i] = nullptr;
            }
            return qxd_fail(ctx, QXD_ENOMEM, "double-float copy of the links or site-diagonal terms: allocation failed");
        }
        made[nmade++] = dst;
        return blas_split_df64(ctx, src, *dst, n, st);
    };
    QXD_TRY(build(&F.Vdf, F.V64));
    QXD_TRY(build(&F.Cdf[0], F.C64[0]));
    if (inverse) QXD_TRY(build(&F.Cdf[1], F.C64[1]));
    return QXD_OK;
}

}  // namespace qxd
