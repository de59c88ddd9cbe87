// Rational functions of Q2 = Dhat^+ Dhat and the determinant factors built on
// them (App. A.1-A.3): the factor P_{k,l} (eq. Pfactor) through its partial
// fractions, the pseudofermion action of a factor (eq. Spf2), the series terms
// of the W_rat exponent (eqs. Wrat2, Wrat3) and the exponent of the W_rtm
// estimate (App. A.3), plus the small-determinant action (Sec. 2.3).
//
// Every shifted inverse comes from one multi-shift CG over all the shifts a
// call needs (FP32 Krylov space, then FP64 defect correction of each shift to
// the requested residual); the assembly and the scalar products run in FP64.
#include <cmath>

#include "blas.h"
#include "ops.h"
#include "qxd_common.cuh"
#include "qxd_internal.h"

namespace qxd {

namespace {

bool rational_ok(const qxd_rational* r) {
    if (!r || !r->nu || !r->mu || r->n < 1 || r->n > kMaxShifts || !std::isfinite(r->A)) return false;
    for (int j = 0; j < r->n; ++j)
        if (!std::isfinite(r->nu[j]) || !std::isfinite(r->mu[j])) return false;
    return true;
}

int check_rational(qxd_ctx* ctx, const qxd_rational* r, const char* what) {
    if (!r || !r->nu || !r->mu) return qxd_fail(ctx, QXD_EARG, std::string(what) + ": NULL rational approximation");
    if (r->n < 1 || r->n > kMaxShifts)
        return qxd_fail(ctx, QXD_EARG, std::string(what) + ": the degree must be 1..32");
    if (!std::isfinite(r->A)) return qxd_fail(ctx, QXD_EARG, std::string(what) + ": A is not finite");
    for (int j = 0; j < r->n; ++j)
        if (!std::isfinite(r->nu[j]) || !std::isfinite(r->mu[j]))
            return qxd_fail(ctx, QXD_EARG, std::string(what) + ": nu and mu must be finite");
    return QXD_OK;
}

int check_range(qxd_ctx* ctx, const qxd_rational* r, int k, int l, const char* what) {
    if (k < 0 || l < k || l >= r->n) return qxd_fail(ctx, QXD_EARG, std::string(what) + ": need 0 <= k <= l < n");
    return QXD_OK;
}

// residues sigma_j (j = k..l) of P_{k,l} - 1 at q2 = -mu_j^2 (App. A.2); false if two
// mu_j^2 of the factor coincide
bool factor_residues_host(const qxd_rational* r, int k, int l, double* sig) {
    for (int j = k; j <= l; ++j) {
        const double p = -r->mu[j] * r->mu[j];
        double s = r->nu[j] * r->nu[j] + p;
        for (int m = k; m <= l; ++m) {
            if (m == j) continue;
            const double den = r->mu[m] * r->mu[m] + p;
            if (den == 0.0) return false;
            s *= (r->nu[m] * r->nu[m] + p) / den;
        }
        sig[j - k] = s;
    }
    return true;
}
int factor_residues(qxd_ctx* ctx, const qxd_rational* r, int k, int l, double* sig) {
    if (!factor_residues_host(r, k, l, sig))
        return qxd_fail(ctx, QXD_EARG, "rational factor: the mu_j^2 must be distinct");
    return QXD_OK;
}

// residues of Ptilde_{k,l} - 1 at q2 = -nu_j^2 (sig) and q2 = -mutilde_j^2 (sigt),
// Ptilde_{k,l}(q2) = prod_j (q2 + mu_j^2)(q2 + nutilde_j^2) / ((q2 + nu_j^2)(q2 + mutilde_j^2));
// false if two poles coincide
bool rtm_residues_host(const qxd_rational* rm, const qxd_rational* rt, int k, int l, double* sig, double* sigt) {
    auto sq = [](double v) { return v * v; };
    for (int j = k; j <= l; ++j) {
        for (int which = 0; which < 2; ++which) {
            const double p = which == 0 ? -sq(rm->nu[j]) : -sq(rt->mu[j]);
            // the factor of j itself without its vanishing denominator
            double s = (sq(rm->mu[j]) + p) * (sq(rt->nu[j]) + p);
            double d = which == 0 ? sq(rt->mu[j]) + p : sq(rm->nu[j]) + p;
            for (int m = k; m <= l; ++m) {
                if (m == j) continue;
                s *= (sq(rm->mu[m]) + p) * (sq(rt->nu[m]) + p);
                d *= (sq(rm->nu[m]) + p) * (sq(rt->mu[m]) + p);
            }
            if (d == 0.0) return false;
            (which == 0 ? sig : sigt)[j - k] = s / d;
        }
    }
    return true;
}
int rtm_residues(qxd_ctx* ctx, const qxd_rational* rm, const qxd_rational* rt, int k, int l, double* sig,
                 double* sigt) {
    if (!rtm_residues_host(rm, rt, k, l, sig, sigt))
        return qxd_fail(ctx, QXD_EARG, "rw_rtm: the poles nu_j^2 and mutilde_j^2 must be distinct");
    return QXD_OK;
}

void add_info(qxd_info* acc, const qxd_info& one) {
    acc->iters += one.iters;
    acc->restarts += one.restarts;
    acc->op_applies += one.op_applies;
    acc->true_relres = std::max(acc->true_relres, one.true_relres);
}

// y += sum_j c_j X_j (FP64 even fields X_j = X + j hb), in groups of kMultiMax
int multi_axpy64(qxd_ctx* ctx, int nj, const double* c, const char* X, void* y, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    for (int j0 = 0; j0 < nj; j0 += kMultiMax) {
        const int kk = std::min(kMultiMax, nj - j0);
        const void* Xp[kMultiMax];
        double cre[kMultiMax], cim[kMultiMax];
        for (int i = 0; i < kk; ++i) {
            Xp[i] = X + (size_t)(j0 + i) * hb;
            cre[i] = c[j0 + i];
            cim[i] = 0.0;
        }
        QXD_TRY(blas_multi_axpy(ctx, 0, 0, n, kk, cre, cim, Xp, y, st));
    }
    return QXD_OK;
}

// Re <a, b> of two FP64 even fields
int dot64(qxd_ctx* ctx, const void* a, const void* b, double* out, cudaStream_t st) {
    QXD_TRY(blas_dot(ctx, 0, 0, 12ull * ctx->g.Vh, a, b, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    *out = ctx->red_host[0];
    return QXD_OK;
}

// out = scale * P_{k,l} b = scale * (b + sum_j sigma_j (Q2 + mu_j^2)^-1 b); X: workspace for
// the l-k+1 solutions.  If S is given, *S = Re <b, P_{k,l} b> (before the scaling).
int factor_apply(qxd_ctx* ctx, int fl, const qxd_rational* r, int k, int l, const qxd_solver* s, const void* b,
                 void* out, char* X, double scale, double* S, qxd_info* acc, cudaStream_t st) {
    const int nj = l - k + 1;
    double sig[kMaxShifts], sh[kMaxShifts];
    QXD_TRY(factor_residues(ctx, r, k, l, sig));
    for (int j = 0; j < nj; ++j) sh[j] = r->mu[k + j] * r->mu[k + j];
    qxd_info one{};
    QXD_TRY(solve_mscg(ctx, fl, nj, sh, s, b, X, &one, st));
    add_info(acc, one);
    const size_t n = 12ull * ctx->g.Vh;
    QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, b, 0.0, 0.0, out, st));
    QXD_TRY(multi_axpy64(ctx, nj, sig, X, out, st));
    if (S) QXD_TRY(dot64(ctx, b, out, S, st));
    if (scale != 1.0) QXD_TRY(blas_axpby(ctx, 0, 0, n, 0.0, 0.0, b, scale, 0.0, out, st));
    return QXD_OK;
}

struct EvenIO {
    const void* din = nullptr;  // canonical input on the device
    void* dout = nullptr;       // canonical output on the device
    bool host_out = false;
};

}  // namespace

// S_sdet per site: log |det| of the two 6x6 blocks of D_oo(x) from an LDL^H
// factorisation (pivots real for a Hermitian block); the sign of the determinant
// is the product of the pivot signs.  One thread per odd site.
__global__ void k_logdet_odd(Geo g, const double2* __restrict__ Doo, double* __restrict__ out, double* __restrict__ neg_out) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= g.Vh) return;
    double acc = 0.0;
    int neg = 0;
    for (int blk = 0; blk < 2; ++blk) {
        double pk[36];
        for (int k = 0; k < 18; ++k) {
            const double2 v = Doo[(size_t)(blk * 18 + k) * g.Vh + h];
            pk[2 * k] = v.x;
            pk[2 * k + 1] = v.y;
        }
        // unpack the Hermitian block (diagonal reals, upper triangle complex)
        cplx<double> a[6][6];
        for (int i = 0; i < 6; ++i) {
            a[i][i] = {pk[i], 0.0};
            for (int j = i + 1; j < 6; ++j) {
                const int o = 6 + 2 * herm_off(i, j);
                a[i][j] = {pk[o], pk[o + 1]};
                a[j][i] = {pk[o], -pk[o + 1]};
            }
        }
        // A = L diag(d) L^H, right-looking elimination on the lower triangle
        for (int c = 0; c < 6; ++c) {
            const double d = a[c][c].re;
            acc += log(fabs(d));
            if (d < 0.0) neg ^= 1;
            const double rd = 1.0 / d;
            for (int i = c + 1; i < 6; ++i) {
                const cplx<double> lic = {a[i][c].re * rd, a[i][c].im * rd};
                for (int j = c + 1; j <= i; ++j) {
                    // a[i][j] -= l_ic d conj(l_jc) = l_ic conj(a[j][c])
                    const cplx<double> ajc = a[j][c];
                    a[i][j].re -= lic.re * ajc.re + lic.im * ajc.im;
                    a[i][j].im -= lic.im * ajc.re - lic.re * ajc.im;
                }
            }
        }
    }
    out[h] = acc;
    neg_out[h] = (double)neg;
}

}  // namespace qxd

using namespace qxd;

extern "C" {

int qxd_rat_apply(qxd_ctx* ctx, int fl, const qxd_rational* r, int k, int l, const qxd_solver* s, const void* in_e,
                  void* out_e, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QXD_TRY(check_rational(ctx, r, "rat_apply"));
    QXD_TRY(check_range(ctx, r, k, l, "rat_apply"));
    if (!s || !in_e || !out_e) return qxd_fail(ctx, QXD_EARG, "rat_apply: NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.Vh * 12 * 16;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    EvenIO io;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, in_e, cb, &io.din, st));
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, out_e, cb, &io.dout, &io.host_out));
    void *b, *o, *X;
    QXD_TRY(qxd_ws(ctx, WS_RAT + 0, hb, &b));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 1, hb, &o));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 2, hb * (l - k + 1), &X));
    QXD_TRY(launch_pack(ctx, 0, io.din, 0, 0, QXD_FP64, b, 1, st));
    qxd_info acc{};
    const int rc = factor_apply(ctx, fl, r, k, l, s, b, o, static_cast<char*>(X), 1.0, nullptr, &acc, st);
    acc.status = rc;
    if (info) *info = acc;
    if (rc != QXD_OK) return rc;
    QXD_TRY(launch_unpack(ctx, QXD_FP64, o, 0, 0, io.dout, 0, 1, st));
    QXD_TRY(finish_out(ctx, out_e, io.dout, cb, io.host_out, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return QXD_OK;
}

int qxd_pf_action(qxd_ctx* ctx, int fl, const qxd_rational* r, int k, int l, const qxd_solver* s, const void* phi_e,
                  double* S, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QXD_TRY(check_rational(ctx, r, "pf_action"));
    QXD_TRY(check_range(ctx, r, k, l, "pf_action"));
    if (!s || !phi_e || !S) return qxd_fail(ctx, QXD_EARG, "pf_action: NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.Vh * 12 * 16;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    const void* din;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, phi_e, cb, &din, st));
    void *b, *o, *X;
    QXD_TRY(qxd_ws(ctx, WS_RAT + 0, hb, &b));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 1, hb, &o));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 2, hb * (l - k + 1), &X));
    QXD_TRY(launch_pack(ctx, 0, din, 0, 0, QXD_FP64, b, 1, st));
    qxd_info acc{};
    const int rc = factor_apply(ctx, fl, r, k, l, s, b, o, static_cast<char*>(X), 1.0, S, &acc, st);
    acc.status = rc;
    if (info) *info = acc;
    return rc;
}

int qxd_rw_rat(qxd_ctx* ctx, int fl, const qxd_rational* r, int u, int v, int nterms, const qxd_solver* s,
               const void* eta_e, double* terms, double* exponent, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QXD_TRY(check_rational(ctx, r, "rw_rat"));
    if (!s || !eta_e || !terms) return qxd_fail(ctx, QXD_EARG, "rw_rat: NULL argument");
    if (u < 1 || v < 1 || u > 64 || v > 64) return qxd_fail(ctx, QXD_EARG, "rw_rat: u and v must be 1..64");
    if (nterms < 1 || nterms > 16) return qxd_fail(ctx, QXD_EARG, "rw_rat: nterms must be 1..16");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.Vh * 12 * 16;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    const size_t n = 12ull * ctx->g.Vh;
    const void* din;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, eta_e, cb, &din, st));
    void *eta, *w, *t0, *t1, *X, *te, *to;
    QXD_TRY(qxd_ws(ctx, WS_RAT + 0, hb, &eta));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 1, hb, &w));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 2, hb * r->n, &X));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 3, hb, &t0));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 4, hb, &t1));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 5, hb, &te));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 6, hb, &to));
    QXD_TRY(launch_pack(ctx, 0, din, 0, 0, QXD_FP64, eta, 1, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(w, eta, hb, cudaMemcpyDeviceToDevice, st));
    qxd_info acc{};
    int rc = QXD_OK;
    double expo = 0.0, cvn = 1.0;
    for (int nt = 1; nt <= nterms && rc == QXD_OK; ++nt) {
        // t = Q2^u R^v w, R = A P_{1,n}
        void* cur = w;
        void* nxt = t0;
        for (int i = 0; i < v && rc == QXD_OK; ++i) {
            rc = factor_apply(ctx, fl, r, 0, r->n - 1, s, cur, nxt, static_cast<char*>(X), r->A, nullptr, &acc, st);
            cur = nxt;
            nxt = (nxt == t0) ? t1 : t0;
        }
        for (int i = 0; i < u && rc == QXD_OK; ++i) {
            rc = op_normal(ctx, fl, 0, 0.0, cur, nxt, te, to, st);
            acc.op_applies += 2;
            cur = nxt;
            nxt = (nxt == t0) ? t1 : t0;
        }
        if (rc != QXD_OK) break;
        // w = Z w = t - w
        QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, cur, -1.0, 0.0, w, st));
        QXD_TRY(dot64(ctx, eta, w, &terms[nt - 1], st));
        cvn *= -(1.0 / v + (nt - 1)) / nt;  // c_{v,n} = (-1)^n (1/v)(1/v+1)...(1/v+n-1) / n!
        expo += cvn * terms[nt - 1];
    }
    acc.status = rc;
    if (info) *info = acc;
    if (rc == QXD_OK && exponent) *exponent = expo;
    return rc;
}

int qxd_rw_rtm(qxd_ctx* ctx, int fl, const qxd_rational* r_mu, const qxd_rational* r_t, int k, int l,
               const qxd_solver* s, const void* eta_e, double* exponent, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    QXD_TRY(check_rational(ctx, r_mu, "rw_rtm"));
    QXD_TRY(check_rational(ctx, r_t, "rw_rtm"));
    if (r_mu->n != r_t->n) return qxd_fail(ctx, QXD_EARG, "rw_rtm: both approximations must have the same degree");
    QXD_TRY(check_range(ctx, r_mu, k, l, "rw_rtm"));
    if (2 * (l - k + 1) > kMaxShifts) return qxd_fail(ctx, QXD_EARG, "rw_rtm: at most 16 factors per call");
    if (!s || !eta_e || !exponent) return qxd_fail(ctx, QXD_EARG, "rw_rtm: NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int nj = l - k + 1;
    double sig[kMaxShifts], sigt[kMaxShifts], sh[kMaxShifts];
    QXD_TRY(rtm_residues(ctx, r_mu, r_t, k, l, sig, sigt));
    for (int j = 0; j < nj; ++j) {
        sh[j] = r_mu->nu[k + j] * r_mu->nu[k + j];
        sh[nj + j] = r_t->mu[k + j] * r_t->mu[k + j];
    }
    const size_t cb = (size_t)ctx->g.Vh * 12 * 16;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    const void* din;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, eta_e, cb, &din, st));
    void *eta, *X;
    QXD_TRY(qxd_ws(ctx, WS_RAT + 0, hb, &eta));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 2, hb * 2 * nj, &X));
    QXD_TRY(launch_pack(ctx, 0, din, 0, 0, QXD_FP64, eta, 1, st));
    qxd_info acc{};
    int rc = solve_mscg(ctx, fl, 2 * nj, sh, s, eta, static_cast<char*>(X), &acc, st);
    acc.status = rc;
    if (info) *info = acc;
    if (rc != QXD_OK) return rc;
    // (sigma_j + sigmatilde_j) <eta, x_j> + sigmatilde_j (nu_j^2 - mutilde_j^2) <x_j, y_j>
    const char* Xc = static_cast<const char*>(X);
    double e = 0.0;
    for (int j = 0; j < nj; ++j) {
        const void* xj = Xc + (size_t)j * hb;
        const void* yj = Xc + (size_t)(nj + j) * hb;
        double ex, xy;
        QXD_TRY(dot64(ctx, eta, xj, &ex, st));
        QXD_TRY(dot64(ctx, xj, yj, &xy, st));
        e += (sig[j] + sigt[j]) * ex + sigt[j] * (sh[j] - sh[nj + j]) * xy;
    }
    *exponent = e;
    return QXD_OK;
}

int qxd_sdet(qxd_ctx* ctx, int fl, double* logdet, int* nneg, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!logdet) return qxd_fail(ctx, QXD_EARG, "sdet: NULL argument");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const Geo& g = ctx->g;
    void *vals, *negs;
    QXD_TRY(qxd_ws(ctx, WS_RAT + 7, sizeof(double) * g.Vh, &vals));
    QXD_TRY(qxd_ws(ctx, WS_RAT + 8, sizeof(double) * g.Vh, &negs));
    const double2* Doo = reinterpret_cast<const double2*>(ctx->fl[fl].C64[0]) + (size_t)36 * g.Vh;
    {
        ProfScope prof(ctx, "logdet_odd", (double)g.Vh * (576 + 16), st);
        k_logdet_odd<<<nblocks(g.Vh, 128), 128, 0, st>>>(g, Doo, static_cast<double*>(vals), static_cast<double*>(negs));
        QXD_CUDA(ctx, cudaGetLastError());
    }
    // deterministic sums of log|det| and of the negative-determinant flags
    QXD_TRY(blas_sum_real(ctx, static_cast<const double*>(vals), g.Vh, 0, st));
    QXD_TRY(blas_sum_real(ctx, static_cast<const double*>(negs), g.Vh, 2, st));
    QXD_TRY(blas_fetch(ctx, 4, st));
    if (ctx->red_host[1] != 0.0) return qxd_fail(ctx, QXD_ENAN, "sdet: a diagonal block has a vanishing leading minor");
    *logdet = ctx->red_host[0];
    if (nneg) *nneg = (int)ctx->red_host[2];
    return QXD_OK;
}

int qxd_rat_residues(const qxd_rational* r, int k, int l, double* sigma) {
    if (!rational_ok(r) || !sigma || k < 0 || l < k || l >= r->n) return QXD_EARG;
    return factor_residues_host(r, k, l, sigma) ? QXD_OK : QXD_EARG;
}

int qxd_rtm_residues(const qxd_rational* r_mu, const qxd_rational* r_t, int k, int l, double* sigma,
                     double* sigma_t) {
    if (!rational_ok(r_mu) || !rational_ok(r_t) || r_mu->n != r_t->n || !sigma || !sigma_t || k < 0 || l < k ||
        l >= r_mu->n)
        return QXD_EARG;
    return rtm_residues_host(r_mu, r_t, k, l, sigma, sigma_t) ? QXD_OK : QXD_EARG;
}

}  // extern "C"
