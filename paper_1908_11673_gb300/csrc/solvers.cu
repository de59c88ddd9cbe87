// Solvers (Sec. 4.4): CG on the normal equations of the even-odd operator
// (CGNE), flexible GCR on Dhat inside FP64 defect correction, and the
// multi-shift CG of the rational approximation (App. A.2).  Host loops drive
// the kernels; scalars come back to the host once or twice per iteration.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "blas.h"
#include "ops.h"
#include "qxd_internal.h"

namespace qxd {

// QXD_VERBOSE=1 in the environment prints the solver scalars to stderr
static bool verbose() {
    static int v = -1;
    if (v < 0) {
        const char* e = std::getenv("QXD_VERBOSE");
        v = (e && *e && *e != '0') ? 1 : 0;
    }
    return v == 1;
}

static int status_of_norm(qxd_ctx* ctx, double nonfinite, const char* where) {
    if (nonfinite != 0.0) return qxd_fail(ctx, QXD_ENAN, std::string("non-finite value in ") + where);
    return QXD_OK;
}

// ---------------------------------------------------------------------------
// r = eta - D x (FP64, full lattice); returns |r|^2 in *rr
int full_residual64(qxd_ctx* ctx, int fl, const Full& eta, const Full& x, const Full& r, const Full& tmp_o,
                    double* rr, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    // r = D x, then r = eta - r
    QXD_TRY(op_Dw(ctx, fl, QXD_FP64, x, r, st));
    QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, eta.e, -1.0, 0.0, r.e, st));
    QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, eta.o, -1.0, 0.0, r.o, st));
    QXD_TRY(blas_norm2(ctx, 0, n, r.e, 0, st));
    QXD_TRY(blas_norm2(ctx, 0, n, r.o, 2, st));
    QXD_TRY(blas_fetch(ctx, 4, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1] + ctx->red_host[3], "residual"));
    *rr = ctx->red_host[0] + ctx->red_host[2];
    (void)tmp_o;
    return QXD_OK;
}

// ---------------------------------------------------------------------------
// CGNE (FP64): even-odd system, CG on Dhat^+ Dhat tracking s = eta_hat - Dhat y.
int solve_cgne64(qxd_ctx* ctx, int fl, const qxd_solver* s, const Full& eta, const Full& x, qxd_info* info,
                 cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, QXD_FP64);
    void *b, *sv, *z, *p, *w, *to, *re, *ro, *de, *dO;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 0, hb, &b));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 1, hb, &sv));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 2, hb, &z));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 3, hb, &p));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 4, hb, &w));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 5, hb, &to));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 6, hb, &re));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 7, hb, &ro));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 8, hb, &de));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 9, hb, &dO));
    Full r{re, ro}, dx{de, dO};
    // |eta|
    QXD_TRY(blas_norm2(ctx, 0, n, eta.e, 0, st));
    QXD_TRY(blas_norm2(ctx, 0, n, eta.o, 2, st));
    QXD_TRY(blas_fetch(ctx, 4, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1] + ctx->red_host[3], "source"));
    const double enorm = std::sqrt(ctx->red_host[0] + ctx->red_host[2]);
    QXD_CUDA(ctx, cudaMemsetAsync(x.e, 0, hb, st));
    QXD_CUDA(ctx, cudaMemsetAsync(x.o, 0, hb, st));
    info->iters = 0;
    info->op_applies = 0;
    info->restarts = 0;
    info->true_relres = 1.0;
    if (enorm == 0.0) {
        info->true_relres = 0.0;
        return QXD_OK;
    }
    // r = eta (x = 0)
    QXD_CUDA(ctx, cudaMemcpyAsync(r.e, eta.e, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r.o, eta.o, hb, cudaMemcpyDeviceToDevice, st));
    const double target = 0.5 * s->tol * enorm;
    for (int restart = 0; restart < 8; ++restart) {
        // eta_hat = r_e - H_eo A_oo^-1 r_o
        QXD_TRY(op_eo_source(ctx, fl, QXD_FP64, r, b, to, st));
        // CGNR on Dhat y = b, y = 0
        QXD_CUDA(ctx, cudaMemsetAsync(dx.e, 0, hb, st));
        QXD_CUDA(ctx, cudaMemcpyAsync(sv, b, hb, cudaMemcpyDeviceToDevice, st));
        QXD_TRY(op_Dhat(ctx, fl, QXD_FP64, 1, sv, z, to, st));
        QXD_CUDA(ctx, cudaMemcpyAsync(p, z, hb, cudaMemcpyDeviceToDevice, st));
        QXD_TRY(blas_norm2(ctx, 0, n, z, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        double zz = ctx->red_host[0];
        info->op_applies += 1;
        while (true) {
            if (info->iters >= s->nmx) break;
            QXD_TRY(op_Dhat(ctx, fl, QXD_FP64, 0, p, w, to, st));
            QXD_TRY(blas_norm2(ctx, 0, n, w, 0, st));
            QXD_TRY(blas_fetch(ctx, 2, st));
            QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "CGNE"));
            const double ww = ctx->red_host[0];
            info->iters += 1;
            info->op_applies += 1;
            if (ww == 0.0) return qxd_fail(ctx, QXD_EBREAKDOWN, "CGNE: |Dhat p| = 0");
            const double alpha = zz / ww;
            QXD_TRY(blas_axpby(ctx, 0, 0, n, alpha, 0.0, p, 1.0, 0.0, dx.e, st));
            QXD_TRY(blas_axpby(ctx, 0, 0, n, -alpha, 0.0, w, 1.0, 0.0, sv, st));
            QXD_TRY(op_Dhat(ctx, fl, QXD_FP64, 1, sv, z, to, st));
            info->op_applies += 1;
            QXD_TRY(blas_norm2(ctx, 0, n, sv, 0, st));
            QXD_TRY(blas_norm2(ctx, 0, n, z, 2, st));
            QXD_TRY(blas_fetch(ctx, 4, st));
            const double ss = ctx->red_host[0];
            const double zz_new = ctx->red_host[2];
            if (verbose() && (info->iters % 50 == 0))
                std::fprintf(stderr, "[qxd cgne] it %d |s|/|eta| %.6e\n", info->iters, std::sqrt(ss) / enorm);
            if (std::sqrt(ss) <= target) break;
            const double beta = zz_new / zz;
            zz = zz_new;
            QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, z, beta, 0.0, p, st));
        }
        // dx_o = A_oo^-1 (r_o - H_oe dx_e);  x += dx
        QXD_TRY(op_odd_reconstruct(ctx, fl, QXD_FP64, r.o, dx.e, dx.o, st));
        QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, dx.e, 1.0, 0.0, x.e, st));
        QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, dx.o, 1.0, 0.0, x.o, st));
        double rr;
        QXD_TRY(full_residual64(ctx, fl, eta, x, r, Full{to, to}, &rr, st));
        info->op_applies += 1;
        info->true_relres = std::sqrt(rr) / enorm;
        if (info->true_relres <= s->tol) return QXD_OK;
        if (info->iters >= s->nmx) break;
        info->restarts += 1;
    }
    return qxd_fail(ctx, QXD_ENOCONV, "CGNE: tolerance not reached within nmx");
}

// ---------------------------------------------------------------------------
// Flexible GCR on Dhat in precision P (even-site vectors), right preconditioner M.
// Solves Dhat e = b to |b - Dhat e| <= rtol |b|; e is overwritten.
// CG on the normal equations in precision P, tracking s = b - Dhat e:
// always convergent (Dhat^+ Dhat is positive definite), used when restarted
// GCR stagnates (a spectrum that surrounds the origin).  e is overwritten.
int cgnr_inner(qxd_ctx* ctx, int fl, int P, const void* b, void* e, int max_iter, double rtol, int* iters,
               cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, P);
    void *sv, *z, *p, *w, *to;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 100, hb, &sv));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 101, hb, &z));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 102, hb, &p));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 103, hb, &w));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 104, hb, &to));
    QXD_CUDA(ctx, cudaMemsetAsync(e, 0, hb, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(sv, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(op_Dhat(ctx, fl, P, 1, sv, z, to, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(p, z, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, P, n, b, 0, st));
    QXD_TRY(blas_norm2(ctx, P, n, z, 2, st));
    QXD_TRY(blas_fetch(ctx, 4, st));
    const double bn = std::sqrt(ctx->red_host[0]);
    double zz = ctx->red_host[2];
    *iters = 0;
    while (*iters < max_iter && zz > 0.0) {
        QXD_TRY(op_Dhat(ctx, fl, P, 0, p, w, to, st));
        QXD_TRY(blas_norm2(ctx, P, n, w, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "CGNR"));
        const double ww = ctx->red_host[0];
        *iters += 1;
        if (!(ww > 0.0)) break;
        const double alpha = zz / ww;
        QXD_TRY(blas_axpby(ctx, P, P, n, alpha, 0.0, p, 1.0, 0.0, e, st));
        QXD_TRY(blas_axpby(ctx, P, P, n, -alpha, 0.0, w, 1.0, 0.0, sv, st));
        QXD_TRY(op_Dhat(ctx, fl, P, 1, sv, z, to, st));
        QXD_TRY(blas_norm2(ctx, P, n, sv, 0, st));
        QXD_TRY(blas_norm2(ctx, P, n, z, 2, st));
        QXD_TRY(blas_fetch(ctx, 4, st));
        if (std::sqrt(ctx->red_host[0]) <= rtol * bn) break;
        const double beta = ctx->red_host[2] / zz;
        zz = ctx->red_host[2];
        QXD_TRY(blas_axpby(ctx, P, P, n, 1.0, 0.0, z, beta, 0.0, p, st));
    }
    return QXD_OK;
}

// Precision of the residual and solution vectors of an inner solve whose
// operator and Krylov basis are stored in precision P: BF16 storage keeps the
// residual and the solution in FP32 (bfloat16 rounding, 2^-9, would swamp the
// recursive residual), FP32 and FP64 use their own precision throughout.
static int vec_prec(int P) { return P == QXD_BF16 ? QXD_FP32 : P; }

// z = M r: r in precision Pv, z in Pb
static int precond_into(qxd_ctx* ctx, int fl, int Pv, int Pb, int kind, const void* r, void* z, void* ztmp,
                        cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    if (Pv == Pb) return apply_precond(ctx, fl, Pv, kind, r, z, st);
    if (kind == QXD_PRECOND_NONE) return blas_axpby(ctx, Pv, Pb, n, 1.0, 0.0, r, 0.0, 0.0, z, st);
    QXD_TRY(apply_precond(ctx, fl, Pv, kind, r, ztmp, st));
    return blas_axpby(ctx, Pv, Pb, n, 1.0, 0.0, ztmp, 0.0, 0.0, z, st);
}

int fgcr_inner(qxd_ctx* ctx, int fl, int P, const qxd_solver* s, const void* b, void* e, int max_iter,
               double rtol, int* iters, bool* stagnated, cudaStream_t st) {
    *stagnated = false;
    const int Pb = P, Pv = vec_prec(P);
    const bool split = Pb != Pv;
    const int nkv = s->nkv < 1 ? 1 : (s->nkv > 64 ? 64 : s->nkv);
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hv = half_bytes(ctx, Pv), hbb = half_bytes(ctx, Pb);
    void *r, *to, *tmp, *ztmp, *tb;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 20, hv, &r));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 21, hbb, &to));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 22, hbb, &tmp));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 23, hv, &ztmp));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 19, hbb, &tb));
    // Krylov basis: two blocks of nkv fields
    void *Zb, *Wb;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 24, hbb * nkv, &Zb));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 25, hbb * nkv, &Wb));
    std::vector<void*> Z(nkv), W(nkv);
    for (int k = 0; k < nkv; ++k) {
        Z[k] = static_cast<char*>(Zb) + (size_t)k * hbb;
        W[k] = static_cast<char*>(Wb) + (size_t)k * hbb;
    }
    QXD_CUDA(ctx, cudaMemsetAsync(e, 0, hv, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hv, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, Pv, n, b, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "GCR source"));
    const double bn = std::sqrt(ctx->red_host[0]);
    *iters = 0;
    if (bn == 0.0) return QXD_OK;
    double rr = bn * bn;
    std::vector<double> Rre(nkv * nkv), Rim(nkv * nkv), are(nkv), aim(nkv), ww(nkv), cre(nkv), cim(nkv);
    std::vector<const void*> Wc(nkv + 1);
    bool done = false;
    // Without a preconditioner the search direction of step k is the residual r_k
    // itself: it is kept in Z[k], and the update r_{k+1} = r_k - a_k w_k is written
    // straight into Z[k+1] (one copy of r per cycle instead of one per step).
    const bool rz = !split && s->precond == QXD_PRECOND_NONE;
    while (!done && *iters < max_iter) {
        int K = 0;
        const double rr_cycle = rr;
        if (rz) QXD_CUDA(ctx, cudaMemcpyAsync(Z[0], r, hbb, cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < nkv; ++k) {
            if (!rz) QXD_TRY(precond_into(ctx, fl, Pv, Pb, s->precond, r, Z[k], ztmp, st));
            const void* rk = rz ? Z[k] : r;  // current residual
            // <W_j, w_k> for j < k and <r, w_k>; without a preconditioner also |w_k|^2,
            // from which |w_k'|^2 of the orthogonalised w_k' follows (the W_j are
            // orthogonal), so that orthogonalisation and residual update run as one pass.
            // In FP32 with up to 8 earlier fields the products come from the operator's
            // own second launch (op_Dhat_dots), which also counts non-finite sites.
            double nonfinite = 0.0;
            if (rz && Pb == QXD_FP32 && k <= kMultiMax) {
                QXD_TRY(op_Dhat_dots(ctx, fl, Z[k], W[k], to, k, W.data(), 0, st));
                QXD_TRY(blas_fetch(ctx, 2 * k + 4, st));
                nonfinite = ctx->red_host[2 * k + 3];
            } else {
                QXD_TRY(op_Dhat(ctx, fl, Pb, 0, Z[k], W[k], to, st));
                for (int j = 0; j < k; ++j) Wc[j] = W[j];
                int nd = k;
                if (!split) Wc[nd++] = rk;
                if (rz) Wc[nd++] = W[k];
                if (nd > 0) QXD_TRY(blas_multi_dot(ctx, Pb, n, nd, Wc.data(), W[k], 0, st));
                if (split) QXD_TRY(blas_dot(ctx, Pv, Pb, n, r, W[k], 2 * k, st));
                QXD_TRY(blas_fetch(ctx, 2 * nd + (split ? 2 : 0), st));
            }
            for (int j = 0; j < k; ++j) {
                Rre[j * nkv + k] = ctx->red_host[2 * j] / ww[j];
                Rim[j * nkv + k] = ctx->red_host[2 * j + 1] / ww[j];
                cre[j] = -Rre[j * nkv + k];
                cim[j] = -Rim[j * nkv + k];
            }
            // <w_k, r> = conj(<r, w_k>); r is orthogonal to the earlier w_j
            const double wr_re = ctx->red_host[2 * k], wr_im = -ctx->red_host[2 * k + 1];
            std::vector<const void*> Wp(W.begin(), W.begin() + k);
            bool fused = false;
            if (rz) {
                // |w_k'|^2 = |w_k|^2 - sum_j |<W_j, w_k>|^2 / |W_j|^2, used unless it cancels
                // to less than a hundredth of |w_k|^2 (then it is summed directly below)
                const double w2 = ctx->red_host[2 * (k + 1)];
                double w2o = w2;
                for (int j = 0; j < k; ++j)
                    w2o -= (ctx->red_host[2 * j] * ctx->red_host[2 * j] + ctx->red_host[2 * j + 1] * ctx->red_host[2 * j + 1]) /
                           ww[j];
                if (std::isfinite(w2o) && w2o > 0.01 * w2) {
                    fused = true;
                    ww[k] = w2o;
                    ctx->red_host[1] = nonfinite;  // non-finite count (the separate dot pass counts none)
                }
            }
            if (!fused) {
                QXD_TRY(blas_multi_axpy_norm(ctx, Pb, n, k, cre.data(), cim.data(), Wp.data(), W[k], 0, st));
                QXD_TRY(blas_fetch(ctx, 2, st));
                ww[k] = ctx->red_host[0];
            }
            if (verbose())
                std::fprintf(stderr, "[qxd gcr] it %d k %d |w|^2 %.6e <w,r> (%.6e, %.6e) rr %.6e nonfinite %g\n", *iters,
                             k, ww[k], wr_re, wr_im, rr, ctx->red_host[1]);
            QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "GCR"));
            if (!(ww[k] > 0.0)) return qxd_fail(ctx, QXD_EBREAKDOWN, "GCR: |w| = 0");
            are[k] = wr_re / ww[k];
            aim[k] = wr_im / ww[k];
            if (fused)
                QXD_TRY(blas_gcr_update(ctx, Pb, n, k, cre.data(), cim.data(), Wp.data(), W[k], -are[k], -aim[k], Z[k],
                                        k + 1 < nkv ? Z[k + 1] : r, st));
            else if (rz) QXD_TRY(blas_axpy3(ctx, Pb, n, -are[k], -aim[k], W[k], Z[k], k + 1 < nkv ? Z[k + 1] : r, st));
            else QXD_TRY(blas_axpby(ctx, Pb, Pv, n, -are[k], -aim[k], W[k], 1.0, 0.0, r, st));
            rr -= (wr_re * wr_re + wr_im * wr_im) / ww[k];
            *iters += 1;
            K = k + 1;
            if (rr <= rtol * rtol * bn * bn || *iters >= max_iter) {
                done = true;
                break;
            }
        }
        // back substitution: c_j = a_j - sum_{k>j} R_jk c_k
        for (int j = K - 1; j >= 0; --j) {
            double sr = are[j], si = aim[j];
            for (int k = j + 1; k < K; ++k) {
                const double rr_ = Rre[j * nkv + k], ri = Rim[j * nkv + k];
                sr -= rr_ * cre[k] - ri * cim[k];
                si -= rr_ * cim[k] + ri * cre[k];
            }
            cre[j] = sr;
            cim[j] = si;
        }
        if (!split) {
            std::vector<const void*> Zp(Z.begin(), Z.begin() + K);
            QXD_TRY(blas_multi_axpy(ctx, Pv, Pv, n, K, cre.data(), cim.data(), Zp.data(), e, st));
        } else {
            for (int k = 0; k < K; ++k) QXD_TRY(blas_axpby(ctx, Pb, Pv, n, cre[k], cim[k], Z[k], 1.0, 0.0, e, st));
        }
        if (!done) {
            // restart: r = b - Dhat e (through the basis precision)
            if (split) {
                QXD_TRY(blas_axpby(ctx, Pv, Pb, n, 1.0, 0.0, e, 0.0, 0.0, tb, st));
                QXD_TRY(op_Dhat(ctx, fl, Pb, 0, tb, tmp, to, st));
            } else {
                QXD_TRY(op_Dhat(ctx, fl, Pb, 0, e, tmp, to, st));
            }
            QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hv, cudaMemcpyDeviceToDevice, st));
            if (!split) {  // r -= tmp and |r|^2 in one pass
                const void* Xp[1] = {tmp};
                const double cr[1] = {-1.0}, ci[1] = {0.0};
                QXD_TRY(blas_multi_axpy_norm(ctx, Pv, n, 1, cr, ci, Xp, r, 0, st));
            } else {
                QXD_TRY(blas_axpby(ctx, Pb, Pv, n, -1.0, 0.0, tmp, 1.0, 0.0, r, st));
                QXD_TRY(blas_norm2(ctx, Pv, n, r, 0, st));
            }
            QXD_TRY(blas_fetch(ctx, 2, st));
            rr = ctx->red_host[0];
            if (rr <= rtol * rtol * bn * bn) done = true;
            // a whole cycle that did not halve the residual norm: restarted GCR
            // stalls (much slower than CG on the normal equations would be)
            if (!done && K == nkv && rr > 0.25 * rr_cycle) {
                *stagnated = true;
                return QXD_OK;
            }
        }
    }
    return QXD_OK;
}

// FP64 defect correction around inner FGCR solves in precision s->inner.
int solve_fgcr_dc(qxd_ctx* ctx, int fl, const qxd_solver* s, const Full& eta, const Full& x, qxd_info* info,
                  cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const int P = s->inner;
    const int Pv = vec_prec(P);  // precision of the inner solve's vectors (FP32 for BF16 storage)
    // Mixed inner precision: the outer loop holds x and D x as double-float fields
    // (FP64 data, FP32-pipe arithmetic, about 48-bit significands; eta is split on the
    // fly), so the residual, its FP32 rounding for the inner solve and its norm come
    // from one pass, and the solution update needs no FP64 arithmetic.  FP64 inner
    // solves keep the outer loop in FP64, and so does a lattice whose double-float
    // copies of the links and site-diagonal terms do not fit in the device memory.
    bool df = P != QXD_FP64;
    if (df && ensure_df64(ctx, fl, st) != QXD_OK) df = false;
    const size_t hb64 = half_bytes(ctx, QXD_FP64);
    const size_t hbP = half_bytes(ctx, Pv);
    void *re, *ro, *t64, *bP, *roP, *tP, *eeP, *eoP, *to2;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 10, hb64, &re));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 11, hb64, &ro));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 12, hb64, &t64));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 13, hbP, &bP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 14, hbP, &roP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 15, hbP, &tP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 16, hbP, &eeP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 17, hbP, &eoP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 18, hbP, &to2));
    Full r{re, ro};
    void *xde = nullptr, *xdo = nullptr, *dxe = nullptr, *dxo = nullptr;
    if (df) {
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 30, hb64, &xde));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 31, hb64, &xdo));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 34, hb64, &dxe));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 35, hb64, &dxo));
    }
    if (df) {  // the source's FP32 rounding for the first inner solve and its norm, one pass per half
        QXD_TRY(blas_f64_to_f32_norm(ctx, eta.e, tP, 0, st));
        QXD_TRY(blas_f64_to_f32_norm(ctx, eta.o, roP, 2, st));
    } else {
        QXD_TRY(blas_norm2(ctx, 0, n, eta.e, 0, st));
        QXD_TRY(blas_norm2(ctx, 0, n, eta.o, 2, st));
    }
    QXD_TRY(blas_fetch(ctx, 4, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1] + ctx->red_host[3], "source"));
    const double enorm = std::sqrt(ctx->red_host[0] + ctx->red_host[2]);
    QXD_CUDA(ctx, cudaMemsetAsync(x.e, 0, hb64, st));
    QXD_CUDA(ctx, cudaMemsetAsync(x.o, 0, hb64, st));
    info->iters = 0;
    info->op_applies = 0;
    info->restarts = 0;
    info->true_relres = 1.0;
    if (enorm == 0.0) {
        info->true_relres = 0.0;
        return QXD_OK;
    }
    if (df) {
        QXD_CUDA(ctx, cudaMemsetAsync(xde, 0, hb64, st));
        QXD_CUDA(ctx, cudaMemsetAsync(xdo, 0, hb64, st));
    } else {
        QXD_CUDA(ctx, cudaMemcpyAsync(r.e, eta.e, hb64, cudaMemcpyDeviceToDevice, st));
        QXD_CUDA(ctx, cudaMemcpyAsync(r.o, eta.o, hb64, cudaMemcpyDeviceToDevice, st));
    }
    // true residual of the current x: relative norm; in the double-float loop it
    // also leaves FP32(eta - D x) in tP, roP for the next inner solve
    auto residual = [&](double* rel) -> int {
        double rr;
        if (df) {
            QXD_TRY(op_Dw(ctx, fl, QXD_DF64, Full{xde, xdo}, Full{dxe, dxo}, st));
            QXD_TRY(blas_df_residual(ctx, eta.e, dxe, tP, 0, st));
            QXD_TRY(blas_df_residual(ctx, eta.o, dxo, roP, 2, st));
            QXD_TRY(blas_fetch(ctx, 4, st));
            QXD_TRY(status_of_norm(ctx, ctx->red_host[1] + ctx->red_host[3], "residual"));
            rr = ctx->red_host[0] + ctx->red_host[2];
        } else {
            QXD_TRY(full_residual64(ctx, fl, eta, x, r, Full{t64, t64}, &rr, st));
        }
        *rel = std::sqrt(rr) / enorm;
        return QXD_OK;
    };
    // the double-float solution goes to the caller's FP64 field
    auto finish = [&]() -> int {
        if (df) {
            QXD_TRY(blas_join_df64(ctx, xde, x.e, n, st));
            QXD_TRY(blas_join_df64(ctx, xdo, x.o, n, st));
        }
        return QXD_OK;
    };
    double relres = 1.0;
    bool use_cgnr = false;
    const double itol = s->inner_tol > 0 ? s->inner_tol : (P == QXD_BF16 ? 5e-3 : (P == QXD_FP32 ? 1e-5 : 1e-10));
    for (int outer = 0; outer < 64; ++outer) {
        if (outer > 0) {
            QXD_TRY(residual(&relres));
            info->op_applies += 1;
            info->true_relres = relres;
            if (verbose()) std::fprintf(stderr, "[qxd dc] outer %d true relres %.6e\n", outer, relres);
            if (relres <= s->tol) return finish();
            info->restarts += 1;
        }
        if (info->iters >= s->nmx) break;
        // even-odd source in precision P: b = r_e - H_eo A_oo^-1 r_o
        if (!df) {
            QXD_TRY(blas_axpby(ctx, 0, Pv, n, 1.0, 0.0, r.e, 0.0, 0.0, tP, st));
            QXD_TRY(blas_axpby(ctx, 0, Pv, n, 1.0, 0.0, r.o, 0.0, 0.0, roP, st));
        }
        QXD_TRY(op_eo_source(ctx, fl, Pv, Full{tP, roP}, bP, to2, st));
        int it = 0;
        const double rtol = std::max(itol, 0.5 * s->tol / relres);
        if (!use_cgnr) {
            bool stag = false;
            QXD_TRY(fgcr_inner(ctx, fl, P, s, bP, eeP, s->nmx - info->iters, rtol, &it, &stag, st));
            info->iters += it;
            info->op_applies += it + 2;
            if (stag) {
                // restarted GCR stalls on this operator: from here on the inner
                // solves run CG on the normal equations, starting again from 0
                use_cgnr = true;
                if (verbose()) std::fprintf(stderr, "[qxd dc] GCR stagnated after %d iterations: CGNR inner\n", it);
            }
        }
        if (use_cgnr) {
            // CGNR runs in the vector precision (FP32 for BF16 storage): it can go to 1e-5
            const double ctol = Pv == QXD_FP64 ? rtol : std::max(1e-5, 0.5 * s->tol / relres);
            QXD_TRY(cgnr_inner(ctx, fl, Pv, bP, eeP, s->nmx - info->iters, ctol, &it, st));
            info->iters += it;
            info->op_applies += 2 * it + 1;
        }
        // e_o = A_oo^-1 (r_o - H_oe e_e);  x += e
        QXD_TRY(op_odd_reconstruct(ctx, fl, Pv, roP, eeP, eoP, st));
        if (df) {
            QXD_TRY(blas_df_add_f32(ctx, eeP, xde, st));
            QXD_TRY(blas_df_add_f32(ctx, eoP, xdo, st));
        } else {
            QXD_TRY(blas_axpby(ctx, Pv, 0, n, 1.0, 0.0, eeP, 1.0, 0.0, x.e, st));
            QXD_TRY(blas_axpby(ctx, Pv, 0, n, 1.0, 0.0, eoP, 1.0, 0.0, x.o, st));
        }
    }
    QXD_TRY(residual(&relres));
    info->true_relres = relres;
    QXD_TRY(finish());
    if (info->true_relres <= s->tol) return QXD_OK;
    return qxd_fail(ctx, QXD_ENOCONV, "FGCR: tolerance not reached within nmx");
}

}  // namespace qxd

namespace qxd {

// out = (Dhat^+ Dhat + sigma) v in precision P (tmp_e, tmp_o scratch)
int op_normal(qxd_ctx* ctx, int fl, int P, double sigma, const void* v, void* out, void* tmp_e, void* tmp_o,
                     cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    QXD_TRY(op_Dhat(ctx, fl, P, 0, v, tmp_e, tmp_o, st));
    QXD_TRY(op_Dhat(ctx, fl, P, 1, tmp_e, out, tmp_o, st));
    if (sigma != 0.0) QXD_TRY(blas_axpby(ctx, P, P, n, sigma, 0.0, v, 1.0, 0.0, out, st));
    return QXD_OK;
}

// CG on (Dhat^+ Dhat + sigma) e = b in precision P; e overwritten; stops at
// |b - (A + sigma) e| <= rtol |b| (recursive residual).
static int cg_shifted(qxd_ctx* ctx, int fl, int P, double sigma, const void* b, void* e, int max_iter, double rtol,
                      int* iters, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, P);
    void *r, *p, *Ap, *te, *to;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 115, hb, &r));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 116, hb, &p));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 117, hb, &Ap));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 118, hb, &te));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 119, hb, &to));
    QXD_CUDA(ctx, cudaMemsetAsync(e, 0, hb, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(p, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, P, n, b, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    const double bn = std::sqrt(ctx->red_host[0]);
    double rr = ctx->red_host[0];
    *iters = 0;
    if (bn == 0.0) return QXD_OK;
    const double mone = -1.0;
    while (*iters < max_iter) {
        QXD_TRY(op_normal(ctx, fl, P, sigma, p, Ap, te, to, st));
        QXD_TRY(blas_dot(ctx, P, P, n, p, Ap, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        const double pAp = ctx->red_host[0];
        *iters += 1;
        if (!(pAp > 0.0)) return qxd_fail(ctx, QXD_EBREAKDOWN, "shifted CG: <p, A p> <= 0");
        const double alpha = rr / pAp;
        QXD_TRY(blas_axpby(ctx, P, P, n, alpha, 0.0, p, 1.0, 0.0, e, st));
        const double ca = -alpha, ci = 0.0;
        const void* Xp[1] = {Ap};
        QXD_TRY(blas_multi_axpy_norm(ctx, P, n, 1, &ca, &ci, Xp, r, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "shifted CG"));
        const double rr_new = ctx->red_host[0];
        if (std::sqrt(rr_new) <= rtol * bn) break;
        QXD_TRY(blas_axpby(ctx, P, P, n, 1.0, 0.0, r, rr_new / rr, 0.0, p, st));
        rr = rr_new;
    }
    (void)mone;
    return QXD_OK;
}

// Multi-shift CG in precision P on (Dhat^+ Dhat + sigma_j) x_j = b (Jegerlehner's
// recursion: one Krylov space built with the smallest shift, the others
// following through the scalars zeta_j).  X: ns fields of precision P (output).
static int mscg_core(qxd_ctx* ctx, int fl, int P, int ns, const double* sigma, const void* b, char* X, int max_iter,
                     double tol, int* iters, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, P);
    void *r, *pb, *Ap, *te, *to, *Pblk;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 110, hb, &r));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 111, hb, &pb));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 112, hb, &Ap));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 113, hb, &te));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 114, hb, &to));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 109, hb * ns, &Pblk));
    char* Pc = static_cast<char*>(Pblk);
    QXD_CUDA(ctx, cudaMemsetAsync(X, 0, hb * ns, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(pb, b, hb, cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j < ns; ++j) QXD_CUDA(ctx, cudaMemcpyAsync(Pc + j * hb, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, P, n, b, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "MSCG source"));
    double rr = ctx->red_host[0];
    const double bn = std::sqrt(rr);
    *iters = 0;
    if (bn == 0.0) return QXD_OK;
    double s0 = sigma[0];
    for (int j = 1; j < ns; ++j) s0 = std::min(s0, sigma[j]);
    std::vector<double> zp(ns, 1.0), z(ns, 1.0), zn(ns, 1.0);
    std::vector<char> active(ns, 1);
    double alpha_prev = 1.0, beta_prev = 0.0;
    while (*iters < max_iter) {
        QXD_TRY(op_normal(ctx, fl, P, s0, pb, Ap, te, to, st));
        QXD_TRY(blas_dot(ctx, P, P, n, pb, Ap, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        const double pAp = ctx->red_host[0];
        *iters += 1;
        if (!(pAp > 0.0)) return qxd_fail(ctx, QXD_EBREAKDOWN, "MSCG: <p, A p> <= 0");
        const double alpha = rr / pAp;
        // r -= alpha A p, |r|^2
        const double ca = -alpha, ci = 0.0;
        const void* Xp[1] = {Ap};
        QXD_TRY(blas_multi_axpy_norm(ctx, P, n, 1, &ca, &ci, Xp, r, 0, st));
        QXD_TRY(blas_fetch(ctx, 2, st));
        QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "MSCG"));
        const double rr_new = ctx->red_host[0];
        const double beta = rr_new / rr;
        ShiftPtrs sp;
        ShiftCoef sc;
        int na = 0;
        for (int j = 0; j < ns; ++j) {
            if (!active[j]) continue;
            const double ds = sigma[j] - s0;
            const double den = alpha * beta_prev * (zp[j] - z[j]) + zp[j] * alpha_prev * (1.0 + ds * alpha);
            zn[j] = z[j] * zp[j] * alpha_prev / den;
            sp.x[na] = X + j * hb;
            sp.p[na] = Pc + j * hb;
            sc.alpha[na] = alpha * zn[j] / z[j];
            sc.zeta[na] = zn[j];
            sc.beta[na] = beta * (zn[j] / z[j]) * (zn[j] / z[j]);
            ++na;
        }
        QXD_TRY(blas_msg_update(ctx, P, n, na, sp, sc, r, st));
        QXD_TRY(blas_axpby(ctx, P, P, n, 1.0, 0.0, r, beta, 0.0, pb, st));
        bool any = false;
        for (int j = 0; j < ns; ++j) {
            if (!active[j]) continue;
            if (std::fabs(zn[j]) * std::sqrt(rr_new) <= tol * bn) active[j] = 0;
            zp[j] = z[j];
            z[j] = zn[j];
            any = any || active[j];
        }
        if (verbose() && (*iters % 50 == 0))
            std::fprintf(stderr, "[qxd mscg] it %d |r|/|b| %.3e\n", *iters, std::sqrt(rr_new) / bn);
        rr = rr_new;
        alpha_prev = alpha;
        beta_prev = beta;
        if (!any) return QXD_OK;
    }
    return QXD_OK;
}

// ---- multi-shift CG with device-resident scalars, captured as a CUDA graph ---------
// The scalars of the recursion (alpha, beta, zeta_j, ...) live in device memory and
// are updated by two one-thread kernels, so an iteration is a fixed sequence of
// launches with no host round trip.  kGraphIters iterations are captured once
// into a graph, which is then replayed; the host reads the number of active
// shifts after each replay.  Iterations after convergence are no-ops (alpha = 0).
constexpr int kGraphIters = 8;

struct MscgDev {
    double rr, alpha, alpha_prev, beta_prev, bn, tol;
    double coef_r[2];  // {-alpha, 0}: r += coef_r[0] A p
    double coef_p[2];  // {1, beta}:   p = r + beta p
    double ds[kMaxShifts], zp[kMaxShifts], z[kMaxShifts], zn[kMaxShifts];
    double aj[kMaxShifts], zj[kMaxShifts], bj[kMaxShifts];
    int active[kMaxShifts], upd[kMaxShifts];
    int nactive, iter;
};

__global__ void k_mscg_alpha(MscgDev* s, const double* __restrict__ red, int ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double pAp = red[0];
    const double alpha = (s->nactive > 0 && pAp > 0.0 && s->rr > 0.0) ? s->rr / pAp : 0.0;
    s->alpha = alpha;
    s->coef_r[0] = -alpha;
    s->coef_r[1] = 0.0;
    for (int j = 0; j < ns; ++j) {
        if (!s->active[j] || alpha == 0.0) {
            s->aj[j] = 0.0;
            continue;
        }
        const double den = alpha * s->beta_prev * (s->zp[j] - s->z[j]) +
                           s->zp[j] * s->alpha_prev * (1.0 + s->ds[j] * alpha);
        s->zn[j] = den != 0.0 ? s->z[j] * s->zp[j] * s->alpha_prev / den : 0.0;
        s->aj[j] = s->z[j] != 0.0 ? alpha * s->zn[j] / s->z[j] : 0.0;
    }
}

__global__ void k_mscg_beta(MscgDev* s, const double* __restrict__ red, int ns) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double rr_new = red[2];
    const bool step = s->alpha != 0.0;
    const double beta = (step && s->rr > 0.0) ? rr_new / s->rr : 0.0;
    int na = 0;
    for (int j = 0; j < ns; ++j) {
        s->upd[j] = step && s->active[j];
        if (!s->upd[j]) continue;
        const double q = s->z[j] != 0.0 ? s->zn[j] / s->z[j] : 0.0;
        s->bj[j] = beta * q * q;
        s->zj[j] = s->zn[j];
        if (fabs(s->zn[j]) * sqrt(rr_new) <= s->tol * s->bn) s->active[j] = 0;
        s->zp[j] = s->z[j];
        s->z[j] = s->zn[j];
    }
    for (int j = 0; j < ns; ++j) na += s->active[j];
    s->nactive = na;
    if (step) {
        s->rr = rr_new;
        s->alpha_prev = s->alpha;
        s->beta_prev = beta;
        s->iter += 1;
    }
    s->coef_p[0] = 1.0;
    s->coef_p[1] = beta;
}

static int mscg_iteration_dev(qxd_ctx* ctx, int fl, int P, int ns, double s0, MscgDev* dstate, const ShiftPtrs& sp,
                              void* r, void* pb, void* Ap, void* te, void* to, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    QXD_TRY(op_normal(ctx, fl, P, s0, pb, Ap, te, to, st));
    QXD_TRY(blas_dot(ctx, P, P, n, pb, Ap, 0, st));
    k_mscg_alpha<<<1, 32, 0, st>>>(dstate, ctx->red_result, ns);
    QXD_CUDA(ctx, cudaGetLastError());
    QXD_TRY(blas_axpy_norm_dev(ctx, P, n, dstate->coef_r, Ap, r, 2, st));
    k_mscg_beta<<<1, 32, 0, st>>>(dstate, ctx->red_result, ns);
    QXD_CUDA(ctx, cudaGetLastError());
    ShiftCoefDev c{dstate->aj, dstate->zj, dstate->bj, dstate->upd};
    QXD_TRY(blas_msg_update_dev(ctx, P, n, ns, sp, c, r, st));
    QXD_TRY(blas_axpby_dev(ctx, P, n, dstate->coef_p, r, pb, st));
    return QXD_OK;
}

static bool graphs_enabled() {
    const char* e = std::getenv("QXD_GRAPHS");
    return !(e && e[0] == '0');
}

static int mscg_core_graph(qxd_ctx* ctx, int fl, int P, int ns, const double* sigma, const void* b, char* X,
                           int max_iter, double tol, int* iters, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, P);
    void *r, *pb, *Ap, *te, *to, *Pblk, *dsv;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 110, hb, &r));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 111, hb, &pb));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 112, hb, &Ap));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 113, hb, &te));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 114, hb, &to));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 109, hb * ns, &Pblk));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 122, sizeof(MscgDev), &dsv));
    MscgDev* dstate = static_cast<MscgDev*>(dsv);
    char* Pc = static_cast<char*>(Pblk);
    QXD_CUDA(ctx, cudaMemsetAsync(X, 0, hb * ns, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(pb, b, hb, cudaMemcpyDeviceToDevice, st));
    for (int j = 0; j < ns; ++j) QXD_CUDA(ctx, cudaMemcpyAsync(Pc + j * hb, b, hb, cudaMemcpyDeviceToDevice, st));
    QXD_TRY(blas_norm2(ctx, P, n, b, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "MSCG source"));
    *iters = 0;
    if (!(ctx->red_host[0] > 0.0)) return QXD_OK;
    double s0 = sigma[0];
    for (int j = 1; j < ns; ++j) s0 = std::min(s0, sigma[j]);
    MscgDev h{};
    h.rr = ctx->red_host[0];
    h.bn = std::sqrt(h.rr);
    h.tol = tol;
    h.alpha_prev = 1.0;
    h.beta_prev = 0.0;
    for (int j = 0; j < ns; ++j) {
        h.ds[j] = sigma[j] - s0;
        h.zp[j] = h.z[j] = 1.0;
        h.active[j] = 1;
    }
    h.nactive = ns;
    QXD_CUDA(ctx, cudaMemcpyAsync(dstate, &h, sizeof h, cudaMemcpyHostToDevice, st));
    ShiftPtrs sp;
    for (int j = 0; j < ns; ++j) {
        sp.x[j] = X + j * hb;
        sp.p[j] = Pc + j * hb;
    }
    // first iteration eagerly (it also settles the autotuned kernel shapes)
    QXD_TRY(mscg_iteration_dev(ctx, fl, P, ns, s0, dstate, sp, r, pb, Ap, te, to, st));
    if (!ctx->cap_stream) QXD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    const int prof_mode = ctx->prof_mode;
    ctx->prof_mode = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = QXD_OK;
    if (cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        ctx->prof_mode = prof_mode;
        return qxd_fail(ctx, QXD_ECUDA, "MSCG: cannot start graph capture");
    }
    for (int k = 0; k < kGraphIters && rc == QXD_OK; ++k)
        rc = mscg_iteration_dev(ctx, fl, P, ns, s0, dstate, sp, r, pb, Ap, te, to, ctx->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ctx->prof_mode = prof_mode;
    if (rc != QXD_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        return qxd_fail(ctx, QXD_ECUDA, "MSCG: graph capture failed");
    }
    size_t nnodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nnodes);
    const double it_bytes = (2 * (1952.0 / 96) + 6 + 4 * ns) * (double)hb;  // rough, for the profile only
    MscgDev* hs = reinterpret_cast<MscgDev*>(ctx->red_host);  // pinned host mirror (large enough)
    static_assert(sizeof(MscgDev) <= kRedSlots * sizeof(double), "state fits the pinned mirror");
    while (true) {
        {
            ProfScope prof(ctx, "mscg_graph", kGraphIters * it_bytes, st, (int)nnodes);
            if (cudaGraphLaunch(exec, st) != cudaSuccess) {
                rc = qxd_fail(ctx, QXD_ECUDA, "MSCG: graph launch failed");
                break;
            }
        }
        if (cudaMemcpyAsync(hs, dstate, sizeof(MscgDev), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = qxd_fail(ctx, QXD_ECUDA, "MSCG: state read failed");
            break;
        }
        *iters = hs->iter;
        if (!std::isfinite(hs->rr)) {
            rc = qxd_fail(ctx, QXD_ENAN, "non-finite value in MSCG");
            break;
        }
        if (verbose()) std::fprintf(stderr, "[qxd mscg-graph] it %d active %d |r|/|b| %.3e\n", hs->iter, hs->nactive,
                                    std::sqrt(hs->rr) / hs->bn);
        if (hs->nactive == 0 || hs->iter >= max_iter || hs->alpha == 0.0) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    return rc;
}

int solve_mscg(qxd_ctx* ctx, int fl, int ns, const double* sigma, const qxd_solver* s, const void* b64, char* X64,
               qxd_info* info, cudaStream_t st) {
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb64 = half_bytes(ctx, QXD_FP64);
    const int P = s->inner == QXD_FP64 ? QXD_FP64 : QXD_FP32;
    info->iters = 0;
    info->restarts = 0;
    int it = 0;
    QXD_TRY(blas_norm2(ctx, 0, n, b64, 0, st));
    QXD_TRY(blas_fetch(ctx, 2, st));
    QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "source"));
    const double bn = std::sqrt(ctx->red_host[0]);
    if (bn == 0.0) {
        QXD_CUDA(ctx, cudaMemsetAsync(X64, 0, hb64 * ns, st));
        info->true_relres = 0.0;
        return QXD_OK;
    }
    if (P == QXD_FP64) {
        if (graphs_enabled()) QXD_TRY(mscg_core_graph(ctx, fl, 0, ns, sigma, b64, X64, s->nmx, 0.5 * s->tol, &it, st));
        else QXD_TRY(mscg_core(ctx, fl, 0, ns, sigma, b64, X64, s->nmx, 0.5 * s->tol, &it, st));
        info->iters += it;
    } else {
        const size_t hbP = half_bytes(ctx, P);
        void *bP, *XP;
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 107, hbP, &bP));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 108, hbP * ns, &XP));
        QXD_TRY(blas_axpby(ctx, 0, P, n, 1.0, 0.0, b64, 0.0, 0.0, bP, st));
        if (graphs_enabled())
            QXD_TRY(mscg_core_graph(ctx, fl, P, ns, sigma, bP, static_cast<char*>(XP), s->nmx, std::max(s->tol, 1e-6),
                                    &it, st));
        else
            QXD_TRY(mscg_core(ctx, fl, P, ns, sigma, bP, static_cast<char*>(XP), s->nmx, std::max(s->tol, 1e-6), &it,
                              st));
        info->iters += it;
        for (int j = 0; j < ns; ++j)
            QXD_TRY(blas_axpby(ctx, P, 0, n, 1.0, 0.0, static_cast<char*>(XP) + j * hbP, 0.0, 0.0, X64 + j * hb64, st));
    }
    // FP64 residual of every shift; FP32 defect correction where it misses tol
    void *r64, *te, *to, *eP, *rP;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 104, hb64, &r64));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 105, hb64, &te));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 106, hb64, &to));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 120, half_bytes(ctx, QXD_FP32), &eP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 121, half_bytes(ctx, QXD_FP32), &rP));
    // With an FP32 Krylov space the residuals b - (Q2 + s_j) x_j are taken on the FP64
    // data in double-float arithmetic (FP32 pipe); they land in FP32 directly for the
    // correction solve.  A plain FP64 run keeps FP64.
    const bool df = P != QXD_FP64;
    void *bdf = nullptr, *xdf = nullptr, *ydf = nullptr, *tdf = nullptr;
    if (df) {
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 36, hb64, &bdf));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 37, hb64, &xdf));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 38, hb64, &ydf));
        QXD_TRY(qxd_ws(ctx, WS_SOLVER + 39, hb64, &tdf));
        QXD_TRY(blas_split_df64(ctx, b64, bdf, n, st));
    }
    double worst = 0.0;
    for (int j = 0; j < ns; ++j) {
        char* xj = X64 + j * hb64;
        for (int pass = 0; pass < 16; ++pass) {
            if (df) {
                QXD_TRY(blas_split_df64(ctx, xj, xdf, n, st));
                QXD_TRY(op_Dhat(ctx, fl, QXD_DF64, 0, xdf, tdf, to, st));
                QXD_TRY(op_Dhat(ctx, fl, QXD_DF64, 1, tdf, ydf, to, st));
                QXD_TRY(blas_df_shift_residual(ctx, bdf, ydf, xdf, sigma[j], rP, 0, st));
            } else {
                QXD_TRY(op_normal(ctx, fl, 0, sigma[j], xj, r64, te, to, st));
                QXD_TRY(blas_axpby(ctx, 0, 0, n, 1.0, 0.0, b64, -1.0, 0.0, r64, st));
                QXD_TRY(blas_norm2(ctx, 0, n, r64, 0, st));
            }
            QXD_TRY(blas_fetch(ctx, 2, st));
            QXD_TRY(status_of_norm(ctx, ctx->red_host[1], "MSCG residual"));
            const double rel = std::sqrt(ctx->red_host[0]) / bn;
            if (verbose()) std::fprintf(stderr, "[qxd mscg] shift %d pass %d relres %.3e\n", j, pass, rel);
            if (rel <= s->tol || info->iters >= s->nmx) {
                worst = std::max(worst, rel);
                break;
            }
            info->restarts += 1;
            if (!df) QXD_TRY(blas_axpby(ctx, 0, 1, n, 1.0, 0.0, r64, 0.0, 0.0, rP, st));
            int ci = 0;
            QXD_TRY(cg_shifted(ctx, fl, 1, sigma[j], rP, eP, s->nmx - info->iters, std::max(1e-5, 0.5 * s->tol / rel),
                               &ci, st));
            info->iters += ci;
            QXD_TRY(blas_axpby(ctx, 1, 0, n, 1.0, 0.0, eP, 1.0, 0.0, xj, st));
            if (pass == 15) worst = std::max(worst, rel);
        }
    }
    info->true_relres = worst;
    if (worst <= s->tol) return QXD_OK;
    return qxd_fail(ctx, QXD_ENOCONV, "MSCG: tolerance not reached within nmx");
}

}  // namespace qxd

namespace qxd {

// ---- batched FGCR: nrhs right-hand sides in lockstep -------------------------------
// Vectors of the batch are stored as blocks of nrhs consecutive half-lattice
// fields, so Dhat is applied to the whole block by one multi-right-hand-side
// launch pair (links and site-diagonal terms read once).  Each right-hand side
// has its own GCR scalars and stops independently (a finished one keeps its
// solution and is no longer updated).
// workspace of the batched inner solve: r, t_o, scratch, the two Krylov bases, one
// preconditioner scratch field and the basis-precision copy of e
struct BatchedWs {
    void *rv, *tov, *tmpv, *Zv, *Wv, *ztmp, *tbv;
};
static int batched_inner_ws(qxd_ctx* ctx, int P, int nkv, int B, BatchedWs* w) {
    const int Pb = P, Pv = vec_prec(P);
    const size_t hb = half_bytes(ctx, Pb), hv = half_bytes(ctx, Pv);
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 130, hv * B, &w->rv));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 131, hb * B, &w->tov));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 132, hb * B, &w->tmpv));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 133, hb * B * nkv, &w->Zv));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 134, hb * B * nkv, &w->Wv));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 135, hv, &w->ztmp));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 136, hb * B, &w->tbv));
    return QXD_OK;
}

static int fgcr_inner_batched(qxd_ctx* ctx, int fl, int P, const qxd_solver* s, const char* b, char* e, int B,
                              int max_iter, const std::vector<double>& rtol, std::vector<int>& iters, bool* stagnated,
                              cudaStream_t st) {
    *stagnated = false;
    const int nkv = s->nkv < 1 ? 1 : (s->nkv > 64 ? 64 : s->nkv);
    const int Pb = P, Pv = vec_prec(P);
    const bool split = Pb != Pv;
    const size_t n = 12ull * ctx->g.Vh;
    const size_t hb = half_bytes(ctx, Pb), hv = half_bytes(ctx, Pv);
    BatchedWs w;
    QXD_TRY(batched_inner_ws(ctx, P, nkv, B, &w));
    void *rv = w.rv, *tov = w.tov, *tmpv = w.tmpv, *Zv = w.Zv, *Wv = w.Wv, *ztmp = w.ztmp, *tbv = w.tbv;
    char* r = static_cast<char*>(rv);
    char* Z = static_cast<char*>(Zv);
    char* W = static_cast<char*>(Wv);
    auto Zk = [&](int k, int j) { return Z + ((size_t)k * B + j) * hb; };
    auto Wk = [&](int k, int j) { return W + ((size_t)k * B + j) * hb; };
    auto Rj = [&](int j) { return r + (size_t)j * hv; };
    QXD_CUDA(ctx, cudaMemsetAsync(e, 0, hv * B, st));
    QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hv * B, cudaMemcpyDeviceToDevice, st));
    std::vector<double> bn(B), rr(B);
    std::vector<char> done(B, 0);
    for (int j = 0; j < B; ++j) QXD_TRY(blas_norm2(ctx, Pv, n, b + j * hv, 2 * j, st));
    QXD_TRY(blas_fetch(ctx, 2 * B, st));
    for (int j = 0; j < B; ++j) {
        QXD_TRY(status_of_norm(ctx, ctx->red_host[2 * j + 1], "GCR source"));
        bn[j] = std::sqrt(ctx->red_host[2 * j]);
        rr[j] = bn[j] * bn[j];
        iters[j] = 0;
        done[j] = bn[j] == 0.0 || rtol[j] >= 1.0;
    }
    std::vector<double> Rre((size_t)B * nkv * nkv), Rim((size_t)B * nkv * nkv), are((size_t)B * nkv),
        aim((size_t)B * nkv), ww((size_t)B * nkv), cre(nkv), cim(nkv);
    std::vector<const void*> Wc(nkv + 1);
    int it = 0;
    auto all_done = [&]() {
        for (int j = 0; j < B; ++j)
            if (!done[j]) return false;
        return true;
    };
    std::vector<double> rr_cycle(B);
    while (!all_done() && it < max_iter) {
        int K = 0;
        for (int j = 0; j < B; ++j) rr_cycle[j] = rr[j];
        std::vector<char> active(done.begin(), done.end());
        for (int j = 0; j < B; ++j) active[j] = !done[j];
        // Without a preconditioner (and one basis precision) the direction of step k is
        // the residual r_k itself, kept in Z_k; the fused step writes r_{k+1} into Z_{k+1}
        // (into r after the last step of a cycle), as in fgcr_inner.
        const bool rz = s->precond == QXD_PRECOND_NONE && !split;
        if (rz) QXD_CUDA(ctx, cudaMemcpyAsync(Zk(0, 0), r, hb * B, cudaMemcpyDeviceToDevice, st));
        for (int k = 0; k < nkv; ++k) {
            if (!rz && s->precond == QXD_PRECOND_NONE) {
                QXD_TRY(blas_axpby(ctx, Pv, Pb, n * B, 1.0, 0.0, r, 0.0, 0.0, Zk(k, 0), st));
            } else if (!rz) {
                for (int j = 0; j < B; ++j)
                    if (active[j] == 1) QXD_TRY(precond_into(ctx, fl, Pv, Pb, s->precond, Rj(j), Zk(k, j), ztmp, st));
            }
            QXD_TRY(op_Dhat(ctx, fl, Pb, 0, Zk(k, 0), Wk(k, 0), tov, st, B));
            // per right-hand side (nv complex slots each): <W_q, w> (q < k), <r, w> and,
            // with rz, |w|^2
            const int nv = k + 1 + (rz ? 1 : 0);
            for (int j = 0; j < B; ++j) {
                if (active[j] != 1) continue;
                for (int q = 0; q < k; ++q) Wc[q] = Wk(q, j);
                int m = k;
                if (!split) Wc[m++] = rz ? static_cast<const void*>(Zk(k, j)) : static_cast<const void*>(Rj(j));
                if (rz) Wc[m++] = Wk(k, j);
                if (m > 0) QXD_TRY(blas_multi_dot(ctx, Pb, n, m, Wc.data(), Wk(k, j), 2 * nv * j, st));
                if (split) QXD_TRY(blas_dot(ctx, Pv, Pb, n, Rj(j), Wk(k, j), 2 * nv * j + 2 * k, st));
            }
            QXD_TRY(blas_fetch(ctx, 2 * nv * B, st));
            std::vector<double> wr_re(B), wr_im(B), w2o(B, 0.0);
            std::vector<char> fused(B, 0);
            for (int j = 0; j < B; ++j) {
                if (active[j] != 1) continue;
                const double* h = ctx->red_host + 2 * nv * j;
                for (int q = 0; q < k; ++q) {
                    const size_t o = ((size_t)j * nkv + q) * nkv + k;
                    Rre[o] = h[2 * q] / ww[(size_t)j * nkv + q];
                    Rim[o] = h[2 * q + 1] / ww[(size_t)j * nkv + q];
                }
                wr_re[j] = h[2 * k];
                wr_im[j] = -h[2 * k + 1];
                if (rz) {
                    // |w'|^2 = |w|^2 - sum_q |<W_q, w>|^2 / |W_q|^2 unless it cancels below 1 %
                    const double w2 = h[2 * (k + 1)];
                    double v = w2;
                    for (int q = 0; q < k; ++q)
                        v -= (h[2 * q] * h[2 * q] + h[2 * q + 1] * h[2 * q + 1]) / ww[(size_t)j * nkv + q];
                    if (std::isfinite(v) && v > 0.01 * w2) {
                        fused[j] = 1;
                        w2o[j] = v;
                    }
                }
            }
            bool need_norm = false;
            for (int j = 0; j < B; ++j) {
                if (active[j] != 1 || fused[j]) continue;
                need_norm = true;
                for (int q = 0; q < k; ++q) {
                    const size_t o = ((size_t)j * nkv + q) * nkv + k;
                    cre[q] = -Rre[o];
                    cim[q] = -Rim[o];
                    Wc[q] = Wk(q, j);
                }
                QXD_TRY(blas_multi_axpy_norm(ctx, Pb, n, k, cre.data(), cim.data(), Wc.data(), Wk(k, j), 2 * j, st));
            }
            if (need_norm) QXD_TRY(blas_fetch(ctx, 2 * B, st));
            for (int j = 0; j < B; ++j) {
                if (active[j] != 1) continue;
                double w2;
                if (fused[j]) {
                    w2 = w2o[j];
                } else {
                    QXD_TRY(status_of_norm(ctx, ctx->red_host[2 * j + 1], "GCR"));
                    w2 = ctx->red_host[2 * j];
                }
                if (!(w2 > 0.0)) return qxd_fail(ctx, QXD_EBREAKDOWN, "GCR: |w| = 0");
                ww[(size_t)j * nkv + k] = w2;
                const double ar = wr_re[j] / w2, ai = wr_im[j] / w2;
                are[(size_t)j * nkv + k] = ar;
                aim[(size_t)j * nkv + k] = ai;
                if (rz) {
                    void* next = k + 1 < nkv ? static_cast<void*>(Zk(k + 1, j)) : static_cast<void*>(Rj(j));
                    if (fused[j]) {
                        for (int q = 0; q < k; ++q) {
                            const size_t o = ((size_t)j * nkv + q) * nkv + k;
                            cre[q] = -Rre[o];
                            cim[q] = -Rim[o];
                            Wc[q] = Wk(q, j);
                        }
                        QXD_TRY(blas_gcr_update(ctx, Pb, n, k, cre.data(), cim.data(), Wc.data(), Wk(k, j), -ar, -ai,
                                                Zk(k, j), next, st));
                    } else {
                        QXD_TRY(blas_axpy3(ctx, Pb, n, -ar, -ai, Wk(k, j), Zk(k, j), next, st));
                    }
                } else {
                    QXD_TRY(blas_axpby(ctx, Pb, Pv, n, -ar, -ai, Wk(k, j), 1.0, 0.0, Rj(j), st));
                }
                rr[j] -= (wr_re[j] * wr_re[j] + wr_im[j] * wr_im[j]) / w2;
                iters[j] += 1;
            }
            ++it;
            K = k + 1;
            bool any = false;
            for (int j = 0; j < B; ++j) {
                if (active[j] && rr[j] <= rtol[j] * rtol[j] * bn[j] * bn[j]) active[j] = 2;  // converged in-cycle
                any = any || active[j] == 1;
            }
            if (!any || it >= max_iter) break;
        }
        // per right-hand side: back substitution and e += sum_k c_k Z_k over the
        // steps it took part in (a right-hand side that stopped in-cycle has K_j < K)
        for (int j = 0; j < B; ++j) {
            if (done[j]) continue;
            int Kj = 0;
            for (int k = 0; k < K; ++k)
                if (ww[(size_t)j * nkv + k] > 0.0) Kj = k + 1;
            for (int q = Kj - 1; q >= 0; --q) {
                double sr = are[(size_t)j * nkv + q], si = aim[(size_t)j * nkv + q];
                for (int k2 = q + 1; k2 < Kj; ++k2) {
                    const size_t o = ((size_t)j * nkv + q) * nkv + k2;
                    sr -= Rre[o] * cre[k2] - Rim[o] * cim[k2];
                    si -= Rre[o] * cim[k2] + Rim[o] * cre[k2];
                }
                cre[q] = sr;
                cim[q] = si;
            }
            if (!split) {
                for (int k = 0; k < Kj; ++k) Wc[k] = Zk(k, j);
                if (Kj > 0)
                    QXD_TRY(blas_multi_axpy(ctx, Pv, Pv, n, Kj, cre.data(), cim.data(), Wc.data(), e + j * hv, st));
            } else {
                for (int k = 0; k < Kj; ++k)
                    QXD_TRY(blas_axpby(ctx, Pb, Pv, n, cre[k], cim[k], Zk(k, j), 1.0, 0.0, e + j * hv, st));
            }
            for (int k = 0; k < nkv; ++k) ww[(size_t)j * nkv + k] = 0.0;
            if (active[j] == 2) done[j] = 1;
        }
        if (all_done() || it >= max_iter) break;
        // restart: r = b - Dhat e for the whole block (through the basis precision)
        if (split) {
            QXD_TRY(blas_axpby(ctx, Pv, Pb, n * B, 1.0, 0.0, e, 0.0, 0.0, tbv, st));
            QXD_TRY(op_Dhat(ctx, fl, Pb, 0, tbv, static_cast<char*>(tmpv), tov, st, B));
        } else {
            QXD_TRY(op_Dhat(ctx, fl, Pb, 0, e, static_cast<char*>(tmpv), tov, st, B));
        }
        QXD_CUDA(ctx, cudaMemcpyAsync(r, b, hv * B, cudaMemcpyDeviceToDevice, st));
        QXD_TRY(blas_axpby(ctx, Pb, Pv, n * B, -1.0, 0.0, tmpv, 1.0, 0.0, r, st));
        for (int j = 0; j < B; ++j) QXD_TRY(blas_norm2(ctx, Pv, n, Rj(j), 2 * j, st));
        QXD_TRY(blas_fetch(ctx, 2 * B, st));
        for (int j = 0; j < B; ++j) {
            if (done[j]) continue;
            rr[j] = ctx->red_host[2 * j];
            if (rr[j] <= rtol[j] * rtol[j] * bn[j] * bn[j]) done[j] = 1;
            // a whole cycle that did not halve the residual norm
            else if (K == nkv && rr[j] > 0.25 * rr_cycle[j]) *stagnated = true;
        }
        if (*stagnated) return QXD_OK;
    }
    return QXD_OK;
}

int solve_fgcr_dc_batched(qxd_ctx* ctx, int fl, const qxd_solver* s, const Full& eta, const Full& x, int B,
                          qxd_info* info, cudaStream_t st) {
    const int nkv = s->nkv < 1 ? 1 : (s->nkv > 64 ? 64 : s->nkv);
    if (2 * (nkv + 1) * B > kRedSlots)
        return qxd_fail(ctx, QXD_EARG, "batched FGCR: nrhs * (nkv + 1) must not exceed 256");
    const size_t n = 12ull * ctx->g.Vh;
    const int P = s->inner;
    const int Pv = vec_prec(P);
    // as in solve_fgcr_dc: with FP32/BF16 inner solves the outer loop holds x and D x as
    // double-float fields (one multi-right-hand-side double-float D_w per outer step);
    // FP64 inner solves keep it in FP64, and so does a lattice whose double-float copies
    // of the links and site-diagonal terms do not fit in the device memory
    bool df = P != QXD_FP64;
    const size_t hb64 = half_bytes(ctx, QXD_FP64), hbP = half_bytes(ctx, Pv);
    // the FP64-sized pair holds x (double-float) or the residual r (FP64 outer loop)
    void *s0, *s1, *bP, *roP, *tP, *eeP, *eoP, *to2;
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 140, hb64 * B, &s0));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 141, hb64 * B, &s1));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 142, hbP * B, &bP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 143, hbP * B, &roP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 144, hbP * B, &tP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 145, hbP * B, &eeP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 146, hbP * B, &eoP));
    QXD_TRY(qxd_ws(ctx, WS_SOLVER + 147, hbP * B, &to2));
    if (df) {
        // the inner solve's workspace first, so that the copies take only what is left
        BatchedWs w;
        QXD_TRY(batched_inner_ws(ctx, P, nkv, B, &w));
        if (ensure_df64(ctx, fl, st) != QXD_OK) df = false;
    }
    void *re = nullptr, *ro = nullptr, *xde = nullptr, *xdo = nullptr;
    if (df) {
        xde = s0;
        xdo = s1;
    } else {
        re = s0;
        ro = s1;
    }
    char* E = static_cast<char*>(eeP);
    auto at = [](void* base, size_t stride, int j) { return static_cast<char*>(base) + (size_t)j * stride; };
    auto cat = [](const void* base, size_t stride, int j) { return static_cast<const char*>(base) + (size_t)j * stride; };
    std::vector<double> enorm(B), relres(B, 1.0);
    for (int j = 0; j < B; ++j) {
        if (df) {  // the sources' FP32 roundings for the first inner solve and their norms
            QXD_TRY(blas_f64_to_f32_norm(ctx, cat(eta.e, hb64, j), at(tP, hbP, j), 4 * j, st));
            QXD_TRY(blas_f64_to_f32_norm(ctx, cat(eta.o, hb64, j), at(roP, hbP, j), 4 * j + 2, st));
        } else {
            QXD_TRY(blas_norm2(ctx, 0, n, cat(eta.e, hb64, j), 4 * j, st));
            QXD_TRY(blas_norm2(ctx, 0, n, cat(eta.o, hb64, j), 4 * j + 2, st));
        }
    }
    QXD_TRY(blas_fetch(ctx, 4 * B, st));
    for (int j = 0; j < B; ++j) {
        QXD_TRY(status_of_norm(ctx, ctx->red_host[4 * j + 1] + ctx->red_host[4 * j + 3], "source"));
        enorm[j] = std::sqrt(ctx->red_host[4 * j] + ctx->red_host[4 * j + 2]);
    }
    QXD_CUDA(ctx, cudaMemsetAsync(x.e, 0, hb64 * B, st));
    QXD_CUDA(ctx, cudaMemsetAsync(x.o, 0, hb64 * B, st));
    if (df) {
        QXD_CUDA(ctx, cudaMemsetAsync(xde, 0, hb64 * B, st));
        QXD_CUDA(ctx, cudaMemsetAsync(xdo, 0, hb64 * B, st));
    } else {
        QXD_CUDA(ctx, cudaMemcpyAsync(re, eta.e, hb64 * B, cudaMemcpyDeviceToDevice, st));
        QXD_CUDA(ctx, cudaMemcpyAsync(ro, eta.o, hb64 * B, cudaMemcpyDeviceToDevice, st));
    }
    // true residuals of the current x: relres[j]; in the double-float loop they also
    // leave FP32(eta - D x) in tP, roP for the next inner solve
    auto residuals = [&](bool* all) -> int {
        if (df) {
            // D x goes to the inner solver's Krylov-basis slot, which is free between inner solves
            void* dx;
            QXD_TRY(qxd_ws(ctx, WS_SOLVER + 133, 2 * hb64 * B, &dx));
            char* dxe = static_cast<char*>(dx);
            char* dxo = dxe + hb64 * B;
            QXD_TRY(op_Dw(ctx, fl, QXD_DF64, Full{xde, xdo}, Full{dxe, dxo}, st, B));
            for (int j = 0; j < B; ++j) {
                QXD_TRY(blas_df_residual(ctx, cat(eta.e, hb64, j), at(dxe, hb64, j), at(tP, hbP, j), 4 * j, st));
                QXD_TRY(blas_df_residual(ctx, cat(eta.o, hb64, j), at(dxo, hb64, j), at(roP, hbP, j), 4 * j + 2, st));
            }
        } else {
            QXD_TRY(op_Dw(ctx, fl, QXD_FP64, x, Full{re, ro}, st, B));
            QXD_TRY(blas_axpby(ctx, 0, 0, n * B, 1.0, 0.0, eta.e, -1.0, 0.0, re, st));
            QXD_TRY(blas_axpby(ctx, 0, 0, n * B, 1.0, 0.0, eta.o, -1.0, 0.0, ro, st));
            for (int j = 0; j < B; ++j) {
                QXD_TRY(blas_norm2(ctx, 0, n, at(re, hb64, j), 4 * j, st));
                QXD_TRY(blas_norm2(ctx, 0, n, at(ro, hb64, j), 4 * j + 2, st));
            }
        }
        QXD_TRY(blas_fetch(ctx, 4 * B, st));
        *all = true;
        for (int j = 0; j < B; ++j) {
            QXD_TRY(status_of_norm(ctx, ctx->red_host[4 * j + 1] + ctx->red_host[4 * j + 3], "residual"));
            relres[j] = enorm[j] > 0 ? std::sqrt(ctx->red_host[4 * j] + ctx->red_host[4 * j + 2]) / enorm[j] : 0.0;
            *all = *all && relres[j] <= s->tol;
        }
        return QXD_OK;
    };
    // the double-float solutions go to the caller's FP64 fields
    auto finish = [&]() -> int {
        if (df)
            for (int j = 0; j < B; ++j) {
                QXD_TRY(blas_join_df64(ctx, at(xde, hb64, j), at(x.e, hb64, j), n, st));
                QXD_TRY(blas_join_df64(ctx, at(xdo, hb64, j), at(x.o, hb64, j), n, st));
            }
        return QXD_OK;
    };
    const double itol = s->inner_tol > 0 ? s->inner_tol : (P == QXD_BF16 ? 5e-3 : (P == QXD_FP32 ? 1e-5 : 1e-10));
    info->iters = 0;
    info->restarts = 0;
    info->op_applies = 0;
    std::vector<int> its(B, 0);
    bool use_cgnr = false;
    for (int outer = 0; outer < 64; ++outer) {
        if (outer > 0) {
            bool all = false;
            QXD_TRY(residuals(&all));
            info->op_applies += B;
            if (verbose()) std::fprintf(stderr, "[qxd dc-batched] outer %d worst relres %.3e\n", outer,
                                        *std::max_element(relres.begin(), relres.end()));
            if (all) break;
            info->restarts += 1;
        }
        if (info->iters >= s->nmx) break;
        if (!df) {
            QXD_TRY(blas_axpby(ctx, 0, Pv, n * B, 1.0, 0.0, re, 0.0, 0.0, tP, st));
            QXD_TRY(blas_axpby(ctx, 0, Pv, n * B, 1.0, 0.0, ro, 0.0, 0.0, roP, st));
        }
        QXD_TRY(op_eo_source(ctx, fl, Pv, Full{tP, roP}, bP, to2, st, B));
        std::vector<double> rtol(B);
        for (int j = 0; j < B; ++j) rtol[j] = relres[j] <= s->tol ? 1.0 : std::max(itol, 0.5 * s->tol / relres[j]);
        int mx = 0;
        if (!use_cgnr) {
            bool stag = false;
            QXD_TRY(fgcr_inner_batched(ctx, fl, P, s, static_cast<char*>(bP), E, B, s->nmx - info->iters, rtol, its,
                                       &stag, st));
            for (int j = 0; j < B; ++j) mx = std::max(mx, its[j]);
            if (stag) {
                // restarted GCR stalls on this operator: from here on CG on the normal
                // equations (FP32 or FP64) for each right-hand side, starting again from 0
                use_cgnr = true;
                if (verbose()) std::fprintf(stderr, "[qxd dc-batched] GCR stagnated: CGNR inner\n");
            }
        }
        if (use_cgnr) {
            for (int j = 0; j < B; ++j) {
                int it = 0;
                if (rtol[j] >= 1.0) {
                    QXD_CUDA(ctx, cudaMemsetAsync(E + j * hbP, 0, hbP, st));
                    continue;
                }
                const double ctol = Pv == QXD_FP64 ? rtol[j] : std::max(1e-5, 0.5 * s->tol / relres[j]);
                QXD_TRY(cgnr_inner(ctx, fl, Pv, static_cast<char*>(bP) + j * hbP, E + j * hbP, s->nmx - info->iters,
                                   ctol, &it, st));
                mx = std::max(mx, 2 * it);
            }
        }
        info->iters += mx;
        info->op_applies += mx * B;
        QXD_TRY(op_odd_reconstruct(ctx, fl, Pv, roP, E, eoP, st, B));
        if (df) {
            for (int j = 0; j < B; ++j) {
                QXD_TRY(blas_df_add_f32(ctx, at(eeP, hbP, j), at(xde, hb64, j), st));
                QXD_TRY(blas_df_add_f32(ctx, at(eoP, hbP, j), at(xdo, hb64, j), st));
            }
        } else {
            QXD_TRY(blas_axpby(ctx, Pv, 0, n * B, 1.0, 0.0, E, 1.0, 0.0, x.e, st));
            QXD_TRY(blas_axpby(ctx, Pv, 0, n * B, 1.0, 0.0, eoP, 1.0, 0.0, x.o, st));
        }
    }
    QXD_TRY(finish());
    double worst = 0.0;
    for (int j = 0; j < B; ++j) worst = std::max(worst, relres[j]);
    info->true_relres = worst;
    if (worst <= s->tol) return QXD_OK;
    return qxd_fail(ctx, QXD_ENOCONV, "batched FGCR: tolerance not reached within nmx");
}

}  // namespace qxd
