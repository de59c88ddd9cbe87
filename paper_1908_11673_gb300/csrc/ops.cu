// Operator compositions (Sec. 2.3): D, Dhat = D_ee - D_eo D_oo^-1 D_oe, the
// even-odd source and the odd-site reconstruction, each as one or two launches
// of the hopping kernel with a fused site-diagonal prologue or epilogue.
#include "blas.h"
#include "ops.h"

namespace qxd {

size_t half_bytes(const qxd_ctx* ctx, int P) {
    const size_t per = (P == QXD_FP64 || P == QXD_DF64) ? 192 : (P == QXD_FP32 ? 96 : 48);
    return per * (size_t)ctx->g.Vh;
}

int op_Dw(qxd_ctx* ctx, int fl, int P, const Full& in, const Full& out, cudaStream_t st, int nrhs) {
    if (P == QXD_DF64) QXD_TRY(ensure_df64(ctx, fl, st));
    HopArgs a{};
    a.c_hop = 1.0;
    a.self_mode = 1;
    a.post_mode = 0;
    a.nrhs = nrhs;
    a.pout = 0;
    a.in_nb = in.o;
    a.in_self = in.e;
    a.out = out.e;
    QXD_TRY(launch_hop(ctx, fl, P, a, st));
    a.pout = 1;
    a.in_nb = in.e;
    a.in_self = in.o;
    a.out = out.o;
    return launch_hop(ctx, fl, P, a, st);
}

int op_Dhat(qxd_ctx* ctx, int fl, int P, int dagger, const void* in_e, void* out_e, void* tmp_o, cudaStream_t st,
            int nrhs) {
    if (P == QXD_DF64) QXD_TRY(ensure_df64(ctx, fl, st, true));
    HopArgs a{};
    a.nrhs = nrhs;
    // tmp_o = A_oo^-1 H_oe (gamma5) in_e
    a.pout = 1;
    a.in_nb = in_e;
    a.in_self = nullptr;
    a.out = tmp_o;
    a.self_mode = 0;
    a.post_mode = 1;
    a.c_hop = 1.0;
    a.g5_nb = dagger;
    QXD_TRY(launch_hop(ctx, fl, P, a, st));
    // out_e = (gamma5) [A_ee (gamma5) in_e - H_eo tmp_o]
    a.pout = 0;
    a.in_nb = tmp_o;
    a.in_self = in_e;
    a.out = out_e;
    a.self_mode = 1;
    a.post_mode = 0;
    a.c_hop = -1.0;
    a.g5_nb = 0;
    a.g5_self = dagger;
    a.g5_out = dagger;
    return launch_hop(ctx, fl, P, a, st);
}

int op_Dhat_dots(qxd_ctx* ctx, int fl, const void* in_e, void* out_e, void* tmp_o, int k, const void* const* W,
                 int slot, cudaStream_t st) {
    HopArgs a{};
    a.nrhs = 1;
    a.pout = 1;
    a.in_nb = in_e;
    a.out = tmp_o;
    a.self_mode = 0;
    a.post_mode = 1;
    a.c_hop = 1.0;
    QXD_TRY(launch_hop(ctx, fl, QXD_FP32, a, st));
    a.pout = 0;
    a.in_nb = tmp_o;
    a.in_self = in_e;
    a.out = out_e;
    a.self_mode = 1;
    a.post_mode = 0;
    a.c_hop = -1.0;
    return launch_hop_dots(ctx, fl, a, k, W, slot, st);
}

int op_eo_source(qxd_ctx* ctx, int fl, int P, const Full& r, void* b_e, void* tmp_o, cudaStream_t st, int nrhs) {
    QXD_TRY(launch_diag(ctx, fl, P, 1, 1, r.o, tmp_o, nrhs, st));
    HopArgs a{};
    a.nrhs = nrhs;
    a.pout = 0;
    a.in_nb = tmp_o;
    a.in_self = r.e;
    a.out = b_e;
    a.self_mode = 2;
    a.post_mode = 0;
    a.c_hop = -1.0;
    return launch_hop(ctx, fl, P, a, st);
}

int op_odd_reconstruct(qxd_ctx* ctx, int fl, int P, const void* r_o, const void* x_e, void* x_o, cudaStream_t st,
                       int nrhs) {
    HopArgs a{};
    a.nrhs = nrhs;
    a.pout = 1;
    a.in_nb = x_e;
    a.in_self = r_o;
    a.out = x_o;
    a.self_mode = 2;
    a.post_mode = 1;
    a.c_hop = -1.0;
    return launch_hop(ctx, fl, P, a, st);
}

int apply_precond(qxd_ctx* ctx, int fl, int P, int kind, const void* r, void* z, cudaStream_t st) {
    if (kind == QXD_PRECOND_NONE) {
        QXD_CUDA(ctx, cudaMemcpyAsync(z, r, half_bytes(ctx, P), cudaMemcpyDeviceToDevice, st));
        return QXD_OK;
    }
    if (kind == QXD_PRECOND_SAP || kind == QXD_PRECOND_DFL) {
        auto even = kind == QXD_PRECOND_SAP ? sap_apply_even : dfl_apply_even;
        if (P == QXD_FP32) return even(ctx, fl, r, z, st);
        void *r32, *z32;
        const size_t n = 12ull * ctx->g.Vh;
        QXD_TRY(qxd_ws(ctx, WS_PTC + 50, half_bytes(ctx, QXD_FP32), &r32));
        QXD_TRY(qxd_ws(ctx, WS_PTC + 51, half_bytes(ctx, QXD_FP32), &z32));
        QXD_TRY(blas_axpby(ctx, P, QXD_FP32, n, 1.0, 0.0, r, 0.0, 0.0, r32, st));
        QXD_TRY(even(ctx, fl, r32, z32, st));
        return blas_axpby(ctx, QXD_FP32, P, n, 1.0, 0.0, z32, 0.0, 0.0, z, st);
    }
    if (kind == QXD_PRECOND_LEARNED) {
        const QxdFlavour& F = ctx->fl[fl];
        if (!F.W) return qxd_fail(ctx, QXD_ESTATE, "learned preconditioner weights not set");
        const float2* W = reinterpret_cast<const float2*>(F.W);
        if (P == QXD_FP32) return ptc_apply_internal(ctx, fl, W, F.nlayers, F.nch, r, z, st, F.wprec);
        // other precisions go through FP32 copies
        void *r32, *z32;
        const size_t n = 12ull * ctx->g.Vh;
        QXD_TRY(qxd_ws(ctx, WS_PTC + 50, half_bytes(ctx, QXD_FP32), &r32));
        QXD_TRY(qxd_ws(ctx, WS_PTC + 51, half_bytes(ctx, QXD_FP32), &z32));
        QXD_TRY(blas_axpby(ctx, P, QXD_FP32, n, 1.0, 0.0, r, 0.0, 0.0, r32, st));
        QXD_TRY(ptc_apply_internal(ctx, fl, W, F.nlayers, F.nch, r32, z32, st, F.wprec));
        return blas_axpby(ctx, QXD_FP32, P, n, 1.0, 0.0, z32, 0.0, 0.0, z, st);
    }
    return qxd_fail(ctx, QXD_EARG, "unknown preconditioner kind");
}

}  // namespace qxd
