// extern "C" entry points of libqxd (declared and documented in include/qxd.h).
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "blas.h"
#include "ops.h"
#include "qxd_internal.h"

using namespace qxd;

int qxd_fail(qxd_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int qxd_ws(qxd_ctx* ctx, int slot, size_t bytes, void** out) {
    if (slot < 0 || slot >= WS_NSLOTS) return qxd_fail(ctx, QXD_EARG, "workspace slot out of range");
    if ((int)ctx->ws_ptr.size() < WS_NSLOTS) {
        ctx->ws_ptr.resize(WS_NSLOTS, nullptr);
        ctx->ws_size.resize(WS_NSLOTS, 0);
    }
    if (ctx->ws_size[slot] < bytes) {
        if (ctx->ws_ptr[slot]) cudaFree(ctx->ws_ptr[slot]);
        ctx->ws_ptr[slot] = nullptr;
        ctx->ws_size[slot] = 0;
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return qxd_fail(ctx, QXD_ENOMEM, "workspace allocation of " + std::to_string(bytes) + " bytes failed");
        }
        ctx->ws_ptr[slot] = p;
        ctx->ws_size[slot] = bytes;
    }
    *out = ctx->ws_ptr[slot];
    return QXD_OK;
}

// ---- profiling -------------------------------------------------------------------
ProfScope::ProfScope(qxd_ctx* c, const char* name, double bytes, cudaStream_t s, int nlaunch) : ctx(c), st(s) {
    if (!ctx || ctx->prof_mode == 0) return;
    auto it = ctx->prof_idx.find(name);
    if (it == ctx->prof_idx.end()) {
        cls = (int)ctx->prof_cls.size();
        ctx->prof_idx[name] = cls;
        ctx->prof_cls.push_back(qxd_ctx::ProfClass{});
        ctx->prof_cls.back().name = name;
    } else {
        cls = it->second;
    }
    ctx->prof_cls[cls].launches += nlaunch;
    ctx->prof_cls[cls].bytes += bytes;
    if (ctx->prof_mode >= 2) {
        for (cudaEvent_t* e : {&a, &b}) {
            if (!ctx->prof_pool.empty()) {
                *e = ctx->prof_pool.back();
                ctx->prof_pool.pop_back();
            } else if (cudaEventCreate(e) != cudaSuccess) {
                cudaGetLastError();
                *e = nullptr;
            }
        }
        if (a) cudaEventRecord(a, st);
    }
}

ProfScope::~ProfScope() {
    if (cls < 0 || !a || !b) return;
    cudaEventRecord(b, st);
    ctx->prof_pending.push_back({cls, a, b});
}

static void prof_resolve(qxd_ctx* ctx) {
    for (auto& p : ctx->prof_pending) {
        float ms = 0.f;
        cudaEventSynchronize(p.b);
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) ctx->prof_cls[p.cls].ms += ms;
        else cudaGetLastError();
        ctx->prof_pool.push_back(p.a);
        ctx->prof_pool.push_back(p.b);
    }
    ctx->prof_pending.clear();
}

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// device view of a caller array: the array itself, or a staged copy of it
int stage_in(qxd_ctx* ctx, int slot, const void* p, size_t bytes, const void** dev, cudaStream_t st) {
    if (is_device_ptr(p)) {
        *dev = p;
        return QXD_OK;
    }
    void* d;
    QXD_TRY(qxd_ws(ctx, slot, bytes, &d));
    QXD_CUDA(ctx, cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, st));
    *dev = d;
    return QXD_OK;
}

int stage_out(qxd_ctx* ctx, int slot, void* p, size_t bytes, void** dev, bool* host) {
    *host = !is_device_ptr(p);
    if (!*host) {
        *dev = p;
        return QXD_OK;
    }
    return qxd_ws(ctx, slot, bytes, dev);
}

int finish_out(qxd_ctx* ctx, void* p, const void* dev, size_t bytes, bool host, cudaStream_t st) {
    if (host) {
        QXD_CUDA(ctx, cudaMemcpyAsync(p, dev, bytes, cudaMemcpyDeviceToHost, st));
        QXD_CUDA(ctx, cudaStreamSynchronize(st));
    }
    return QXD_OK;
}

int check_fl(qxd_ctx* ctx, int fl) {
    if (!ctx) return QXD_EARG;
    if (fl < 0 || fl >= QXD_MAX_FLAVOURS) return qxd_fail(ctx, QXD_EARG, "flavour id out of range 0..7");
    if (!ctx->links_set) return qxd_fail(ctx, QXD_ESTATE, "qxd_set_links has not been called");
    if (!ctx->fl[fl].set) return qxd_fail(ctx, QXD_ESTATE, "qxd_set_clover has not been called for this flavour");
    return QXD_OK;
}

bool make_geo(const qxd_geom* g, Geo* G) {
    for (int mu = 0; mu < 4; ++mu)
        if (g->L[mu] < 2 || (g->L[mu] & 1)) return false;
    if (g->cstar < 0 || g->cstar > 3) return false;
    if (g->cstar > 0 && (g->theta[1] != 0.0 || g->theta[2] != 0.0 || g->theta[3] != 0.0)) return false;
    if (g->tbc != QXD_TBC_PERIODIC && g->tbc != QXD_TBC_OPEN) return false;
    if (g->tbc == QXD_TBC_OPEN && (g->theta[0] != 0.0 || !std::isfinite(g->cF))) return false;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) V *= g->L[mu];
    if (g->cstar) V *= 2;
    if (V / 2 > 0x7fffffffLL / 36) return false;  // 32-bit half-lattice indexing
    G->N[0] = g->L[0];
    G->N[1] = g->cstar ? 2 * g->L[1] : g->L[1];
    G->N[2] = g->L[2];
    G->N[3] = g->L[3];
    G->L1 = g->L[1];
    G->cstar = g->cstar;
    G->V = V;
    G->Vh = (int)(V / 2);
    G->open0 = g->tbc == QXD_TBC_OPEN;
    return true;
}

static void free_flavour(QxdFlavour& F) {
    cudaFree(F.V64);
    cudaFree(F.Z32);
    for (int k = 0; k < 2; ++k) {
        cudaFree(F.C64[k]);
        cudaFree(F.C32[k]);
        cudaFree(F.Cdf[k]);
    }
    cudaFree(F.Vdf);
    cudaFree(F.W);
    cudaFree(F.dfl_basis);
    cudaFree(F.dfl_A);
    cudaFree(F.dfl_nbr);
    cudaFree(F.dfl_stat);
    F = QxdFlavour{};
}

extern "C" {

int qxd_create(const qxd_geom* g, int device, qxd_ctx** out) {
    if (!g || !out) return QXD_EARG;
    *out = nullptr;
    Geo G;
    if (!make_geo(g, &G)) return QXD_EARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return QXD_ECUDA;
    }
    qxd_ctx* ctx = new (std::nothrow) qxd_ctx();
    if (!ctx) return QXD_ENOMEM;
    ctx->geom = *g;
    ctx->device = device;
    ctx->g = G;
    cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, device);
    const size_t Vh = G.Vh;
    bool ok = cudaMalloc(&ctx->U64, 2 * 36 * Vh * sizeof(double2)) == cudaSuccess &&
              cudaMalloc(&ctx->A64, 2 * 4 * Vh * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&ctx->U32, 2 * 12 * Vh * sizeof(float4)) == cudaSuccess &&
              cudaMalloc(&ctx->red_partials, kPartials * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&ctx->red_result, kRedSlots * sizeof(double)) == cudaSuccess &&
              cudaMalloc(&ctx->dev_flag, sizeof(int)) == cudaSuccess &&
              cudaMalloc(&ctx->red_ticket, sizeof(unsigned)) == cudaSuccess &&
              cudaMemset(ctx->red_ticket, 0, sizeof(unsigned)) == cudaSuccess &&
              cudaMallocHost(&ctx->red_host, kRedSlots * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        qxd_destroy(ctx);
        return QXD_ENOMEM;
    }
    *out = ctx;
    return QXD_OK;
}

void qxd_destroy(qxd_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    cudaFree(ctx->U64);
    cudaFree(ctx->A64);
    cudaFree(ctx->U32);
    for (auto& F : ctx->fl) free_flavour(F);
    for (void* p : ctx->ws_ptr) cudaFree(p);
    prof_resolve(ctx);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    cudaFree(ctx->red_partials);
    cudaFree(ctx->red_result);
    cudaFree(ctx->dev_flag);
    cudaFree(ctx->red_ticket);
    cudaFreeHost(ctx->red_host);
    delete ctx;
}

int qxd_set_links(qxd_ctx* ctx, const double* U, const double* A, double invqel, void* stream) {
    if (!ctx) return QXD_EARG;
    if (!U || !A) return qxd_fail(ctx, QXD_EARG, "set_links: NULL field");
    (void)invqel;
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t Vp = (size_t)ctx->geom.L[0] * ctx->geom.L[1] * ctx->geom.L[2] * ctx->geom.L[3];
    const void *dU, *dA;
    QXD_TRY(stage_in(ctx, WS_STAGE_U, U, Vp * 4 * 9 * 16, &dU, st));
    QXD_TRY(stage_in(ctx, WS_STAGE_A, A, Vp * 4 * 8, &dA, st));
    for (auto& F : ctx->fl) free_flavour(F);
    QXD_TRY(launch_set_links(ctx, static_cast<const double2*>(dU), static_cast<const double*>(dA), st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    ctx->links_set = true;
    return QXD_OK;
}

int qxd_set_clover(qxd_ctx* ctx, int fl, const qxd_flavour* f, void* stream) {
    if (!ctx) return QXD_EARG;
    if (fl < 0 || fl >= QXD_MAX_FLAVOURS) return qxd_fail(ctx, QXD_EARG, "flavour id out of range 0..7");
    if (!f || !(f->kappa > 0.0)) return qxd_fail(ctx, QXD_EARG, "set_clover: kappa must be positive");
    if (!ctx->links_set) return qxd_fail(ctx, QXD_ESTATE, "qxd_set_links has not been called");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    QxdFlavour& F = ctx->fl[fl];
    const size_t Vh = ctx->g.Vh;
    if (!F.V64) {
        bool ok = cudaMalloc(&F.V64, 2 * 36 * Vh * sizeof(double2)) == cudaSuccess &&
                  cudaMalloc(&F.Z32, 2 * 2 * Vh * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&F.C64[0], 2 * 36 * Vh * sizeof(double2)) == cudaSuccess &&
                  cudaMalloc(&F.C64[1], 2 * 36 * Vh * sizeof(double2)) == cudaSuccess &&
                  cudaMalloc(&F.C32[0], 2 * 18 * Vh * sizeof(float4)) == cudaSuccess &&
                  cudaMalloc(&F.C32[1], 2 * 18 * Vh * sizeof(float4)) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            free_flavour(F);
            return qxd_fail(ctx, QXD_ENOMEM, "set_clover: allocation failed");
        }
    }
    F.f = *f;
    F.set = false;
    // double-float copies and a deflation subspace belong to the operator they were built for
    cudaFree(F.Vdf);
    cudaFree(F.Cdf[0]);
    cudaFree(F.Cdf[1]);
    F.Vdf = nullptr;
    F.Cdf[0] = F.Cdf[1] = nullptr;
    dfl_free(F);
    QXD_TRY(launch_set_flavour(ctx, fl, st));
    F.set = true;
    return QXD_OK;
}

int qxd_apply_Dw(qxd_ctx* ctx, int fl, int prec, const void* in, void* out, int nrhs, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (prec < 0 || prec > 3) return qxd_fail(ctx, QXD_EARG, "apply_Dw: precision must be 0, 1, 2 or 3");
    if (nrhs < 1 || !in || !out) return qxd_fail(ctx, QXD_EARG, "apply_Dw: bad arguments");
    if (prec == QXD_DF64 && nrhs != 1) return qxd_fail(ctx, QXD_EARG, "apply_Dw: QXD_DF64 takes one right-hand side");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int cprec = (prec == QXD_FP64 || prec == QXD_DF64) ? 0 : 1;
    const size_t cbytes = (size_t)nrhs * ctx->g.V * 12 * (cprec == 0 ? 16 : 8);
    const void* din;
    void* dout;
    bool host_out;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, in, cbytes, &din, st));
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, out, cbytes, &dout, &host_out));
    const size_t hb = half_bytes(ctx, prec) * nrhs;
    void *ie, *io, *oe, *oo;
    QXD_TRY(qxd_ws(ctx, WS_T0, hb, &ie));
    QXD_TRY(qxd_ws(ctx, WS_T1, hb, &io));
    QXD_TRY(qxd_ws(ctx, WS_T2, hb, &oe));
    QXD_TRY(qxd_ws(ctx, WS_T3, hb, &oo));
    // double-float: FP64 layout converted in place (the two layouts share their 16-byte chunks)
    const int iprec = prec == QXD_DF64 ? QXD_FP64 : prec;
    QXD_TRY(launch_pack(ctx, cprec, din, 1, 0, iprec, ie, nrhs, st));
    QXD_TRY(launch_pack(ctx, cprec, din, 1, 1, iprec, io, nrhs, st));
    if (prec == QXD_DF64) {
        QXD_TRY(blas_split_df64(ctx, ie, ie, 12ull * ctx->g.Vh, st));
        QXD_TRY(blas_split_df64(ctx, io, io, 12ull * ctx->g.Vh, st));
    }
    QXD_TRY(op_Dw(ctx, fl, prec, Full{ie, io}, Full{oe, oo}, st, nrhs));
    if (prec == QXD_DF64) {
        QXD_TRY(blas_join_df64(ctx, oe, oe, 12ull * ctx->g.Vh, st));
        QXD_TRY(blas_join_df64(ctx, oo, oo, 12ull * ctx->g.Vh, st));
    }
    QXD_TRY(launch_unpack(ctx, iprec, oe, 0, cprec, dout, 1, nrhs, st));
    QXD_TRY(launch_unpack(ctx, iprec, oo, 1, cprec, dout, 1, nrhs, st));
    return finish_out(ctx, out, dout, cbytes, host_out, st);
}

int qxd_apply_Dhat_eo(qxd_ctx* ctx, int fl, int prec, int dagger, const void* in_e, void* out_e, int nrhs,
                      void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (prec < 0 || prec > 2) return qxd_fail(ctx, QXD_EARG, "apply_Dhat_eo: precision must be 0, 1 or 2");
    if (nrhs < 1 || !in_e || !out_e) return qxd_fail(ctx, QXD_EARG, "apply_Dhat_eo: bad arguments");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int cprec = prec == QXD_FP64 ? 0 : 1;
    const size_t cbytes = (size_t)nrhs * ctx->g.Vh * 12 * (cprec == 0 ? 16 : 8);
    const void* din;
    void* dout;
    bool host_out;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, in_e, cbytes, &din, st));
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, out_e, cbytes, &dout, &host_out));
    const size_t hb = half_bytes(ctx, prec) * nrhs;
    void *ie, *to, *oe;
    QXD_TRY(qxd_ws(ctx, WS_T0, hb, &ie));
    QXD_TRY(qxd_ws(ctx, WS_T1, hb, &to));
    QXD_TRY(qxd_ws(ctx, WS_T2, hb, &oe));
    QXD_TRY(launch_pack(ctx, cprec, din, 0, 0, prec, ie, nrhs, st));
    QXD_TRY(op_Dhat(ctx, fl, prec, dagger ? 1 : 0, ie, oe, to, st, nrhs));
    QXD_TRY(launch_unpack(ctx, prec, oe, 0, cprec, dout, 0, nrhs, st));
    return finish_out(ctx, out_e, dout, cbytes, host_out, st);
}

int qxd_solve(qxd_ctx* ctx, int fl, const qxd_solver* s, const void* eta, void* psi, int nrhs, qxd_info* info,
              void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!s || !eta || !psi || nrhs < 1) return qxd_fail(ctx, QXD_EARG, "solve: bad arguments");
    if (!(s->tol > 0.0) || s->nmx < 1) return qxd_fail(ctx, QXD_EARG, "solve: tol and nmx must be positive");
    if (s->kind != QXD_CGNE && s->kind != QXD_FGCR) return qxd_fail(ctx, QXD_EARG, "solve: kind must be CGNE or FGCR");
    if (s->kind == QXD_FGCR && (s->inner < 0 || s->inner > 2))
        return qxd_fail(ctx, QXD_EARG, "solve: inner precision must be 0, 1 or 2");
    if (s->precond == QXD_PRECOND_LEARNED && !ctx->fl[fl].W)
        return qxd_fail(ctx, QXD_ESTATE, "solve: learned preconditioner weights not set");
    if (s->precond < 0 || s->precond > QXD_PRECOND_DFL) return qxd_fail(ctx, QXD_EARG, "solve: unknown preconditioner");
    if (s->precond == QXD_PRECOND_SAP) QXD_TRY(sap_check(ctx));
    if (s->precond == QXD_PRECOND_DFL && !ctx->fl[fl].dfl_basis)
        return qxd_fail(ctx, QXD_ESTATE, "solve: deflation subspace not set up (qxd_dfl_setup)");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cbytes = (size_t)nrhs * ctx->g.V * 12 * 16;
    const void* din;
    void* dout;
    bool host_out;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, eta, cbytes, &din, st));
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, psi, cbytes, &dout, &host_out));
    const size_t hb = half_bytes(ctx, QXD_FP64);
    void *ee, *eo, *xe, *xo;
    QXD_TRY(qxd_ws(ctx, WS_T4, hb, &ee));
    QXD_TRY(qxd_ws(ctx, WS_T5, hb, &eo));
    QXD_TRY(qxd_ws(ctx, WS_T6, hb, &xe));
    QXD_TRY(qxd_ws(ctx, WS_T7, hb, &xo));
    qxd_info local{};
    int worst = QXD_OK;
    if (s->kind == QXD_FGCR && nrhs > 1) {
        // all right-hand sides in lockstep: one multi-RHS operator launch per iteration
        void *bee, *beo, *bxe, *bxo;
        QXD_TRY(qxd_ws(ctx, WS_T4, hb * nrhs, &bee));
        QXD_TRY(qxd_ws(ctx, WS_T5, hb * nrhs, &beo));
        QXD_TRY(qxd_ws(ctx, WS_T6, hb * nrhs, &bxe));
        QXD_TRY(qxd_ws(ctx, WS_T7, hb * nrhs, &bxo));
        QXD_TRY(launch_pack(ctx, 0, din, 1, 0, QXD_FP64, bee, nrhs, st));
        QXD_TRY(launch_pack(ctx, 0, din, 1, 1, QXD_FP64, beo, nrhs, st));
        int rc = solve_fgcr_dc_batched(ctx, fl, s, Full{bee, beo}, Full{bxe, bxo}, nrhs, &local, st);
        local.status = rc;
        if (info) *info = local;
        if (rc != QXD_OK && rc != QXD_ENOCONV) return rc;
        QXD_TRY(launch_unpack(ctx, QXD_FP64, bxe, 0, 0, dout, 1, nrhs, st));
        QXD_TRY(launch_unpack(ctx, QXD_FP64, bxo, 1, 0, dout, 1, nrhs, st));
        QXD_TRY(finish_out(ctx, psi, dout, cbytes, host_out, st));
        QXD_CUDA(ctx, cudaStreamSynchronize(st));
        if (s->precond == QXD_PRECOND_DFL) QXD_TRY(dfl_status(ctx, fl, nullptr, nullptr, st));
        return rc;
    }
    for (int r = 0; r < nrhs; ++r) {
        const char* src = static_cast<const char*>(din) + (size_t)r * ctx->g.V * 12 * 16;
        char* dst = static_cast<char*>(dout) + (size_t)r * ctx->g.V * 12 * 16;
        QXD_TRY(launch_pack(ctx, 0, src, 1, 0, QXD_FP64, ee, 1, st));
        QXD_TRY(launch_pack(ctx, 0, src, 1, 1, QXD_FP64, eo, 1, st));
        local = qxd_info{};
        int rc = (s->kind == QXD_CGNE) ? solve_cgne64(ctx, fl, s, Full{ee, eo}, Full{xe, xo}, &local, st)
                                       : solve_fgcr_dc(ctx, fl, s, Full{ee, eo}, Full{xe, xo}, &local, st);
        local.status = rc;
        if (rc != QXD_OK && rc != QXD_ENOCONV) {
            if (info) *info = local;
            return rc;
        }
        if (rc != QXD_OK) worst = rc;
        QXD_TRY(launch_unpack(ctx, QXD_FP64, xe, 0, 0, dst, 1, 1, st));
        QXD_TRY(launch_unpack(ctx, QXD_FP64, xo, 1, 0, dst, 1, 1, st));
    }
    if (info) {
        *info = local;
        info->status = worst;
    }
    QXD_TRY(finish_out(ctx, psi, dout, cbytes, host_out, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    if (s->precond == QXD_PRECOND_DFL) QXD_TRY(dfl_status(ctx, fl, nullptr, nullptr, st));
    return worst;
}

int qxd_solve_multishift(qxd_ctx* ctx, int fl, int nshift, const double* sigma, const qxd_solver* s,
                         const void* phi_e, void* x_e, qxd_info* info, void* stream) {
    QXD_TRY(check_fl(ctx, fl));
    if (!s || !sigma || !phi_e || !x_e) return qxd_fail(ctx, QXD_EARG, "solve_multishift: NULL argument");
    if (nshift < 1 || nshift > kMaxShifts) return qxd_fail(ctx, QXD_EARG, "solve_multishift: nshift must be 1..32");
    for (int j = 0; j < nshift; ++j)
        if (!(sigma[j] >= 0.0) || !std::isfinite(sigma[j]))
            return qxd_fail(ctx, QXD_EARG, "solve_multishift: shifts must be finite and >= 0");
    if (!(s->tol > 0.0) || s->nmx < 1) return qxd_fail(ctx, QXD_EARG, "solve_multishift: tol and nmx must be positive");
    if (s->inner != QXD_FP64 && s->inner != QXD_FP32)
        return qxd_fail(ctx, QXD_EARG, "solve_multishift: inner precision must be FP64 or FP32");
    cudaSetDevice(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cb = (size_t)ctx->g.Vh * 12 * 16;
    const void* din;
    void* dout;
    bool host_out;
    QXD_TRY(stage_in(ctx, WS_STAGE_IN, phi_e, cb, &din, st));
    QXD_TRY(stage_out(ctx, WS_STAGE_OUT, x_e, cb * nshift, &dout, &host_out));
    const size_t hb = half_bytes(ctx, QXD_FP64);
    void *b64, *X64;
    QXD_TRY(qxd_ws(ctx, WS_T8, hb, &b64));
    QXD_TRY(qxd_ws(ctx, WS_T9, hb * nshift, &X64));
    QXD_TRY(launch_pack(ctx, 0, din, 0, 0, QXD_FP64, b64, 1, st));
    qxd_info local{};
    int rc = solve_mscg(ctx, fl, nshift, sigma, s, b64, static_cast<char*>(X64), &local, st);
    local.status = rc;
    if (info) *info = local;
    if (rc != QXD_OK && rc != QXD_ENOCONV) return rc;
    QXD_TRY(launch_unpack(ctx, QXD_FP64, X64, 0, 0, dout, 0, nshift, st));
    QXD_TRY(finish_out(ctx, x_e, dout, cb * nshift, host_out, st));
    QXD_CUDA(ctx, cudaStreamSynchronize(st));
    return rc;
}

int qxd_profile(qxd_ctx* ctx, int mode) {
    if (!ctx) return QXD_EARG;
    if (mode < 0 || mode > 2) return qxd_fail(ctx, QXD_EARG, "profile: mode must be 0, 1 or 2");
    cudaSetDevice(ctx->device);
    prof_resolve(ctx);
    ctx->prof_cls.clear();
    ctx->prof_idx.clear();
    ctx->prof_mode = mode;
    return QXD_OK;
}

int qxd_profile_entry(qxd_ctx* ctx, int i, char* name, int len, long long* launches, double* ms, double* bytes) {
    if (!ctx) return QXD_EARG;
    cudaSetDevice(ctx->device);
    prof_resolve(ctx);
    if (i < 0 || i >= (int)ctx->prof_cls.size()) return QXD_EARG;
    const auto& c = ctx->prof_cls[i];
    if (name && len > 0) {
        std::strncpy(name, c.name.c_str(), (size_t)len - 1);
        name[len - 1] = 0;
    }
    if (launches) *launches = c.launches;
    if (ms) *ms = c.ms;
    if (bytes) *bytes = c.bytes;
    return QXD_OK;
}

const char* qxd_last_error(qxd_ctx* ctx) {
    if (!ctx) return "NULL context";
    return ctx->err.c_str();
}

long long qxd_volume(const qxd_ctx* ctx) { return ctx ? ctx->g.V : 0; }

}  // extern "C"
