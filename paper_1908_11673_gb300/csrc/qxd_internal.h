// Host-side context of libqxd and helpers shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/qxd.h"
#include "qxd_common.cuh"

#define QXD_MAX_FLAVOURS 8

struct QxdFlavour {
    bool set = false;
    qxd_flavour f{};
    double2* V64 = nullptr;    // [p][36][Vh]   V = U z^qhat (boundary phase folded in)
    float4* Z32 = nullptr;     // [p][2][Vh]    z^qhat (boundary phase folded in)
    double2* C64[2] = {nullptr, nullptr};  // [p][36][Vh]  diag term, inverse
    float4* C32[2] = {nullptr, nullptr};   // [p][18][Vh]
    float4* Vdf = nullptr;                 // [p][36][Vh]  V64 as double-float pairs (on first use)
    float4* Cdf[2] = {nullptr, nullptr};   // [p][36][Vh]  C64[0] as double-float pairs (on first use; [1] unused)
    // learned preconditioner
    void* W = nullptr;         // device weights (complex float [layers][cout][cin][9][4][4])
    int nlayers = 0, nch = 0;
    int wprec = QXD_BF16;      // precision of the network's channel mixing inside FGCR
    // deflation subspace (qxd_dfl_setup)
    float4* dfl_basis = nullptr;  // [Ns] full FP32 fields, block-orthonormal
    float2* dfl_A = nullptr;      // little operator [Nb][9][Ns][Ns]
    int* dfl_nbr = nullptr;       // block neighbours [Nb][9]
    void* dfl_stat = nullptr;     // status of the little-system solves (steps, residual, barrier error)
    int dfl_Ns = 0, dfl_cnmx = 0, dfl_cnkv = 0;
    double dfl_ctol = 0.0;
};

struct qxd_ctx {
    qxd_geom geom{};
    qxd::Geo g{};
    int device = 0;
    std::string err;
    bool links_set = false;
    double2* U64 = nullptr;    // [p][36][Vh] SU(3) links, all simulated sites
    double* A64 = nullptr;     // [p][4][Vh]  photon field (mirror: -A)
    float4* U32 = nullptr;     // [p][12][Vh] two rows of U per direction
    QxdFlavour fl[QXD_MAX_FLAVOURS];
    // workspace: named device buffers, grown on demand, freed in qxd_destroy
    std::vector<void*> ws_ptr;
    std::vector<size_t> ws_size;
    double* red_partials = nullptr;  // reduction scratch (per-block partial sums)
    double* red_result = nullptr;    // reduction results (device)
    unsigned* red_ticket = nullptr;  // last-block ticket of the reductions (0 between launches)
    double* red_host = nullptr;      // pinned host mirror of the results
    int* dev_flag = nullptr;         // device error flag (singular block, non-finite)
    int nsm = 0;
    // kernel profiling (qxd_profile): 0 off, 1 count launches, 2 count and time
    int prof_mode = 0;
    struct ProfClass {
        std::string name;
        long long launches = 0;
        double bytes = 0.0;
        double ms = 0.0;
    };
    struct ProfPending {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<ProfClass> prof_cls;
    std::map<std::string, int> prof_idx;
    std::vector<ProfPending> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    // autotuned (rhs per thread, threads per block) of the multi-RHS hopping kernel,
    // keyed by (precision, self mode, post mode, nrhs, V/2)
    std::map<std::tuple<int, int, int, int, long long>, std::pair<int, int>> tune_hop;
    cudaStream_t cap_stream = nullptr;  // library stream for CUDA-graph capture
    int sap_ncy = 5, sap_nmr = 5;       // SAP preconditioner parameters (qxd_set_sap)
};

// Brackets one kernel launch when profiling is on: counts it under `name` with
// its algorithmic DRAM bytes and, in timing mode, records CUDA events around it
// on the launching stream.
struct ProfScope {
    qxd_ctx* ctx;
    int cls = -1;
    cudaEvent_t b = nullptr;
    cudaEvent_t a = nullptr;
    cudaStream_t st;
    ProfScope(qxd_ctx* c, const char* name, double bytes, cudaStream_t s, int nlaunch = 1);
    ~ProfScope();
};

// error helpers ------------------------------------------------------------------
int qxd_fail(qxd_ctx* ctx, int code, const std::string& msg);

#define QXD_CUDA(ctx, expr)                                                              \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess)                                                           \
            return qxd_fail(ctx, QXD_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

#define QXD_TRY(expr)              \
    do {                           \
        int _s = (expr);           \
        if (_s != QXD_OK) return _s; \
    } while (0)

// workspace slot `slot` with at least `bytes` bytes (device memory)
int qxd_ws(qxd_ctx* ctx, int slot, size_t bytes, void** out);

// caller arrays at the C ABI (api.cu): a device view of an input (the array
// itself when it is device memory, else a copy staged in workspace `slot`); a
// device destination for an output and whether it must be copied back to the
// host afterwards (finish_out, which then synchronises); flavour-state checks
int stage_in(qxd_ctx* ctx, int slot, const void* p, size_t bytes, const void** dev, cudaStream_t st);
int stage_out(qxd_ctx* ctx, int slot, void* p, size_t bytes, void** dev, bool* host);
int finish_out(qxd_ctx* ctx, void* p, const void* dev, size_t bytes, bool host, cudaStream_t st);
int check_fl(qxd_ctx* ctx, int fl);
// simulated-lattice geometry of a qxd_geom; false if the geometry is invalid
bool make_geo(const qxd_geom* g, qxd::Geo* G);

// workspace slots
enum {
    WS_STAGE_IN = 0, WS_STAGE_OUT, WS_STAGE_U, WS_STAGE_A,
    WS_T0, WS_T1, WS_T2, WS_T3, WS_T4, WS_T5, WS_T6, WS_T7, WS_T8, WS_T9,
    WS_SOLVER = 32,   // solver vectors start here (up to 128 slots)
    WS_PTC = 192,
    WS_SAP = 272,
    WS_RAT = 288,
    WS_DFL = 300,
    WS_NSLOTS = 320
};

// kernels launched from other translation units ------------------------------------
namespace qxd {

constexpr int kThreads = 128;
inline int nblocks(long long n, int threads = kThreads) { return (int)((n + threads - 1) / threads); }

// fields.cu
int launch_set_links(qxd_ctx* ctx, const double2* U, const double* A, cudaStream_t st);
int launch_set_flavour(qxd_ctx* ctx, int fl, cudaStream_t st);

// hop kernels (dirac.cu).  A half-lattice hop producing parity `pout`:
//   out = POST( SELF + c_hop * H_{pout, 1-pout} in_nb )
// SELF: 0 none, 1 diag-term * in_self, 2 in_self; POST: 0 none, 1 diag-term inverse.
// g5 flags multiply the neighbour input, the self input or the output by gamma5.
struct HopArgs {
    int pout;
    const void* in_nb;
    const void* in_self;
    void* out;
    int self_mode;
    int post_mode;
    double c_hop;
    int g5_nb, g5_self, g5_out;
    int nrhs;        // right-hand sides stored one after the other (stride = chunks*Vh)
};
int launch_hop(qxd_ctx* ctx, int fl, int prec, const HopArgs& a, cudaStream_t st);
// out = (diag term or its inverse) * in on parity p (inv = 0 or 1), optional gamma5
int launch_diag(qxd_ctx* ctx, int fl, int prec, int p, int inv, const void* in, void* out, int nrhs,
                cudaStream_t st);

// layout.cu: canonical [site][4][3] complex <-> internal half-lattice fields
// canonical full-lattice (cfull=1, V sites) or half-lattice (cfull=0, Vh sites of parity p)
int launch_pack(qxd_ctx* ctx, int prec_in_canon, const void* canon, int cfull, int p, int prec_int,
                void* internal, int nrhs, cudaStream_t st);
int launch_unpack(qxd_ctx* ctx, int prec_int, const void* internal, int p, int prec_out_canon, void* canon,
                  int cfull, int nrhs, cudaStream_t st);

}  // namespace qxd
