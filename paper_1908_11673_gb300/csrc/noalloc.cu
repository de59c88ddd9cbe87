// qxd_apply_Dhat_eo_noalloc: the even-odd operator for callers that must not
// allocate device memory during the call.  Its three half-lattice temporaries
// (packed input, odd intermediate, packed output) live in one file-scope device
// array instead of the context's workspace, which qxd_apply_Dhat_eo grows with
// cudaMalloc on first use.
#include <mutex>

#include "hop.cuh"
#include "ops.h"
#include "qxd_internal.h"

using namespace qxd;

namespace {

// Largest half-lattice this entry point accepts, and the scratch it needs:
// three half-lattice fields in the widest (FP64) internal layout.
constexpr long long kNoallocMaxVh = 32768;
constexpr size_t kNoallocFieldBytes = 192ull * kNoallocMaxVh;  // one FP64 half-lattice field
constexpr size_t kNoallocBytes = 3 * kNoallocFieldBytes;       // 18 MiB

// Held by every GPU that loads this library, until the process exits.
static __device__ __align__(256) unsigned char g_dhat_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (which must be current).
// Looked up once per device; the first call therefore talks to the driver.
int scratch_address(qxd_ctx* ctx, int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return qxd_fail(ctx, QXD_EARG, "noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dhat_scratch);
        if (e != cudaSuccess || !p)
            return qxd_fail(ctx, QXD_ECUDA, std::string("noalloc: cudaGetSymbolAddress failed: ") +
                                                cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[device]);
    return QXD_OK;
}

// true for device (or managed) memory of `device` itself; memory of another GPU
// is refused, since the kernels would then read and write it over the peer link
bool on_device(const void* p, int device) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == device;
}

// Turns the hop autotuner off on this thread for the lifetime of the object: a
// first call for a new (precision, lattice) key would otherwise time candidate
// launch shapes, which creates events and waits for them on the host.
struct NoAutotune {
    bool saved;
    NoAutotune() : saved(t_no_autotune) { t_no_autotune = true; }
    ~NoAutotune() { t_no_autotune = saved; }
};

}  // namespace

extern "C" int qxd_apply_Dhat_eo_noalloc(qxd_ctx* ctx, int fl, int prec, int dagger, const void* in_e, void* out_e,
                                         void* stream) {
    if (!ctx) return QXD_EARG;
    if (fl < 0 || fl >= QXD_MAX_FLAVOURS) return qxd_fail(ctx, QXD_EARG, "flavour id out of range 0..7");
    if (!ctx->links_set || !ctx->fl[fl].set)
        return qxd_fail(ctx, QXD_ESTATE, "apply_Dhat_eo_noalloc: links and SW term must be set first");
    if (prec < 0 || prec > 2) return qxd_fail(ctx, QXD_EARG, "apply_Dhat_eo_noalloc: precision must be 0, 1 or 2");
    if (ctx->g.Vh > kNoallocMaxVh)
        return qxd_fail(ctx, QXD_EARG, "apply_Dhat_eo_noalloc: lattice has " + std::to_string(ctx->g.Vh) +
                                           " even sites; this entry point handles at most 32768");
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        cudaGetLastError();
        return qxd_fail(ctx, QXD_ECUDA, "apply_Dhat_eo_noalloc: cannot select the context's device");
    }
    if (!in_e || !out_e || !on_device(in_e, ctx->device) || !on_device(out_e, ctx->device))
        return qxd_fail(ctx, QXD_EARG,
                        "apply_Dhat_eo_noalloc: in_e and out_e must be device arrays of the context's GPU");
    unsigned char* scratch;
    QXD_TRY(scratch_address(ctx, ctx->device, &scratch));
    // three consecutive half-lattice fields; every kernel below overwrites its
    // whole output, so nothing has to be cleared between calls
    void* ie = scratch;
    void* to = scratch + kNoallocFieldBytes;
    void* oe = scratch + 2 * kNoallocFieldBytes;
    cudaStream_t st = (cudaStream_t)stream;
    const int cprec = prec == QXD_FP64 ? 0 : 1;
    NoAutotune frozen;
    QXD_TRY(launch_pack(ctx, cprec, in_e, 0, 0, prec, ie, 1, st));
    QXD_TRY(op_Dhat(ctx, fl, prec, dagger ? 1 : 0, ie, oe, to, st, 1));
    QXD_TRY(launch_unpack(ctx, prec, oe, 0, cprec, out_e, 0, 1, st));
    return QXD_OK;
}
