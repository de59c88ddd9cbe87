// Vector-kernel interface used by the solvers (blas.cu).  Fields are flat
// arrays of n complex numbers in precision 0 (FP64), 1 (FP32) or 2 (BF16).
// Reductions write their FP64 results to ctx->red_result[slot ...]; blas_fetch
// copies the first nslots results to ctx->red_host and synchronises the stream.
#pragma once

#include "qxd_internal.h"

namespace qxd {

constexpr int kMultiMax = 8;
constexpr int kRedSlots = 512;
constexpr int kMaxRedBlocks = 1024;
constexpr int kPartials = 2 * kMultiMax * kMaxRedBlocks;

struct MultiPtr {
    const void* p[kMultiMax];
};
struct MultiCoef {
    double re[kMultiMax];
    double im[kMultiMax];
};

// Same-precision operations treat a field as a flat array (any n); operations
// between two precisions work site by site on whole half-lattice fields
// (n a multiple of 12 V/2), because the flat complex order of the internal
// layout depends on the precision.
// result[slot], result[slot+1] = Re, Im <a, b> = sum conj(a) b (pa == pb)
int blas_dot(qxd_ctx* ctx, int pa, int pb, size_t n, const void* a, const void* b, int slot, cudaStream_t st);
// result[slot] = |a|^2 over finite entries, result[slot+1] = number of non-finite entries
int blas_norm2(qxd_ctx* ctx, int p, size_t n, const void* a, int slot, cudaStream_t st);
// Double-float conversions over n complex numbers (16-byte chunks): FP64 -> double-float
// and double-float -> FP64 (in == out allowed for both)
int blas_split_df64(qxd_ctx* ctx, const void* in, void* out, size_t n, cudaStream_t st);

int blas_join_df64(qxd_ctx* ctx, const void* in, void* out, size_t n, cudaStream_t st);
// The mixed solver's outer loop on half-lattice fields (FP32 pipe only): with eta FP64
// and dx double-float, r32 = FP32(eta - dx) with result[slot] = |r|^2, result[slot+1] =
// non-finite sites; x += e32; r32 = FP32(x) for a double-float x; r32 = FP32(x) for an
// FP64 x with result[slot] = |x|^2 (about 2^-23 relative), result[slot+1] = non-finite sites
int blas_df_residual(qxd_ctx* ctx, const void* eta, const void* dx, void* r32, int slot, cudaStream_t st);
int blas_f64_to_f32_norm(qxd_ctx* ctx, const void* x, void* r32, int slot, cudaStream_t st);
int blas_df_add_f32(qxd_ctx* ctx, const void* e32, void* x, cudaStream_t st);
int blas_df_to_f32(qxd_ctx* ctx, const void* x, void* r32, cudaStream_t st);
// r32 = FP32(b - y - sigma x), b, y, x double-float; result[slot] = |r|^2, [slot+1] = non-finite sites
int blas_df_shift_residual(qxd_ctx* ctx, const void* b, const void* y, const void* x, double sigma, void* r32,
                           int slot, cudaStream_t st);
// result[slot] = sum of the finite entries of the real FP64 array a[n], result[slot+1] = count of the others
int blas_sum_real(qxd_ctx* ctx, const double* a, size_t n, int slot, cudaStream_t st);
// result[slot + 2j], [slot + 2j + 1] = <W_j, v>, j < k
int blas_multi_dot(qxd_ctx* ctx, int p, size_t n, int k, const void* const* W, const void* v, int slot,
                   cudaStream_t st);
// y = a x + b y
int blas_axpby(qxd_ctx* ctx, int px, int py, size_t n, double ar, double ai, const void* x, double br, double bi,
               void* y, cudaStream_t st);
// z = x + a w (same precision, out of place)
// GCR step in one pass: w += sum_{j<k} (cre_j + i cim_j) X_j, then z = x + (ar + i ai) w
// (same precision P, k <= 8; z may not alias w or the X_j)
int blas_gcr_update(qxd_ctx* ctx, int p, size_t n, int k, const double* cre, const double* cim,
                    const void* const* X, void* w, double ar, double ai, const void* x, void* z, cudaStream_t st);
int blas_axpy3(qxd_ctx* ctx, int p, size_t n, double ar, double ai, const void* w, const void* x, void* z,
               cudaStream_t st);
// y += sum_j c_j X_j  (px == py)
int blas_multi_axpy(qxd_ctx* ctx, int px, int py, size_t n, int k, const double* cre, const double* cim,
                    const void* const* X, void* y, cudaStream_t st);
// y += sum_j c_j X_j, then result[slot] = |y|^2, result[slot+1] = non-finite count
int blas_multi_axpy_norm(qxd_ctx* ctx, int p, size_t n, int k, const double* cre, const double* cim,
                         const void* const* X, void* y, int slot, cudaStream_t st);
int blas_fetch(qxd_ctx* ctx, int nslots, cudaStream_t st);

// Variants whose scalars live in device memory (no host round trip; usable
// inside captured CUDA graphs):
// y = c[0] x + c[1] y  (real coefficients read from the device array c)
int blas_axpby_dev(qxd_ctx* ctx, int P, size_t n, const double* c, const void* x, void* y, cudaStream_t st);
// y += c[0] x, then result[slot] = |y|^2
int blas_axpy_norm_dev(qxd_ctx* ctx, int P, size_t n, const double* c, const void* x, void* y, int slot,
                       cudaStream_t st);

}  // namespace qxd

namespace qxd {

constexpr int kMaxShifts = 32;

// Fused multi-shift CG update over the active shifts j < ns (one pass over r):
//   x_j += alpha_j p_j;   p_j = zeta_j r + beta_j p_j
struct ShiftPtrs {
    void* x[kMaxShifts];
    void* p[kMaxShifts];
};
struct ShiftCoef {
    double alpha[kMaxShifts];
    double zeta[kMaxShifts];
    double beta[kMaxShifts];
};
int blas_msg_update(qxd_ctx* ctx, int P, size_t n, int ns, const ShiftPtrs& ptr, const ShiftCoef& c, const void* r,
                    cudaStream_t st);

// Same update with coefficients in device memory: for j < ns with upd[j] != 0,
// x_j += alpha[j] p_j; p_j = zeta[j] r + beta[j] p_j
struct ShiftCoefDev {
    const double* alpha;
    const double* zeta;
    const double* beta;
    const int* upd;
};
int blas_msg_update_dev(qxd_ctx* ctx, int P, size_t n, int ns, const ShiftPtrs& ptr, const ShiftCoefDev& c,
                        const void* r, cudaStream_t st);

}  // namespace qxd
