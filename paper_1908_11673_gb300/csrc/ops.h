// Operator compositions built from the hopping and site-diagonal kernels.
#pragma once

#include "qxd_internal.h"

namespace qxd {

// a full-lattice field as its even and odd halves (internal layout)
struct Full {
    void* e;
    void* o;
};

// bytes of one half-lattice field in precision P (0 FP64, 1 FP32, 2 BF16)
size_t half_bytes(const qxd_ctx* ctx, int P);

// double-float copies of the flavour's FP64 links and site-diagonal term, and with
// inverse = true of the inverse term too (fields.cu), built on first use
int ensure_df64(qxd_ctx* ctx, int fl, cudaStream_t st, bool inverse = false);
// out = D in (eq. dirac):  out_e = A_ee in_e + H_eo in_o,  out_o = A_oo in_o + H_oe in_e
int op_Dw(qxd_ctx* ctx, int fl, int P, const Full& in, const Full& out, cudaStream_t st, int nrhs = 1);
// out_e = Dhat in_e = A_ee in_e - H_eo A_oo^-1 H_oe in_e (dagger: gamma5 Dhat gamma5); tmp_o: odd scratch
int op_Dhat(qxd_ctx* ctx, int fl, int P, int dagger, const void* in_e, void* out_e, void* tmp_o, cudaStream_t st,
            int nrhs = 1);
// Dhat on FP32 even fields (no dagger, one right-hand side) with the inner products of
// a GCR step fused into the second half: result[slot + 2j, +1] = <W_j, out_e> (j < k <= 8),
// [slot + 2k, +1] = <in_e, out_e>, [slot + 2k + 2] = |out_e|^2 over finite sites,
// [slot + 2k + 3] = number of sites where it is not finite
int op_Dhat_dots(qxd_ctx* ctx, int fl, const void* in_e, void* out_e, void* tmp_o, int k, const void* const* W,
                 int slot, cudaStream_t st);
int launch_hop_dots(qxd_ctx* ctx, int fl, const HopArgs& a, int k, const void* const* W, int slot, cudaStream_t st);
// b_e = r_e - H_eo A_oo^-1 r_o  (even-odd preconditioned source)
int op_eo_source(qxd_ctx* ctx, int fl, int P, const Full& r, void* b_e, void* tmp_o, cudaStream_t st, int nrhs = 1);
// x_o = A_oo^-1 (r_o - H_oe x_e)
int op_odd_reconstruct(qxd_ctx* ctx, int fl, int P, const void* r_o, const void* x_e, void* x_o, cudaStream_t st,
                       int nrhs = 1);
// z = M r (identity or the learned preconditioner)
int apply_precond(qxd_ctx* ctx, int fl, int P, int kind, const void* r, void* z, cudaStream_t st);

// learned preconditioner (ptc.cu): z_e = (M r_e)_e on FP32 internal even fields, the
// channel mixing in FP32 (prec QXD_FP32) or on the tensor cores in bfloat16 (QXD_BF16)
int ptc_apply_internal(qxd_ctx* ctx, int fl, const float2* W, int nlayers, int nch, const void* r_e, void* z_e,
                       cudaStream_t st, int prec = QXD_FP32);

// SAP preconditioner (sap.cu): z_e = (M_SAP (r_e, 0))_e on FP32 internal even fields
int sap_apply_even(qxd_ctx* ctx, int fl, const void* r_e, void* z_e, cudaStream_t st);
// psi = M_SAP eta on full FP32 fields (even half, odd half; psi distinct from eta)
int sap_apply_full(qxd_ctx* ctx, int fl, const float4* eta, float4* psi, cudaStream_t st);
int sap_check(qxd_ctx* ctx);

// deflation (deflation.cu): out = M_dfl v on full FP32 fields (coarse GCR iterations and
// residual reported if the pointers are given); z_e = (M_dfl (r_e, 0))_e on FP32 even fields
int dfl_apply_full(qxd_ctx* ctx, int fl, const float4* v, float4* out, int* citers, double* crel, cudaStream_t st);
int dfl_apply_even(qxd_ctx* ctx, int fl, const void* r_e, void* z_e, cudaStream_t st);
int dfl_status(qxd_ctx* ctx, int fl, int* iters, double* relres, cudaStream_t st);
void dfl_free(QxdFlavour& F);

// solvers.cu
int solve_cgne64(qxd_ctx* ctx, int fl, const qxd_solver* s, const Full& eta, const Full& x, qxd_info* info,
                 cudaStream_t st);
// out = (Dhat^+ Dhat + sigma) v in precision P; tmp_e, tmp_o: even and odd scratch
int op_normal(qxd_ctx* ctx, int fl, int P, double sigma, const void* v, void* out, void* tmp_e, void* tmp_o,
              cudaStream_t st);
// multi-shift CG: b64 even FP64 field, X64 ns consecutive FP64 even fields (output)
int solve_mscg(qxd_ctx* ctx, int fl, int ns, const double* sigma, const qxd_solver* s, const void* b64, char* X64,
               qxd_info* info, cudaStream_t st);
// FGCR + defect correction for nrhs right-hand sides in lockstep (one multi-RHS
// operator launch per iteration); eta, x: nrhs consecutive fields per parity
int solve_fgcr_dc_batched(qxd_ctx* ctx, int fl, const qxd_solver* s, const Full& eta, const Full& x, int nrhs,
                          qxd_info* info, cudaStream_t st);
int solve_fgcr_dc(qxd_ctx* ctx, int fl, const qxd_solver* s, const Full& eta, const Full& x, qxd_info* info,
                  cudaStream_t st);

}  // namespace qxd
