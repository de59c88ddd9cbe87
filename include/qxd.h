/*
 * qxd.h - C ABI of libqxd: the O(a)-improved Wilson-Dirac operator with
 * combined SU(3) x U(1) links, SU(3) and U(1) Sheikholeslami-Wohlert terms,
 * even-odd preconditioning, phase-periodic and C* boundary conditions, and
 * the solvers built on it, on one NVIDIA GB300 (sm_103a).
 *
 * Definitions follow openQ*D (Campos et al., arXiv:1908.11673):
 *   operator           Sec. 2.3, eqs. dirac, wilson-dirac, frw-covder, bkw-covder
 *   SW term            Sec. 2.3, eq. sw-term and the U(1) field tensor below it
 *   even-odd operator  Sec. 2.3, definition of D-hat
 *   C* boundaries      Sec. 2.1, eqs. cstar-bc, ext-periodic-bc, ext-shifted-bc
 *   solvers            Sec. 4.4 (CG, MSCG, GCR); shifts of App. A.1/A.2
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice.  mu = 0 is time.  The physical lattice is L0 x L1 x L2 x L3.  With
 *   C* in `cstar` >= 1 directions (turned on in the order 1, 2, 3) the simulated
 *   lattice is the extended lattice L0 x 2L1 x L2 x L3; otherwise it is the
 *   physical one.  V = number of simulated sites, V_e = V_o = V/2.
 * Site order.  Lexicographic over the simulated lattice, x0 slowest:
 *   idx = ((x0*N1 + x1)*N2 + x2)*N3 + x3  (N = simulated extents).
 *   Parity = (x0+x1+x2+x3) mod 2, 0 = even.  Because N3 is even, an even-site
 *   (odd-site) vector lists the even (odd) sites in lexicographic order, and
 *   site idx sits at position idx/2.
 * Spinors.  [site][spin 4][colour 3] complex, interleaved (re, im).  FP64 entry
 *   points take complex128 (double pairs), FP32 ones complex64 (float pairs).
 *   Several right-hand sides are stored one after the other: [nrhs][V or V/2][4][3].
 * Gamma matrices.  Chiral basis: gamma_0 = [[0,-1],[-1,0]],
 *   gamma_k = [[0,-i s_k],[i s_k,0]] (s_k Pauli matrices), gamma_5 = diag(1,1,-1,-1);
 *   sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu].
 * Pointers.  Every array argument may be host memory or device memory of the
 *   context's GPU; the library looks at each pointer (cudaPointerGetAttributes)
 *   and stages host arrays through its own device buffers.  The caller owns all
 *   arrays it passes; the library owns its internal copies of links, SW terms
 *   and workspace and frees them in qxd_destroy.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Operator
 *   applications on device arrays are asynchronous on that stream; calls that
 *   take or return host arrays, and all solves, synchronise it before returning.
 * Errors.  Every call returns a qxd_status; 0 is success.  No C++ exception
 *   crosses the ABI.  qxd_last_error() gives a message for the last failure on
 *   a context.  Arguments are checked before any launch.
 */
#ifndef QXD_H
#define QXD_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QXD_OK = 0,
    QXD_EARG = 1,        /* invalid argument (geometry, sizes, flavour id, precision) */
    QXD_ENOCONV = 2,     /* solver reached nmx without meeting its tolerance */
    QXD_EBREAKDOWN = 3,  /* Krylov breakdown (zero denominator) */
    QXD_ENAN = 4,        /* non-finite value in a source or during a solve */
    QXD_ECUDA = 5,       /* CUDA runtime error */
    QXD_ENOMEM = 6,      /* device allocation failed */
    QXD_ESTATE = 7       /* call out of order (e.g. operator before set_links/set_clover) */
} qxd_status;

/* QXD_DF64: FP64 data (complex128 at the interface) with double-float arithmetic
 * (each real an unevaluated sum of two floats, about 48 significant bits) on the
 * FP32 pipe; qxd_apply_Dw only (one right-hand side), and the outer residual of
 * the FGCR solver. */
typedef enum { QXD_FP64 = 0, QXD_FP32 = 1, QXD_BF16 = 2, QXD_DF64 = 3 } qxd_prec;

typedef enum { QXD_CGNE = 0, QXD_FGCR = 1, QXD_MSCG = 2 } qxd_solver_kind;

typedef enum { QXD_PRECOND_NONE = 0, QXD_PRECOND_LEARNED = 1, QXD_PRECOND_SAP = 2, QXD_PRECOND_DFL = 3 } qxd_precond_kind;

/* Geometry (Sec. 2.1).  Every L[mu] must be even and >= 2.
 * cstar in 0..3: C* boundary conditions in directions 1..cstar.
 * theta[mu]: fermion phase psi(x + L_mu e_mu) = exp(i theta_mu) psi(x)
 * (eq. periodic-bc-quark); theta[0] = pi gives antiperiodic time.  With
 * cstar > 0 the spatial phases theta[1..3] must be 0 (Sec. 2.1).
 * tbc: time boundary, QXD_TBC_PERIODIC (phase theta[0]) or QXD_TBC_OPEN.  The
 *   paper lists open boundaries in time among those of eq. dirac (term dD_b,
 *   Sec. 2.3) and defers their definition to openQCD (Luescher and Schaefer,
 *   Comput. Phys. Commun. 184 (2013) 519); this library implements: the lattice
 *   ends at x0 = 0 and x0 = L0 - 1, no hop crosses between them, the clover
 *   leaves (SU(3) and U(1)) whose plaquette would cross are absent from the SW
 *   term, and dD_b psi(x) = (cF - 1)(delta_{x0,0} + delta_{x0,L0-1}) psi(x).
 *   With QXD_TBC_OPEN theta[0] must be 0.
 * cF: boundary improvement coefficient of dD_b (1 = tree level, dD_b = 0);
 *   used only with QXD_TBC_OPEN. */
typedef enum { QXD_TBC_PERIODIC = 0, QXD_TBC_OPEN = 1 } qxd_tbc;

typedef struct {
    int L[4];
    int cstar;
    double theta[4];
    int tbc;
    double cF;
} qxd_geom;

/* One quark flavour (input-file section [Flavour n], App. C):
 * qhat = q/qel (integer charge), kappa (a m0 = 1/(2 kappa) - 4),
 * su3csw, u1csw = SW coefficients of eq. sw-term. */
typedef struct {
    int qhat;
    double kappa;
    double su3csw;
    double u1csw;
} qxd_flavour;

/* Solver parameters.
 * kind   : QXD_CGNE  - CG on Dhat^+ Dhat in FP64 (the plain FP64 solver);
 *          QXD_FGCR  - flexible GCR on Dhat in precision `inner`, restarted every
 *                      nkv steps, inside FP64 defect correction;
 *          QXD_MSCG  - multi-shift CG (only with qxd_solve_multishift).
 * tol    : target true relative residual |eta - D psi| / |eta| (FP64, full lattice)
 *          for qxd_solve, |phi - (Dhat^+Dhat + s_j) x_j| / |phi| for each shift j.
 * nmx    : maximum number of operator applications of the Krylov solver
 *          (for defect correction: summed over the inner solves).
 * nkv    : GCR restart length (1..64).
 * inner  : precision of the inner Krylov solver (QXD_FP32 or QXD_BF16 storage;
 *          QXD_FP64 makes FGCR a plain FP64 solver).
 * inner_tol : relative residual reduction requested from each inner solve
 *          (0 selects 1e-5 for FP32 and 5e-3 for BF16 storage).
 * precond: right preconditioner of FGCR: QXD_PRECOND_NONE, QXD_PRECOND_LEARNED (the network of
 *          qxd_set_precond_weights) or QXD_PRECOND_SAP (Schwarz alternating procedure, see
 *          qxd_set_sap; needs every simulated extent to be a multiple of 8) or
 *          QXD_PRECOND_DFL (inexact deflation with SAP, see qxd_dfl_setup). */
typedef struct {
    int kind;
    double tol;
    int nmx;
    int nkv;
    int inner;
    double inner_tol;
    int precond;
} qxd_solver;

/* Solver report.  true_relres is always recomputed from the returned solution with
 * the FP64 operator data: in FP64 arithmetic for CGNE and for FGCR with FP64 inner
 * solves, in double-float arithmetic (QXD_DF64, about 48-bit significands) for the
 * mixed-precision FGCR.  op_applies counts applications of Dhat (or D) in any precision. */
typedef struct {
    int status;
    int iters;
    int restarts;
    int op_applies;
    double true_relres;
} qxd_info;

typedef struct qxd_ctx qxd_ctx;

/* Create a context on CUDA device `device` for geometry `g`.
 * Errors: QXD_EARG for an odd or non-positive extent, cstar outside 0..3, a
 * non-zero spatial theta with cstar > 0, tbc outside 0..1, or an open time
 * boundary with theta[0] != 0 or a non-finite cF; QXD_ECUDA if the device is
 * unusable. */
int qxd_create(const qxd_geom* g, int device, qxd_ctx** out);

/* Free every device buffer of the context.  NULL is allowed. */
void qxd_destroy(qxd_ctx* ctx);

/* Load the gauge field given on the PHYSICAL lattice (Sec. 2):
 *   U: complex128 [Vphys][4][3][3] SU(3) links U_mu(x) (row-major colour matrix),
 *   A: float64   [Vphys][4] photon field A_mu(x), z_mu(x) = exp(i A_mu(x)).
 * With C* the mirror half is filled by the library from the orbifold
 * constraint U(x + L1 e1) = U(x)^*, A(x + L1 e1) = -A(x) (eq. cstar-bc-gauge).
 * invqel = 1/qel (elementary charge) is kept for reference; the operator does not
 * depend on it (q Ahat = qhat (i/4) Im sum z_{mu nu}).
 * Invalidates every SW term set before.  Synchronises `stream`. */
int qxd_set_links(qxd_ctx* ctx, const double* U, const double* A, double invqel, void* stream);

/* Build, for flavour slot fl (0..7), the hopping phases z^qhat (with the
 * boundary phases folded in), the site-diagonal term 1/(2 kappa) + dD_sw + dD_b
 * (eq. sw-term; two Hermitian 6x6 chiral blocks per site) and its inverse on
 * every site, in FP64 with FP32 and BF16 copies.
 * Errors: QXD_ESTATE before qxd_set_links; QXD_EARG for fl outside 0..7 or
 * kappa <= 0; QXD_ENAN if a diagonal block is singular.  Synchronises `stream`. */
int qxd_set_clover(qxd_ctx* ctx, int fl, const qxd_flavour* f, void* stream);

/* out = D in on the full simulated lattice (eq. dirac; dD_b = 0 unless the time
 * boundary is open, see qxd_geom), for nrhs
 * right-hand sides.  in, out: [nrhs][V][4][3] complex128 (prec = QXD_FP64) or
 * complex64 (QXD_FP32, and QXD_BF16 which stores spinors in bfloat16 inside the
 * kernel and accumulates in FP32); QXD_DF64: complex128 like QXD_FP64, arithmetic in
 * double-float, nrhs = 1.  in and out must not overlap. */
int qxd_apply_Dw(qxd_ctx* ctx, int fl, int prec, const void* in, void* out, int nrhs, void* stream);

/* out_e = Dhat in_e = (D_ee - D_eo D_oo^-1 D_oe) in_e (Sec. 2.3) on even-site
 * vectors [nrhs][V/2][4][3].  If dagger != 0 applies Dhat^+ = gamma5 Dhat gamma5. */
int qxd_apply_Dhat_eo(qxd_ctx* ctx, int fl, int prec, int dagger, const void* in_e, void* out_e,
                      int nrhs, void* stream);

/* Solve D psi = eta on the full lattice (complex128 [nrhs][V][4][3]) to the true
 * relative residual s->tol.  CGNE: even-odd system, CG on Dhat^+ Dhat in FP64,
 * odd sites reconstructed, one right-hand side after the other.  FGCR: FP64
 * defect correction whose inner solves run flexible GCR on Dhat in precision
 * s->inner; with nrhs > 1 all right-hand sides run in lockstep, every iteration
 * applying Dhat to the whole batch in one multi-right-hand-side launch
 * (2 nrhs (nkv + 1) <= 512).  info (may be NULL) receives the report (for a batch:
 * inner iterations of the slowest right-hand side, true_relres the worst).
 * Returns QXD_ENOCONV if any right-hand side misses the tolerance within nmx. */
int qxd_solve(qxd_ctx* ctx, int fl, const qxd_solver* s, const void* eta, void* psi, int nrhs,
              qxd_info* info, void* stream);

/* Multi-shift CG (Sec. 4.4 MSCG; App. A.2): x_j = (Dhat^+ Dhat + sigma[j])^-1 phi_e
 * for j = 0..nshift-1 (1 <= nshift <= 32, sigma[j] >= 0), phi_e and each x_j
 * complex128 [V/2][4][3]; x_e holds the nshift solutions one after the other.
 * s->inner = QXD_FP64 runs the Krylov space in FP64; QXD_FP32 runs it with the
 * FP32 operator and then refines each shift by FP64 defect correction. */
int qxd_solve_multishift(qxd_ctx* ctx, int fl, int nshift, const double* sigma, const qxd_solver* s,
                         const void* phi_e, void* x_e, qxd_info* info, void* stream);

/* Rational approximation of order [n, n] in q2 (App. A.1, eq. ratfunc):
 *   rho(q2) = A prod_{j=0..n-1} (q2 + nu[j]^2) / (q2 + mu[j]^2),   1 <= n <= 32.
 * The coefficients are inputs: the paper obtains them from a separate minmax
 * program.  Factor ranges k..l below are 0-based and inclusive (the paper's
 * j = k+1 .. l+1).  The mu[j]^2 of a factor must be pairwise distinct. */
typedef struct {
    int n;
    double A;
    const double* nu;
    const double* mu;
} qxd_rational;

/* out_e = P_{k,l} in_e with P_{k,l} = prod_{j=k..l} (Q2 + nu_j^2) / (Q2 + mu_j^2),
 * Q2 = Dhat^+ Dhat (App. A.2, eq. Pfactor), evaluated through its partial fractions
 * P_{k,l} = 1 + sum_j sigma_j (Q2 + mu_j^2)^-1 with one multi-shift CG (solver
 * parameters as in qxd_solve_multishift: each shift to relative residual s->tol).
 * in_e, out_e: complex128 [V/2][4][3], host or device; the full R = A P_{0,n-1}.
 * info (may be NULL): CG iterations and the worst shift residual. */
int qxd_rat_apply(qxd_ctx* ctx, int fl, const qxd_rational* r, int k, int l, const qxd_solver* s,
                  const void* in_e, void* out_e, qxd_info* info, void* stream);

/* Pseudofermion action of the factor P_{k,l} (App. A.2, eqs. Spf, Spf2):
 * *S = (phi, phi) + sum_{j=k..l} sigma_j (phi, (Q2 + mu_j^2)^-1 phi) = (phi, P_{k,l} phi),
 * phi_e complex128 [V/2][4][3] (host or device), sums in FP64. */
int qxd_pf_action(qxd_ctx* ctx, int fl, const qxd_rational* r, int k, int l, const qxd_solver* s,
                  const void* phi_e, double* S, qxd_info* info, void* stream);

/* Stochastic estimate of the reweighting factor W_rat = det[Q2^alpha R] with
 * alpha = u/v (App. A.3, eqs. Wrat2, Wrat3): Z = Q2^u R^v - 1, R = A P_{0,n-1};
 * terms[i] = (eta, Z^(i+1) eta) for i < nterms (1..16), and *exponent (may be NULL)
 * = sum_i c_{v,i+1} terms[i], c_{v,n} the Taylor coefficients of (1 + Z)^(-1/v);
 * one source eta gives the estimate exp(-*exponent).  Each power of Z costs v
 * multi-shift solves and u applications of Q2. */
int qxd_rw_rat(qxd_ctx* ctx, int fl, const qxd_rational* r, int u, int v, int nterms, const qxd_solver* s,
               const void* eta_e, double* terms, double* exponent, qxd_info* info, void* stream);

/* Exponent of the stochastic estimate of det Ptilde_{k,l}^-1, the factor k..l of
 * the reweighting factor W_rtm = det[R^-1 R_mu] (App. A.3):
 *   *exponent = (eta, [Ptilde_{k,l} - 1] eta),
 *   Ptilde_{k,l} = prod_j (Q2 + mu_j^2)(Q2 + nutilde_j^2) / ((Q2 + nu_j^2)(Q2 + mutilde_j^2)),
 * with (nu, mu) from r_mu (the approximation of (Q2 + muhat^2)^-alpha) and
 * (nutilde, mutilde) from r_t (that of Q2^-alpha), both of the same degree;
 * l - k + 1 <= 16.  Evaluated in the combined form the paper recommends for
 * stability: sum_j (sigma_j + sigmatilde_j) (eta, x_j)
 * + sigmatilde_j (nu_j^2 - mutilde_j^2) (x_j, y_j), x_j = (Q2 + nu_j^2)^-1 eta,
 * y_j = (Q2 + mutilde_j^2)^-1 eta, all from one multi-shift CG. */
int qxd_rw_rtm(qxd_ctx* ctx, int fl, const qxd_rational* r_mu, const qxd_rational* r_t, int k, int l,
               const qxd_solver* s, const void* eta_e, double* exponent, qxd_info* info, void* stream);

/* Small-determinant action (Sec. 2.3; det D = det D_oo det Dhat):
 * *logdet = sum over odd sites x of log |det D_oo(x)|, D_oo(x) = 1/(2 kappa) + dD_sw
 * (12x12), in FP64 from an LDL^H factorisation of each 6x6 chiral block;
 * S_sdet = -alpha_f *logdet for a flavour of weight alpha_f.  *nneg (may be NULL)
 * receives the number of odd sites with a negative determinant.  QXD_ENAN if a
 * block has a vanishing leading minor.  Synchronises `stream`. */
int qxd_sdet(qxd_ctx* ctx, int fl, double* logdet, int* nneg, void* stream);

/* Dhat for callers that cannot allocate device memory during the call.  The
 * paper has no counterpart; this is an interface convenience.  Some callers own
 * all device memory through their own pool allocator and have nothing left for
 * the library, and cudaMalloc synchronises the whole device, which a tight
 * asynchronous loop cannot afford.  qxd_apply_Dhat_eo grows the context's
 * workspace with cudaMalloc on first use.  This entry point computes the same
 * out_e = Dhat in_e (dagger: Dhat^+), with the same kernels, for one
 * right-hand side, and allocates nothing.  Its temporaries are held in one
 * file-scope device array of 18 MiB.  Every GPU that loads the library holds
 * that array until the process exits.
 *  - Maximum size: V/2 <= 32768 even sites (e.g. 16^4, or 8x(2x8)x8x16 with C*);
 *    larger lattices return QXD_EARG.
 *  - in_e and out_e must be device arrays of the context's GPU ([V/2][4][3]
 *    complex128 for QXD_FP64, complex64 for QXD_FP32 and QXD_BF16); host arrays
 *    and arrays on another GPU return QXD_EARG (staging would allocate).
 *  - The first call on a device looks up the array's device address with the
 *    CUDA runtime.  Make that first call before any stream capture.
 *  - The call never runs the launch-shape autotuner of qxd_apply_Dhat_eo (which
 *    times candidate shapes and waits for them on the host): it uses the shape
 *    that an earlier qxd_apply_Dhat_eo on the same context and lattice tuned,
 *    else a fixed default shape.  The result is the same either way.
 *  - Every call, from any context on the device, uses the same array.  Calls
 *    whose work overlaps on the GPU (different streams, or different threads)
 *    race and give wrong results.  Serialise them.  Each call overwrites the
 *    whole array region it reads, so no state carries over between calls.
 *  - Asynchronous on `stream`, like qxd_apply_Dhat_eo on device arrays. */
int qxd_apply_Dhat_eo_noalloc(qxd_ctx* ctx, int fl, int prec, int dagger, const void* in_e, void* out_e,
                              void* stream);

/* Learned preconditioner weights for flavour fl (used by FGCR with
 * QXD_PRECOND_LEARNED), and the precision of the network's channel mixing inside
 * the solver: QXD_FP32 (CUDA cores, FP32) or QXD_BF16 (tensor cores: transports and
 * weights rounded to bfloat16, FP32 accumulation; layers with at most 8 input and 8
 * output channels, wider ones run in FP32).  The network M has nlayers gauge-covariant layers
 *   psi'_c(x) = sum_{c'} sum_{d=0..8} W[l][c][c'][d] T_d psi_{c'}(x),
 * T_0 = 1, T_{1+mu} psi(x) = V_mu(x) psi(x+mu), T_{5+mu} psi(x) = V_mu(x-mu)^+ psi(x-mu),
 * with V = U z^qhat and the boundary conditions of D; channel counts
 * 1 -> nch -> ... -> nch -> 1.  W: float32 complex, per layer
 * [cout][cin][9][4][4] spin matrices (interleaved re, im), layers one after the
 * other.  The network is not part of the paper. */
int qxd_set_precond_weights(qxd_ctx* ctx, int fl, const float* W, int nlayers, int nch, int prec);

/* ---- SAP preconditioner (Sec. 4.1 and 4.4: SAP+GCR) ----
 * Blocks of 4^4 sites coloured like a checkerboard; one application M eta runs
 * ncy cycles over the two colours, each block solving its Dirichlet block system
 * (hops leaving the block dropped) approximately by nmr minimal-residual steps on
 * the block's even-odd system, for the residual rho = eta - D psi taken on the
 * block at the start of its colour's sweep.  FGCR on Dhat uses z_e = (M (r_e, 0))_e (Dhat^-1 = (D^-1)_ee).
 * Arithmetic in FP32. */

/* Set ncy and nmr (1..64 each; default 5 and 5, the paper's values). */
int qxd_set_sap(qxd_ctx* ctx, int ncy, int nmr);

/* out = M in on the full lattice, complex64 [V][4][3] (host or device arrays).
 * QXD_EARG unless every simulated extent is a multiple of 8 (an even number of blocks,
 * so that blocks of one colour never touch).  Synchronises `stream`. */
int qxd_sap_apply(qxd_ctx* ctx, int fl, const void* in, void* out, void* stream);

/* ---- inexact deflation with SAP (Sec. 4.4: DFL+SAP+GCR) ----
 * One deflation subspace per flavour slot, hence per charge.  Blocks are the SAP
 * blocks (4^4; every simulated extent a multiple of 8).  The subspace is built
 * from Ns given random fields: ninv times phi_k <- M_sap phi_k (SAP with the
 * context's ncy, nmr), each time followed by Gram-Schmidt of the restrictions
 * phi_k|_B on every block B.  P c = sum_{B,k} c_{B,k} phi_k|_B, P^+ its adjoint,
 * A = P^+ D P the little Dirac operator.  The preconditioner is
 *   M_dfl v = P A^-1 P^+ v + M_sap (v - D P A^-1 P^+ v),
 * with A^-1 from GCR on the block grid (restart cnkv, at most cnmx steps, relative
 * residual ctol); FGCR on Dhat uses z_e = (M_dfl (r_e, 0))_e.  FP32 throughout. */
typedef struct {
    int Ns;       /* vectors per block, 1..32 */
    int ninv;     /* inverse-iteration steps with SAP, 0..64 */
    double ctol;  /* relative residual of the little-system solves */
    int cnmx;     /* maximum GCR steps of a little-system solve */
    int cnkv;     /* GCR restart length of the little-system solver, 1..32 */
} qxd_dfl_params;

/* Build the subspace and A for flavour fl.  seeds: complex64 [Ns][V][4][3] random
 * start fields (host or device).  Replaces an earlier subspace of fl; dropped when
 * the links or the SW term of fl change.  QXD_EARG for bad parameters or a lattice
 * SAP does not support.  Synchronises `stream`. */
int qxd_dfl_setup(qxd_ctx* ctx, int fl, const qxd_dfl_params* p, const void* seeds, void* stream);

/* Basis field phi_k (block-orthonormal), complex64 [V][4][3] (host or device). */
int qxd_dfl_basis(qxd_ctx* ctx, int fl, int k, void* out, void* stream);

/* The little operator: A_out (may be NULL) complex64 [Nb][9][Ns][Ns] with
 * A_out[B][s][l][k] = <phi_k|_B, D phi_l|_{B_s}>; nbr_out (may be NULL) int [Nb][9]
 * the block B_s of slot s (0: B; 1 + 2 mu: across the +mu face; 2 + 2 mu: across
 * the -mu face); *nblocks (may be NULL) = Nb.  Blocks are numbered
 * lexicographically by block coordinates, x0 slowest. */
int qxd_dfl_little(qxd_ctx* ctx, int fl, void* A_out, int* nbr_out, int* nblocks, void* stream);

/* out = M_dfl in on the full lattice, complex64 [V][4][3] (host or device).
 * info (may be NULL): iters and true_relres of the little-system GCR. */
int qxd_dfl_apply(qxd_ctx* ctx, int fl, const void* in, void* out, qxd_info* info, void* stream);

/* ---- learned preconditioner: inference and training (not part of the paper) ----
 * The network M and its weight layout are those of qxd_set_precond_weights.
 * Even-site fields below are complex64 [V/2][4][3] in the canonical order;
 * every array may be host or device memory. */

/* out_e = (M in_e)_e: the network applied to in_e embedded in the full lattice
 * (zero on odd sites), restricted to the even sites; channel mixing in prec
 * (QXD_FP32 or QXD_BF16, as in qxd_set_precond_weights).  Synchronises `stream`;
 * QXD_ECUDA if a tensor-core completion wait timed out. */
int qxd_ptc_apply(qxd_ctx* ctx, int fl, int prec, const float* W, int nlayers, int nch, const void* in_e,
                  void* out_e, void* stream);

/* Loss over npairs pairs (r, e: [npairs][V/2][4][3] complex64) into *loss:
 * kind 0, Euclidean error: L = sum_i |(M r_i)_e - e_i|^2 / |e_i|^2;
 * kind 1, residual norm:   L = sum_i |r_i - Dhat (M r_i)_e|^2 / |r_i|^2 (with Dhat the
 * FP32 operator; for pairs with Dhat e_i = r_i the error of M r_i in the norm |Dhat .|);
 * and, if grad != NULL, its gradient
 * G = dL/dW^* (Wirtinger; the gradient with respect to the real and imaginary
 * parts of W is 2 Re G, 2 Im G), complex float32 in the layout of W. */
int qxd_ptc_loss_grad(qxd_ctx* ctx, int fl, const float* W, int nlayers, int nch, const void* r, const void* e,
                      int npairs, int kind, double* loss, float* grad, void* stream);

/* nsteps steps of Adam (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * loss above (kind as there), each over `batch` pairs taken in turn from the npairs given.  W is
 * updated in place; m, v are the Adam moments (same size as W, zero at the
 * start of training) and *t the step counter, all carried between calls so
 * that training can alternate gauge fields (one context per field).
 * losses (may be NULL) receives the mean loss of each step. */
int qxd_ptc_train(qxd_ctx* ctx, int fl, float* W, float* m, float* v, int nlayers, int nch, const void* r,
                  const void* e, int npairs, int batch, int nsteps, double lr, int kind, int* t, double* losses,
                  void* stream);

/* Training pairs from the plain FP64 solver: CG on the normal equations of
 * Dhat x = b (b: complex128 [V/2][4][3]) run to |b - Dhat x| <= 1e-10 |b|; at
 * iterations k = stride, 2 stride, ... the pair r = b - Dhat x_k, e = x* - x_k is
 * recorded (x* the converged solution), npairs pairs into r_out, e_out
 * (complex64 [npairs][V/2][4][3]).  QXD_ENOCONV if the solve does not
 * converge, QXD_EARG if it converges before npairs * stride iterations. */
int qxd_ptc_record_pairs(qxd_ctx* ctx, int fl, const void* b, int npairs, int stride, void* r_out, void* e_out,
                         void* stream);

/* Kernel profiling for benchmarks (not part of the paper).  mode 0: off;
 * 1: count the library's kernel launches by class; 2: also time each launch with
 * a CUDA event pair recorded on its launching stream.  Every call resets the
 * counters.  Timing adds two event records per launch and nothing else. */
int qxd_profile(qxd_ctx* ctx, int mode);

/* Class i (0-based, in order of first launch) of the profile: its name, launch
 * count, summed device time in ms (mode 2; synchronises the recorded events)
 * and summed algorithmic DRAM bytes (every input and output array element
 * counted once per launch: the roofline numerator).  QXD_EARG past the last class. */
int qxd_profile_entry(qxd_ctx* ctx, int i, char* name, int len, long long* launches, double* ms, double* bytes);

/* ---- host-only helpers (no device, no context) ----
 * The partial-fraction residues the rational functions above use:
 * sigma[j-k] = (nu_j^2 - mu_j^2) prod_{m != j} (nu_m^2 - mu_j^2) / (mu_m^2 - mu_j^2),
 * j = k..l, of P_{k,l} (App. A.2), and the residues (sigma, sigma_t) of Ptilde_{k,l} - 1 at
 * q2 = -nu_j^2 and q2 = -mutilde_j^2 (App. A.3, W_rtm).  QXD_EARG for bad arguments or
 * coinciding poles. */
int qxd_rat_residues(const qxd_rational* r, int k, int l, double* sigma);
int qxd_rtm_residues(const qxd_rational* r_mu, const qxd_rational* r_t, int k, int l, double* sigma,
                     double* sigma_t);

/* The 4^4 block grid of SAP and deflation for geometry g: *nblocks (may be NULL) = Nb,
 * nbr_out (may be NULL) int [Nb][9] as in qxd_dfl_little.  QXD_EARG for an invalid
 * geometry or a simulated extent that is not a multiple of 8. */
int qxd_block_neighbours(const qxd_geom* g, int* nbr_out, int* nblocks);

/* Message describing the last failing call on ctx (never NULL). */
const char* qxd_last_error(qxd_ctx* ctx);

/* Number of simulated sites V of the context (0 for NULL). */
long long qxd_volume(const qxd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* QXD_H */
