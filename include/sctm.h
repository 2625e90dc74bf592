/*
 * sctm.h -- C ABI of the GB300 split-CTMRG library (libsctm.so).
 *
 * Split corner-transfer renormalization group for the triple-layer PEPS-PEPO-PEPS network of a
 * 3D classical model (Xu, Lin & Zhang, arXiv:2506.19339): the free-energy density
 *     f = -T (ln kappa_num - ln kappa_den)                        (Sec. II, Eq. "free energy expression")
 * and its gradient g = 2 df/dA-bar                               (Sec. II, Eq. "gradient expression")
 * from converged split-CTM environments (Sec. III) of the numerator <psi|T|psi> and of the norm
 * <psi|psi>.  All compute runs in CUDA kernels on one GPU; cuSOLVER is used for the FP64 SVDs.
 *
 * Conventions shared by every entry point
 *   - Tensors are dense, row-major, FP64.
 *       PEPS  A[s,u,l,d,r]          shape (p, D, D, D, D)      (bra = A, real)
 *       PEPO  O[s_up,s_dn,u,l,d,r]  shape (p, p, d, d, d, d)   (s_dn joins the ket, s_up the bra)
 *   - Pointer arguments documented as "host or device" are inspected with
 *     cudaPointerGetAttributes; either kind is accepted.  The library never keeps or frees a
 *     caller's pointer: inputs are copied, outputs are written.
 *   - Every call returns an sctm_status and never aborts; a context-level message is available
 *     from sctm_last_error().  A NULL context returns SCTM_EINVAL.
 *   - Calls on one context are not thread-safe; different contexts are independent.
 *   - Results are deterministic: the same inputs and options give the same bits on the same GPU
 *     (all reductions have a fixed order).  In SCTM_PREC_F64EMU the kernel of each contraction
 *     shape is chosen by timing (sctm_autotune_info) once per process and device: contexts of one
 *     process agree bit for bit, two processes may differ in the last bits (both FP64-accurate).
 */
#ifndef SCTM_H
#define SCTM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sctm_ctx sctm_ctx;

typedef enum {
    SCTM_OK = 0,
    SCTM_EINVAL = 1,     /* bad argument (NULL pointer, size out of range, unknown option)      */
    SCTM_ECUDA = 2,      /* a CUDA runtime call or kernel launch failed                          */
    SCTM_ECUSOLVER = 3,  /* a cuSOLVER call failed or did not converge                           */
    SCTM_ENOMEM = 4,     /* device memory allocation failed                                      */
    SCTM_ENOCONV = 5,    /* iteration limit reached before ||S[i+1]-S[i]||_2 < tol (Sec. III.D)  */
    SCTM_ENUMERIC = 6,   /* kappa <= 0, a non-finite value, or an all-zero spectrum              */
    SCTM_ETIMEOUT = 7    /* a bounded device-side wait ran out (tensor-core kernels)             */
} sctm_status;

/* Arithmetic of the move contractions (corner and edge absorption, half patches, rho_B rho_T,
 * renormalisation; Sec. III).  Projector formation, SVDs, normalisations, the spectrum, the local
 * contractions and the free-energy ratio are FP64 in every mode.  The TF32 / BF16 forms iterate
 * with a raised pseudo-inverse cutoff and finish in FP64 (sctm_iterate); SCTM_PREC_F64EMU is
 * FP64-accurate and runs a contraction on the tensor cores where an autotuner, run when the
 * context is created, measured the emulation faster than the FP64 kernels for that contraction
 * shape (sctm_autotune_info); elsewhere the FP64 kernels. */
enum {
    SCTM_PREC_FP64 = 0,    /* all contractions in FP64                                         */
    SCTM_PREC_TF32 = 1,    /* contractions on tensor cores, TF32 inputs, FP32 accumulation     */
    SCTM_PREC_TF32X3 = 2,  /* TF32 with hi/lo split products (hi*hi + hi*lo + lo*hi)            */
    SCTM_PREC_BF16 = 3,    /* contractions on tensor cores, BF16 inputs, FP32 accumulation     */
    SCTM_PREC_BF16X3 = 4,  /* BF16 with hi/lo split products                                   */
    SCTM_PREC_F64EMU = 5   /* FP64-accurate: eight 7-bit BF16 digits per operand element, exact */
                           /* FP32 level sums on the tensor cores, FP64 recombination           */
};

/* Gradient returned by sctm_grad:
 *   SCTM_GRAD_ENV      the paper's gradient (Sec. II, Eq. "gradient expression"): twice the
 *                      derivative of f with respect to the bra tensor with the environment held
 *                      fixed, g = -2T (E_num/Z11_num - E_den/Z11_den)
 *   SCTM_GRAD_ADJOINT  the derivative of the converged free energy itself, d f / d A (both the
 *                      ket and the bra slot, and the environment's dependence on A), by implicit
 *                      differentiation of the split-CTMRG fixed point.  The paper has no such
 *                      gradient; the two agree as chi grows (the environment part vanishes at
 *                      the exact fixed point). */
enum { SCTM_GRAD_ENV = 0, SCTM_GRAD_ADJOINT = 1 };
/* FP64 SVD of the projector matrices (Eq. "projector construction"):
 *   SCTM_SVD_QR       cuSOLVER gesvd (bidiagonalisation + QR iteration), the reference path: its
 *                     singular vectors stay accurate down to the pseudo-inverse cutoff
 *   SCTM_SVD_POLAR    cuSOLVER gesvdp (polar decomposition + symmetric eigensolver): about 3x
 *                     faster at n = 512 with the same singular values, but less accurate vectors
 *                     for the smallest kept singular values (f moves at the 1e-10 level)
 *   SCTM_SVD_PARTIAL  the partial SVD of Sec. III (largest chi triplets by an iterative
 *                     solver): the first solve of each projector after a cold start is gesvd,
 *                     every later one a subspace-iteration step warm-started from the previous
 *                     iteration's right singular subspace (chi + p columns, p = chi/4, at
 *                     least 8, reduced to keep chi + p <= 160 where chi <= 152) with a
 *                     Rayleigh-Ritz (Jacobi) extraction, about 25 kernel launches instead of
 *                     thousands.  Projectors whose subspace would exceed 160 columns stay on
 *                     gesvd; above 112 columns the k x k kernels use a global scratch buffer.
 *                     The fixed point is the same as SCTM_SVD_QR's; a trajectory from a cold
 *                     start differs at the level of the subspace error of the early iterations.
 *                     sctm_env_import and a reset start cold again.
 *   SCTM_SVD_PARTIAL_RANDOM  as SCTM_SVD_PARTIAL, but the cold solve is two subspace steps
 *                     from a pseudo-random (SplitMix64) subspace instead of gesvd, and the
 *                     chi x chi spectrum of the convergence test (Sec. III.D) uses the same
 *                     Jacobi kernel: no cuSOLVER call at all for chi <= 160.  Same fixed
 *                     point; from a cold start the first iterations' projectors carry the
 *                     random start's subspace error, which the later warm steps remove. */
enum { SCTM_SVD_QR = 0, SCTM_SVD_POLAR = 1, SCTM_SVD_PARTIAL = 2, SCTM_SVD_PARTIAL_RANDOM = 3 };
enum { SCTM_NET_NUM = 0, SCTM_NET_DEN = 1 };          /* <psi|T|psi> and <psi|psi>            */
/* Contraction method of the triple-layer network:
 *   SCTM_METHOD_SPLIT    the paper's split-CTMRG (Sec. III): three edge layers per side, two-stage
 *                        truncation with six projector pairs per move
 *   SCTM_METHOD_REDUCED  the reduced method it is compared with (Sec. II, Fig. 3; Sec. IV.A): A,
 *                        O and A-bar fused into one tensor of bond D d D, standard directional
 *                        CTMRG with one projector pair per move from the two-by-two patch.  FP64
 *                        only (precision must be SCTM_PREC_FP64), environment gradient only; its
 *                        edge tensors are exported in the ket slots (leg m = D d D, grouped
 *                        (A, O, A-bar)), the int and bra slots are empty; cold start
 *                        C = e_0 e_0^T, T[0][0][:] = 1.
 *   SCTM_METHOD_SPLIT_D2 the D2-symmetric split-CTMRG (Sec. III.B, Eq. "Symmetry constraints"):
 *                        for a PEPS whose virtual legs are D4-invariant and a PEPO invariant under
 *                        the reflection about the main diagonal (O[t,s,u,l,d,r] = O[t,s,l,u,r,d])
 *                        and the 180-degree rotation with s_up <-> s_dn
 *                        (O[t,s,u,l,d,r] = O[s,t,d,r,u,l]), checked at creation to 1e-12 of
 *                        max|O| (else SCTM_EINVAL).  The environment is C1, C4 and the left edge
 *                        T4^{k,i,b}; C3 = C1 = C1^T, C2 = C4 = C4^T, T1 = T4, T2 = T3 = T4 with
 *                        ket <-> bra and its two chain bonds exchanged.  One iteration is one
 *                        set of six projector pairs (the left move's; the opposite boundary's
 *                        stage-1 pairs are the images of this boundary's under the 180-degree
 *                        rotation, P^R_1T = P_1B, P^R_2T = P_3B, P^R_3T = P_2B and the same
 *                        with T <-> B, Appendix, so each iteration takes six SVDs instead of 36):
 *                        T4 is renormalised as in the left move, and C1 and C4 each absorb one
 *                        column and one row at once with both legs truncated by the alpha pair,
 *                        then are symmetrised.  The PEPS is
 *                        replaced by its D4 group average on entry (sctm_create, sctm_set_peps)
 *                        and sctm_grad returns the group average of the gradient.  Environment
 *                        gradient only.  sctm_move accepts SCTM_MOVE_LEFT only (one symmetric
 *                        iteration); sctm_env_export writes all sixteen slots (the derived ones
 *                        from the constraints), sctm_env_import reads C1, C4 and T4 and
 *                        symmetrises the corners. */
enum { SCTM_METHOD_SPLIT = 0, SCTM_METHOD_REDUCED = 1, SCTM_METHOD_SPLIT_D2 = 2 };
/* Patch of the stage-2 alpha projector (projector 4, Appendix):
 *   SCTM_P4_FULL  the 2x2-cell patch (both columns, the bra lines renormalised by projector 1 of
 *                 this and of the opposite boundary), cost O(chi^3 D^4 d)
 *   SCTM_P4_HALF  the 2x1-cell patch: the two enlarged left corners (C1 and C4 each with one
 *                 column and one row absorbed), the bra lines of both their legs renormalised by
 *                 projector 1 -- on the column cut by the up / down moves' projector 1, which the
 *                 D2 symmetry gives as the transposed P_1T / P_1B, and which the directional
 *                 split method computes in each move from the same environment (two more SVD
 *                 pipelines per move; environment gradient only) (in the down move's frame ket
 *                 and bra trade places, so the lower corner's column-cut projector acts on its
 *                 ket line).  Cost O(chi^3 D^3 d^3); not with SCTM_METHOD_REDUCED. */
enum { SCTM_P4_FULL = 0, SCTM_P4_HALF = 1 };
enum { SCTM_MOVE_LEFT = 0, SCTM_MOVE_RIGHT = 1, SCTM_MOVE_UP = 2, SCTM_MOVE_DOWN = 3 };

/* Kernel of the k x k Jacobi SVD that closes each warm step of the partial SVD (svd_mode
 * SCTM_SVD_PARTIAL / SCTM_SVD_PARTIAL_RANDOM, and the convergence spectrum in the latter mode):
 * SCTM_JACOBI_CTA runs it in one CTA (one SM's FP64 pipe); SCTM_JACOBI_CLUSTER splits the rows of
 * the iterated matrices over a cluster of 8 CTAs where 32 <= k + (k mod 2) <= 128 (measured at
 * k = 80: 1.9 -> 0.9 ms warm, 5.2 -> 2.8 ms cold), and uses the one-CTA kernel elsewhere.  Both
 * compute the same decomposition to rounding; the rounding differs (the cluster sums each dot
 * product in another order), and the iteration count to a tolerance moves with it. */
enum { SCTM_JACOBI_CTA = 0, SCTM_JACOBI_CLUSTER = 1 };

typedef struct {
    double T;                     /* temperature; f = -T (...), g = -2T (...)               */
    int D;                        /* PEPS virtual bond dimension, >= 1                      */
    int p;                        /* physical dimension (2 for Ising), >= 1                 */
    int d;                        /* PEPO in-plane bond dimension (2 for Ising), >= 1       */
    int precision;                /* SCTM_PREC_*                                            */
    int grad_mode;                /* SCTM_GRAD_ENV or SCTM_GRAD_ADJOINT                     */
    double svd_cutoff;            /* pseudo-inverse cutoff s_k/s_1 (default 1e-12)          */
    unsigned long long init_seed; /* SplitMix64 seed of the cold-start environment (0)      */
    int batch;                    /* reserved, must be 1                                    */
    void* cuda_stream;            /* cudaStream_t for all work, NULL = legacy default       */
    int svd_mode;                 /* SCTM_SVD_* (default SCTM_SVD_QR)                       */
    int method;                   /* SCTM_METHOD_SPLIT (default), _REDUCED or _SPLIT_D2     */
    int p4_mode;                  /* SCTM_P4_FULL (default) or SCTM_P4_HALF (not REDUCED)   */
    int jacobi;                   /* SCTM_JACOBI_CTA (default) or SCTM_JACOBI_CLUSTER       */
} sctm_opts;

/* Fill *o with the defaults: T=1, D=2, p=2, d=2, FP64, env gradient, cutoff 1e-12, seed 0,
 * batch 1, default stream, QR SVD, the directional split method, full projector 4, the one-CTA
 * Jacobi kernel.  Returns
 * SCTM_EINVAL for NULL. */
sctm_status sctm_default_opts(sctm_opts* o);

/* sctm_create -- the problem statement of Sec. II: a PEPS tensor A, a PEPO tensor O and the
 * environment bond dimension chi.
 *   peps  host or device, p*D^4 doubles, layout A[s,u,l,d,r]                 (copied)
 *   pepo  host or device, p^2*d^4 doubles, layout O[s_up,s_dn,u,l,d,r]        (copied)
 *   chi   environment bond dimension, 1 <= chi <= 4096
 *   o     options (NULL = defaults); o->D, o->p, o->d give the shapes
 *   out   receives the new context (NULL on failure)
 * Allocates every device buffer of both networks (numerator with O, norm with the identity
 * PEPO), builds the execution plans and writes the cold-start environment (SplitMix64, Sec. III
 * gives no initialisation).  Errors: EINVAL (shapes, NULL), ENOMEM, ECUDA, ECUSOLVER. */
sctm_status sctm_create(const double* peps, const double* pepo, int chi, const sctm_opts* o,
                        sctm_ctx** out);

/* sctm_set_peps -- replace A (host or device pointer, p*D^4 doubles, copied).  With
 * reset_env != 0 the environments go back to the cold start; otherwise the current
 * environments are kept as a warm start.  Errors: EINVAL, ECUDA. */
sctm_status sctm_set_peps(sctm_ctx* ctx, const double* peps, int reset_env);

/* sctm_iterate -- power iteration of both environments (Sec. III.B: left, right, up, down
 * moves per iteration; Sec. III.D: stop once ||S[i+1]-S[i]||_2 < tol for the singular values S
 * of rho_eff = C1 C2 C3 C4 / Tr).  Each network stops on its own.  tol <= 0 runs exactly
 * max_it iterations.  *it_done (may be NULL) = the larger iteration count of the two networks;
 * *last_dS (may be NULL) = the larger final ||dS||_2.  Returns SCTM_ENOCONV when tol > 0 and a
 * network did not converge within max_it (the environments are still updated).
 * Mixed forms (o->precision != SCTM_PREC_FP64): each call starts in the context's form and
 * stays in it while ||dS|| falls, then polishes in FP64 once ||dS|| is below the form's level
 * (TF32 1e-4, BF16 1e-3, TF32 hi/lo 1e-6, BF16 hi/lo 1e-5) or has not halved in three
 * iterations; convergence is only declared on FP64 iterations.  The pseudo-inverse cutoff is
 * raised to the form's floor (1e-3, 1e-2, 1e-4, 1e-3) while the form is in use.
 * Errors: ENUMERIC (non-finite spectrum change or projector matrix), ETIMEOUT (a bounded wait
 * of the tensor-core kernel ran out), ECUSOLVER, ECUDA. */
sctm_status sctm_iterate(sctm_ctx* ctx, int max_it, double tol, int* it_done, double* last_dS);

/* sctm_free_energy -- f per 3D site in FP64 from the current environments (Sec. II):
 * kappa = Z11 Z00 / (Z10 Z01) per network, f = -T (ln kappa_num - ln kappa_den).
 *   f  host pointer to one double.
 * Returns SCTM_ENUMERIC if a kappa is <= 0 or not finite (f is then NaN), SCTM_ENOCONV if the
 * last sctm_iterate did not converge (f is still written). */
sctm_status sctm_free_energy(sctm_ctx* ctx, double* f);

/* sctm_grad -- the environment gradient g = -2T (E_num/Z11_num - E_den/Z11_den) (Sec. II,
 * Fig. 4(c): E = Z11 with A-bar removed).
 *   g  host or device pointer to p*D^4 doubles (layout of A), caller-owned.
 * Same status rules as sctm_free_energy. */
sctm_status sctm_grad(sctm_ctx* ctx, double* g);

/* sctm_set_grad_mode -- choose what sctm_grad returns (SCTM_GRAD_ENV or SCTM_GRAD_ADJOINT), and
 * for the adjoint the relative residual tol (0 < tol < 1, default 1e-10), the largest number of
 * matrix-vector products (>= 1, default 400) of its linear solve, and svd_grad_cutoff in [0, 1)
 * (default 1e-6): kept singular values below svd_grad_cutoff s_0 are held fixed in the SVD
 * backward.  Their projector columns are rounding-level directions whose exact sensitivities
 * (through S^-1/2 and 1 / (s_j^2 - s_i^2)) are huge and cancel in f; carried through, they make
 * the linear system numerically useless at large chi (measured at D=4, chi=64: no GMRES progress
 * without the cutoff, a relative residual of 1e-10 with 1e-6).  0 differentiates every kept value.
 * The adjoint gradient: with E* = F(E*, A) the converged environment of a network (F one
 * iteration: left, right, up, down moves, Sec. III.B) and ln kappa its per-site value (Sec. II),
 *     d ln kappa / dA = d ln kappa / dA |_E + lambda^T dF/dA,   (I - J^T) lambda = d ln kappa / dE,
 * J = dF/dE at E*, and d f / dA = -T (d ln kappa_num / dA - d ln kappa_den / dA).  sctm_grad then
 * (i) runs one more iteration of each network with full SVDs, keeping every intermediate and a
 * copy of each move's input (checkpointed recompute), (ii) solves for lambda by restarted GMRES,
 * each product with J^T one pass of the hand-written backward plans (contractions transposed on
 * the same kernels, the truncated-SVD backward from the full singular basis with a Lorentzian
 * broadening of 1e-12 s_0^2, the normalisation's backward), (iii) applies dF/dA^T.  Everything
 * runs in FP64 on the GPU.  The first adjoint call builds the backward plans (about as much
 * device memory again as the forward plans).  sctm_grad returns SCTM_ENOCONV (with g written)
 * if the solve stopped above tol; the environment is left one iteration further.
 * Errors: EINVAL (mode, tol, max_matvecs). */
sctm_status sctm_set_grad_mode(sctm_ctx* ctx, int mode, double tol, int max_matvecs,
                               double svd_grad_cutoff);

/* sctm_adjoint_info -- statistics of the last adjoint gradient: matvecs[0..1] the products with
 * J^T of the numerator and norm networks' solves, residual[0..1] their final relative residuals
 * |w - (I - J^T) lambda| / |w|.  Either pointer may be NULL. */
sctm_status sctm_adjoint_info(sctm_ctx* ctx, int* matvecs, double* residual);

/* sctm_destroy -- release every resource of the context.  NULL-safe (returns SCTM_OK). */
sctm_status sctm_destroy(sctm_ctx* ctx);

/* sctm_ising_pepo -- host helper: the Ising PEPO at temperature T (Sec. II, Sec. IV): the
 * six-leg delta tensor with sqrt(W), W = [[e^b, e^-b], [e^-b, e^b]], b = 1/T, on every leg.
 *   O64  host pointer to 64 doubles, layout O[s_up,s_dn,u,l,d,r].  T <= 0 -> SCTM_EINVAL;
 *   T = +inf gives the b = 0 tensor. */
sctm_status sctm_ising_pepo(double T, double* O64);

/* sctm_last_error -- message of the last failing call on ctx ("" if none; a static message
 * for NULL).  The pointer stays valid until the next call on ctx. */
const char* sctm_last_error(const sctm_ctx* ctx);

/* ---- inspection and checkpoint / resume -------------------------------------------------- */

/* Number of doubles of one network's environment in the export layout:
 * C1, C2, C3, C4 (chi x chi each), then T1^{ket,int,bra}, T2^{...}, T3^{...}, T4^{...}
 * (chi x chi x m each, m = D for ket/bra, d for int; d = 1 for the norm network).
 * Returns 0 for a NULL context or an unknown network. */
size_t sctm_env_size(const sctm_ctx* ctx, int network);

/* Copy one network's environment to / from a host buffer of sctm_env_size() doubles.  Leg
 * order (Sec. III.A): C1[h,v] (h to the top chain, v to the left chain), C2[h,v] (top, right),
 * C3[h,v] (bottom, right), C4[h,v] (bottom, left); T1[a,b,m] (left bond, right bond, leg down
 * into the site), T2[a,b,m] (up, down, leg left), T3[a,b,m] (left, right, leg up), T4[a,b,m]
 * (up, down, leg right); each tensor row-major.  import overwrites the current environment
 * (warm start).  Errors: EINVAL (network, NULL, n too small), ECUDA. */
sctm_status sctm_env_export(sctm_ctx* ctx, int network, double* host_buf, size_t n);
sctm_status sctm_env_import(sctm_ctx* ctx, int network, const double* host_buf, size_t n);

/* sctm_move -- run one directional move (SCTM_MOVE_*) of one network (Sec. III.B), without a
 * convergence check.  For inspection and tests. */
sctm_status sctm_move(sctm_ctx* ctx, int network, int direction);

/* sctm_spectrum -- the chi singular values of rho_eff of one network (Sec. III.D), descending,
 * into a host buffer of chi doubles. */
sctm_status sctm_spectrum(sctm_ctx* ctx, int network, double* S);

/* sctm_iterate_batch -- sctm_iterate on `count` independent contexts at once (the batched
 * sweep: several temperatures or PEPS of one (D, chi)).  Each context is driven from its own host
 * thread on its own streams (give each context its own cuda_stream at creation, otherwise their
 * work serialises on the shared stream).  status[i], it_done[i], last_dS[i] (host arrays of
 * `count`, any may be NULL) receive each context's results.  Returns SCTM_OK if every context
 * returned SCTM_OK, SCTM_ENOCONV if the worst was ENOCONV, else the first error status. */
sctm_status sctm_iterate_batch(sctm_ctx* const* ctxs, int count, int max_it, double tol,
                               int* status, int* it_done, double* last_dS);

/* sctm_autotune_info -- for an SCTM_PREC_F64EMU context: how many of one network's
 * FP64-accurate move contractions run on the emulation kernel (*emu) out of those that may
 * (*eligible), as chosen at creation by timing both kernels once per contraction shape (shapes
 * below 4 MFLOP stay on the FP64 kernels; the decisions are kept per device and shape for the
 * life of the process).  Both are 0 for other forms.  Either pointer may be NULL.
 * Errors: EINVAL (NULL ctx, bad network). */
sctm_status sctm_autotune_info(sctm_ctx* ctx, int network, int* emu, int* eligible);

/* sctm_device_bytes -- device memory held by the context (all of it is allocated at create). */
size_t sctm_device_bytes(const sctm_ctx* ctx);

/* sctm_local_values -- the local contractions of one network from its current environment
 * (Sec. II, Fig. 4(b)): out[0..3] = Z00, Z10, Z01, Z11 and out[4] = ln kappa,
 * kappa = Z11 Z00 / (Z10 Z01) (NaN when kappa <= 0).  Host buffer of 5 doubles.  Each Z depends
 * on the normalisation of the environment tensors; kappa does not.  For inspection and tests. */
sctm_status sctm_local_values(sctm_ctx* ctx, int network, double* out5);

/* sctm_set_profiling -- mode 1 records CUDA events around every contraction kernel and every
 * SVD (no host synchronisation is added; the events are read after each iteration); the
 * concurrent streams share the GPU, so an event pair then also counts time the launch spent
 * waiting behind other streams' work.  Mode 2 does the same with the execution serialised (every
 * step on the caller's stream, the parallel sub-plans and the two networks one after the other),
 * so each event pair measures that launch alone: per-kernel durations, at the cost of overlap.
 * Mode 0 (the default, or 1 from creation when the environment variable SCTM_PROFILE=1 is set)
 * turns both off.  Errors: EINVAL (other modes). */
sctm_status sctm_set_profiling(sctm_ctx* ctx, int on);

/* sctm_profile -- counters since creation or the last reset (reset != 0 zeroes them after
 * reading).  Any output pointer may be NULL.
 *   ctr_ms, ctr_launches, ctr_flops  device time, launches and algorithmic FLOPs (2 M N K per
 *                                    contraction) of the contraction kernel (profiling only)
 *   svd_ms, svd_calls                device time and count of the cuSOLVER SVDs (profiling only)
 *   kernel_launches                  launches of this library's own kernels (always counted) */
sctm_status sctm_profile(sctm_ctx* ctx, double* ctr_ms, long long* ctr_launches,
                         long long* ctr_flops, double* svd_ms, long long* svd_calls,
                         long long* kernel_launches, int reset);

/* Contraction kernels, for sctm_profile_kernel. */
enum {
    SCTM_KERNEL_F64 = 0,     /* tiled FP64 kernel (64 x 64 or 32 x 32 tiles, split K)              */
    SCTM_KERNEL_SKINNY = 1,  /* FP64, one output row per thread (N <= 32, K <= 64)                 */
    SCTM_KERNEL_TC = 2,      /* tensor cores, TF32 / BF16 (hi/lo) forms                             */
    SCTM_KERNEL_F64EMU = 3,  /* tensor cores, FP64 emulation                                        */
    SCTM_KERNEL_JACOBI = 4,  /* partial SVD: one-CTA Jacobi SVD of the k x k Rayleigh-Ritz matrix   */
    SCTM_KERNEL_CHOL = 5     /* partial SVD: one-CTA Cholesky-QR pass (flops and bytes not counted)  */
};

/* sctm_profile_kernel -- the profiling counters of one contraction kernel (SCTM_KERNEL_*) since
 * creation or the last reset of sctm_profile: summed CUDA-event time around its launches,
 * launches, algorithmic FLOPs (2 M N K per contraction) and minimum bytes (8 (MK + KN + MN) per
 * contraction: each operand read once, the output written once).  Any pointer may be NULL.
 * Errors: EINVAL (NULL ctx, bad kernel). */
sctm_status sctm_profile_kernel(sctm_ctx* ctx, int kernel, double* ms, long long* launches,
                                long long* flops, long long* bytes);

/* sctm_jacobi_svd -- B = U diag(S) W^T for a k x k column-major device matrix B, by the one-sided
 * Jacobi SVD that closes each warm step of the partial SVD (the k x k Rayleigh-Ritz matrix of the
 * subspace iteration; Sec. III, partial SVD by an iterative solver).  FP32 sweeps, then FP64 sweeps
 * to rounding level.  variant SCTM_JACOBI_CTA runs it in one CTA; SCTM_JACOBI_CLUSTER splits the
 * rows of the iterated matrices over a cluster of 8 CTAs (8 SMs' FP64 pipes; the engine's choice
 * for 32 <= k + (k mod 2) <= 128).  Diagnostic entry point: the engine calls the kernels itself.
 *   B            device pointer, k x k column-major, FP64 (read only)
 *   k            1 <= k <= 160 (SCTM_JACOBI_CTA); 31 <= k <= 128 (SCTM_JACOBI_CLUSTER)
 *   S            device, k values, decreasing
 *   U, W         device, k x k column-major, columns in the order of S (signs unfixed)
 *   cuda_stream  stream of the current device (NULL = legacy default); synchronised on return
 * Pointers of the host or of another device, or sizes out of range: SCTM_EINVAL.  Returns
 * SCTM_OK, SCTM_ECUSOLVER if the FP64 sweep limit was reached (the results are then the last
 * sweep's), SCTM_ENOMEM or SCTM_ECUDA.  It allocates (and frees) a status word, and for
 * SCTM_JACOBI_CTA above k = 112 one k x k scratch matrix. */
sctm_status sctm_jacobi_svd(const double* B, int k, double* S, double* U, double* W, int variant,
                            void* cuda_stream);

/* sctm_chol_orth -- one pass of the column-scaled, shifted Cholesky QR that orthonormalises the
 * partial SVD's subspace bases (Sec. III, partial SVD by an iterative solver): for the k x k
 * Gram matrix G = Y^T Y (column-major, symmetric), D = diag(G)^1/2, D^-1 G D^-1 + shift I = F^T F
 * (upper F; pivots <= 1e-20 give a zero row), T = D^-1 F^-1 (upper triangular, column-major), so
 * that Y T has orthonormal columns up to the shift and rounding.  variant SCTM_CHOL_CTA runs it
 * in one CTA; SCTM_CHOL_CLUSTER on a cluster of 8 CTAs (the engine's choice for 32 <= k <= 128),
 * with bit-identical results.  Diagnostic entry point: the engine calls the kernels itself.
 *   G      device, k x k, FP64 (read only);  T  device, k x k (written)
 *   k      1 <= k <= 160 (SCTM_CHOL_CTA); 32 <= k <= 128 (SCTM_CHOL_CLUSTER);  shift >= 0
 *   cuda_stream  stream of the current device (NULL = legacy default); synchronised on return
 * Pointers of the host or of another device, or sizes out of range: SCTM_EINVAL.  Returns
 * SCTM_OK, SCTM_ENOMEM (SCTM_CHOL_CTA above k = 112 allocates one k x k scratch matrix) or
 * SCTM_ECUDA. */
enum { SCTM_CHOL_CTA = 0, SCTM_CHOL_CLUSTER = 1 };
sctm_status sctm_chol_orth(const double* G, int k, double shift, double* T, int variant,
                           void* cuda_stream);

/* sctm_gemm -- O = X Y for row-major device matrices X (M x K), Y (K x N), O (M x N), run by the
 * library's contraction kernels in the arithmetic `precision` (SCTM_PREC_*): the FP64 kernel, or
 * the tensor-core kernel with TF32 / BF16 operands (optionally hi/lo split) and FP32
 * accumulation, the forms the move contractions of Sec. III take in the mixed modes.  The
 * elementwise error is bounded by c (|X||Y|)_ij with c about 2^-11 (TF32), 2^-8 (BF16), 2^-21
 * (TF32X3), 2^-16 (BF16X3) and the FP64 rounding for SCTM_PREC_FP64.
 *   X, Y, O      device pointers of the current device (host pointers, and memory of another
 *                GPU: SCTM_EINVAL); caller-owned
 *   M, N, K      >= 1, M*N*... each below 2^31 elements
 *   cuda_stream  cudaStream_t of the current device (NULL = legacy default; a stream of another
 *                device: SCTM_EINVAL); the call synchronises it before
 *                returning (it allocates and frees its index tables and split-K buffer)
 * Returns SCTM_OK, SCTM_EINVAL, SCTM_ENOMEM, SCTM_ECUDA, or SCTM_ETIMEOUT if a bounded wait of
 * the tensor-core kernel ran out (the result is then invalid). */
sctm_status sctm_gemm(const double* X, const double* Y, double* O, int M, int N, int K,
                      int precision, void* cuda_stream);

/* sctm_gemm_noalloc -- O = X Y in FP64 for row-major device matrices X (M x K), Y (K x N),
 * O (M x N), computed by a variant of the library's contraction kernel that allocates nothing.
 * The paper has no counterpart; it exists for callers that cannot allocate device memory: code
 * whose device memory is owned by another allocator that must not be bypassed, code that may not
 * trigger the device-wide synchronisation a cudaMalloc/cudaFree can imply, or code that runs where
 * the runtime's allocator is unavailable.  The context-based entry points allocate all their
 * buffers in sctm_create; this one uses no context.
 *   X, Y, O      device pointers of the current device (host pointers, and memory of another
 *                GPU, are rejected with SCTM_EINVAL); caller-owned
 *   M, N, K      >= 1; M*N must not exceed 2^21 (SCTM_EINVAL otherwise)
 *   cuda_stream  cudaStream_t of the current device for the work (NULL = legacy default stream;
 *                a stream of another device: SCTM_EINVAL)
 * The split-K partial sums live in one 16 MiB file-scope device array that every device loading
 * the library holds until exit.  All calls share it: calls whose work overlaps on a GPU (several
 * streams or host threads at once) race and must be serialised by the caller.  It keeps the last
 * call's contents, every value read is written earlier by the same call.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress, with that device current)
 * and keeps it for the life of the process; make that first call before any stream capture on
 * the device.  A cudaDeviceReset of the device invalidates the kept address: do not call this
 * entry point on that device again in the same process.  No cudaMalloc, cudaFree or allocating
 * library routine is called.  The result is deterministic (fixed summation order).
 * Returns SCTM_OK, SCTM_EINVAL, or SCTM_ECUDA (launch or lookup failure, or a CUDA error left
 * pending by earlier work, which is then reported without launching and left for its owner). */
sctm_status sctm_gemm_noalloc(const double* X, const double* Y, double* O, int M, int N, int K,
                              void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* SCTM_H */
