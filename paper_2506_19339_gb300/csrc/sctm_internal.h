// Internal declarations of the split-CTMRG runtime (kernels + plan executor).
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sctm.h"

namespace sctm {

// ---------------------------------------------------------------------------------------------
// Contraction launch descriptor.  A contraction O[b][m][n] = sum_k X[b][m][k] Y[b][k][n] over
// multi-indices whose element offsets are read from gather tables (one table per operand and
// index group), so any permutation of the stored legs is folded into the tile loads and the
// epilogue store: no transpose kernel ever touches memory.
// ---------------------------------------------------------------------------------------------
struct CtrLaunch {
    const double* X = nullptr;
    const double* Y = nullptr;
    double* O = nullptr;
    const int* xm = nullptr;  // [M] offsets of X along the m group
    const int* xk = nullptr;  // [K]
    const int* yk = nullptr;  // [K]
    const int* yn = nullptr;  // [N]
    const int* om = nullptr;  // [M]
    const int* on = nullptr;  // [N]
    const int* xb = nullptr;  // [nb] batch offsets (nullptr when nb == 1)
    const int* yb = nullptr;
    const int* ob = nullptr;
    int M = 1, N = 1, K = 1, nb = 1;
    const double* rowscale = nullptr;  // optional O[m][n] *= rowscale[m]
    const double* colscale = nullptr;  // optional O[m][n] *= colscale[n]
    double* partial = nullptr;         // split-K workspace, nb*splits*M*N doubles
    int splits = 1;
    int kchunk = 1;
    int precision = 0;                 // SCTM_PREC_*
    int tile = 64;                     // CTA output tile: 64 x 64 or 32 x 32 (FP64 kernel)
    int* err = nullptr;                // set to 1 by the tensor-core kernel on a wait timeout
    int tc_splits = 1, tc_kchunk = 1;  // split-K of the tensor-core kernel (128 x 64 tiles)
    double* scale_ws = nullptr;        // 2 * kScaleBlocks doubles: per-block max |X|, max |Y|
    void* pack_x = nullptr;            // tensor-core operands, converted once per launch into
    void* pack_y = nullptr;            //   hi (then lo) tiles in shared-memory image order
    int* rexp = nullptr;               // nb * (M + N) row / column exponents (SCTM_PREC_F64EMU)
    int accumulate = 0;                // FP64 kernels: O += result instead of O = result
    // tensor-core kernels: spin limit of the first mbarrier wait of each CTA (-1 = the normal
    // bound).  0 makes that wait give up at once, which exercises the timeout path (drain, error
    // flag, SCTM_ETIMEOUT) without a hang or a fault; used by the tests only.
    int first_wait_limit = -1;
};
// bytes of the packed tensor-core operands (hi and lo, TF32: the largest form)
size_t tc_pack_bytes_x(const CtrLaunch& a);
size_t tc_pack_bytes_y(const CtrLaunch& a);
// FP64 emulation on the tensor cores (ctr_emu.cu)
void launch_ctr_emu(const CtrLaunch& a, cudaStream_t s);
size_t emu_pack_bytes_x(const CtrLaunch& a);
size_t emu_pack_bytes_y(const CtrLaunch& a);
size_t emu_exp_ints(const CtrLaunch& a);
constexpr int kScaleBlocks = 152;       // blocks of the operand max-abs pass (one per SM)

void launch_ctr(const CtrLaunch& a, cudaStream_t s);
// shapes that launch_ctr (FP64) runs on the one-row-per-thread kernel
bool ctr_is_skinny(const CtrLaunch& a);
// tensor-core variant (a.precision = SCTM_PREC_TF32 / TF32X3 / BF16 / BF16X3), 128 x 64 tiles
void launch_ctr_tc(const CtrLaunch& a, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// auxiliary kernels
// ---------------------------------------------------------------------------------------------
struct NormItem {          // dst[i0*s0+i1*s1+i2*s2] = src[i] / ||src||_F, i row-major over d0,d1,d2
    const double* src;
    double* dst;
    int d0, d1, d2;
    long long s0, s1, s2;
};
void launch_normalize(const NormItem* items_dev, int count, cudaStream_t s);

void launch_splitmix_fill(double* p, long long n, unsigned long long seed, unsigned long long slot,
                          cudaStream_t s);
void launch_scalevec(const double* S, int k, double cutoff, double* out, cudaStream_t s);
// vt = 1: V holds V^T (gesvd layout); vt = 0: V holds the right vectors as columns
void launch_signfix(double* U, double* V, int n, int k, int vt, cudaStream_t s);
void launch_copy(const double* src, double* dst, long long n, cudaStream_t s);
// partial SVD (psvd.cu): column-scaled Cholesky QR pass, one-CTA Jacobi SVD, V^T -> columns
constexpr int kPsvdSmemK = 112;  // subspaces up to this size keep all k x k work in shared memory
constexpr int kPsvdMaxK = 160;   // largest subspace: above kPsvdSmemK one k x k matrix of each
                                 // one-CTA kernel lives in a global scratch buffer
// Cholesky-QR pass on the k x k Gram matrix G: the cluster kernel where chol_cluster_fits(k)
// (bit-identical to the one-CTA kernel; SCTM_CHOL=cta in the environment forces the one-CTA
// kernel), the one-CTA kernel otherwise (Xg: its global scratch above kPsvdSmemK, else null)
void launch_chol_orth(const double* G, int k, double shift, double* T, double* Xg,
                      cudaStream_t s);
void launch_chol_orth_cta(const double* G, int k, double shift, double* T, double* Xg,
                          cudaStream_t s);
bool chol_cluster_fits(int k);  // 32 <= k <= 128
void launch_chol_orth_cluster(const double* G, int k, double shift, double* T, cudaStream_t s);
void launch_refill(double* V, int n, int k, const double* S, unsigned long long seed,
                   cudaStream_t s);
// Jacobi SVD of the k x k matrix B: the cluster kernel if `cluster` and jacobi_cluster_fits(k),
// the one-CTA kernel otherwise; Vg: global scratch of the one-CTA kernel above kPsvdSmemK
// (kp (kp + 1) doubles), else null
void launch_jacobi_svd(const double* B, int k, double* S, double* U, double* W, int* info,
                       double* Vg, bool cluster, cudaStream_t s);
void launch_jacobi_svd_cta(const double* B, int k, double* S, double* U, double* W, int* info,
                           double* Vg, cudaStream_t s);
bool jacobi_cluster_fits(int k);  // 32 <= k + (k & 1) <= 128
void launch_jacobi_svd_cluster(const double* B, int k, double* S, double* U, double* W, int* info,
                               cudaStream_t s);
void launch_vt_columns(const double* VT, double* Vout, int n, int k, cudaStream_t s);
void launch_zero(double* p, long long n, cudaStream_t s);
void launch_symmetrize(double* X, int n, cudaStream_t s);   // X <- (X + X^T) / 2, n x n
// D4 group average of A[s, u, l, d, r] over its four virtual legs (out != in)
void launch_d4_project(const double* in, double* out, int p, int D, cudaStream_t s);
// flag[0] = 1 if any of p[0..n) is NaN or infinite, else 0
void launch_check_finite(const double* p, long long n, int* flag, cudaStream_t s);
// p[i] <- 0 where p[i] is not finite, and *flag <- 1 if any was (flag is never cleared here)
void launch_sanitize(double* p, long long n, int* flag, cudaStream_t s);
void launch_spectrum_update(const double* Sraw, const double* rho, int chi, double* S_old,
                            double* dS_out, cudaStream_t s);
// lnk[0] = ln(Z11 Z00 / (Z10 Z01)) (NaN if the ratio is <= 0 or not finite), lnk[1] = Z11
void launch_lnkappa(const double* Z00, const double* Z10, const double* Z01, const double* Z11,
                    double* lnk, cudaStream_t s);
// out[0] = -T (lnk_num - lnk_den)
void launch_free_energy(const double* lnk_num, const double* lnk_den, double T, double* out,
                        cudaStream_t s);
// g = -T (dnum - dden): the adjoint gradient from the two networks' d ln kappa / dA
void launch_adj_combine(const double* dnum, const double* dden, double T, int n, double* g,
                        cudaStream_t s);
// g = -2T (Enum / Z11num - Eden / Z11den)
void launch_grad_combine(const double* Enum, const double* lnk_num, const double* Eden,
                         const double* lnk_den, double T, int n, double* g, cudaStream_t s);

}  // namespace sctm
