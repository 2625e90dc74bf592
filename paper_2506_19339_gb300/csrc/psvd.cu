// Kernels of the partial SVD (Sec. III: the largest chi singular triplets of the projector
// matrix M by an iterative solver instead of a full decomposition).
//
// The projector matrix changes little from one CTMRG iteration to the next, so its leading
// right singular subspace of the previous iteration (k = chi + oversampling columns) is a warm
// start.  One warm solve is a two-sided subspace iteration step with a Rayleigh-Ritz
// extraction:
//     Y = M V_prev,    Q_y = orth(Y)       (left subspace)
//     Z = M^T Q_y,     Q_z = orth(Z)       (right subspace, one step of M^T M further)
//     B = Z^T Q_z = Q_y^T M Q_z  (k x k),  B = U_B S V_B^T
//     M ~ (Q_y U_B) S (Q_z V_B)^T.
// The products with M, the Gram matrices and the basis updates run on the contraction kernel;
// the kernels here do the k x k work, each in one CTA, and (further down) each also on a
// thread-block cluster of 8 CTAs that spreads the FP64 work over 8 SMs:
//   * chol_orth_kernel: one pass of column-scaled Cholesky QR.  With G = Y^T Y and D the column
//     norms, D^-1 G D^-1 + shift I = R^T R; it returns T = D^-1 R^-1, so that Y T is orthonormal
//     up to the shift and rounding.  Column scaling keeps the relative accuracy of small
//     columns (Y ~ U S in the warm regime).  Columns of the tail directions are dominated by the
//     change of M since the last iteration and can be numerically dependent; the shift
//     (Fukaya et al.'s shifted Cholesky QR: 11 (n k + k (k + 1)) u on the unit-diagonal scaled
//     Gram matrix) keeps the factorisation positive definite, so three passes -- shifted,
//     shifted, plain -- give an orthonormal basis without dropping columns.  A column that is
//     exactly zero stays zero (pivot below 1e-20); refill_kernel puts a pseudo-random vector in
//     its place before the next solve.
//   * jacobi_svd_kernel: one-sided (Hestenes) Jacobi SVD of B, round-robin ordering of the
//     k(k-1)/2 column pairs.  FP64 arithmetic is scarce on this GPU (about 1/64 of FP32), so the
//     sweeps run first in FP32 (which converges W to about 1e-6), W is re-orthonormalised in FP64
//     (Cholesky of W^T W), A = B W is formed in FP64 and FP64 sweeps finish from there: Jacobi
//     converges quadratically, so one or two FP64 sweeps reach rounding level.  B's columns are
//     the rows of the triangular factor of Z, graded by the singular values, which is the
//     ordering under which one-sided Jacobi converges fastest.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "sctm_internal.h"

namespace sctm {

namespace cg = cooperative_groups;

namespace {

constexpr int kPsvdThreads = 512;
constexpr int kJacobiMaxSweeps32 = 12;
// FP64 sweeps: distinct values converge quadratically (two sweeps after the FP32 phase); values
// graded down to ~1e-12 of the largest, which the FP32 phase cannot resolve, measured up to 17
// sweeps in a host simulation.  Reaching the limit is reported (SCTM_ECUSOLVER).
constexpr int kJacobiMaxSweeps64 = 30;
constexpr double kPivotFloor = 1e-20;

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// In-place right-looking Cholesky of the symmetric k x k matrix in R (row-major, upper triangle
// used).  Rows are left unscaled: on return the upper factor is F[j][c] = R[j][c] * rinv[j]
// (c >= j), F[j][j] = R[j][j] * rinv[j] = sqrt(pivot j).  Pivots at or below kPivotFloor give
// rinv = 0 (a zero row).  The reciprocal square root is taken by one thread: FP64 is scarce on
// this GPU and a redundant evaluation by every thread costs as much as the update.
__device__ void block_cholesky(double* R, double* rinv, int k) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            const double piv = R[j * k + j];
            rinv[j] = piv > kPivotFloor ? 1.0 / sqrt(piv) : 0.0;
        }
        __syncthreads();
        const double ri = rinv[j];
        const double r2 = ri * ri;
        const int lane = tid & 31, nw = nt >> 5;
        for (int a = j + 1 + (tid >> 5); a < k; a += nw) {
            const double fa = R[j * k + a] * r2;
            for (int b = a + lane; b < k; b += 32) R[a * k + b] -= fa * R[j * k + b];
        }
        __syncthreads();
    }
}

// Scratch of one Jacobi round, one entry per column pair.
struct RoundScratch {
    double* c;   // cosine of each pair's rotation (as the sweep's type)
    double* s;   // sine (as the sweep's type)
    int* act;    // 1 if the pair rotates
    int* pi;     // the pair's columns i, j (this round)
    int* pj;
};

// One sweep of one-sided Jacobi rotations over all column pairs (circle-method rounds) of the
// kp x kp column-major matrix A (leading dimension ld), accumulating into V (same layout).  Per
// round: thread q < kp/2 forms pair q's three dot products and its rotation (one pair per
// thread, so the FP64 square roots and divisions are not repeated across a warp), then every
// thread applies the rotations, one (pair, row) element at a time.  Pairs with
// |a_i . a_j| <= tol |a_i| |a_j| are left alone.  Returns (to every thread) the largest
// |a_i . a_j| / (|a_i| |a_j|) seen.
template <typename F>
__device__ float jacobi_sweep(F* A, F* V, int kp, int ld, F tol, RoundScratch rs, float* s_max) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int np = kp / 2;
    if (tid == 0) *s_max = 0.0f;
    float wmax = 0.0f;
    for (int round = 0; round < kp - 1; ++round) {
        for (int q = tid; q < np; q += nt) {
            const int p0 = q, p1 = kp - 1 - q;
            const int i = p0 == 0 ? 0 : 1 + (p0 - 1 + round) % (kp - 1);
            const int j = 1 + (p1 - 1 + round) % (kp - 1);
            const F* ai = A + (long long)i * ld;
            const F* aj = A + (long long)j * ld;
            F al = 0, be = 0, ga = 0;
            for (int r = 0; r < kp; ++r) {
                const F x = ai[r], y = aj[r];
                al = fma(x, x, al);
                be = fma(y, y, be);
                ga = fma(x, y, ga);
            }
            int act = 0;
            F c = 1, sn = 0;
            if (al > F(0) && be > F(0)) {
                const F rel = fabs(ga) / (sqrt(al) * sqrt(be));
                wmax = fmaxf(wmax, (float)rel);
                if (rel > tol) {
                    const F zeta = (be - al) / (F(2) * ga);
                    const F t = (zeta >= F(0) ? F(1) : F(-1)) / (fabs(zeta) + sqrt(F(1) + zeta * zeta));
                    c = F(1) / sqrt(F(1) + t * t);
                    sn = c * t;
                    act = 1;
                }
            }
            // stored in the sweep's own type (np doubles of room hold np values of either):
            // a float <-> double conversion runs on the FP64 pipe of this GPU
            reinterpret_cast<F*>(rs.c)[q] = c;
            reinterpret_cast<F*>(rs.s)[q] = sn;
            rs.act[q] = act;
            rs.pi[q] = i;
            rs.pj[q] = j;
        }
        __syncthreads();
        // rotations: warp per pair, lane per row (no integer division in the inner loop)
        for (int q = tid >> 5; q < np; q += nt >> 5) {
            if (!rs.act[q]) continue;
            const F c = reinterpret_cast<const F*>(rs.c)[q], sn = reinterpret_cast<const F*>(rs.s)[q];
            F* ai = A + (long long)rs.pi[q] * ld;
            F* aj = A + (long long)rs.pj[q] * ld;
            F* vi = V + (long long)rs.pi[q] * ld;
            F* vj = V + (long long)rs.pj[q] * ld;
            for (int r = tid & 31; r < kp; r += 32) {
                const F x = ai[r], y = aj[r];
                ai[r] = c * x - sn * y;
                aj[r] = sn * x + c * y;
                const F u = vi[r], w = vj[r];
                vi[r] = c * u - sn * w;
                vj[r] = sn * u + c * w;
            }
        }
        __syncthreads();
    }
    // relative values are non-negative, so their float bits order as integers
    for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (lane == 0) atomicMax((int*)s_max, __float_as_int(wmax));
    __syncthreads();
    const float r = *s_max;
    __syncthreads();
    return r;
}

}  // namespace

// G (k x k, column-major G[i + j k]) -> T (k x k, column-major, upper triangular) with Y T
// orthonormal (up to the shift) for the Y that gave G = Y^T Y.  Shared memory: chol_orth_smem(k).
//
// This SM retires two FP64 lane-operations per cycle, so the kernel is organised around few
// FP64 instructions and few block barriers: a blocked right-looking Cholesky (warp 0 factors a
// block of kCholNB rows -- pivots, the block's own rows, its scaled pivot rows -- under warp
// synchronisation only; then every warp applies the block's kCholNB rank-one terms to the
// trailing rows at once: two barriers per block instead of two per row), the factor's rows
// scaled once, and the inverse factor by column back substitution with a warp per column.
constexpr int kCholNB = 16;

__global__ void __launch_bounds__(kPsvdThreads)
    chol_orth_kernel(const double* __restrict__ G, int k, double shift, double* __restrict__ T,
                     double* Xg) {
    extern __shared__ double sm[];
    double* R = sm;                        // row-major k x k: scaled Gram, then the factor rows
    double* X = Xg ? Xg : sm + k * k;      // row-major k x k: F^-1 (global above kPsvdSmemK)
    double* d = sm + (Xg ? 1 : 2) * k * k; // reciprocal column norms
    double* rinv = d + k;                  // reciprocal pivots
    double* P = X;                         // kCholNB x k scaled pivot rows (X is free until then)
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    for (int i = tid; i < k; i += nt) {  // d = 1 / column norm (0 for a zero column)
        const double g = G[i + (long long)i * k];
        d[i] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
    }
    __syncthreads();
    // G is a Gram matrix, symmetric bit for bit (each entry sums the same products in the same
    // order), so the row-major R can be read from G's column-major storage element for element
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        R[e] = G[e] * d[i] * d[j] + ((i == j && d[i] > 0.0) ? shift : 0.0);
    }
    __syncthreads();
    // Cholesky R = F^T F of the upper triangle, rows left unscaled: F[j][c] = R[j][c] rinv[j]
    // (c >= j).  A pivot at or below kPivotFloor gives rinv = 0 (a zero row).
    for (int j0 = 0; j0 < k; j0 += kCholNB) {
        const int j1 = min(j0 + kCholNB, k);
        if (warp == 0) {
            for (int j = j0; j < j1; ++j) {
                double ri = 0.0;
                if (lane == 0) {
                    const double piv = R[j * k + j];
                    ri = piv > kPivotFloor ? 1.0 / sqrt(piv) : 0.0;
                    rinv[j] = ri;
                }
                ri = __shfl_sync(0xffffffffu, ri, 0);
                const double r2 = ri * ri;
                for (int a = j + 1; a < j1; ++a) {  // the block's own later rows, all columns
                    const double fa = R[j * k + a] * r2;
                    for (int b = a + lane; b < k; b += 32) R[a * k + b] -= fa * R[j * k + b];
                }
                for (int b = j1 + lane; b < k; b += 32) P[(j - j0) * k + b] = R[j * k + b] * r2;
                __syncwarp();
            }
        }
        __syncthreads();
        // trailing rows a >= j1: R[a][b] -= sum_j P[j][a] R[j][b], the same terms in the same
        // order as one rank-one update per pivot
        const int nb = j1 - j0;
        for (int a = j1 + warp; a < k; a += nw) {
            double pa[kCholNB];
#pragma unroll
            for (int q = 0; q < kCholNB; ++q) pa[q] = q < nb ? P[q * k + a] : 0.0;
            for (int b = a + lane; b < k; b += 32) {
                double acc = R[a * k + b];
#pragma unroll
                for (int q = 0; q < kCholNB; ++q)
                    if (q < nb) acc -= pa[q] * R[(j0 + q) * k + b];
                R[a * k + b] = acc;
            }
        }
        __syncthreads();
    }
    // F's off-diagonal part, transposed into R's unused lower triangle: R[l][r] = F[r][l] =
    // R[r][l] rinv[r] (r < l), so that the columns of F the back substitution walks are rows
    for (int e = tid; e < k * k; e += nt) {
        const int l = e / k, r = e % k;
        if (r < l) R[e] = R[r * k + l] * rinv[r];
    }
    __syncthreads();
    // X = F^-1, stored by columns (X[c k + r] = (F^-1)[r][c]), column c by back substitution
    // (F[l][l] = 1 / rinv[l]): x = e_c, then for l = c down to 0: x_l <- x_l rinv[l] and
    // x_r -= F[r][l] x_l for r < l.  A warp per column; its lanes walk r, so both the column of
    // X and the column of F they touch are consecutive in shared memory.
    for (int c = warp; c < k; c += nw) {
        double* x = X + (long long)c * k;
        for (int r = lane; r < k; r += 32) x[r] = r == c ? 1.0 : 0.0;
        __syncwarp();
        for (int l = c; l >= 0; --l) {
            const double xl = x[l] * rinv[l];
            __syncwarp();
            if (lane == 0) x[l] = xl;
            const double* fl = R + (long long)l * k;  // F[r][l] for r < l
            for (int r = lane; r < l; r += 32) x[r] -= fl[r] * xl;
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {  // T = D^-1 F^-1, column-major
        const int i = e % k, j = e / k;
        T[e] = j >= i ? X[e] * d[i] : 0.0;
    }
}

// ---------------------------------------------------------------------------------------------
// The same Cholesky-QR pass spread over a thread-block cluster of kCcCluster CTAs.
//
// CTA c holds rows [c rp, (c + 1) rp) of the scaled Gram matrix R (rp = ceil(k / 8)).  The
// factorisation goes panel by panel, a panel being one CTA's rows: the owner factors its rows
// (each pivot's rank-one update applied to the panel's later rows), one cluster barrier, and
// every later CTA applies the panel's rank-one updates to its own rows, reading the panel's rows
// from the owner's shared memory.  Each element R[a][b] receives the updates of the pivots
// j < a in pivot order, each as one fused multiply-add with the factor R[j][a] rinv[j]^2 -- the
// operations of chol_orth_kernel in the same order -- so the factor is bit-identical.  Then every
// CTA gathers F (upper triangle, transposed) and the reciprocal pivots, and computes the columns
// c = rank, rank + 8, ... of F^-1 by the same back substitution (a warp per column), writing its
// columns of T = D^-1 F^-1.
// ---------------------------------------------------------------------------------------------
constexpr int kCcCluster = 8;
constexpr int kCcThreads = 256;
constexpr int kCcMinK = 32;
constexpr int kCcMaxK = 128;

namespace {
struct CcLayout {  // shared-memory carve-up of one CTA, in doubles from the base
    int k, rp;
    long long rl, ft, d, rinv, xcol, pl, prinv, doubles;
    __host__ __device__ explicit CcLayout(int k_) : k(k_) {
        rp = (k + kCcCluster - 1) / kCcCluster;
        rl = 0;                             // own rows of R, row-major (stride k)
        ft = rl + (long long)rp * k;        // F transposed: ft[l k + r] = F[r][l], r < l
        d = ft + (long long)k * k;          // reciprocal column norms
        rinv = d + k;                       // reciprocal pivots (all rows after the gather)
        xcol = rinv + k;                    // one column of F^-1 per warp
        pl = xcol + (long long)(kCcThreads / 32) * k;  // a copy of the current panel's rows
        prinv = pl + (long long)rp * k;     //   and of their reciprocal pivots
        doubles = prinv + rp;
    }
    __host__ __device__ size_t bytes() const { return (size_t)doubles * sizeof(double); }
};
}  // namespace

__global__ void __cluster_dims__(kCcCluster, 1, 1) __launch_bounds__(kCcThreads)
    chol_orth_cluster_kernel(const double* __restrict__ G, int k, double shift,
                             double* __restrict__ T) {
    cg::cluster_group cluster = cg::this_cluster();
    const CcLayout L(k);
    if (k < 1 || k > kCcMaxK) return;  // uniform over the cluster (the launcher checks)
    extern __shared__ double sm[];
    const int crank = (int)cluster.block_rank();
    const int rp = L.rp;
    const int row0 = min(k, crank * rp);
    const int nr = min(k, row0 + rp) - row0;
    double* Rl = sm + L.rl;
    double* Ft = sm + L.ft;
    double* d = sm + L.d;
    double* rinv = sm + L.rinv;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    for (int i = tid; i < k; i += nt) {  // d = 1 / column norm (0 for a zero column)
        const double g = G[i + (long long)i * k];
        d[i] = g > 0.0 ? 1.0 / sqrt(g) : 0.0;
    }
    __syncthreads();
    // own rows of the scaled Gram matrix plus the shift (G symmetric bit for bit: row a is read
    // as G's column a)
    for (int e = tid; e < nr * k; e += nt) {
        const int a = row0 + e / k, b = e % k;
        Rl[e] = G[b + (long long)a * k] * d[a] * d[b] + ((a == b && d[a] > 0.0) ? shift : 0.0);
    }
    __syncthreads();
    for (int p = 0; p < kCcCluster; ++p) {
        const int p0 = min(k, p * rp), p1 = min(k, p0 + rp);
        if (crank == p) {  // factor this CTA's rows: pivot j, then its update of rows j+1 .. p1-1
            for (int j = p0; j < p1; ++j) {
                const int lj = j - row0;
                if (tid == 0) {
                    const double piv = Rl[lj * k + j];
                    rinv[j] = piv > kPivotFloor ? 1.0 / sqrt(piv) : 0.0;
                }
                __syncthreads();
                const double ri = rinv[j];
                const double r2 = ri * ri;
                for (int e = tid; e < (p1 - j - 1) * k; e += nt) {
                    const int a = j + 1 + e / k, b = e % k;
                    if (b < a) continue;
                    const double fa = Rl[lj * k + a] * r2;
                    Rl[(a - row0) * k + b] -= fa * Rl[lj * k + b];
                }
                __syncthreads();
            }
        }
        cluster.sync();  // panel p is final (its rows are never written again)
        if (crank > p && p1 > p0) {
            // the panel's rows and pivots, copied from the owner's shared memory
            double* Pl = sm + L.pl;
            double* Pr = sm + L.prinv;
            const double* Rp = cluster.map_shared_rank(Rl, p);
            const double* rinvp = cluster.map_shared_rank(rinv, p);
            for (int e = tid; e < (p1 - p0) * k; e += nt) Pl[e] = Rp[e];
            for (int j = tid; j < p1 - p0; j += nt) Pr[j] = rinvp[p0 + j];
            __syncthreads();
            for (int e = tid; e < nr * k; e += nt) {
                const int a = row0 + e / k, b = e % k;
                if (b < a) continue;
                double acc = Rl[e];
                for (int j = 0; j < p1 - p0; ++j) {
                    const double ri = Pr[j];
                    const double pa = Pl[j * k + a] * (ri * ri);
                    acc -= pa * Pl[j * k + b];
                }
                Rl[e] = acc;
            }
            __syncthreads();
        }
    }
    // gather every reciprocal pivot and F's off-diagonal part, transposed:
    // Ft[l k + r] = F[r][l] = R[r][l] rinv[r] (r < l)
    for (int j = tid; j < k; j += nt) {
        const int o = j / rp;
        if (o != crank) rinv[j] = cluster.map_shared_rank(rinv, o)[j];
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        const int l = e / k, r = e % k;
        if (r < l) {
            const int o = r / rp;
            Ft[e] = cluster.map_shared_rank(Rl, o)[(r - o * rp) * k + l] * rinv[r];
        }
    }
    __syncthreads();
    // columns c = crank, crank + 8, ... of X = F^-1 by back substitution (the one-CTA kernel's
    // order), then T = D^-1 X
    double* x = sm + L.xcol + (long long)warp * k;
    for (int c = crank + kCcCluster * warp; c < k; c += kCcCluster * nw) {
        for (int r = lane; r < k; r += 32) x[r] = r == c ? 1.0 : 0.0;
        __syncwarp();
        for (int l = c; l >= 0; --l) {
            const double xl = x[l] * rinv[l];
            __syncwarp();
            if (lane == 0) x[l] = xl;
            const double* fl = Ft + (long long)l * k;
            for (int r = lane; r < l; r += 32) x[r] -= fl[r] * xl;
            __syncwarp();
        }
        for (int i = lane; i < k; i += 32) T[i + (long long)c * k] = c >= i ? x[i] * d[i] : 0.0;
        __syncwarp();
    }
    cluster.sync();  // no CTA exits while another may still read its shared memory
}

// SVD of B (k x k, column-major): B W = A with orthogonal columns, B = U S W^T, U = A S^-1.
// Writes S (k, decreasing), U and W (k x k, column-major, columns in the order of S).
// info: 0, or 1 if the FP64 sweep limit was reached.  kp = k rounded up to even (an odd k gets a
// zero column that is never rotated); columns are stored with the odd leading dimension
// ld = kp + 1 so that the threads of the dot-product phase, which read different columns, hit
// different shared-memory banks.  Shared memory: jacobi_svd_smem(k).
__global__ void __launch_bounds__(kPsvdThreads)
    jacobi_svd_kernel(const double* __restrict__ B, int k, double* __restrict__ S,
                      double* __restrict__ U, double* __restrict__ W, int* info, double* Vg) {
    extern __shared__ double sm[];
    const int kp = k + (k & 1), ld = kp + 1, np = kp / 2;
    double* A = sm;                        // FP64 phase: column j at A + j ld
    double* V = Vg ? Vg : sm + kp * ld;    // W, column j at V + j ld (global above kPsvdSmemK)
    float* A32 = (float*)A;                // FP32 phase: both FP32 matrices inside A's space
    float* V32 = A32 + kp * ld;
    double* sig = sm + (Vg ? 1 : 2) * kp * ld;
    RoundScratch rs;
    rs.c = sig + kp;
    rs.s = rs.c + np;
    int* rank = (int*)(rs.s + np);
    rs.act = rank + kp;
    rs.pi = rs.act + np;
    rs.pj = rs.pi + np;
    __shared__ float s_max;
    __shared__ int s_exp;
    __shared__ double s_wmax[kPsvdThreads / 32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    int bad = 0;

    // 0. scale: B 2^-ex has entries below 1 in magnitude (exact; FP32 squares stay in range)
    {
        double m = 0.0;
        for (int e = tid; e < k * k; e += nt) m = fmax(m, fabs(B[e]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_wmax[warp] = m;
        __syncthreads();
        if (tid == 0) {
            double mm = 0.0;
            for (int w = 0; w < nw; ++w) mm = fmax(mm, s_wmax[w]);
            int e2 = 0;
            if (mm > 0.0 && isfinite(mm)) frexp(mm, &e2);  // mm < 2^e2
            s_exp = e2;
        }
        __syncthreads();
    }
    const int ex = s_exp;
    // 1. FP32 sweeps on B 2^-ex, until no pair is above the FP32 rounding level of a kp-term dot
    //    product
    for (int e = tid; e < kp * kp; e += nt) {
        const int r = e % kp, c = e / kp;
        A32[c * ld + r] = (r < k && c < k) ? (float)ldexp(B[r + (long long)c * k], -ex) : 0.0f;
        V32[c * ld + r] = (r == c) ? 1.0f : 0.0f;
    }
    __syncthreads();
    const float tol32 = 4.0f * (float)kp * 5.9604645e-8f;
    bool w_is_identity = false;  // the first FP32 sweep found every pair orthogonal: W = I
    for (int sw = 0; sw < kJacobiMaxSweeps32; ++sw)
        if (jacobi_sweep<float>(A32, V32, kp, ld, tol32, rs, &s_max) <= tol32) {
            w_is_identity = sw == 0;  // no rotation was made (uniform: s_max is shared)
            break;
        }
    if (w_is_identity) {
        // a warm solve whose B already has orthogonal columns to FP32 accuracy: W = I and
        // A = B 2^-ex exactly, which steps 2 and 3 below would also produce
        __syncthreads();
        for (int e = tid; e < kp * kp; e += nt) {
            const int r = e % kp, c = e / kp;
            V[c * ld + r] = r == c ? 1.0 : 0.0;
            A[c * ld + r] = (r < k && c < k) ? ldexp(B[r + (long long)c * k], -ex) : 0.0;
        }
        __syncthreads();
    } else {
    // 2. W = V32 in FP64, re-orthonormalised: W <- W F^-1 with F^T F = W^T W
    for (int e = tid; e < kp * kp; e += nt) {
        const int r = e % kp, c = e / kp;
        V[c * ld + r] = (double)V32[c * ld + r];
    }
    __syncthreads();
    for (int e = tid; e < kp * kp; e += nt) {  // A (row-major, stride kp) = W^T W
        const int i = e / kp, j = e % kp;
        double v = 0.0;
        for (int l = 0; l < kp; ++l) v = fma(V[i * ld + l], V[j * ld + l], v);
        A[e] = v;
    }
    __syncthreads();
    double* rinv = sig;  // reciprocal pivots, until the singular values are written
    block_cholesky(A, rinv, kp);
    // row r of W: x F = w_r in place (forward substitution), F[i][j] = A[i][j] rinv[i]
    for (int r = tid; r < kp; r += nt) {
        for (int j = 0; j < kp; ++j) {
            double acc = V[j * ld + r];
            for (int i = 0; i < j; ++i) acc -= V[i * ld + r] * (A[i * kp + j] * rinv[i]);
            V[j * ld + r] = acc * rinv[j];
        }
    }
    __syncthreads();
    // 3. A = B W 2^-ex in FP64
    for (int e = tid; e < kp * kp; e += nt) {
        const int r = e % kp, c = e / kp;
        double v = 0.0;
        if (r < k)
            for (int l = 0; l < k; ++l) v = fma(B[r + (long long)l * k], V[c * ld + l], v);
        A[c * ld + r] = ldexp(v, -ex);
    }
    __syncthreads();
    }
    // 4. FP64 sweeps; tol64 = kp eps is the rounding level of a kp-term dot product.  Jacobi
    //    converges quadratically, so a sweep whose largest relative off-diagonal value was below
    //    1e-6 leaves them near 1e-12: it is the last (one FP64 sweep costs about 1.5 ms of the
    //    SM's FP64 pipe at k = 80, most of a warm solve)
    const double tol64 = (double)kp * 2.220446049250313e-16;
    {
        int sw = 0;
        for (; sw < kJacobiMaxSweeps64; ++sw) {
            const float mx = jacobi_sweep<double>(A, V, kp, ld, tol64, rs, &s_max);
            if (mx <= tol64 || mx < 1e-6f) break;
        }
        if (sw >= kJacobiMaxSweeps64) bad = 1;
    }
    // 5. singular values = column norms, ranks by decreasing value (ties: lower index first)
    for (int c = warp; c < k; c += nw) {
        double v = 0.0;
        for (int r = lane; r < kp; r += 32) v = fma(A[c * ld + r], A[c * ld + r], v);
        v = warp_allsum(v);
        if (lane == 0) sig[c] = sqrt(v);  // of B 2^-ex
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        int rk = 0;
        for (int o = 0; o < k; ++o)
            if (sig[o] > sig[c] || (sig[o] == sig[c] && o < c)) ++rk;
        rank[c] = rk;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        const int r = e % k, c = e / k;
        const int dst = r + rank[c] * k;
        const double sc = sig[c];
        U[dst] = sc > 0.0 ? A[c * ld + r] / sc : 0.0;
        W[dst] = V[c * ld + r];
    }
    for (int c = tid; c < k; c += nt) S[rank[c]] = ldexp(sig[c], ex);
    if (tid == 0 && info) *info = bad;
}

// ---------------------------------------------------------------------------------------------
// The same one-sided Jacobi SVD spread over a thread-block cluster of kJcCluster CTAs.
//
// One SM retires two FP64 lane-operations per cycle, so the one-CTA kernel above is bound by its
// SM's FP64 pipe (about 1.5 ms per FP64 sweep at k = 80).  Here the rows of A (= B W) and of W
// are split across the cluster: CTA c keeps rows [c rows_per, (c + 1) rows_per) of both in its
// shared memory.  A round of the circle method then costs, per CTA, the dot products and the
// rotations of its own rows only:
//   1. every CTA forms, for each of the kp/2 pairs of the round, the three partial dot products
//      a_i.a_i, a_j.a_j, a_i.a_j over its rows (one buffer of 3 kp/2 values, two alternating
//      buffers so that a round's writes never meet the previous round's reads);
//   2. one cluster barrier; every CTA reads the partial sums of all CTAs through distributed
//      shared memory and adds them in cluster-rank order, so every CTA holds bit-identical sums
//      and computes bit-identical rotations (FP64 angles, the formulas of jacobi_sweep) and
//      bit-identical convergence decisions: the loops stay in step without further exchange;
//   3. every CTA rotates its own rows of A and W.
// W's re-orthonormalisation after the FP32 sweeps is two Newton-Schulz steps
// W <- W (3 I - W^T W) / 2 (the Gram matrix reduced over the cluster: a reduce-scatter and an
// all-gather through distributed shared memory), A = B W reads the rows of W from their owners,
// and the singular values are column norms summed over the cluster.  Results agree with the
// one-CTA kernel to rounding (the dot products are summed in another order).
// ---------------------------------------------------------------------------------------------
constexpr int kJcCluster = 8;                      // CTAs per cluster (the portable maximum)
constexpr int kJcThreads = 256;
constexpr int kJcMaxKp = 128;                      // the k x k Gram matrix fits in shared memory
constexpr int kJcMaxRows = kJcMaxKp / kJcCluster;  // rows of A and W per CTA, at most
constexpr int kJcMinKp = 32;                       // smaller orders stay on the one-CTA kernel
constexpr int kJcNsSteps = 2;                      // Newton-Schulz steps (1e-5 -> 1e-10 -> eps)

namespace {

struct JcLayout {  // shared-memory carve-up of one CTA, in doubles from the base
    int kp, np, rows_per, un, slice_n;
    long long al, vl, un_off, slice, part, cpart, sig, rc, rsn, ints;
    long long doubles;
    __host__ __device__ explicit JcLayout(int k) {
        kp = k + (k & 1);
        np = kp / 2;
        rows_per = (kp + kJcCluster - 1) / kJcCluster;
        un = kp * kp > rows_per * kp ? kp * kp : rows_per * kp;
        slice_n = (kp * kp + kJcCluster - 1) / kJcCluster;
        al = 0;
        vl = al + (long long)rows_per * kp;
        un_off = vl + (long long)rows_per * kp;
        slice = un_off + un;
        part = slice + slice_n;  // 2 buffers x 3 values x np pairs
        cpart = part + 3LL * kp;
        sig = cpart + kp;
        rc = sig + kp;
        rsn = rc + np;
        ints = rsn + np;         // rank[kp], act[np], pi[np], pj[np]
        doubles = ints;
    }
    __host__ __device__ size_t bytes() const {
        return (size_t)doubles * sizeof(double) + (size_t)(kp + 3 * np) * sizeof(int);
    }
};

// One sweep over all column pairs of the kp x kp matrix whose rows [row0, row0 + nr) this CTA
// holds (Al, Vl: row-major, row stride kp).  part: two alternating buffers of 3 np values of F;
// buf selects the one the next round writes.  Returns to every thread of every CTA the largest
// relative off-diagonal value |a_i . a_j| / (|a_i| |a_j|) of the sweep (identical in all CTAs).
template <typename F>
__device__ float cluster_sweep(cg::cluster_group& cluster, F* Al, F* Vl, int nr, int kp, F tol,
                               F* part, int& buf, RoundScratch rs, float* s_max) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const int np = kp / 2;
    if (tid == 0) *s_max = 0.0f;
    float wmax = 0.0f;
    for (int round = 0; round < kp - 1; ++round) {
        F* pb = part + (long long)buf * 3 * np;
        // 1. partial dot products of this CTA's rows
        for (int q = tid; q < np; q += nt) {
            const int p0 = q, p1 = kp - 1 - q;
            const int i = p0 == 0 ? 0 : 1 + (p0 - 1 + round) % (kp - 1);
            const int j = 1 + (p1 - 1 + round) % (kp - 1);
            F al = 0, be = 0, ga = 0;
            for (int r = 0; r < nr; ++r) {
                const F x = Al[r * kp + i], y = Al[r * kp + j];
                al = fma(x, x, al);
                be = fma(y, y, be);
                ga = fma(x, y, ga);
            }
            pb[3 * q] = al;
            pb[3 * q + 1] = be;
            pb[3 * q + 2] = ga;
            rs.pi[q] = i;
            rs.pj[q] = j;
        }
        cluster.sync();
        // 2. the cluster's sums in rank order, then the rotation of every pair (in every CTA)
        for (int q = tid; q < np; q += nt) {
            F al = 0, be = 0, ga = 0;
            for (int src = 0; src < kJcCluster; ++src) {
                const F* rp = cluster.map_shared_rank(pb, src);
                al += rp[3 * q];
                be += rp[3 * q + 1];
                ga += rp[3 * q + 2];
            }
            int act = 0;
            F c = 1, sn = 0;
            if (al > F(0) && be > F(0)) {
                const F rel = fabs(ga) / (sqrt(al) * sqrt(be));
                wmax = fmaxf(wmax, (float)rel);
                if (rel > tol) {
                    const F zeta = (be - al) / (F(2) * ga);
                    const F t = (zeta >= F(0) ? F(1) : F(-1)) / (fabs(zeta) + sqrt(F(1) + zeta * zeta));
                    c = F(1) / sqrt(F(1) + t * t);
                    sn = c * t;
                    act = 1;
                }
            }
            reinterpret_cast<F*>(rs.c)[q] = c;
            reinterpret_cast<F*>(rs.s)[q] = sn;
            rs.act[q] = act;
        }
        __syncthreads();
        // 3. rotations of this CTA's rows of A and W, one (pair, row) element per thread
        for (int e = tid; e < np * nr; e += nt) {
            const int q = e % np, r = e / np;
            if (!rs.act[q]) continue;
            const F c = reinterpret_cast<const F*>(rs.c)[q], sn = reinterpret_cast<const F*>(rs.s)[q];
            F* a = Al + r * kp;
            F* v = Vl + r * kp;
            const int i = rs.pi[q], j = rs.pj[q];
            const F x = a[i], y = a[j];
            a[i] = c * x - sn * y;
            a[j] = sn * x + c * y;
            const F u = v[i], w = v[j];
            v[i] = c * u - sn * w;
            v[j] = sn * u + c * w;
        }
        __syncthreads();
        buf ^= 1;
    }
    for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    if (lane == 0) atomicMax((int*)s_max, __float_as_int(wmax));
    __syncthreads();
    const float r = *s_max;
    __syncthreads();
    return r;
}

}  // namespace

// B (k x k, column-major) -> S (k, decreasing), U, W (k x k, column-major, columns in the order
// of S) with B = U diag(S) W^T; info: 0, or 1 if the FP64 sweep limit was reached.  Launched as
// one cluster of kJcCluster CTAs; kJcMinKp <= k + (k & 1) <= kJcMaxKp.  Shared memory:
// JcLayout(k).bytes().  Every loop that contains a cluster barrier runs the same number of times
// in every CTA (its trip count depends only on k and on values every CTA computes identically).
__global__ void __cluster_dims__(kJcCluster, 1, 1) __launch_bounds__(kJcThreads)
    jacobi_svd_cluster_kernel(const double* __restrict__ B, int k, double* __restrict__ S,
                              double* __restrict__ U, double* __restrict__ W, int* info) {
    cg::cluster_group cluster = cg::this_cluster();
    const JcLayout L(k);
    const int kp = L.kp, np = L.np, rows_per = L.rows_per;
    if (kp < 2 || kp > kJcMaxKp) return;  // uniform over the cluster (the launcher checks)
    extern __shared__ double sm[];
    const int crank = (int)cluster.block_rank();
    const int row0 = min(kp, crank * rows_per);
    const int nr = min(kp, row0 + rows_per) - row0;  // rows of this CTA (0 for trailing CTAs)
    double* Al = sm + L.al;
    double* Vl = sm + L.vl;
    double* Un = sm + L.un_off;  // FP32 rows, then the Gram matrix, then B's rows
    double* slice = sm + L.slice;
    double* part = sm + L.part;
    double* cpart = sm + L.cpart;
    double* sig = sm + L.sig;
    RoundScratch rs;
    rs.c = sm + L.rc;
    rs.s = sm + L.rsn;
    int* rank = (int*)(sm + L.ints);
    rs.act = rank + kp;
    rs.pi = rs.act + np;
    rs.pj = rs.pi + np;
    float* A32 = (float*)Un;
    float* V32 = A32 + rows_per * kp;
    __shared__ float s_max;
    __shared__ int s_exp;
    __shared__ double s_wmax[kJcThreads / 32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    int bad = 0, buf = 0;

    // 0. scale: B 2^-ex has entries below 1 in magnitude (every CTA reads all of B)
    {
        double m = 0.0;
        for (int e = tid; e < k * k; e += nt) m = fmax(m, fabs(B[e]));
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_wmax[warp] = m;
        __syncthreads();
        if (tid == 0) {
            double mm = 0.0;
            for (int w = 0; w < nw; ++w) mm = fmax(mm, s_wmax[w]);
            int e2 = 0;
            if (mm > 0.0 && isfinite(mm)) frexp(mm, &e2);
            s_exp = e2;
        }
        __syncthreads();
    }
    const int ex = s_exp;
    // 1. FP32 sweeps on this CTA's rows of B 2^-ex
    for (int e = tid; e < nr * kp; e += nt) {
        const int r = e / kp, c = e % kp, rg = row0 + r;
        A32[e] = (rg < k && c < k) ? (float)ldexp(B[rg + (long long)c * k], -ex) : 0.0f;
        V32[e] = rg == c ? 1.0f : 0.0f;
    }
    __syncthreads();
    const float tol32 = 4.0f * (float)kp * 5.9604645e-8f;
    bool w_is_identity = false;
    for (int sw = 0; sw < kJacobiMaxSweeps32; ++sw)
        if (cluster_sweep<float>(cluster, A32, V32, nr, kp, tol32, (float*)part, buf, rs, &s_max) <=
            tol32) {
            w_is_identity = sw == 0;
            break;
        }
    // every CTA is past its last read of the FP32 partial sums before any buffer is reused
    cluster.sync();
    buf = 0;
    if (w_is_identity) {
        for (int e = tid; e < nr * kp; e += nt) {
            const int r = e / kp, c = e % kp, rg = row0 + r;
            Vl[e] = rg == c ? 1.0 : 0.0;
            Al[e] = (rg < k && c < k) ? ldexp(B[rg + (long long)c * k], -ex) : 0.0;
        }
        __syncthreads();
    } else {
        // 2. W in FP64, re-orthonormalised by Newton-Schulz steps W <- W (3 I - X) / 2,
        //    X = W^T W summed over the cluster
        for (int e = tid; e < nr * kp; e += nt) Vl[e] = (double)V32[e];
        __syncthreads();
        const int kk = kp * kp;
        const int e0 = min(kk, crank * L.slice_n), e1 = min(kk, e0 + L.slice_n);
        for (int step = 0; step < kJcNsSteps; ++step) {
            for (int e = tid; e < kk; e += nt) {  // this CTA's rows' share of X (row-major)
                const int a = e / kp, b = e % kp;
                double v = 0.0;
                for (int r = 0; r < nr; ++r) v = fma(Vl[r * kp + a], Vl[r * kp + b], v);
                Un[e] = v;
            }
            cluster.sync();
            for (int e = e0 + tid; e < e1; e += nt) {  // reduce-scatter, rank order
                double v = 0.0;
                for (int src = 0; src < kJcCluster; ++src) v += cluster.map_shared_rank(Un, src)[e];
                slice[e - e0] = v;
            }
            cluster.sync();
            for (int e = tid; e < kk; e += nt) {  // all-gather of the summed slices
                const int o = e / L.slice_n;
                Un[e] = cluster.map_shared_rank(slice, o)[e - o * L.slice_n];
            }
            __syncthreads();
            for (int e = tid; e < nr * kp; e += nt) {
                const int r = e / kp, c = e % kp;
                double v = 0.0;
                for (int m = 0; m < kp; ++m) v = fma(Vl[r * kp + m], Un[m * kp + c], v);
                Al[e] = 1.5 * Vl[e] - 0.5 * v;
            }
            __syncthreads();
            for (int e = tid; e < nr * kp; e += nt) Vl[e] = Al[e];
            __syncthreads();
        }
        // 3. A = B W 2^-ex on this CTA's rows; W's rows are read from the CTAs that hold them
        cluster.sync();  // every CTA's W is final
        double* Bl = Un;
        for (int e = tid; e < nr * kp; e += nt) {
            const int r = e / kp, m = e % kp, rg = row0 + r;
            Bl[e] = (rg < k && m < k) ? B[rg + (long long)m * k] : 0.0;
        }
        __syncthreads();
        for (int c = tid; c < kp; c += nt) {
            double acc[kJcMaxRows];
#pragma unroll
            for (int r = 0; r < kJcMaxRows; ++r) acc[r] = 0.0;
            for (int m = 0; m < kp; ++m) {
                const int o = m / rows_per;
                const double w = cluster.map_shared_rank(Vl, o)[(m - o * rows_per) * kp + c];
#pragma unroll
                for (int r = 0; r < kJcMaxRows; ++r)
                    if (r < nr) acc[r] = fma(Bl[r * kp + m], w, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kJcMaxRows; ++r)
                if (r < nr) Al[r * kp + c] = ldexp(acc[r], -ex);
        }
        __syncthreads();
    }
    cluster.sync();  // no CTA rotates its W before every CTA has read it
    // 4. FP64 sweeps (stopping rule of the one-CTA kernel)
    const double tol64 = (double)kp * 2.220446049250313e-16;
    {
        int sw = 0;
        for (; sw < kJacobiMaxSweeps64; ++sw) {
            const float mx = cluster_sweep<double>(cluster, Al, Vl, nr, kp, tol64, part, buf, rs,
                                                   &s_max);
            if (mx <= tol64 || mx < 1e-6f) break;
        }
        if (sw >= kJacobiMaxSweeps64) bad = 1;
    }
    // 5. singular values = column norms summed over the cluster; ranks by decreasing value
    for (int c = tid; c < kp; c += nt) {
        double v = 0.0;
        for (int r = 0; r < nr; ++r) v = fma(Al[r * kp + c], Al[r * kp + c], v);
        cpart[c] = v;
    }
    cluster.sync();
    for (int c = tid; c < k; c += nt) {
        double v = 0.0;
        for (int src = 0; src < kJcCluster; ++src) v += cluster.map_shared_rank(cpart, src)[c];
        sig[c] = sqrt(v);  // of B 2^-ex
    }
    __syncthreads();
    for (int c = tid; c < k; c += nt) {
        int rk = 0;
        for (int o = 0; o < k; ++o)
            if (sig[o] > sig[c] || (sig[o] == sig[c] && o < c)) ++rk;
        rank[c] = rk;
    }
    __syncthreads();
    for (int e = tid; e < nr * k; e += nt) {
        const int r = e / k, c = e % k, rg = row0 + r;
        if (rg >= k) continue;
        const int dst = rg + rank[c] * k;
        const double sc = sig[c];
        U[dst] = sc > 0.0 ? Al[r * kp + c] / sc : 0.0;
        W[dst] = Vl[r * kp + c];
    }
    if (crank == 0) {
        for (int c = tid; c < k; c += nt) S[rank[c]] = ldexp(sig[c], ex);
        if (tid == 0 && info) *info = bad;
    }
    cluster.sync();  // no CTA exits while another may still read its shared memory
}

// Vout[r + c n] = VT[c + r n] for c < k: the first k right singular vectors of gesvd's V^T as
// columns.
__global__ void vt_columns_kernel(const double* __restrict__ VT, double* __restrict__ Vout, int n,
                                  int k) {
    const long long total = (long long)n * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        Vout[e] = VT[c + (long long)r * n];
    }
}

// Columns c with S[c] == 0 (a zero column of the subspace basis; every column when S is null)
// get uniform [-1, 1) entries from SplitMix64 (Steele, Lea, Flood 2014) at counter c n + r.
__global__ void refill_kernel(double* __restrict__ V, int n, int k, const double* __restrict__ S,
                              unsigned long long seed) {
    const int c = blockIdx.x;
    if (c >= k || (S && S[c] != 0.0)) return;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        unsigned long long z = seed + ((unsigned long long)c * n + r + 1ULL) * 0x9E3779B97F4A7C15ULL;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        V[r + (long long)c * n] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
}

void launch_refill(double* V, int n, int k, const double* S, unsigned long long seed,
                   cudaStream_t s) {
    refill_kernel<<<k, 256, 0, s>>>(V, n, k, S, seed);
}

size_t chol_orth_smem(int k, bool global_x) {
    return (size_t)((global_x ? 1 : 2) * k * k + 2 * k) * sizeof(double);
}
size_t jacobi_svd_smem(int k, bool global_v) {  // A (and W), S, the round scratch, the ranks
    const int kp = k + (k & 1), ld = kp + 1, np = kp / 2;
    return (size_t)((global_v ? 1 : 2) * kp * ld + kp + 2 * np) * sizeof(double) +
           (size_t)(kp + 3 * np) * sizeof(int);
}

// The one-CTA kernels are bound by the FP64 throughput of their SM, which every warp resident on
// that SM shares.  Contraction CTAs of other streams would otherwise fill the rest of the SM and
// take most of that throughput, so these launches request enough shared memory (220 KB) that
// nothing else fits beside them: each runs on an SM of its own.  SCTM_SHARED_SM=1 requests only
// what the kernel uses (for comparison).
constexpr size_t kExclusiveSmem = 220 * 1024;

static size_t one_cta_smem(size_t need) {
    static const bool shared = [] {
        const char* v = getenv("SCTM_SHARED_SM");
        return v && v[0] == '1';
    }();
    return shared ? need : std::max(need, kExclusiveSmem);
}

bool chol_cluster_fits(int k) { return k >= kCcMinK && k <= kCcMaxK; }

void launch_chol_orth_cluster(const double* G, int k, double shift, double* T, cudaStream_t s) {
    const size_t smem = one_cta_smem(CcLayout(k).bytes());
    static std::once_flag once;
    std::call_once(once, [] {
        const size_t mx = std::max(CcLayout(kCcMaxK).bytes(), kExclusiveSmem);
        cudaFuncSetAttribute(chol_orth_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mx);
    });
    chol_orth_cluster_kernel<<<kCcCluster, kCcThreads, smem, s>>>(G, k, shift, T);
}

// The engine's Cholesky-QR pass: the cluster kernel where the order fits it (bit-identical
// results), unless SCTM_CHOL=cta selects the one-CTA kernel everywhere (for comparison).
static bool cluster_chol_enabled() {
    static const bool on = [] {
        const char* v = getenv("SCTM_CHOL");
        return !(v && v[0] == 'c' && v[1] == 't' && v[2] == 'a');
    }();
    return on;
}

void launch_chol_orth(const double* G, int k, double shift, double* T, double* Xg,
                      cudaStream_t s) {
    if (cluster_chol_enabled() && chol_cluster_fits(k)) {
        launch_chol_orth_cluster(G, k, shift, T, s);
        return;
    }
    launch_chol_orth_cta(G, k, shift, T, Xg, s);
}

void launch_chol_orth_cta(const double* G, int k, double shift, double* T, double* Xg,
                          cudaStream_t s) {
    const size_t smem = one_cta_smem(chol_orth_smem(k, Xg != nullptr));
    static std::once_flag once;
    std::call_once(once, [] {
        // the largest request: all in shared memory at kPsvdSmemK, or X in global at kPsvdMaxK
        const size_t mx = std::max({chol_orth_smem(kPsvdSmemK, false), chol_orth_smem(kPsvdMaxK, true),
                                    kExclusiveSmem});
        cudaFuncSetAttribute(chol_orth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    });
    chol_orth_kernel<<<1, kPsvdThreads, smem, s>>>(G, k, shift, T, Xg);
}

bool jacobi_cluster_fits(int k) {
    const int kp = k + (k & 1);
    return kp >= kJcMinKp && kp <= kJcMaxKp;
}

void launch_jacobi_svd_cluster(const double* B, int k, double* S, double* U, double* W, int* info,
                               cudaStream_t s) {
    const size_t smem = one_cta_smem(JcLayout(k).bytes());
    static std::once_flag once;
    std::call_once(once, [] {
        const size_t mx = std::max(JcLayout(kJcMaxKp).bytes(), kExclusiveSmem);
        cudaFuncSetAttribute(jacobi_svd_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)mx);
    });
    jacobi_svd_cluster_kernel<<<kJcCluster, kJcThreads, smem, s>>>(B, k, S, U, W, info);
}

void launch_jacobi_svd(const double* B, int k, double* S, double* U, double* W, int* info,
                       double* Vg, bool cluster, cudaStream_t s) {
    if (cluster && jacobi_cluster_fits(k)) {
        launch_jacobi_svd_cluster(B, k, S, U, W, info, s);
        return;
    }
    launch_jacobi_svd_cta(B, k, S, U, W, info, Vg, s);
}

void launch_jacobi_svd_cta(const double* B, int k, double* S, double* U, double* W, int* info,
                           double* Vg, cudaStream_t s) {
    const size_t smem = one_cta_smem(jacobi_svd_smem(k, Vg != nullptr));
    static std::once_flag once;
    std::call_once(once, [] {
        const size_t mx = std::max({jacobi_svd_smem(kPsvdSmemK, false),
                                    jacobi_svd_smem(kPsvdMaxK, true), kExclusiveSmem});
        cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    });
    jacobi_svd_kernel<<<1, kPsvdThreads, smem, s>>>(B, k, S, U, W, info, Vg);
}

void launch_vt_columns(const double* VT, double* Vout, int n, int k, cudaStream_t s) {
    const long long total = (long long)n * k;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 2048);
    vt_columns_kernel<<<std::max(blocks, 1), 256, 0, s>>>(VT, Vout, n, k);
}

}  // namespace sctm
