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
// the kernels here do the k x k work in one CTA each:
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
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "sctm_internal.h"

namespace sctm {

namespace {

constexpr int kPsvdThreads = 512;
constexpr int kJacobiMaxSweeps32 = 12;
constexpr int kJacobiMaxSweeps64 = 20;
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

void launch_chol_orth(const double* G, int k, double shift, double* T, double* Xg,
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

void launch_jacobi_svd(const double* B, int k, double* S, double* U, double* W, int* info,
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
