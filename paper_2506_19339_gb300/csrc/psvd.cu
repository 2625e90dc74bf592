// Kernels of the partial SVD (Sec. III: the largest chi singular triplets of the projector
// matrix M by an iterative solver instead of a full decomposition).
//
// The projector matrix changes little from one CTMRG iteration to the next, so its leading
// right singular subspace of the previous iteration (k = chi + oversampling columns) is a warm
// start.  One warm solve is a two-sided subspace iteration step with a Rayleigh-Ritz
// extraction:
//     Y = M V_prev,  Y = Q_y R_y          (Q_y: orthonormal basis of the left subspace)
//     Z = M^T Q_y,   Z = Q_z R_z          (Q_z: improved right subspace)
//     Q_y^T M Q_z = R_z^T;  R_z = U_r S W^T (k x k SVD)
//     M ~ (Q_y W) S (Q_z U_r)^T           left vectors Q_y W, right vectors Q_z U_r.
// The products with M and the basis updates run on the contraction kernel; the two kernels here
// do the k x k work in one CTA each:
//   * chol_orth_kernel: one pass of column-scaled Cholesky QR.  With G = Y^T Y and D the column
//     norms, G = D (R^T R) D; it returns T = D^-1 R^-1 (so that Y T is orthonormal) and the
//     triangular factor R D (times the previous pass's factor).  The columns of Y are close to
//     orthogonal in the warm regime (Y ~ U S), so the scaled Gram matrix is close to the identity
//     and the factorisation keeps the relative accuracy of small columns; a second pass restores
//     orthogonality to rounding.  Columns whose scaled pivot falls below 1e-20 are dependent:
//     their basis column and factor row are set to zero.
//   * jacobi_svd_kernel: one-sided (Hestenes) Jacobi SVD of the k x k factor, round-robin
//     ordering of the k(k-1)/2 column pairs, sweeps until no pair is rotated (bounded), output
//     sorted by decreasing singular value.
#include <algorithm>
#include <mutex>

#include "sctm_internal.h"

namespace sctm {

namespace {

constexpr int kPsvdThreads = 512;
constexpr int kJacobiMaxSweeps = 40;
constexpr double kPivotFloor = 1e-20;

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace

// G (k x k, column-major G[i + j k]) -> T (k x k, column-major, upper triangular) with Y T
// orthonormal for the Y that gave G = Y^T Y, and Rout = R D Rprev (Rprev == nullptr: R D).
// Shared memory: 2 k^2 + k doubles.
__global__ void __launch_bounds__(kPsvdThreads)
    chol_orth_kernel(const double* __restrict__ G, int k, const double* __restrict__ Rprev,
                     double* __restrict__ T, double* __restrict__ Rout) {
    extern __shared__ double sm[];
    double* R = sm;              // row-major k x k: scaled Gram, then the Cholesky factor (upper)
    double* X = sm + k * k;      // row-major k x k: R^-1
    double* d = sm + 2 * k * k;  // column norms
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < k; i += nt) {
        const double g = G[i + (long long)i * k];
        d[i] = g > 0.0 ? sqrt(g) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        const double di = d[i], dj = d[j];
        R[e] = (di > 0.0 && dj > 0.0) ? G[i + (long long)j * k] / (di * dj) : 0.0;
    }
    __syncthreads();
    // right-looking Cholesky, upper factor in the upper triangle of R (row j = R_j,:)
    for (int j = 0; j < k; ++j) {
        const double piv = R[j * k + j];
        const double rjj = piv > kPivotFloor ? sqrt(piv) : 0.0;
        __syncthreads();
        for (int c = j + tid; c < k; c += nt) R[j * k + c] = rjj > 0.0 ? R[j * k + c] / rjj : 0.0;
        __syncthreads();
        const int m = k - j - 1;  // trailing (j+1..k-1)^2 block, upper part
        for (int e = tid; e < m * m; e += nt) {
            const int a = j + 1 + e / m, b = j + 1 + e % m;
            if (b >= a) R[a * k + b] -= R[j * k + a] * R[j * k + b];
        }
        __syncthreads();
    }
    // X = R^-1 by back substitution, one column per thread; rows of dependent columns are zero
    for (int c = tid; c < k; c += nt) {
        for (int r = k - 1; r >= 0; --r) {
            double x = 0.0;
            if (r <= c && R[r * k + r] > 0.0) {
                double acc = (r == c) ? 1.0 : 0.0;
                for (int l = r + 1; l <= c; ++l) acc -= R[r * k + l] * X[l * k + c];
                x = acc / R[r * k + r];
            }
            X[r * k + c] = x;
        }
    }
    __syncthreads();
    // T = D^-1 R^-1 ; Rout = R D Rprev
    for (int e = tid; e < k * k; e += nt) {
        const int i = e % k, j = e / k;  // column-major output index
        T[e] = (d[i] > 0.0 && j >= i) ? X[i * k + j] / d[i] : 0.0;
        double v = 0.0;
        if (Rprev) {
            for (int l = i; l < k; ++l) v += R[i * k + l] * d[l] * Rprev[l + (long long)j * k];
        } else if (j >= i) {
            v = R[i * k + j] * d[j];
        }
        Rout[e] = v;
    }
}

// One-sided Jacobi SVD of B (k x k, column-major): B W = A with orthogonal columns, B = U S W^T,
// U = A S^-1.  Writes S (k, decreasing), U and W (k x k, column-major, columns in the order of
// S).  info: 0, or 1 if the sweep limit was reached.  Shared memory: 2 kp^2 + 2 kp doubles,
// kp = k rounded up to even (an odd k gets a zero column that is never rotated).
__global__ void __launch_bounds__(kPsvdThreads)
    jacobi_svd_kernel(const double* __restrict__ B, int k, double* __restrict__ S,
                      double* __restrict__ U, double* __restrict__ W, int* info) {
    extern __shared__ double sm[];
    const int kp = k + (k & 1);
    double* A = sm;                // column j at A + j kp
    double* V = sm + kp * kp;      // column j at V + j kp
    double* sig = sm + 2 * kp * kp;
    int* rank = (int*)(sig + kp);
    __shared__ int s_rot;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5,
              nw = nt >> 5;
    for (int e = tid; e < kp * kp; e += nt) {
        const int r = e % kp, c = e / kp;
        A[e] = (r < k && c < k) ? B[r + (long long)c * k] : 0.0;
        V[e] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    // a pair is rotated while |a_i . a_j| > tol |a_i| |a_j|; tol = 4 sqrt(kp) eps sits above the
    // rounding level of the dot products of orthogonal columns, so the sweeps terminate
    const double tol = 4.0 * sqrt((double)kp) * 2.220446049250313e-16;
    int sweep = 0;
    for (; sweep < kJacobiMaxSweeps; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < kp - 1; ++round) {
            // circle method: position 0 fixed, positions 1..kp-1 rotate by `round`
            for (int q = warp; q < kp / 2; q += nw) {
                const int p0 = q, p1 = kp - 1 - q;
                const int i = p0 == 0 ? 0 : 1 + (p0 - 1 + round) % (kp - 1);
                const int j = 1 + (p1 - 1 + round) % (kp - 1);
                double* ai = A + (long long)i * kp;
                double* aj = A + (long long)j * kp;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int r = lane; r < kp; r += 32) {
                    const double x = ai[r], y = aj[r];
                    al = fma(x, x, al);
                    be = fma(y, y, be);
                    ga = fma(x, y, ga);
                }
                al = warp_allsum(al);
                be = warp_allsum(be);
                ga = warp_allsum(ga);
                if (ga != 0.0 && al > 0.0 && be > 0.0 && fabs(ga) > tol * sqrt(al * be)) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                    double* vi = V + (long long)i * kp;
                    double* vj = V + (long long)j * kp;
                    for (int r = lane; r < kp; r += 32) {
                        const double x = ai[r], y = aj[r];
                        ai[r] = c * x - s * y;
                        aj[r] = s * x + c * y;
                        const double u = vi[r], w = vj[r];
                        vi[r] = c * u - s * w;
                        vj[r] = s * u + c * w;
                    }
                    if (lane == 0) s_rot = 1;
                }
            }
            __syncthreads();
        }
        if (s_rot == 0) break;
        __syncthreads();
    }
    // singular values = column norms, ranks by decreasing value (ties: lower index first)
    for (int c = warp; c < k; c += nw) {
        double v = 0.0;
        for (int r = lane; r < kp; r += 32) v = fma(A[c * kp + r], A[c * kp + r], v);
        v = warp_allsum(v);
        if (lane == 0) sig[c] = sqrt(v);
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
        U[dst] = sc > 0.0 ? A[c * kp + r] / sc : 0.0;
        W[dst] = V[c * kp + r];
    }
    for (int c = tid; c < k; c += nt) S[rank[c]] = sig[c];
    if (tid == 0 && info) *info = sweep >= kJacobiMaxSweeps ? 1 : 0;
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

size_t chol_orth_smem(int k) { return (size_t)(2 * k * k + k) * sizeof(double); }
size_t jacobi_svd_smem(int k) {
    const int kp = k + (k & 1);
    return (size_t)(2 * kp * kp + kp) * sizeof(double) + (size_t)kp * sizeof(int);
}

void launch_chol_orth(const double* G, int k, const double* Rprev, double* T, double* Rout,
                      cudaStream_t s) {
    const size_t smem = chol_orth_smem(k);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(chol_orth_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)chol_orth_smem(kPsvdMaxK));
    });
    chol_orth_kernel<<<1, kPsvdThreads, smem, s>>>(G, k, Rprev, T, Rout);
}

void launch_jacobi_svd(const double* B, int k, double* S, double* U, double* W, int* info,
                       cudaStream_t s) {
    const size_t smem = jacobi_svd_smem(k);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(jacobi_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)jacobi_svd_smem(kPsvdMaxK));
    });
    jacobi_svd_kernel<<<1, kPsvdThreads, smem, s>>>(B, k, S, U, W, info);
}

void launch_vt_columns(const double* VT, double* Vout, int n, int k, cudaStream_t s) {
    const long long total = (long long)n * k;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 2048);
    vt_columns_kernel<<<std::max(blocks, 1), 256, 0, s>>>(VT, Vout, n, k);
}

}  // namespace sctm
