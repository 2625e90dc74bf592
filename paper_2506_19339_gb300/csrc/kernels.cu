// CUDA kernels of the split-CTMRG runtime: the gather-table contraction (FP64) and the FP64
// auxiliary kernels (normalisation, SVD sign gauge, pseudo-inverse scales, cold start,
// convergence spectrum, free energy, gradient).
#include "sctm_internal.h"

#include <cmath>

namespace sctm {

// ---------------------------------------------------------------------------------------------
// FP64 contraction: 64x64 (or 32x32) output tile per CTA, 256 threads, 4x4 (2x2) register tile
// per thread, K in chunks of 16.  Operand tiles are gathered through the offset tables into shared memory, so the
// leg permutation of each operand is paid inside the load (Sec. III's contractions have every
// operand in a different leg order).  Split-K writes partial tiles that a second kernel sums in
// a fixed order (deterministic, no atomics).
// ---------------------------------------------------------------------------------------------
namespace {
constexpr int BK = 16, NT = 256;
}

// TM x TN outputs per thread on a 16 x 16 thread grid: a (16 TM) x (16 TN) tile per CTA.  Every
// output element accumulates over K in the same order (chunks of 16, then sequentially) whatever
// the tile size, so the tile choice does not change the result.
template <int TM, int TN>
__global__ void __launch_bounds__(NT) ctr_f64_kernel(const CtrLaunch a) {
    constexpr int BM = 16 * TM, BN = 16 * TN;
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    __shared__ int sxm[BM];
    __shared__ int syn[BN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int z = blockIdx.z;
    const int b = z / a.splits, sp = z % a.splits;
    const long long xbo = a.xb ? a.xb[b] : 0;
    const long long ybo = a.yb ? a.yb[b] : 0;

    if (tid < BM) {
        sxm[tid] = (m0 + tid < a.M) ? a.xm[m0 + tid] : -1;
    } else if (tid < BM + BN) {
        const int j = tid - BM;
        syn[j] = (n0 + j < a.N) ? a.yn[n0 + j] : -1;
    }
    __syncthreads();

    const int kbeg = sp * a.kchunk;
    const int kend = min(a.K, kbeg + a.kchunk);
    double acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int q = 0; q < BM * BK / NT; ++q) {
            const int e = tid + NT * q;
            const int kk = e % BK, mm = e / BK;
            const int k = k0 + kk;
            const int om_ = sxm[mm];
            double v = 0.0;
            if (om_ >= 0 && k < kend) v = a.X[xbo + om_ + a.xk[k]];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int q = 0; q < BN * BK / NT; ++q) {
            const int e = tid + NT * q;
            const int nn = e % BN, kk = e / BN;
            const int k = k0 + kk;
            const int on_ = syn[nn];
            double v = 0.0;
            if (on_ >= 0 && k < kend) v = a.Y[ybo + a.yk[k] + on_];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double av[TM], bv[TN];
#pragma unroll
            for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }

    if (a.splits > 1) {
        double* P = a.partial + (long long)z * a.M * a.N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int m = m0 + ty + 16 * i;
            if (m >= a.M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                const int n = n0 + tx + 16 * j;
                if (n < a.N) P[(long long)m * a.N + n] = acc[i][j];
            }
        }
        return;
    }
    const long long obo = a.ob ? a.ob[b] : 0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= a.M) continue;
        const double rs = a.rowscale ? a.rowscale[m] : 1.0;
        const long long om_ = obo + a.om[m];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= a.N) continue;
            double v = acc[i][j] * rs;
            if (a.colscale) v *= a.colscale[n];
            double* dst = a.O + om_ + a.on[n];
            *dst = a.accumulate ? *dst + v : v;
        }
    }
}

__global__ void ctr_splitk_reduce_kernel(const CtrLaunch a) {
    const long long MN = (long long)a.M * a.N;
    const long long total = MN * a.nb;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(t / MN);
        const long long r = t - (long long)b * MN;
        const int m = (int)(r / a.N), n = (int)(r - (long long)m * a.N);
        double v = 0.0;
        const double* P = a.partial + (long long)b * a.splits * MN + r;
        for (int s = 0; s < a.splits; ++s) v += P[(long long)s * MN];
        if (a.rowscale) v *= a.rowscale[m];
        if (a.colscale) v *= a.colscale[n];
        const long long obo = a.ob ? a.ob[b] : 0;
        double* dst = a.O + obo + a.om[m] + a.on[n];
        *dst = a.accumulate ? *dst + v : v;
    }
}

// Skinny contractions (N <= 32 outputs per row, K <= 64, one K range): one thread per output row
// keeps its N accumulators in registers, Y[b] is staged once per block in shared memory.  The
// 64 x 64 tiles of ctr_f64_kernel would spend most of their FMAs on padding for these shapes
// (N = 2..32 against a 64-wide tile), which are memory-bound.  The K loop runs in increasing k
// with one FMA per term, as in ctr_f64_kernel, so the result is bitwise the same.
constexpr int kSkinnyN = 32, kSkinnyK = 64, kSkinnyRows = 256;
__global__ void __launch_bounds__(kSkinnyRows) ctr_skinny_kernel(const CtrLaunch a) {
    __shared__ double ys[kSkinnyK * kSkinnyN];
    const int b = blockIdx.y;
    const long long ybo = a.yb ? a.yb[b] : 0;
    for (int e = threadIdx.x; e < a.K * a.N; e += blockDim.x) {
        const int k = e / a.N, n = e - k * a.N;
        ys[k * kSkinnyN + n] = a.Y[ybo + a.yk[k] + a.yn[n]];
    }
    __syncthreads();
    const long long xbo = a.xb ? a.xb[b] : 0;
    const long long obo = a.ob ? a.ob[b] : 0;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < a.M; m += gridDim.x * blockDim.x) {
        double acc[kSkinnyN];
#pragma unroll
        for (int n = 0; n < kSkinnyN; ++n) acc[n] = 0.0;
        const long long xr = xbo + a.xm[m];
        for (int k = 0; k < a.K; ++k) {
            const double x = a.X[xr + a.xk[k]];
#pragma unroll
            for (int n = 0; n < kSkinnyN; ++n)
                if (n < a.N) acc[n] = fma(x, ys[k * kSkinnyN + n], acc[n]);
        }
        const double rs = a.rowscale ? a.rowscale[m] : 1.0;
        const long long om_ = obo + a.om[m];
#pragma unroll
        for (int n = 0; n < kSkinnyN; ++n) {
            if (n >= a.N) continue;
            double v = acc[n] * rs;
            if (a.colscale) v *= a.colscale[n];
            double* dst = a.O + om_ + a.on[n];
            *dst = a.accumulate ? *dst + v : v;
        }
    }
}

bool ctr_is_skinny(const CtrLaunch& a) {
    return a.N <= kSkinnyN && a.K <= kSkinnyK && a.nb <= 65535;
}

void launch_ctr(const CtrLaunch& a0, cudaStream_t s) {
    if (a0.precision != SCTM_PREC_FP64) {
        CtrLaunch a = a0;
        a.splits = a0.tc_splits;
        a.kchunk = a0.tc_kchunk;
        launch_ctr_tc(a, s);
        if (a.splits > 1) {
            const long long total = (long long)a.M * a.N * a.nb;
            int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
            ctr_splitk_reduce_kernel<<<blocks, 256, 0, s>>>(a);
        }
        return;
    }
    const CtrLaunch& a = a0;
    if (ctr_is_skinny(a)) {
        const int bx = (int)std::min<long long>((a.M + kSkinnyRows - 1) / kSkinnyRows, 65535);
        dim3 grid(std::max(bx, 1), a.nb);
        ctr_skinny_kernel<<<grid, kSkinnyRows, 0, s>>>(a);
        return;
    }
    const int bm = a.tile, bn = a.tile;
    dim3 grid((a.N + bn - 1) / bn, (a.M + bm - 1) / bm, a.nb * a.splits);
    if (a.tile == 32)
        ctr_f64_kernel<2, 2><<<grid, NT, 0, s>>>(a);
    else
        ctr_f64_kernel<4, 4><<<grid, NT, 0, s>>>(a);
    if (a.splits > 1) {
        const long long total = (long long)a.M * a.N * a.nb;
        int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
        ctr_splitk_reduce_kernel<<<blocks, 256, 0, s>>>(a);
    }
}

// ---------------------------------------------------------------------------------------------
// block reductions (fixed order: warp shuffle tree, then warp 0 over the warp partials)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v) {
    __shared__ double ws[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    double t = (threadIdx.x < nw) ? ws[threadIdx.x] : 0.0;
    if (w == 0) t = warp_sum(t);
    __shared__ double res;
    if (threadIdx.x == 0) res = t;
    __syncthreads();
    const double out = res;
    __syncthreads();
    return out;
}

// Frobenius normalisation of each environment tensor after a move, written through a strided
// destination view (this is where a relabelled frame writes back into the stored layout).
__global__ void normalize_kernel(const NormItem* items) {
    const NormItem it = items[blockIdx.x];
    const long long n = (long long)it.d0 * it.d1 * it.d2;
    double ss = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) ss += it.src[i] * it.src[i];
    const double tot = block_sum(ss);
    const double inv = tot > 0.0 ? 1.0 / sqrt(tot) : 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const int i2 = (int)(i % it.d2);
        const long long r = i / it.d2;
        const int i1 = (int)(r % it.d1);
        const int i0 = (int)(r / it.d1);
        it.dst[i0 * it.s0 + i1 * it.s1 + i2 * it.s2] = it.src[i] * inv;
    }
}

void launch_normalize(const NormItem* items_dev, int count, cudaStream_t s) {
    normalize_kernel<<<count, 1024, 0, s>>>(items_dev);
}

// SplitMix64 (Steele, Lea & Flood 2014): entry j of slot q is the (c+1)-th output of the
// generator started at `seed`, c = q * 2^32 + j, mapped to [0,1) with its top 53 bits.
__global__ void splitmix_kernel(double* p, long long n, unsigned long long seed,
                                unsigned long long slot) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const unsigned long long c = (slot << 32) + (unsigned long long)j;
    unsigned long long z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    p[j] = (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

void launch_splitmix_fill(double* p, long long n, unsigned long long seed, unsigned long long slot,
                          cudaStream_t s) {
    splitmix_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, n, seed, slot);
}

// (S~^1/2)^+ of Eq. "projector construction 2": 1/sqrt(s_c) for s_c > cutoff * s_0, else 0.
__global__ void scalevec_kernel(const double* S, int k, double cutoff, double* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    const double s0 = S[0], sc = S[c];
    out[c] = (sc > cutoff * s0 && sc > 0.0) ? 1.0 / sqrt(sc) : 0.0;
}

void launch_scalevec(const double* S, int k, double cutoff, double* out, cudaStream_t s) {
    scalevec_kernel<<<(k + 127) / 128, 128, 0, s>>>(S, k, cutoff, out);
}

// SVD sign gauge: flip (u_c, v_c) so that the largest-magnitude entry of u_c (first index on a
// tie) is positive.  U and V are n x n column-major with the singular vectors as columns (cuSOLVER
// layout); one CTA per column.
__global__ void signfix_kernel(double* U, double* V, int n, int vt) {
    const int c = blockIdx.x;
    double* u = U + (long long)c * n;
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = fabs(u[i]);
        if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    __shared__ double sv[256];
    __shared__ int si[256];
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double v2 = sv[threadIdx.x + o];
            const int i2 = si[threadIdx.x + o];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    const int imax = si[0];
    const bool flip = (imax < n) && (u[imax] < 0.0);
    __syncthreads();
    if (!flip) return;
    // right vector c: column c of V, or row c of V^T (gesvd layout, column-major)
    const long long v0 = vt ? c : (long long)c * n, vs = vt ? n : 1;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        u[i] = -u[i];
        V[v0 + i * vs] = -V[v0 + i * vs];
    }
}

void launch_signfix(double* U, double* V, int n, int k, int vt, cudaStream_t s) {
    signfix_kernel<<<k, 256, 0, s>>>(U, V, n, vt);
}

__global__ void copy_kernel(const double* src, double* dst, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

void launch_copy(const double* src, double* dst, long long n, cudaStream_t s) {
    int blocks = (int)std::min<long long>((n + 255) / 256, 2048);
    copy_kernel<<<std::max(blocks, 1), 256, 0, s>>>(src, dst, n);
}

// C <- (C + C^T) / 2 in place, n x n row-major: one thread per pair (i < j), the diagonal kept
// (the symmetric split-CTMRG corners, Sec. III.B, Eq. "Symmetry constraints")
__global__ void symmetrize_kernel(double* X, int n) {
    const long long m = (long long)n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < m;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n), j = (int)(idx % n);
        if (i >= j) continue;
        const double v = 0.5 * (X[(long long)i * n + j] + X[(long long)j * n + i]);
        X[(long long)i * n + j] = v;
        X[(long long)j * n + i] = v;
    }
}

void launch_symmetrize(double* X, int n, cudaStream_t s) {
    const long long m = (long long)n * n;
    int blocks = (int)std::min<long long>((m + 255) / 256, 1024);
    symmetrize_kernel<<<std::max(blocks, 1), 256, 0, s>>>(X, n);
}

// Average of A[s, u, l, d, r] over the square's symmetry group D4 acting on the virtual legs
// (Sec. III.B: the PEPS and its gradient kept in the D4-invariant subspace).  The group maps the
// output index (i0, i1, i2, i3) of the legs in cyclic order u, l, d, r to the inputs
// (i_k, i_k+1, i_k+2, i_k+3) (rotations) and (i_k, i_k-1, i_k-2, i_k-3) (reflections), k = 0..3,
// indices mod 4.
__global__ void d4_project_kernel(const double* in, double* out, int p, int D) {
    const long long D2 = (long long)D * D, D4 = D2 * D2;
    const long long n = (long long)p * D4;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long s = idx / D4;
        long long r = idx - s * D4;
        int c[4];
        for (int q = 3; q >= 0; --q) {
            c[q] = (int)(r % D);
            r /= D;
        }
        double acc = 0.0;
        for (int k = 0; k < 4; ++k)
            for (int dir = 1; dir >= -1; dir -= 2) {
                long long off = 0;
                for (int q = 0; q < 4; ++q) off = off * D + c[(k + dir * q + 8) & 3];
                acc += in[s * D4 + off];
            }
        out[idx] = 0.125 * acc;
    }
}

void launch_d4_project(const double* in, double* out, int p, int D, cudaStream_t s) {
    const long long n = (long long)p * D * D * D * D;
    int blocks = (int)std::min<long long>((n + 255) / 256, 2048);
    d4_project_kernel<<<std::max(blocks, 1), 256, 0, s>>>(in, out, p, D);
}

__global__ void zero_kernel(double* p, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = 0.0;
}

void launch_zero(double* p, long long n, cudaStream_t s) {
    int blocks = (int)std::min<long long>((n + 255) / 256, 2048);
    zero_kernel<<<std::max(blocks, 1), 256, 0, s>>>(p, n);
}

__global__ void check_finite_kernel(const double* p, long long n, int* flag) {
    int bad = 0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) bad |= !isfinite(p[i]);
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) flag[0] = bad;
}

void launch_check_finite(const double* p, long long n, int* flag, cudaStream_t s) {
    check_finite_kernel<<<1, 256, 0, s>>>(p, n, flag);
}

__global__ void sanitize_kernel(double* p, long long n, int* flag) {
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!isfinite(p[i])) {
            p[i] = 0.0;
            bad = 1;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

void launch_sanitize(double* p, long long n, int* flag, cudaStream_t s) {
    const int blocks = (int)std::min<long long>((n + 255) / 256, 1024);
    sanitize_kernel<<<std::max(blocks, 1), 256, 0, s>>>(p, n, flag);
}

// Convergence (Sec. III.D): S = singular values of rho_eff / Tr(rho_eff); dS = ||S - S_old||_2;
// S_old <- S.  rho is chi x chi column-major (only its diagonal is read here, for the trace).
__global__ void spectrum_update_kernel(const double* Sraw, const double* rho, int chi,
                                       double* S_old, double* dS_out) {
    double tr = 0.0;
    for (int i = threadIdx.x; i < chi; i += blockDim.x) tr += rho[(long long)i * chi + i];
    tr = block_sum(tr);
    const double inv = (tr != 0.0) ? 1.0 / fabs(tr) : 0.0;
    double d2 = 0.0;
    for (int i = threadIdx.x; i < chi; i += blockDim.x) {
        const double s = Sraw[i] * inv;
        const double diff = s - S_old[i];
        d2 += diff * diff;
    }
    d2 = block_sum(d2);
    for (int i = threadIdx.x; i < chi; i += blockDim.x) S_old[i] = Sraw[i] * inv;
    if (threadIdx.x == 0) dS_out[0] = (tr != 0.0 && isfinite(tr)) ? sqrt(d2) : NAN;
}

void launch_spectrum_update(const double* Sraw, const double* rho, int chi, double* S_old,
                            double* dS_out, cudaStream_t s) {
    spectrum_update_kernel<<<1, 256, 0, s>>>(Sraw, rho, chi, S_old, dS_out);
}

__global__ void lnkappa_kernel(const double* Z00, const double* Z10, const double* Z01,
                               const double* Z11, double* lnk) {
    const double kappa = Z11[0] * Z00[0] / (Z10[0] * Z01[0]);
    lnk[0] = (isfinite(kappa) && kappa > 0.0) ? log(kappa) : NAN;
    lnk[1] = Z11[0];
}

void launch_lnkappa(const double* Z00, const double* Z10, const double* Z01, const double* Z11,
                    double* lnk, cudaStream_t s) {
    lnkappa_kernel<<<1, 1, 0, s>>>(Z00, Z10, Z01, Z11, lnk);
}

__global__ void free_energy_kernel(const double* lnk_num, const double* lnk_den, double T,
                                   double* out) {
    out[0] = -T * (lnk_num[0] - lnk_den[0]);
}

void launch_free_energy(const double* lnk_num, const double* lnk_den, double T, double* out,
                        cudaStream_t s) {
    free_energy_kernel<<<1, 1, 0, s>>>(lnk_num, lnk_den, T, out);
}

__global__ void grad_combine_kernel(const double* Enum, const double* lnk_num, const double* Eden,
                                    const double* lnk_den, double T, int n, double* g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double zn = lnk_num[1], zd = lnk_den[1];
    g[i] = -2.0 * T * (Enum[i] / zn - Eden[i] / zd);
}

void launch_grad_combine(const double* Enum, const double* lnk_num, const double* Eden,
                         const double* lnk_den, double T, int n, double* g, cudaStream_t s) {
    grad_combine_kernel<<<(n + 255) / 256, 256, 0, s>>>(Enum, lnk_num, Eden, lnk_den, T, n, g);
}

}  // namespace sctm
