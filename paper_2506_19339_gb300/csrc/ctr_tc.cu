// Tensor-core (tcgen05) variant of the gather-table contraction, for the mixed-precision forms:
// TF32 or BF16 operands with FP32 accumulation in tensor memory, optionally with hi/lo split
// products (x = hi + lo; hi*hi + hi*lo + lo*hi) that recover most of the FP32 input precision.
//
// Each launch first finds max |X| and max |Y| (ctr_maxabs_kernel), then converts both operands
// once (ctr_pack_kernel): gathered through the offset tables (the leg permutation is folded into
// this pass, as in the FP64 kernel), scaled by a power of two into the format's range, split into
// hi/lo and written as tiles whose bytes are already in the shared-memory image order: K-major,
// no-swizzle canonical layout (8-row x 16-byte core matrices: K-adjacent core matrices 128 B
// apart, M/N-adjacent ones (32 * elem / 16) * 128 B apart).  FP64 arithmetic is scarce on this
// GPU, so it is spent once per operand element rather than once per tile that reads it.
// One CTA = 128 threads = 4 warps computes a 128 x 64 output tile (one tcgen05.mma of M=128,
// N=64 per K-step).  Per K chunk of 32 the threads copy the packed tiles to shared memory with
// 16-byte moves; one thread issues the MMAs and commits them to an mbarrier that every thread
// waits on before the shared tiles are reused.  The epilogue reads the accumulator
// with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = tile rows) and scatters FP64 results
// through the output tables.  Every wait is bounded: on timeout the kernel records an error,
// drains, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sctm_internal.h"

namespace sctm {

namespace {

constexpr int TBM = 128, TBN = 64, TBK = 32, TNT = 128;
constexpr int kTmemCols = 64;                 // FP32 accumulator columns (= TBN)
constexpr long long kSpinLimit = 1LL << 20;   // bounded mbarrier wait (about a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading (K) byte offset >> 4
// (16-29), stride (M/N) byte offset >> 4 (32-45), descriptor version 1 (46-47), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32 / kind::f16: D = F32 (bits 4-5 = 1), A and B format
// (bits 7-9, 10-12: F16 0, BF16 1, TF32 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <bool BF16>
struct Op {
    using T = uint32_t;  // tf32 bits
    static constexpr int kElem = 4;
    static constexpr uint32_t kFmt = 2;
    static constexpr int kMmaK = 8;
    __device__ static void split(double x, uint32_t& hi, uint32_t& lo) {
        const float f = (float)x;
        uint32_t h;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
        h &= 0xFFFFE000u;  // keep sign, exponent and the 10 TF32 mantissa bits
        const float r = (float)(x - (double)__uint_as_float(h));
        uint32_t l;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
        hi = h;
        lo = l & 0xFFFFE000u;
    }
};

template <>
struct Op<true> {
    using T = unsigned short;  // bf16 bits
    static constexpr int kElem = 2;
    static constexpr uint32_t kFmt = 1;
    static constexpr int kMmaK = 16;
    __device__ static void split(double x, unsigned short& hi, unsigned short& lo) {
        const __nv_bfloat16 h = __double2bfloat16(x);
        const __nv_bfloat16 l = __double2bfloat16(x - (double)__bfloat162float(h));
        hi = *reinterpret_cast<const unsigned short*>(&h);
        lo = *reinterpret_cast<const unsigned short*>(&l);
    }
};

// Row r and K index k of element e of a (rows x TBK) K-major tile stored in the canonical
// no-swizzle core-matrix layout, where element e sits at byte e * E:
//   byte(r, k) = ((r / 8) * CHUNKS + k / T) * 128 + (r % 8) * 16 + (k % T) * E,
// T = 16 / E elements per 16-byte core-matrix row, CHUNKS = TBK / T core matrices along K.
template <int E>
__device__ __forceinline__ void tile_pos(int e, int& r, int& k) {
    constexpr int T = 16 / E;
    constexpr int CHUNKS = TBK / T;
    const int kin = e % T, rin = (e / T) % 8, chunk = (e / (8 * T)) % CHUNKS,
              group = e / (8 * T * CHUNKS);
    r = group * 8 + rin;
    k = chunk * T + kin;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kSpinLimit) {
    for (long long i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// one tcgen05.mma (single-thread issue): D[tmem] (+)= A[da] * B[db]^T, accumulate iff acc != 0
template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t acc);
template <>
__device__ __forceinline__ void mma<false>(uint32_t tmem, uint64_t da, uint64_t db,
                                           uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
template <>
__device__ __forceinline__ void mma<true>(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                          uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

}  // namespace

// Per-block maxima of |X| (blocks 0 .. kScaleBlocks-1) and |Y| (the next kScaleBlocks) over the
// elements the contraction reads, through its gather tables.  FP32 and its TF32 / BF16 subsets
// cover about 1e-38 .. 3e38, while the FP64 tensors of a large network can sit far below that
// (projector matrices of ~1e-35 at D=4, chi=64 with a normalised PEPS), so the tensor-core
// kernel scales each operand by a power of two taken from these maxima.
__global__ void __launch_bounds__(256) ctr_maxabs_kernel(const CtrLaunch a) {
    const bool isY = blockIdx.x >= kScaleBlocks;
    const int blk = isY ? blockIdx.x - kScaleBlocks : blockIdx.x;
    const int R = isY ? a.N : a.M;
    const long long rows = (long long)R * a.nb;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    double m = 0.0;
    // warp per (batch, row), lanes along K: no division in the inner loop
    for (long long w = (long long)blk * nwb + wib; w < rows; w += (long long)kScaleBlocks * nwb) {
        const int b = (int)(w / R), r = (int)(w - (long long)b * R);
        if (isY) {
            const long long base = (a.yb ? a.yb[b] : 0) + a.yn[r];
            for (int k = lane; k < a.K; k += 32) m = fmax(m, fabs(a.Y[base + a.yk[k]]));
        } else {
            const long long base = (a.xb ? a.xb[b] : 0) + a.xm[r];
            for (int k = lane; k < a.K; k += 32) m = fmax(m, fabs(a.X[base + a.xk[k]]));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ double wm[8];
    if (lane == 0) wm[wib] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = 0.0;
        for (int w = 0; w < nwb; ++w) mm = fmax(mm, wm[w]);
        a.scale_ws[blockIdx.x] = mm;
    }
}

// power-of-two exponent e with max < 2^e (0 for a zero or non-finite maximum)
__device__ __forceinline__ int scale_exponent(double mx) {
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
    return e;
}

// Elements per packed tile and tile counts: X in 128-row tiles, Y in 64-row tiles, K in chunks of
// 32, zero-padded; tile (b, r, c) of an operand with R row tiles and C chunks starts at element
// ((b R + r) C + c) * rows * 32, and inside it element e sits where the shared-memory image puts
// it (tile_pos).  The lo tiles follow all hi tiles.
__host__ __device__ inline long long tc_tiles_x(const CtrLaunch& a) {
    return (long long)a.nb * ((a.M + TBM - 1) / TBM) * ((a.K + TBK - 1) / TBK);
}
__host__ __device__ inline long long tc_tiles_y(const CtrLaunch& a) {
    return (long long)a.nb * ((a.N + TBN - 1) / TBN) * ((a.K + TBK - 1) / TBK);
}

// Convert both operands once: gather through the tables, scale by the power of two from the
// max-abs pass, split into hi (and lo) in the tensor-core format, and write the tiles in
// shared-memory image order, so that the contraction kernel only copies bytes.
template <bool BF16, bool X3>
__global__ void __launch_bounds__(256) ctr_pack_kernel(const CtrLaunch a) {
    using O = Op<BF16>;
    using T = typename O::T;
    constexpr int E = O::kElem;
    __shared__ double wm[2][8];
    double mx = 0.0, my = 0.0;
    for (int i = threadIdx.x; i < kScaleBlocks; i += blockDim.x) {
        mx = fmax(mx, a.scale_ws[i]);
        my = fmax(my, a.scale_ws[kScaleBlocks + i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
    }
    if ((threadIdx.x & 31) == 0) {
        wm[0][threadIdx.x >> 5] = mx;
        wm[1][threadIdx.x >> 5] = my;
    }
    __syncthreads();
    mx = my = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        mx = fmax(mx, wm[0][w]);
        my = fmax(my, wm[1][w]);
    }
    const double sx = ldexp(1.0, -scale_exponent(mx)), sy = ldexp(1.0, -scale_exponent(my));
    const int nkc = (a.K + TBK - 1) / TBK;
    const long long tx = tc_tiles_x(a), ty = tc_tiles_y(a);
    const long long nx = tx * (TBM * TBK), ny = ty * (TBN * TBK);
    T* xh = (T*)a.pack_x;
    T* yh = (T*)a.pack_y;
    // block per tile (X tiles, then Y tiles), threads over the tile's elements: the tile is
    // decoded once per thread, the element position by tile_pos (compile-time divisors)
    for (long long tile = blockIdx.x; tile < tx + ty; tile += gridDim.x) {
        const bool isY = tile >= tx;
        const long long t = isY ? tile - tx : tile;
        const int rows = isY ? TBN : TBM;
        const int c = (int)(t % nkc);
        const long long br = t / nkc;
        const int nrt = isY ? (a.N + TBN - 1) / TBN : (a.M + TBM - 1) / TBM;
        const int r = (int)(br % nrt), b = (int)(br / nrt);
        const long long xbo = (!isY && a.xb) ? a.xb[b] : 0, ybo = (isY && a.yb) ? a.yb[b] : 0;
        T* dst = (isY ? yh : xh) + t * (long long)(rows * TBK);
        const long long lo_off = isY ? ny : nx;
        for (int e = threadIdx.x; e < rows * TBK; e += blockDim.x) {
            int rr, kk;
            tile_pos<E>(e, rr, kk);
            const int row = r * rows + rr, k = c * TBK + kk;
            double v = 0.0;
            if (isY) {
                if (row < a.N && k < a.K) v = a.Y[ybo + a.yk[k] + a.yn[row]] * sy;
            } else {
                if (row < a.M && k < a.K) v = a.X[xbo + a.xm[row] + a.xk[k]] * sx;
            }
            T hi, lo;
            O::split(v, hi, lo);
            dst[e] = hi;
            if (X3) dst[lo_off + e] = lo;
        }
    }
}

template <bool BF16, bool X3>
__global__ void __launch_bounds__(TNT) ctr_tc_kernel(const CtrLaunch a) {
    using O = Op<BF16>;
    using T = typename O::T;
    constexpr int E = O::kElem;
    constexpr uint32_t A_BYTES = TBM * TBK * E, B_BYTES = TBN * TBK * E;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + A_BYTES;
    unsigned char* b_hi = smem + 2 * A_BYTES;
    unsigned char* b_lo = smem + 2 * A_BYTES + B_BYTES;
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;
    __shared__ double s_mx[2][TNT / 32];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
    const int z = blockIdx.z;
    const int b = z / a.splits, sp = z % a.splits;

    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t bar = smem_u32(&mbar);
    // the packed operands were scaled by 2^-ex, 2^-ey (exact, max |.| < 1); the product is scaled
    // back by 2^(ex + ey) in FP64 before it is stored
    {
        double mx = 0.0, my = 0.0;
        for (int i = tid; i < kScaleBlocks; i += TNT) {
            mx = fmax(mx, a.scale_ws[i]);
            my = fmax(my, a.scale_ws[kScaleBlocks + i]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
        }
        if (lane == 0) {
            s_mx[0][warp] = mx;
            s_mx[1][warp] = my;
        }
        __syncthreads();
    }
    double mxa = 0.0, mya = 0.0;
#pragma unroll
    for (int w = 0; w < TNT / 32; ++w) {
        mxa = fmax(mxa, s_mx[0][w]);
        mya = fmax(mya, s_mx[1][w]);
    }
    const int ex = scale_exponent(mxa), ey = scale_exponent(mya);
    const double sxy = ldexp(1.0, ex + ey);

    const int kbeg = sp * a.kchunk;
    const int kend = min(a.K, kbeg + a.kchunk);
    constexpr uint32_t idesc = instr_desc(O::kFmt, TBM, TBN);
    constexpr uint32_t LBO = 128, A_SBO = (TBK * E / 16) * 128, B_SBO = A_SBO;
    uint32_t phase = 0, fail_phase = 0;
    bool first = true;
    bool ok = true;
    const int nkc = (a.K + TBK - 1) / TBK;
    const long long xtiles = tc_tiles_x(a), ytiles = tc_tiles_y(a);

    for (int k0 = kbeg; k0 < kend && ok; k0 += TBK) {
        // copy the packed tiles (already in shared-memory image order) with 16-byte moves
        {
            const int kc = k0 / TBK;
            const long long xt = ((long long)b * gridDim.y + blockIdx.y) * nkc + kc;
            const long long yt = ((long long)b * gridDim.x + blockIdx.x) * nkc + kc;
            const uint4* gx = reinterpret_cast<const uint4*>(
                reinterpret_cast<const unsigned char*>(a.pack_x) + xt * A_BYTES);
            const uint4* gy = reinterpret_cast<const uint4*>(
                reinterpret_cast<const unsigned char*>(a.pack_y) + yt * B_BYTES);
            uint4* sa = reinterpret_cast<uint4*>(a_hi);
            uint4* sb = reinterpret_cast<uint4*>(b_hi);
            constexpr int NA = A_BYTES / 16, NB = B_BYTES / 16;
#pragma unroll
            for (int i = tid; i < NA; i += TNT) sa[i] = gx[i];
#pragma unroll
            for (int i = tid; i < NB; i += TNT) sb[i] = gy[i];
            if (X3) {
                const uint4* gxl = reinterpret_cast<const uint4*>(
                    reinterpret_cast<const unsigned char*>(a.pack_x) + (xtiles + xt) * A_BYTES);
                const uint4* gyl = reinterpret_cast<const uint4*>(
                    reinterpret_cast<const unsigned char*>(a.pack_y) + (ytiles + yt) * B_BYTES);
                uint4* sal = reinterpret_cast<uint4*>(a_lo);
                uint4* sbl = reinterpret_cast<uint4*>(b_lo);
#pragma unroll
                for (int i = tid; i < NA; i += TNT) sal[i] = gxl[i];
#pragma unroll
                for (int i = tid; i < NB; i += TNT) sbl[i] = gyl[i];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo);
            const uint32_t bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
            for (int s = 0; s < TBK / O::kMmaK; ++s) {
                const uint32_t step = s * (O::kMmaK * E / 16) * 128;  // core matrices per K-step
                const uint64_t dah = smem_desc(ah + step, LBO, A_SBO);
                const uint64_t dbh = smem_desc(bh + step, LBO, B_SBO);
                mma<BF16>(tmem, dah, dbh, idesc, first ? 0u : 1u);
                first = false;
                if (X3) {
                    const uint64_t dal = smem_desc(al + step, LBO, A_SBO);
                    const uint64_t dbl = smem_desc(bl + step, LBO, B_SBO);
                    mma<BF16>(tmem, dah, dbl, idesc, 1u);
                    mma<BF16>(tmem, dal, dbh, idesc, 1u);
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    bar)
                : "memory");
        }
        first = false;
        // every thread waits for the MMAs before the tiles are overwritten
        if (!mbar_wait(bar, phase, (k0 == kbeg && a.first_wait_limit >= 0) ? a.first_wait_limit
                                                                              : kSpinLimit)) {
            ok = false;
            s_fail = 1;
            fail_phase = phase;
        }
        phase ^= 1u;
        __syncthreads();
        if (s_fail) ok = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");

    if (ok && !first) {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (tile rows), 16 columns at a time
        const int m = m0 + warp * 32 + lane;
        const bool mrow = m < a.M;
        const double rs = (mrow && a.rowscale) ? a.rowscale[m] : 1.0;
        const long long obo = a.ob ? a.ob[b] : 0;
#pragma unroll
        for (int c0 = 0; c0 < TBN; c0 += 16) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
                "%10, %11, %12, %13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (mrow) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n >= a.N) continue;
                    const double v = (double)__uint_as_float(r[j]) * sxy;
                    if (a.splits > 1) {
                        a.partial[((long long)z * a.M + m) * a.N + n] = v;
                    } else {
                        double w = v * rs;
                        if (a.colscale) w *= a.colscale[n];
                        a.O[obo + a.om[m] + a.on[n]] = w;
                    }
                }
            }
        }
    } else if (ok && first) {
        // empty K range: the contraction (or this split's part of it) is zero
        const int m = m0 + warp * 32 + lane;
        if (m < a.M) {
            const long long obo = a.ob ? a.ob[b] : 0;
            for (int n = n0; n < min(a.N, n0 + TBN); ++n) {
                if (a.splits > 1)
                    a.partial[((long long)z * a.M + m) * a.N + n] = 0.0;
                else
                    a.O[obo + a.om[m] + a.on[n]] = 0.0;
            }
        }
    }
    if (!ok) {
        // drain: wait (bounded) for the MMAs still in flight before the tensor memory is freed
        mbar_wait(bar, fail_phase);
        if (tid == 0 && a.err) atomicExch(a.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols));
    }
}

size_t tc_pack_bytes_x(const CtrLaunch& a) { return (size_t)tc_tiles_x(a) * TBM * TBK * 4 * 2; }
size_t tc_pack_bytes_y(const CtrLaunch& a) { return (size_t)tc_tiles_y(a) * TBN * TBK * 4 * 2; }

template <bool BF16, bool X3>
static void launch_tc(const CtrLaunch& a, cudaStream_t s) {
    {
        const long long tiles = tc_tiles_x(a) + tc_tiles_y(a);
        const int blocks = (int)std::min<long long>(tiles, 8192);
        ctr_pack_kernel<BF16, X3><<<std::max(blocks, 1), 256, 0, s>>>(a);
    }
    constexpr int E = BF16 ? 2 : 4;
    // hi and lo tiles of A and B; at least 32 KB so that at most 7 CTAs share an SM and their
    // 64-column tensor-memory allocations (7 x 64 <= 512) never wait on one another
    const size_t smem = std::max<size_t>(2 * (size_t)(TBM + TBN) * TBK * E, 32768);
    static std::once_flag attr_once;
    std::call_once(attr_once, [&] {
        cudaFuncSetAttribute(ctr_tc_kernel<BF16, X3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    });
    dim3 grid((a.N + TBN - 1) / TBN, (a.M + TBM - 1) / TBM, a.nb * a.splits);
    ctr_tc_kernel<BF16, X3><<<grid, TNT, smem, s>>>(a);
}

void launch_ctr_tc(const CtrLaunch& a, cudaStream_t s) {
    if (a.precision == SCTM_PREC_F64EMU) {
        launch_ctr_emu(a, s);
        return;
    }
    ctr_maxabs_kernel<<<2 * kScaleBlocks, 256, 0, s>>>(a);
    switch (a.precision) {
        case SCTM_PREC_TF32: launch_tc<false, false>(a, s); break;
        case SCTM_PREC_TF32X3: launch_tc<false, true>(a, s); break;
        case SCTM_PREC_BF16: launch_tc<true, false>(a, s); break;
        default: launch_tc<true, true>(a, s); break;
    }
}

}  // namespace sctm
