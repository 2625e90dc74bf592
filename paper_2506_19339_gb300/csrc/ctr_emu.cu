// FP64-accurate contraction on the BF16 tensor cores (SCTM_PREC_F64EMU): an Ozaki-type
// error-free split.  Each row of X (each column of Y) is scaled by a power of two 2^-e with
// max |.| < 1 over K; an element x then becomes the 56-bit integer N = trunc(x 2^(56-e)), written
// as eight signed 7-bit digits a_1..a_8 (|a_t| <= 127, exact in BF16):
//     x = 2^e sum_t a_t 2^(-7t)      (up to 2^-56 of the row maximum).
// A product x y = 2^(ex+ey) sum_{t,u} a_t b_u 2^(-7(t+u)); the 36 digit pairs with t + u <= 9 are
// kept (the rest lie below 2^-63 of the leading term).  Pairs of one level L = t + u share a
// tensor-memory accumulator (8 levels x 64 FP32 columns = the whole 512-column tensor memory):
// a level sum over K blocks of 128 is an integer below 8 * 127^2 * 128 < 2^24, so FP32
// accumulation in the tensor core is exact.  After each K block the four leading level sums
// (L = 0..3) are read back (tcgen05.ld), combined exactly into one 64-bit integer (below 2^46)
// and added to a 64-bit integer accumulator, and their MMAs restart the accumulators.  The four
// trailing levels (L = 4..7) weigh 2^-28 and less of the leading one: they accumulate in FP32 in
// the tensor memory over all of K (rounding 2^-24 of their sum, below 2^-52 of the product
// bound) and are read once at the end.  FP64 arithmetic is spent once per operand element (the
// digit split) and a few times per output element, none per K block: this GPU's FP64 rate is a
// small fraction of its integer and FP32 rates.
//
// Data movement: the digit split writes, per (row tile, K chunk of 32), the eight digit tiles
// contiguously in the shared-memory image order (K-major, no swizzle), so one K chunk of the A
// operand is a single 64 KB bulk copy and of the B operand a single 32 KB one.  The contraction
// kernel keeps two such chunks in flight (cp.async.bulk into a two-stage shared-memory ring,
// completion counted on an mbarrier per stage), one thread issues the 72 MMAs of a chunk
// (36 digit pairs x 2 K-steps of 16) as soon as its stage has landed, and refills the stage
// once a tcgen05.commit reports those MMAs done, so loads overlap the tensor-core work.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sctm_internal.h"

namespace sctm {

namespace {

constexpr int EBM = 128, EBN = 64, EBK = 32, ENT = 256;
constexpr int kColsPerThread = EBN / 2;  // warps w and w + 4 share TMEM lanes 32 (w % 4)..
constexpr int kDigits = 8;                   // slices per operand element
constexpr int kLevels = 8;                   // levels L = t + u - 2 = 0..7
constexpr int kBlockChunks = 4;              // K block of 4 x 32 = 128 between read-backs
constexpr int kEmuTmemCols = kLevels * EBN;  // 512
constexpr long long kEmuSpinLimit = 1LL << 20;
constexpr uint32_t kSliceA = EBM * EBK * 2, kSliceB = EBN * EBK * 2;  // bytes per BF16 slice tile
constexpr uint32_t kChunkA = kDigits * kSliceA, kChunkB = kDigits * kSliceB;  // 64 KB, 32 KB
constexpr uint32_t kStageBytes = kChunkA + kChunkB;
constexpr int kStages = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// kind::f16 instruction descriptor: D = F32, A = B = BF16, K-major, N = 64, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((EBN >> 3) << 17) | ((EBM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kEmuSpinLimit) {
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

// The integer value of an FP32 number that holds an exact integer of magnitude below 2^24 (a
// level sum), decoded from its IEEE-754 fields with integer operations only: on this GPU the
// float-to-integer conversion instruction shares the slow FP64 pipe, and the level read-back
// converts 128 values per thread per K block.
__device__ __forceinline__ int level_to_int(float f) {
    const unsigned u = __float_as_uint(f);
    const int e = (int)((u >> 23) & 0xFFu);  // biased exponent: 0 for zero, 127..150 otherwise
    const int mag = e == 0 ? 0 : (int)((0x800000u | (u & 0x7FFFFFu)) >> (150 - e));
    return (u >> 31) ? -mag : mag;
}

// 2^e as a double for a frexp exponent of a finite double (e in [-1073, 1024]): built from its
// bits in one or two normal factors, so that a product by it is the exact scaling ldexp would do
// (up to the rounding of a subnormal result)
__device__ __forceinline__ double pow2_lo(int e) {  // e in [-1022, 1023]
    return __longlong_as_double((long long)(e + 1023) << 52);
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// one bulk (non-tensor) copy global -> shared, completion counted on the mbarrier in bytes;
// both addresses 16-byte aligned and the size a multiple of 16
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
}

// element e of a (rows x 32) BF16 tile in the no-swizzle K-major core-matrix image (byte e * 2)
__device__ __forceinline__ void tile_pos_bf16(int e, int& r, int& k) {
    const int kin = e % 8, rin = (e / 8) % 8, chunk = (e / 64) % 4, group = e / 256;
    r = group * 8 + rin;
    k = chunk * 8 + kin;
}

__host__ __device__ inline long long emu_tiles_x(const CtrLaunch& a) {
    return (long long)a.nb * ((a.M + EBM - 1) / EBM) * ((a.K + EBK - 1) / EBK);
}
__host__ __device__ inline long long emu_tiles_y(const CtrLaunch& a) {
    return (long long)a.nb * ((a.N + EBN - 1) / EBN) * ((a.K + EBK - 1) / EBK);
}

}  // namespace

// Row exponents: ex[b M + m] with max_k |X[b][m][k]| < 2^ex (0 for a zero row), and likewise
// ey[b N + n] over the columns of Y.  A warp per row, lanes along K.
__global__ void __launch_bounds__(256) emu_rowexp_kernel(const CtrLaunch a, int* ex, int* ey) {
    const int lane = threadIdx.x & 31;
    const long long wpg = (long long)gridDim.x * (blockDim.x >> 5);
    const long long rx = (long long)a.nb * a.M, ry = (long long)a.nb * a.N;
    for (long long w = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); w < rx + ry;
         w += wpg) {
        const bool isY = w >= rx;
        const long long q = isY ? w - rx : w;
        const int R = isY ? a.N : a.M;
        const int b = (int)(q / R), r = (int)(q - (long long)b * R);
        // max |x| as the largest bit pattern of |x| (non-negative doubles order as integers):
        // integer operations only, the FP64 pipe of this GPU being slow
        unsigned long long m = 0;
        if (isY) {
            const long long base = (a.yb ? a.yb[b] : 0) + a.yn[r];
            for (int k = lane; k < a.K; k += 32)
                m = max(m, (unsigned long long)__double_as_longlong(a.Y[base + a.yk[k]]) &
                               0x7FFFFFFFFFFFFFFFull);
        } else {
            const long long base = (a.xb ? a.xb[b] : 0) + a.xm[r];
            for (int k = lane; k < a.K; k += 32)
                m = max(m, (unsigned long long)__double_as_longlong(a.X[base + a.xk[k]]) &
                               0x7FFFFFFFFFFFFFFFull);
        }
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            int e = 0;
            const double md = __longlong_as_double((long long)m);
            if (md > 0.0 && isfinite(md)) frexp(md, &e);
            (isY ? ey : ex)[q] = e;
        }
    }
}

// Digit split of both operands into kDigits BF16 slices, tiles in shared-memory image order;
// tile t (over batch, row tile, K chunk) holds its kDigits digit tiles contiguously, digit d at
// (t kDigits + d) x (tile bytes).  A block per tile.
__global__ void __launch_bounds__(256) emu_pack_kernel(const CtrLaunch a, const int* ex,
                                                       const int* ey) {
    const int nkc = (a.K + EBK - 1) / EBK;
    const long long tx = emu_tiles_x(a), ty = emu_tiles_y(a);
    unsigned short* xp = (unsigned short*)a.pack_x;
    unsigned short* yp = (unsigned short*)a.pack_y;
    for (long long tile = blockIdx.x; tile < tx + ty; tile += gridDim.x) {
        const bool isY = tile >= tx;
        const long long t = isY ? tile - tx : tile;
        const int rows = isY ? EBN : EBM;
        const int c = (int)(t % nkc);
        const long long br = t / nkc;
        const int nrt = isY ? (a.N + EBN - 1) / EBN : (a.M + EBM - 1) / EBM;
        const int r = (int)(br % nrt), b = (int)(br / nrt);
        const long long slice = rows * EBK;
        unsigned short* dst = (isY ? yp : xp) + t * (long long)(kDigits * rows * EBK);
        for (int e = threadIdx.x; e < rows * EBK; e += blockDim.x) {
            int rr, kk;
            tile_pos_bf16(e, rr, kk);
            const int row = r * rows + rr, k = c * EBK + kk;
            double v = 0.0;
            int er = 0;
            if (isY) {
                if (row < a.N && k < a.K) {
                    v = a.Y[(a.yb ? a.yb[b] : 0) + a.yk[k] + a.yn[row]];
                    er = ey[(long long)b * a.N + row];
                }
            } else {
                if (row < a.M && k < a.K) {
                    v = a.X[(a.xb ? a.xb[b] : 0) + a.xm[row] + a.xk[k]];
                    er = ex[(long long)b * a.M + row];
                }
            }
            // |v| < 2^er, so N = trunc(|v| 2^(56 - er)) < 2^56 (exact to 2^-56 of the row
            // maximum), taken from the IEEE-754 fields of v: |v| = mant 2^(E' - 1075)
            const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
            const unsigned neg = (unsigned)(bits >> 63);
            const int E = (int)((bits >> 52) & 0x7FFull);
            const unsigned long long mant =
                (bits & 0xFFFFFFFFFFFFFull) | (E ? 0x10000000000000ull : 0ull);
            const int sh = (E ? E : 1) - 1075 + 56 - er;
            const unsigned long long mag =
                sh >= 0 ? (mant << sh) : (sh > -64 ? (mant >> (-sh)) : 0ull);
#pragma unroll
            for (int d = 0; d < kDigits; ++d) {
                // the 7-bit digit as a BF16 bit pattern (exact): sign, exponent 127 + p with
                // p = floor(log2 digit), the digit's bits below its leading one as mantissa
                const unsigned chunk = (unsigned)((mag >> (7 * (kDigits - 1 - d))) & 127ull);
                unsigned short h = 0;
                if (chunk) {
                    const int p = 31 - __clz(chunk);
                    h = (unsigned short)((neg << 15) | ((127u + p) << 7) |
                                         ((chunk << (7 - p)) & 0x7Fu));
                }
                dst[d * slice + e] = h;
            }
        }
    }
}

__global__ void __launch_bounds__(ENT, 1) emu_ctr_kernel(const CtrLaunch a, const int* ex,
                                                         const int* ey) {
    extern __shared__ __align__(1024) unsigned char smem[];  // kStages x (A chunk, B chunk)
    __shared__ __align__(8) unsigned long long full_bar[kStages], mma_bar[kStages], acc_bar, drain_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * EBM, n0 = blockIdx.x * EBN;
    const int z = blockIdx.z;
    const int b = z / a.splits, sp = z % a.splits;
    const int kbeg = sp * a.kchunk;
    const int kend = min(a.K, kbeg + a.kchunk);
    const int nch = kend > kbeg ? (kend - kbeg + EBK - 1) / EBK : 0;  // K chunks of this CTA
    const int cfirst = kbeg / EBK;                                    // kchunk is a multiple of EBK
    const int nkc = (a.K + EBK - 1) / EBK;
    if (tid == 0) {
        s_fail = 0;
        for (int s = 0; s < kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_bar[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_bar)));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&drain_bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kEmuTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const long long xt0 = ((long long)b * gridDim.y + blockIdx.y) * nkc + cfirst;
    const long long yt0 = ((long long)b * gridDim.x + blockIdx.x) * nkc + cfirst;
    const unsigned char* gx = reinterpret_cast<const unsigned char*>(a.pack_x);
    const unsigned char* gy = reinterpret_cast<const unsigned char*>(a.pack_y);
    constexpr uint32_t LBO = 128, SBO = (EBK * 2 / 16) * 128;

    // producer state (thread 0): phases of the stage barriers and the loads still in flight
    uint32_t fph[kStages] = {0, 0}, mph[kStages] = {0, 0}, aph = 0;
    bool pending[kStages] = {false, false};
    auto issue_load = [&](int c, int s) {
        const uint32_t fb = smem_u32(&full_bar[s]);
        const uint32_t dst = smem_u32(smem + (size_t)s * kStageBytes);
        mbar_expect_tx(fb, kStageBytes);
        bulk_load(dst, gx + (xt0 + c) * (long long)kChunkA, kChunkA, fb);
        bulk_load(dst + kChunkA, gy + (yt0 + c) * (long long)kChunkB, kChunkB, fb);
        pending[s] = true;
    };
    if (tid == 0)
        for (int c = 0; c < nch && c < kStages; ++c) issue_load(c, c);

    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows) and columns (w / 4) x 32 .. + 31
    const int quarter = warp & 3, colhalf = warp >> 2;
    long long acc[kColsPerThread];  // levels 0-3, in units of level 3, exact
#pragma unroll
    for (int j = 0; j < kColsPerThread; ++j) acc[j] = 0;

    for (int c = 0; c < nch; ++c) {
        const int s = c % kStages;
        const bool fresh = (c % kBlockChunks) == 0;  // first chunk of a K block
        if (tid == 0 && !s_fail) {
            const long long lim =
                (c == 0 && a.first_wait_limit >= 0) ? a.first_wait_limit : kEmuSpinLimit;
            if (!mbar_wait(smem_u32(&full_bar[s]), fph[s], lim)) {
                s_fail = 1;
            } else {
                fph[s] ^= 1u;
                pending[s] = false;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sa = smem_u32(smem + (size_t)s * kStageBytes);
                const uint32_t sb = sa + kChunkA;
                for (int da = 0; da < kDigits; ++da) {
                    for (int db = 0; db + da < kLevels; ++db) {
                        const int L = da + db;
                        const uint32_t ta = tmem + (uint32_t)(L * EBN);
                        // a level's first MMA (da == 0, st == 0) of a K block (levels 0-3) or of
                        // the whole contraction (levels 4-7) starts its accumulator
                        const bool start = da == 0 && (L < kLevels / 2 ? fresh : c == 0);
#pragma unroll
                        for (int st = 0; st < EBK / 16; ++st) {
                            const uint32_t step = st * 256;  // 16 BF16 along K = 2 core matrices
                            const uint64_t dA = smem_desc(sa + da * kSliceA + step, LBO, SBO);
                            const uint64_t dB = smem_desc(sb + db * kSliceB + step, LBO, SBO);
                            mma_bf16(ta, dA, dB, (start && st == 0) ? 0u : 1u);
                        }
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&mma_bar[s]))
                    : "memory");
                if (c + kStages < nch) {
                    // the stage is free once these MMAs have read it
                    if (!mbar_wait(smem_u32(&mma_bar[s]), mph[s])) {
                        s_fail = 1;
                    } else {
                        mph[s] ^= 1u;
                        issue_load(c + kStages, s);
                    }
                }
            }
        }
        if ((c % kBlockChunks) == kBlockChunks - 1 || c == nch - 1) {
            // end of a K block: the level sums are complete once every MMA issued so far is done
            if (tid == 0 && !s_fail) {
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        smem_u32(&acc_bar))
                    : "memory");
            }
            __syncthreads();
            if (s_fail) break;
            if (!mbar_wait(smem_u32(&acc_bar), aph)) atomicExch(&s_fail, 1);
            aph ^= 1u;
            __syncthreads();
            if (s_fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // the leading level sums are exact integers (|S| < 2^24): S_0 2^21 + S_1 2^14 +
            // S_2 2^7 + S_3 (below 2^46) is added exactly to the 64-bit accumulator
#pragma unroll
            for (int cb = 0; cb < kColsPerThread; cb += 8) {
                uint32_t r[4][8];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                                           (uint32_t)(q * EBN + colhalf * kColsPerThread + cb);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, "
                        "%7}, [%8];"
                        : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]),
                          "=r"(r[q][4]), "=r"(r[q][5]), "=r"(r[q][6]), "=r"(r[q][7])
                        : "r"(taddr));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    long long v = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        v = v * 128 + (long long)level_to_int(__uint_as_float(r[q][j]));
                    acc[cb + j] += v;
                }
            }
            // the next block's MMAs overwrite the accumulators only after every warp has read them
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
    }

    // the trailing levels 4-7 (FP32 sums over all of K, weights 2^-49 .. 2^-70 relative to the
    // accumulator's unit 2^-35): read once, combined in FP64 with the exact leading part
    double res[kColsPerThread];
    if (!s_fail) {
#pragma unroll
        for (int cb = 0; cb < kColsPerThread; cb += 8) {
            uint32_t r[4][8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) +
                                       (uint32_t)((4 + q) * EBN + colhalf * kColsPerThread + cb);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, "
                    "%7}, [%8];"
                    : "=r"(r[q][0]), "=r"(r[q][1]), "=r"(r[q][2]), "=r"(r[q][3]),
                      "=r"(r[q][4]), "=r"(r[q][5]), "=r"(r[q][6]), "=r"(r[q][7])
                    : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // S_4 2^21 + S_5 2^14 + S_6 2^7 + S_7 in FP32: its relative rounding (3 x 2^-24)
                // is below 2^-50 of the product bound, since this part weighs 2^-28 of it
                float lo = __uint_as_float(r[0][j]);
#pragma unroll
                for (int q = 1; q < 4; ++q) lo = fmaf(lo, 128.0f, __uint_as_float(r[q][j]));
                res[cb + j] = fma((double)lo, 0x1p-63, (double)acc[cb + j] * 0x1p-35);
            }
        }
    }

    if (!s_fail) {
        const int m = m0 + quarter * 32 + lane;
        if (m < a.M) {
            // exponents of frexp on finite doubles lie in [-1073, 1024]: split each into two
            // normal powers of two
            const int erow = ex[(long long)b * a.M + m];
            const double er1 = pow2_lo(erow / 2), er2 = pow2_lo(erow - erow / 2);
            const double rs = a.rowscale ? a.rowscale[m] : 1.0;
            const long long obo = a.ob ? a.ob[b] : 0;
#pragma unroll
            for (int j = 0; j < kColsPerThread; ++j) {
                const int n = n0 + colhalf * kColsPerThread + j;
                if (n >= a.N) continue;
                const int ec = ey[(long long)b * a.N + n], et = erow + ec;
                // one multiplication by 2^(erow + ec) when that is a normal power of two
                const double v = (et >= -1022 && et <= 1023)
                                     ? res[j] * pow2_lo(et)
                                     : res[j] * er1 * pow2_lo(ec / 2) * er2 * pow2_lo(ec - ec / 2);
                if (a.splits > 1) {
                    a.partial[((long long)z * a.M + m) * a.N + n] = v;
                } else {
                    double w = v * rs;
                    if (a.colscale) w *= a.colscale[n];
                    a.O[obo + a.om[m] + a.on[n]] = w;
                }
            }
        }
    } else if (tid == 0) {
        // drain (bounded) before the shared memory and the tensor memory are released: the bulk
        // copies still in flight, then every MMA this thread issued (a commit to a barrier used
        // for nothing else arrives once all of them have completed)
        for (int s = 0; s < kStages; ++s)
            if (pending[s]) mbar_wait(smem_u32(&full_bar[s]), fph[s]);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&drain_bar))
            : "memory");
        mbar_wait(smem_u32(&drain_bar), 0u);
        if (a.err) atomicExch(a.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kEmuTmemCols));
    }
}

size_t emu_pack_bytes_x(const CtrLaunch& a) { return (size_t)emu_tiles_x(a) * kDigits * kSliceA; }
size_t emu_pack_bytes_y(const CtrLaunch& a) { return (size_t)emu_tiles_y(a) * kDigits * kSliceB; }
size_t emu_exp_ints(const CtrLaunch& a) { return (size_t)a.nb * (a.M + a.N); }

void launch_ctr_emu(const CtrLaunch& a, cudaStream_t s) {
    int* ex = a.rexp;
    int* ey = a.rexp + (long long)a.nb * a.M;
    {
        const long long rows = (long long)a.nb * (a.M + a.N);
        const int blocks = (int)std::min<long long>((rows + 7) / 8, 4096);
        emu_rowexp_kernel<<<std::max(blocks, 1), 256, 0, s>>>(a, ex, ey);
    }
    {
        const long long tiles = emu_tiles_x(a) + emu_tiles_y(a);
        emu_pack_kernel<<<(int)std::min<long long>(std::max<long long>(tiles, 1), 8192), 256, 0, s>>>(
            a, ex, ey);
    }
    // two stages of 96 KB: one CTA per SM, which owns the whole tensor memory
    const size_t smem = (size_t)kStages * kStageBytes;
    static std::once_flag once;
    std::call_once(once, [&] {
        cudaFuncSetAttribute(emu_ctr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    dim3 grid((a.N + EBN - 1) / EBN, (a.M + EBM - 1) / EBM, a.nb * a.splits);
    emu_ctr_kernel<<<grid, ENT, smem, s>>>(a, ex, ey);
}

}  // namespace sctm
