// FP64-accurate contraction on the BF16 tensor cores (SCTM_PREC_F64EMU): an Ozaki-type
// error-free split.  Each row of X (each column of Y) is scaled by a power of two 2^-e with
// max |.| < 1 over K; an element x then becomes the 56-bit integer N = trunc(x 2^(56-e)), written
// as eight signed 7-bit digits a_1..a_8 (|a_t| <= 127, exact in BF16):
//     x = 2^e sum_t a_t 2^(-7t)      (up to 2^-56 of the row maximum).
// A product x y = 2^(ex+ey) sum_{t,u} a_t b_u 2^(-7(t+u)); the 36 digit pairs with t + u <= 9 are
// kept (the rest lie below 2^-63 of the leading term).  Pairs of one level L = t + u share a
// tensor-memory accumulator (8 levels x 64 FP32 columns = the whole 512-column tensor memory):
// a level sum over K blocks of 128 is an integer below 8 * 127^2 * 128 < 2^24, so FP32
// accumulation in the tensor core is exact.  After each K block the eight level sums are read
// back (tcgen05.ld) and added into FP64 registers with their weights 2^(-7L), and the block's
// MMAs restart the accumulators.  FP64 arithmetic is spent once per operand element (the digit
// split) and once per output element and level per 128 K, not per multiply-add.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "sctm_internal.h"

namespace sctm {

namespace {

constexpr int EBM = 128, EBN = 64, EBK = 32, ENT = 128;
constexpr int kDigits = 8;                   // slices per operand element
constexpr int kLevels = 8;                   // levels L = t + u - 2 = 0..7
constexpr int kBlockChunks = 4;              // K block of 4 x 32 = 128 between read-backs
constexpr int kEmuTmemCols = kLevels * EBN;  // 512
constexpr long long kEmuSpinLimit = 1LL << 20;
constexpr uint32_t kSliceA = EBM * EBK * 2, kSliceB = EBN * EBK * 2;  // bytes per BF16 slice tile

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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kEmuSpinLimit; ++i) {
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
        double m = 0.0;
        if (isY) {
            const long long base = (a.yb ? a.yb[b] : 0) + a.yn[r];
            for (int k = lane; k < a.K; k += 32) m = fmax(m, fabs(a.Y[base + a.yk[k]]));
        } else {
            const long long base = (a.xb ? a.xb[b] : 0) + a.xm[r];
            for (int k = lane; k < a.K; k += 32) m = fmax(m, fabs(a.X[base + a.xk[k]]));
        }
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            int e = 0;
            if (m > 0.0 && isfinite(m)) frexp(m, &e);
            (isY ? ey : ex)[q] = e;
        }
    }
}

// Digit split of both operands into kDigits BF16 slices, tiles in shared-memory image order
// (slice-major: all tiles of digit 1, then digit 2, ...).  A block per tile.
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
        const long long slice = (isY ? ty : tx) * (long long)(rows * EBK);
        unsigned short* dst = (isY ? yp : xp) + t * (long long)(rows * EBK);
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
            // |v| < 2^er, so |N| < 2^56 and the truncation is exact to 2^-56 of the row maximum
            const long long N = __double2ll_rz(ldexp(v, 56 - er));
            const unsigned long long mag = (unsigned long long)(N < 0 ? -N : N);
            const float sgn = N < 0 ? -1.0f : 1.0f;
#pragma unroll
            for (int d = 0; d < kDigits; ++d) {
                const int chunk = (int)((mag >> (7 * (kDigits - 1 - d))) & 127ull);
                const __nv_bfloat16 h = __float2bfloat16_rn(sgn * (float)chunk);  // exact
                dst[d * slice + e] = *reinterpret_cast<const unsigned short*>(&h);
            }
        }
    }
}

__global__ void __launch_bounds__(ENT) emu_ctr_kernel(const CtrLaunch a, const int* ex,
                                                      const int* ey) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sa = smem;                       // kDigits A slices
    unsigned char* sb = smem + kDigits * kSliceA;   // kDigits B slices
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * EBM, n0 = blockIdx.x * EBN;
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
                     "r"(kEmuTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t bar = smem_u32(&mbar);

    const int kbeg = sp * a.kchunk;
    const int kend = min(a.K, kbeg + a.kchunk);
    const int nkc = (a.K + EBK - 1) / EBK;
    const long long xtiles = emu_tiles_x(a), ytiles = emu_tiles_y(a);
    constexpr uint32_t LBO = 128, SBO = (EBK * 2 / 16) * 128;
    uint32_t phase = 0, fail_phase = 0;
    bool ok = true;
    double acc[EBN];
#pragma unroll
    for (int j = 0; j < EBN; ++j) acc[j] = 0.0;

    for (int kb = kbeg; kb < kend && ok; kb += kBlockChunks * EBK) {
        const int kbend = min(kend, kb + kBlockChunks * EBK);
        bool fresh = true;  // the block's first MMA into each level starts that accumulator
        for (int k0 = kb; k0 < kbend && ok; k0 += EBK) {
            {
                const int kc = k0 / EBK;
                const long long xt = ((long long)b * gridDim.y + blockIdx.y) * nkc + kc;
                const long long yt = ((long long)b * gridDim.x + blockIdx.x) * nkc + kc;
#pragma unroll
                for (int d = 0; d < kDigits; ++d) {
                    const uint4* gx = reinterpret_cast<const uint4*>(
                        reinterpret_cast<const unsigned char*>(a.pack_x) +
                        ((long long)d * xtiles + xt) * kSliceA);
                    const uint4* gy = reinterpret_cast<const uint4*>(
                        reinterpret_cast<const unsigned char*>(a.pack_y) +
                        ((long long)d * ytiles + yt) * kSliceB);
                    uint4* dx = reinterpret_cast<uint4*>(sa + d * kSliceA);
                    uint4* dy = reinterpret_cast<uint4*>(sb + d * kSliceB);
                    for (int i = tid; i < (int)(kSliceA / 16); i += ENT) dx[i] = gx[i];
                    for (int i = tid; i < (int)(kSliceB / 16); i += ENT) dy[i] = gy[i];
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int da = 0; da < kDigits; ++da) {
                    for (int db = 0; db + da < kLevels; ++db) {
                        const int L = da + db;
                        const uint32_t ta = tmem + (uint32_t)(L * EBN);
#pragma unroll
                        for (int s = 0; s < EBK / 16; ++s) {
                            const uint32_t step = s * 256;  // 16 BF16 along K = 2 core matrices
                            const uint64_t dA = smem_desc(smem_u32(sa + da * kSliceA) + step, LBO, SBO);
                            const uint64_t dB = smem_desc(smem_u32(sb + db * kSliceB) + step, LBO, SBO);
                            // first MMA into level L in this block: da == 0 holds every level's
                            // first pair (db = L), issued before any other pair of that level
                            mma_bf16(ta, dA, dB, (fresh && da == 0 && s == 0) ? 0u : 1u);
                        }
                    }
                }
                asm volatile(
                    "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        bar)
                    : "memory");
            }
            fresh = false;
            if (!mbar_wait(bar, phase)) {
                ok = false;
                s_fail = 1;
                fail_phase = phase;
            }
            phase ^= 1u;
            __syncthreads();
            if (s_fail) ok = false;
        }
        if (!ok) break;
        // read back the eight level sums of this K block into the FP64 accumulators
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
        for (int L = 0; L < kLevels; ++L) {
            const double w = ldexp(1.0, -7 * (L + 2));
#pragma unroll
            for (int c0 = 0; c0 < EBN; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(L * EBN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
                    "%9, %10, %11, %12, %13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; ++j) acc[c0 + j] = fma((double)__uint_as_float(r[j]), w, acc[c0 + j]);
            }
        }
        // the next block's MMAs overwrite the accumulators only after every warp has read them
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }

    if (ok) {
        const int m = m0 + warp * 32 + lane;
        if (m < a.M) {
            const int erow = ex[(long long)b * a.M + m];
            const double rs = a.rowscale ? a.rowscale[m] : 1.0;
            const long long obo = a.ob ? a.ob[b] : 0;
#pragma unroll
            for (int j = 0; j < EBN; ++j) {
                const int n = n0 + j;
                if (n >= a.N) continue;
                const double v = ldexp(acc[j], erow + ey[(long long)b * a.N + n]);
                if (a.splits > 1) {
                    a.partial[((long long)z * a.M + m) * a.N + n] = v;
                } else {
                    double w = v * rs;
                    if (a.colscale) w *= a.colscale[n];
                    a.O[obo + a.om[m] + a.on[n]] = w;
                }
            }
        }
    } else {
        mbar_wait(bar, fail_phase);  // drain (bounded) before the tensor memory is freed
        if (tid == 0 && a.err) atomicExch(a.err, 1);
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
    // > 114 KB of shared memory: one CTA per SM, which owns the whole tensor memory
    const size_t smem = std::max<size_t>(kDigits * (kSliceA + kSliceB), 120 * 1024);
    static std::once_flag once;
    std::call_once(once, [&] {
        cudaFuncSetAttribute(emu_ctr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    dim3 grid((a.N + EBN - 1) / EBN, (a.M + EBM - 1) / EBM, a.nb * a.splits);
    emu_ctr_kernel<<<grid, ENT, smem, s>>>(a, ex, ey);
}

}  // namespace sctm
