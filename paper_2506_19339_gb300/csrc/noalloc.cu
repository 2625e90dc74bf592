// sctm_gemm_noalloc: the library's FP64 contraction for plain row-major operands, for callers
// that cannot allocate device memory.  The split-K partial sums, which the context-based path
// keeps in a buffer it allocates when a plan is built, live here in one file-scope device array.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "sctm.h"

namespace {

// Maximum number of doubles of split-K partial sums (16 MiB); also the largest M*N accepted.
constexpr long long kScratchDoubles = 1LL << 21;
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_scratch[kScratchDoubles];

// O = X Y with X (M x K), Y (K x N), O (M x N) row-major.  Same tiling as the gather-table
// contraction: 64 x 64 tile per CTA, 4 x 4 per thread, K in chunks of 16.  With splits > 1, CTA z
// covers K range [z*kchunk, (z+1)*kchunk) and writes its tile to part + z*M*N.
__global__ void __launch_bounds__(NT) gemm_rowmajor_kernel(const double* __restrict__ X,
                                                            const double* __restrict__ Y,
                                                            double* __restrict__ O, int M, int N,
                                                            int K, int splits, int kchunk,
                                                            double* part) {
    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, z = blockIdx.z;
    const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + NT * q, kk = e & (BK - 1), mm = e >> 4;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < kend) ? X[(long long)m * K + k] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + NT * q, nn = e & (BN - 1), kk = e >> 6;
            const int n = n0 + nn, k = k0 + kk;
            Bs[kk][nn] = (n < N && k < kend) ? Y[(long long)k * N + n] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* dst = splits > 1 ? part + (long long)z * M * N : O;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n < N) dst[(long long)m * N + n] = acc[i][j];
        }
    }
}

// O[m][n] = sum over the splits, in split order (deterministic).
__global__ void splitk_sum_kernel(const double* part, double* O, long long MN, int splits) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < MN;
         t += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int s = 0; s < splits; ++s) v += part[(long long)s * MN + t];
        O[t] = v;
    }
}

std::mutex g_setup_mutex;
double* g_scratch_dev[kMaxDevices] = {nullptr};

// True if p is device (or managed) memory that belongs to device `dev`.  Memory of another GPU
// is rejected: the kernel runs on the current device, and reaching another GPU's memory without
// peer access would fault instead of returning an error.
bool is_device_pointer_on(const void* p, int dev) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clears only the error this query itself raised
        return false;
    }
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == dev;
}

// True if the stream is the legacy / per-thread default stream or was created on `dev`.
bool stream_on(cudaStream_t s, int dev) {
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return true;
    int sd = -1;
    if (cudaStreamGetDevice(s, &sd) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return sd == dev;
}

}  // namespace

extern "C" sctm_status sctm_gemm_noalloc(const double* X, const double* Y, double* O, int M, int N,
                                         int K, void* cuda_stream) {
    if (!X || !Y || !O || M < 1 || N < 1 || K < 1) return SCTM_EINVAL;
    if ((long long)M * N > kScratchDoubles) return SCTM_EINVAL;  // M*N above 2^21 doubles
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SCTM_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!is_device_pointer_on(X, dev) || !is_device_pointer_on(Y, dev) ||
        !is_device_pointer_on(O, dev) || !stream_on(s, dev))
        return SCTM_EINVAL;
    // An error left pending by earlier, unrelated work is not this call's: report it without
    // launching and without clearing it.
    if (cudaPeekAtLastError() != cudaSuccess) return SCTM_ECUDA;
    double* scratch = nullptr;
    {
        // Once per device, with that device current: the scratch array's device address.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_dev[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SCTM_ECUDA;
            }
            g_scratch_dev[dev] = (double*)p;
        }
        scratch = g_scratch_dev[dev];
    }
    const long long MN = (long long)M * N;
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    int splits = 1, kchunk = K;
    if (tiles < 152 && K > 256) {
        long long want = std::min<long long>(std::max<long long>(304 / tiles, 1), (K + 127) / 128);
        want = std::min<long long>(want, 128);
        want = std::min<long long>(want, kScratchDoubles / MN);  // partials must fit the array
        if (want > 1) {
            kchunk = (int)((K + want - 1) / want);
            kchunk = ((kchunk + BK - 1) / BK) * BK;
            splits = (K + kchunk - 1) / kchunk;
        }
        if (splits <= 1) {
            splits = 1;
            kchunk = K;
        }
    }
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, splits);
    gemm_rowmajor_kernel<<<grid, NT, 0, s>>>(X, Y, O, M, N, K, splits, kchunk, scratch);
    if (splits > 1) {
        const int blocks = (int)std::min<long long>((MN + 255) / 256, 4096);
        splitk_sum_kernel<<<blocks, 256, 0, s>>>(scratch, O, MN, splits);
    }
    // no error was pending before the launches, so any error now is theirs
    return cudaGetLastError() == cudaSuccess ? SCTM_OK : SCTM_ECUDA;
}
