// Throughput of the packed-integer operations an inter-task cell update can be built from on
// sm_103a: the int16x2 DPX max-plus form used by the kernels, and the 4 x 8-bit SIMD forms an
// int8 first tier would need (Section 4.2: 8-bit lanes first, recompute wider on overflow).
// Every thread runs 8 independent chains of one operation; the rate is operations (calls) per
// second over the whole GPU.  Prints one JSON object.  Used by `bench.py --workload simd_rates`.
#include <cstdio>

#include <cuda_runtime.h>

namespace {

constexpr int kChains = 8;

template <int kOp>
__device__ __forceinline__ unsigned apply(unsigned a, unsigned b, unsigned c) {
    if constexpr (kOp == 0) return __viaddmax_s16x2(a, b, c);   // max(a + b, c), 2 x int16
    if constexpr (kOp == 1) return __vmaxs4(a, c);              // max, 4 x int8
    if constexpr (kOp == 2) return __vaddss4(a, b);             // saturating add, 4 x int8
    if constexpr (kOp == 3) return __vsubss4(a, b);             // saturating subtract, 4 x int8
    return __viaddmax_s32(a, b, c);                             // max(a + b, c), int32
}

template <int kOp>
__global__ void k_rate(unsigned* out, unsigned seed, unsigned b, int iters) {
    unsigned acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = seed * (threadIdx.x + 1) + 977u * i;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = apply<kOp>(acc[i], b, acc[(i + 3) % kChains]);
    }
    unsigned r = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) r ^= acc[i];
    out[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = r;
}

template <int kOp>
float time_op(unsigned* d, int blocks, int threads, int iters) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_rate<kOp><<<blocks, threads>>>(d, 3u, 0x01020304u, iters);   // warm-up
    cudaEventRecord(e0);
    k_rate<kOp><<<blocks, threads>>>(d, 7u, 0x01020304u, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms;
}

}  // namespace

int main() {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, 0) != cudaSuccess) {
        std::printf("{\"error\": \"no CUDA device\"}\n");
        return 1;
    }
    const int sms = pr.multiProcessorCount, threads = 256, blocks = sms * 4, iters = 1 << 14;
    unsigned* d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned) * blocks * threads) != cudaSuccess) {
        std::printf("{\"error\": \"cudaMalloc failed\"}\n");
        return 1;
    }
    const double calls = static_cast<double>(blocks) * threads * iters * kChains;
    const float ms[5] = {time_op<0>(d, blocks, threads, iters), time_op<1>(d, blocks, threads, iters),
                         time_op<2>(d, blocks, threads, iters), time_op<3>(d, blocks, threads, iters),
                         time_op<4>(d, blocks, threads, iters)};
    const char* names[5] = {"viaddmax_s16x2", "vmaxs4", "vaddss4", "vsubss4", "viaddmax_s32"};
    const cudaError_t e = cudaGetLastError();
    cudaFree(d);
    if (e != cudaSuccess) {
        std::printf("{\"error\": \"%s\"}\n", cudaGetErrorString(e));
        return 1;
    }
    double rate[5];
    for (int i = 0; i < 5; ++i) rate[i] = calls / (ms[i] * 1e-3);
    // Cell-update cost: int16x2 DPX = 5.5 operations per 2 cells; an int8x4 saturating update =
    // 5 saturating adds/subtracts + 6 maxima per 4 cells (x, X - Goe, H - Goe, E, F, best).
    const double cells_i16 = 2.0 * rate[0] / 5.5;
    const double cells_i8 = 4.0 / (5.0 / rate[2] + 6.0 / rate[1]);
    std::printf("{\"sms\": %d, \"calls_per_launch\": %.0f, \"rates_per_s\": {", sms, calls);
    for (int i = 0; i < 5; ++i) std::printf("%s\"%s\": %.4e", i ? ", " : "", names[i], rate[i]);
    std::printf("}, \"cell_updates_per_s\": {\"int16x2_dpx\": %.4e, \"int8x4_simd\": %.4e}}\n",
                cells_i16, cells_i8);
    return 0;
}
