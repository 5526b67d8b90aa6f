// alu_rate.cu -- measured throughput of the 32-bit Shoup modular multiply
// (a w mod b in [0, 2b), three 32-bit multiplies), the operation the inverse
// NTTs of the tensor stage are made of: a reference rate for the integer
// roofline beside the one derived from unit counts and clocks.
#include "device_math.cuh"
#include "launch.h"

namespace sfhe {

namespace {
constexpr int RATE_CHAINS = 8;     // independent multiply chains per thread
constexpr int RATE_ITERS = 4096;   // multiplies per chain
constexpr int RATE_THREADS = 256;

__global__ void __launch_bounds__(RATE_THREADS) k_mulmod32_rate(u32* out, u32 b, u32 w, u32 ws)
{
    u32 x[RATE_CHAINS];
#pragma unroll
    for (int c = 0; c < RATE_CHAINS; c++) x[c] = (threadIdx.x * 7919u + c * 104729u + blockIdx.x) % b;
    for (int i = 0; i < RATE_ITERS; i++) {
#pragma unroll
        for (int c = 0; c < RATE_CHAINS; c++) x[c] = shoup32_lazy(x[c], w, ws, b);
    }
    u32 acc = 0;
#pragma unroll
    for (int c = 0; c < RATE_CHAINS; c++) acc ^= x[c];
    out[(size_t)blockIdx.x * RATE_THREADS + threadIdx.x] = acc;
}
}  // namespace

cudaError_t measure_mulmod32(u32 b, u32 w, u32 ws, double* per_s, cudaStream_t s)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mulmod32_rate, RATE_THREADS, 0);
    if (e != cudaSuccess) return e;
    const int grid = sms * per_sm;
    u32* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaMallocAsync((void**)&out, (size_t)grid * RATE_THREADS * 4, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    if (e == cudaSuccess) {
        k_mulmod32_rate<<<grid, RATE_THREADS, 0, s>>>(out, b, w, ws);  // warm-up
        cudaEventRecord(e0, s);
        k_mulmod32_rate<<<grid, RATE_THREADS, 0, s>>>(out, b, w, ws);
        cudaEventRecord(e1, s);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (out) cudaFreeAsync(out, s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    *per_s = ms > 0.f ? (double)grid * RATE_THREADS * RATE_CHAINS * RATE_ITERS / (ms * 1e-3) : 0.0;
    return cudaSuccess;
}

}  // namespace sfhe
