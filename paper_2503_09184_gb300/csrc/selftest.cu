// selftest.cu -- exercises the bounded device wait and its status word
// without any fault: one thread waits on an mbarrier that nothing arrives
// at, gives up after `tries` attempts or `limit_ns` nanoseconds and flags the
// workspace's status word exactly as the persistent kernel does when a bulk
// copy does not complete.
#include "device_math.cuh"
#include "launch.h"

namespace sfhe {

namespace {
__global__ void k_wait_selftest(unsigned* queue, u32 tries, u64 limit_ns)
{
    __shared__ __align__(8) u64 bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    fence_mbar_init();
    if (!mbar_wait(&bar, 0, tries, limit_ns)) atomicExch(queue + 1, 1u);
}
}  // namespace

cudaError_t launch_wait_selftest(unsigned* queue, u32 tries, u64 limit_ns, cudaStream_t s)
{
    k_wait_selftest<<<1, 32, 0, s>>>(queue, tries, limit_ns);
    return cudaGetLastError();
}

}  // namespace sfhe
