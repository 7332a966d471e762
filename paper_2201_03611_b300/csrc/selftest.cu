// Exercise of the bounded-wait path on the GPU without any fault: one warp waits on a
// shared-memory mbarrier whose phase nothing completes. The wait is the kernels' own bounded
// poll loop (mbar_wait), so it gives up after max_spins polls, the warp records that it gave up
// and returns, and the context stays usable.
#include <cuda_runtime.h>

#include "harris_common.cuh"
#include "shine.h"
#include "shine_host.h"

namespace shine {
namespace {

__global__ void bounded_wait_probe(int max_spins, int* result) {
    __shared__ __align__(8) uint64_t bar;
    const int lane = threadIdx.x & 31;
    const uint32_t b = smem_u32(&bar);
    if (lane == 0) mbar_init(b, 1);  // one arrival expected; none ever comes
    mbar_init_fence();
    __syncwarp();
    const bool ok = __all_sync(kFull, mbar_wait(b, 0u, max_spins));
    if (lane == 0) *result = ok ? 0 : 1;
}

}  // namespace
}  // namespace shine

using namespace shine;

extern "C" shine_status shine_selftest_bounded_wait(int32_t max_spins, int* result, void* stream) {
    if (!result || max_spins < 1 || max_spins > (1 << 22)) return SHINE_ERR_INVALID_ARG;
    if (!aligned_to(result, 4)) return SHINE_ERR_ALIGNMENT;
    bounded_wait_probe<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(max_spins, result);
    return cuda_status(cudaPeekAtLastError());
}
