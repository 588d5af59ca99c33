// Self-test of the bounded device-side wait that every pipelined kernel of this
// library uses (tc::mbar_wait): one thread waits on an mbarrier that nothing
// completes. The wait must give up once its time limit has passed, record
// CORR_ETIMEOUT in the status word and return, so that a lost arrival ends a kernel
// with an error code instead of a hang; afterwards one arrival must still complete
// the barrier's phase. Nothing here faults or traps.
#include "internal.h"
#include "tc_ptx.cuh"

namespace corr {
namespace {

// status[0]: the word the wait records its time-out in (CORR_ETIMEOUT expected);
// status[1]: 1 if the first wait returned true (it cannot complete), 2 if the
// barrier did not complete after the arrival, 0 otherwise;
// status[2..3]: elapsed nanoseconds of the first wait (low, high words).
__global__ void k_wait_selftest(int *status, unsigned long long limit_ns) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    const uint32_t b = tc::smem_u32(&bar);
    tc::mbar_init(b, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint64_t t0 = tc::global_ns();
    // phase 0 needs one arrival and gets none
    const bool done = tc::mbar_wait(b, 0u, &abort_flag, status, limit_ns);
    const uint64_t dt = tc::global_ns() - t0;
    int bad = done ? 1 : 0;
    // one arrival completes phase 0: the wait (abort flag ignored) returns at once
    tc::mbar_arrive(b);
    if (!tc::mbar_wait(b, 0u, &abort_flag, status + 1, limit_ns, false)) bad = 2;
    status[1] = bad;
    status[2] = (int)(uint32_t)dt;
    status[3] = (int)(uint32_t)(dt >> 32);
}

}  // namespace

corr_status selftest_bounded_wait(uint64_t limit_ns) {
    int *d = nullptr;
    if (cudaMalloc(&d, 4 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return CORR_ENOMEM;
    }
    int h[4] = {0, 0, 0, 0};
    corr_status r = CORR_OK;
    if (cudaMemset(d, 0, 4 * sizeof(int)) != cudaSuccess) r = CORR_ECUDA;
    if (r == CORR_OK) {
        k_wait_selftest<<<1, 32>>>(d, (unsigned long long)limit_ns);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess)
            r = CORR_ECUDA;
    }
    cudaFree(d);
    if (r != CORR_OK) return r;
    const uint64_t dt = (uint64_t)(uint32_t)h[2] | ((uint64_t)(uint32_t)h[3] << 32);
    // the wait gave up (not earlier than its limit), recorded the time-out, and the
    // barrier completed afterwards
    if (h[0] != CORR_ETIMEOUT || h[1] != 0 || dt < limit_ns) return CORR_ESTATE;
    return CORR_OK;
}

}  // namespace corr
