// Self-test of the bounded device waits (failure detection, no counterpart in the paper).
//
// The library's kernels never spin without a limit: every wait on an mbarrier phase, on a
// shared-memory counter or on a message from the partner CTA of a cluster gives up after the
// handle's limit (oras_options.wait_ms), records DEV_TIMEOUT in the handle's device status
// flags and lets the kernel return, so the context stays usable and the host call reports
// ORAS_ERR_DEVICE_TIMEOUT.  This kernel runs each of those wait primitives on a condition that
// nothing will ever satisfy (a barrier nobody arrives on, a counter nobody increments), so the
// whole path -- the wait giving up, the flag, the host reading it -- is exercised without
// breaking any real kernel and without faulting the GPU.
#include "dev.cuh"

namespace oras {

// One warp; lane 0 waits.  status[ST_DETAIL] gets one bit per primitive that gave up:
// 1 = CTA-scope mbarrier phase, 2 = cluster-scope acquire on an mbarrier, 4 = counter.
__global__ void k_wait_selftest(int32_t* status, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int counter;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);  // expects one arrival, which never comes
    counter = 0;         // never incremented
    fence_mbar_init();
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  int gave_up = 0;
  if (!mbar_wait(&bar, 0, false, limit_ns)) gave_up |= 1;
  if (!mbar_wait(&bar, 0, true, limit_ns)) gave_up |= 2;
  if (!wait_counter(&counter, 1, limit_ns)) gave_up |= 4;
  if (gave_up) {
    atomicExch(&status[ST_ERR], DEV_TIMEOUT);
    atomicOr(&status[ST_DETAIL], gave_up);
  }
}

int launch_wait_selftest(const oras_handle* h) {
  k_wait_selftest<<<1, 32, 0, h->dev.stream>>>(h->dev.status, wait_limit_ns(h));
  count_launches(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace oras
