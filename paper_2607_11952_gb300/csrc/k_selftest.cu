// Failure-detection self-test: the sweep's bounded mbarrier wait, run on a
// phase that nothing completes, so that the timeout path (status bit, normal
// return, FA_ERR_TIMEOUT on the host) can be exercised without a fault.
#include "fa_internal.cuh"
#include "sweep_dev.cuh"

namespace fa {

// One thread waits, through the same bounded wait the sweep uses, on an
// mbarrier phase that nothing completes (expected arrival count 1, no
// arrival): the wait gives up after its time limit and the kernel records
// ST_TIMEOUT, as it would for a TMA stage or a peer's exchange that never
// lands.  Nothing is faulted; the kernel returns normally.
__global__ void k_wait_selftest(int* status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t a = smem_u32(&bar);
  mbar_init(a, 1u);
  fence_mbar_init();
  if (!mbar_wait_bounded(a, 0u)) atomicOr(status, ST_TIMEOUT);
}

fa_status launch_wait_selftest(int* status, cudaStream_t s) {
  k_wait_selftest<<<1, 1, 0, s>>>(status);
  FA_LAUNCHED("k_wait_selftest");
  return FA_OK;
}

}  // namespace fa
