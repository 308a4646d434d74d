// Failure-detection self-test of the bounded device waits.
//
// The library's device waits (the cooperative PCG's grid barrier polling a generation word, the
// staged dense kernel waiting on an mbarrier for its bulk copies, the persistent batched solve
// waiting for a work-queue slot to be published) give up after a bounded number of polls and
// report an error the host turns into BF_ERR_TIMEOUT, so a lost participant cannot hang the GPU.
// These kernels make each kind of wait run out on purpose, with the same helpers and a short
// limit: a generation word that nothing advances, an mbarrier that nothing arrives on, a slot
// flag that nothing sets.  Nothing faults and nothing is left in flight: no copy was issued, the
// wait just ends.
#include "bf_internal.cuh"

namespace bf {

// One thread polls a word nothing changes; err = 1 when the wait gave up.
__global__ void k_selftest_word(const unsigned *word, int *err, long long limit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  __shared__ int abort_flag;
  abort_flag = 0;
  const bool changed = wait_change((const volatile unsigned *)word, 0u, (const volatile int *)&abort_flag, limit, 64);
  *err = changed ? 0 : 1;
}

// An mbarrier expecting one arrival that never comes; every thread waits (bounded); err = 1 when
// the wait gave up.
__global__ void k_selftest_mbarrier(int *err, long long limit) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned barp = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barp) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool done = mbar_wait(barp, 0, limit);
  __syncthreads();
  if (threadIdx.x == 0) *err = done ? 0 : 1;
}

// One thread waits for a work-queue slot flag (the word) nothing publishes; err = 1 when the wait
// gave up.
__global__ void k_selftest_slot(const unsigned *word, int *err, long long limit) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  __shared__ int abort_flag;
  abort_flag = 0;
  const bool published = wait_published((const int *)word, (const volatile int *)&abort_flag, limit);
  *err = published ? 0 : 1;
}

int launch_selftest_wait(int which, const unsigned *word, int *err, long long limit, cudaStream_t st) {
  if (which == 0)
    k_selftest_word<<<1, 32, 0, st>>>(word, err, limit);
  else if (which == 1)
    k_selftest_mbarrier<<<1, 128, 0, st>>>(err, limit);
  else
    k_selftest_slot<<<1, 32, 0, st>>>(word, err, limit);
  return 1;
}

}  // namespace bf
