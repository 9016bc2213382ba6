// Grid-wide barrier for kernels launched cooperatively (every block
// resident), with a bounded wait: shared by the persistent CG and the fused
// set-up kernel.
#pragma once

#include <cuda_runtime.h>

#include "kernels.h"

namespace efgp {

namespace gsync {

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int arrive_acq_rel(unsigned int* p) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

}  // namespace gsync

// Grid barrier on a generation counter.  Thread 0 of every block arrives
// (release of everything the block wrote, ordered before it by the block
// barrier); the last arrival resets the count and publishes the next
// generation (release), the others poll the generation (acquire), bounded.
// Returns false if this block gave up or another block reported an error.
__device__ __forceinline__ bool grid_barrier(GridBarrier* gb, unsigned int nblocks, unsigned int& gen, long long limit) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int arrived = gsync::arrive_acq_rel(&gb->count);
    if (arrived == nblocks - 1) {
      gb->count = 0u;
      gsync::st_release(&gb->gen, gen + 1u);
    } else {
      long long i = 0;
      for (; i < limit; ++i) {
        if (gsync::ld_acquire(&gb->gen) != gen) break;
        if (gsync::ld_relaxed_i(&gb->err)) { ok = 0; break; }
      }
      if (i == limit) {
        atomicOr(&gb->err, 1);
        ok = 0;
      }
    }
    if (ok && gsync::ld_relaxed_i(&gb->err)) ok = 0;
    gen += 1u;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace efgp
