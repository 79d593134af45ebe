// frank_instance.cu -- one instantiation of the bit-sliced kernel; compiled once
// per K (number of propensity planes) with -DBITSSA_K=<K> so that the
// instantiations build in parallel.
#include <cuda_runtime.h>

#include "frank_kernel.cuh"
#include "frank_tail.cuh"

#ifndef BITSSA_K
#error "compile with -DBITSSA_K=<planes>"
#endif

#define BITSSA_CAT2(a, b) a##b
#define BITSSA_CAT(a, b) BITSSA_CAT2(a, b)

namespace bitssa {

// variant: bit 0 = batch (ensemble table), bit 1 = product clock (SSA_P64), bit 2 = the
// state-following bound (FrankLaunch::adapt)
namespace {
template <typename F>
int with_kernel(int variant, F f) {
  switch (variant & 7) {
    case 0: return f(frank_kernel<BITSSA_K, false, false, false>);
    case 1: return f(frank_kernel<BITSSA_K, true, false, false>);
    case 2: return f(frank_kernel<BITSSA_K, false, true, false>);
    case 3: return f(frank_kernel<BITSSA_K, true, true, false>);
    case 4: return f(frank_kernel<BITSSA_K, false, false, true>);
    case 5: return f(frank_kernel<BITSSA_K, true, false, true>);
    case 6: return f(frank_kernel<BITSSA_K, false, true, true>);
    default: return f(frank_kernel<BITSSA_K, true, true, true>);
  }
}
}  // namespace

int BITSSA_CAT(frank_launch_k, BITSSA_K)(const FrankLaunch& p, int grid, int block, int smem,
                                          void* stream) {
  const cudaStream_t st = (cudaStream_t)stream;
  const int variant = (p.ens_table ? 1 : 0) | (p.precision == kP64 ? 2 : 0) | (p.adapt ? 4 : 0);
  return with_kernel(variant, [&](auto kern) {
    kern<<<grid, block, smem, st>>>(p);
    return (int)cudaGetLastError();
  });
}

// Occupancy at `smem` bytes of dynamic shared memory; lifts the kernel's dynamic shared-memory
// limit first when the request exceeds the default 48 KB (the staging rows of a snapshot dump).
int BITSSA_CAT(frank_occupancy_k, BITSSA_K)(int variant, int block, int smem, int* blocks) {
  return with_kernel(variant, [&](auto kern) {
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return (int)e;
    }
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, block, (size_t)smem);
  });
}

int BITSSA_CAT(frank_regs_k, BITSSA_K)(int variant) {
  return with_kernel(variant, [&](auto kern) {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, kern) == cudaSuccess ? a.numRegs : -1;
  });
}

}  // namespace bitssa
