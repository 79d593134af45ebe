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
// state-following bound (FrankLaunch::adapt), bit 3 = per-run clocks (FrankLaunch::lane_clock,
// single ensembles only: variants 8 and 10)
namespace {
template <typename F>
int with_kernel(int variant, F f) {
  switch (variant & 15) {
    case 0: return f(frank_kernel<BITSSA_K, false, false, false>);
    case 1: return f(frank_kernel<BITSSA_K, true, false, false>);
    case 2: return f(frank_kernel<BITSSA_K, false, true, false>);
    case 3: return f(frank_kernel<BITSSA_K, true, true, false>);
    case 4: return f(frank_kernel<BITSSA_K, false, false, true>);
    case 5: return f(frank_kernel<BITSSA_K, true, false, true>);
    case 6: return f(frank_kernel<BITSSA_K, false, true, true>);
    case 7: return f(frank_kernel<BITSSA_K, true, true, true>);
    case 8: return f(frank_kernel<BITSSA_K, false, false, false, true>);
    default: return f(frank_kernel<BITSSA_K, false, true, false, true>);
  }
}
}  // namespace

int BITSSA_CAT(frank_launch_k, BITSSA_K)(const FrankLaunch& p, int grid, int block, int smem,
                                          void* stream) {
  const cudaStream_t st = (cudaStream_t)stream;
  const int variant = (p.ens_table ? 1 : 0) | (p.precision == kP64 ? 2 : 0) | (p.adapt ? 4 : 0) |
                      (p.lane_clock ? 8 : 0);
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
      if (e != cudaSuccess) {
        cudaGetLastError();  // the caller reports it; leave no error pending for later calls
        return (int)e;
      }
    }
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, block, (size_t)smem);
    if (e != cudaSuccess) cudaGetLastError();
    return (int)e;
  });
}

int BITSSA_CAT(frank_regs_k, BITSSA_K)(int variant) {
  return with_kernel(variant, [&](auto kern) {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, kern) == cudaSuccess ? a.numRegs : -1;
  });
}

}  // namespace bitssa
