// frank_trio_instance.cu -- one instantiation of the three-warp bit-sliced kernel,
// compiled once per K with -DBITSSA_K=<K> like frank_instance.cu.
#include <cuda_runtime.h>

#include "frank_trio.cuh"

#ifndef BITSSA_K
#error "compile with -DBITSSA_K=<planes>"
#endif

#define BITSSA_CAT2(a, b) a##b
#define BITSSA_CAT(a, b) BITSSA_CAT2(a, b)

namespace bitssa {

namespace {
// variant: bit 0 = batch (ensemble table), bit 1 = product clock (SSA_P64)
template <typename F>
int with_trio_kernel(int variant, F f) {
  switch (variant & 3) {
    case 0: return f(frank_trio_kernel<BITSSA_K, false, false>);
    case 1: return f(frank_trio_kernel<BITSSA_K, true, false>);
    case 2: return f(frank_trio_kernel<BITSSA_K, false, true>);
    default: return f(frank_trio_kernel<BITSSA_K, true, true>);
  }
}
}  // namespace

int BITSSA_CAT(frank_trio_launch_k, BITSSA_K)(const FrankLaunch& p, int grid, int smem, void* stream) {
  const int variant = (p.ens_table ? 1 : 0) | (p.precision == kP64 ? 2 : 0);
  return with_trio_kernel(variant, [&](auto kern) {
    kern<<<grid, kTrioBlock, smem, (cudaStream_t)stream>>>(p);
    return (int)cudaGetLastError();
  });
}

int BITSSA_CAT(frank_trio_occupancy_k, BITSSA_K)(int variant, int smem, int* blocks) {
  return with_trio_kernel(variant, [&](auto kern) {
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, kTrioBlock, (size_t)smem);
  });
}

int BITSSA_CAT(frank_trio_regs_k, BITSSA_K)(int variant) {
  return with_trio_kernel(variant, [&](auto kern) {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, kern) == cudaSuccess ? a.numRegs : -1;
  });
}

}  // namespace bitssa
