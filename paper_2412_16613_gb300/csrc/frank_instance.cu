// frank_instance.cu -- one instantiation of the bit-sliced kernel; compiled once
// per K (number of propensity planes) with -DBITSSA_K=<K> so that the
// instantiations build in parallel.
#include <cuda_runtime.h>

#include "frank_kernel.cuh"

#ifndef BITSSA_K
#error "compile with -DBITSSA_K=<planes>"
#endif

#define BITSSA_CAT2(a, b) a##b
#define BITSSA_CAT(a, b) BITSSA_CAT2(a, b)

namespace bitssa {

int BITSSA_CAT(frank_launch_k, BITSSA_K)(const FrankLaunch& p, int grid, int block, int smem,
                                          void* stream) {
  if (p.ens_table) frank_kernel<BITSSA_K, true><<<grid, block, smem, (cudaStream_t)stream>>>(p);
  else frank_kernel<BITSSA_K, false><<<grid, block, smem, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

int BITSSA_CAT(frank_occupancy_k, BITSSA_K)(int batch, int block, int smem, int* blocks) {
  if (batch)
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, frank_kernel<BITSSA_K, true>,
                                                              block, (size_t)smem);
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, frank_kernel<BITSSA_K, false>,
                                                            block, (size_t)smem);
}

int BITSSA_CAT(frank_regs_k, BITSSA_K)(int batch) {
  cudaFuncAttributes a;
  const cudaError_t err = batch ? cudaFuncGetAttributes(&a, frank_kernel<BITSSA_K, true>)
                                : cudaFuncGetAttributes(&a, frank_kernel<BITSSA_K, false>);
  return err == cudaSuccess ? a.numRegs : -1;
}

}  // namespace bitssa
