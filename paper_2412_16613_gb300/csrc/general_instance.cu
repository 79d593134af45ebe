// general_instance.cu -- one instantiation of the general-network bit-sliced kernels (planes in
// shared memory; planes in registers up to kRegMaxK); compiled once per K (number of propensity
// planes) with -DBITSSA_K=<K>.
#include <cuda_runtime.h>

#include "general_reg.cuh"

#ifndef BITSSA_K
#error "compile with -DBITSSA_K=<planes>"
#endif

#define BITSSA_CAT2(a, b) a##b
#define BITSSA_CAT(a, b) BITSSA_CAT2(a, b)

namespace bitssa {

// variant: bit 0 = batch (ensemble table), bit 1 = product clock (SSA_P64), bit 2 = planes in
// registers (p.net.regs at launch)
namespace {
template <bool REG, bool BATCH, bool PROD>
constexpr auto general_entry() {
  if constexpr (REG && BITSSA_K <= kRegMaxK) return general_reg_kernel<BITSSA_K, BATCH, PROD>;
  else return general_kernel<BITSSA_K, BATCH, PROD>;
}
}  // namespace

int BITSSA_CAT(general_launch_k, BITSSA_K)(const FrankLaunch& p, int grid, int block, int smem,
                                            void* stream) {
  const cudaStream_t st = (cudaStream_t)stream;
  const bool prod = p.precision == kP64;
  if (p.net.regs && BITSSA_K > kRegMaxK) return (int)cudaErrorInvalidValue;
  if (p.net.regs) {
    if (p.ens_table) {
      if (prod) general_entry<true, true, true>()<<<grid, block, smem, st>>>(p);
      else general_entry<true, true, false>()<<<grid, block, smem, st>>>(p);
    } else {
      if (prod) general_entry<true, false, true>()<<<grid, block, smem, st>>>(p);
      else general_entry<true, false, false>()<<<grid, block, smem, st>>>(p);
    }
  } else if (p.ens_table) {
    if (prod) general_kernel<BITSSA_K, true, true><<<grid, block, smem, st>>>(p);
    else general_kernel<BITSSA_K, true, false><<<grid, block, smem, st>>>(p);
  } else {
    if (prod) general_kernel<BITSSA_K, false, true><<<grid, block, smem, st>>>(p);
    else general_kernel<BITSSA_K, false, false><<<grid, block, smem, st>>>(p);
  }
  return (int)cudaGetLastError();
}

namespace {
template <typename F>
int with_kernel(int variant, F f) {
  switch (variant & 7) {
    case 0: return f(general_kernel<BITSSA_K, false, false>);
    case 1: return f(general_kernel<BITSSA_K, true, false>);
    case 2: return f(general_kernel<BITSSA_K, false, true>);
    case 3: return f(general_kernel<BITSSA_K, true, true>);
    case 4: return f(general_entry<true, false, false>());
    case 5: return f(general_entry<true, true, false>());
    case 6: return f(general_entry<true, false, true>());
    default: return f(general_entry<true, true, true>());
  }
}
}  // namespace

// Occupancy at `smem` bytes of dynamic shared memory; lifts the kernel's dynamic shared-memory
// limit first when the request exceeds the default 48 KB.
int BITSSA_CAT(general_occupancy_k, BITSSA_K)(int variant, int block, int smem, int* blocks) {
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

int BITSSA_CAT(general_regs_k, BITSSA_K)(int variant) {
  return with_kernel(variant, [&](auto kern) {
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, kern) == cudaSuccess ? a.numRegs : -1;
  });
}

}  // namespace bitssa
