// lattice_instance.cu -- one instantiation of the lattice kernel; compiled once per plane count
// with -DBITSSA_LAT_P=<P> (4, 8, 12, 16) so that the instantiations build in parallel.
#include <cuda_runtime.h>

#include "lattice_kernel.cuh"

#ifndef BITSSA_LAT_P
#error "compile with -DBITSSA_LAT_P=<planes>"
#endif

#define BITSSA_CAT2(a, b) a##b
#define BITSSA_CAT(a, b) BITSSA_CAT2(a, b)

namespace bitssa {

// Draw planes of the instantiation: 2 P + 8, at most the stream's 32.  The host takes a wider
// instantiation when some cap the run may reach needs more.
constexpr int kLatKW = 2 * BITSSA_LAT_P + 8 > 32 ? 32 : 2 * BITSSA_LAT_P + 8;

int BITSSA_CAT(lattice_launch_p, BITSSA_LAT_P)(const LatticeLaunch& p, int grid, int block, int smem, void* stream) {
  auto kern = lattice_kernel<BITSSA_LAT_P, kLatKW>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return (int)e;
    }
  }
  kern<<<grid, block, smem, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

int BITSSA_CAT(lattice_kw_p, BITSSA_LAT_P)() { return kLatKW; }

int BITSSA_CAT(lattice_occupancy_p, BITSSA_LAT_P)(int block, int smem, int* blocks) {
  auto kern = lattice_kernel<BITSSA_LAT_P, kLatKW>;
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return (int)e;
    }
  }
  const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, block, (size_t)smem);
  if (e != cudaSuccess) cudaGetLastError();
  return (int)e;
}

}  // namespace bitssa
