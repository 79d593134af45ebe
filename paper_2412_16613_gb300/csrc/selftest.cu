// selftest.cu -- the test and measurement entry points of include/bitssa_test.h.
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>
#include <vector>

#include "../../include/bitssa_test.h"
#include "bitslice.cuh"
#include "philox.cuh"

using namespace bitssa;

namespace {

__global__ void philox_kernel(const uint4* ctr, const uint2* key, uint4* out, long long n, int which) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (which == 0) out[i] = philox4x32_10(ctr[i], PhiloxKey{key[i].x, key[i].y});
  else out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

// One thread per group of 32 lanes: transpose the operands into planes, apply
// the primitive, transpose the result back.
__global__ void bitslice_kernel(int op, const long long* x, const long long* y, long long* out, long long n) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 32 >= n) return;
  uint32_t X[8], Y[8];
  bs::broadcast(X, 0);
  bs::broadcast(Y, 0);
  for (int l = 0; l < 32; ++l) {
    bs::set_lane(X, l, x[g * 32 + l]);
    bs::set_lane(Y, l, y[g * 32 + l]);
  }
  if (op == 0 || op == 1) {
    uint32_t R[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) R[i] = bs::plane<false>(X, i);
    if (op == 0) {
      uint32_t T[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) T[i] = bs::plane<false>(Y, i);
      bs::add_signed(R, T, 0u);
    } else {
      uint32_t T[9];  // -y = ~y + 1
#pragma unroll
      for (int i = 0; i < 9; ++i) T[i] = ~bs::plane<false>(Y, i);
      bs::add_signed(R, T, 0xFFFFFFFFu);
    }
    for (int l = 0; l < 32; ++l) out[g * 32 + l] = op == 0 ? bs::lane_value<false>(R, l) : bs::lane_value<true>(R, l);
  } else if (op == 2) {
    const uint32_t lt = bs::less_than(X, Y);
    for (int l = 0; l < 32; ++l) out[g * 32 + l] = (lt >> l) & 1u;
  } else if (op == 3) {
    uint32_t R[16];
    bs::multiply(R, X, Y);
    for (int l = 0; l < 32; ++l) out[g * 32 + l] = bs::lane_value<false>(R, l);
  } else {
    uint32_t R[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) R[i] = bs::plane<false>(X, i);
    const uint32_t m1 = Y[0] & ~Y[1], m2 = ~Y[0] & Y[1], m3 = Y[0] & Y[1];
    bs::add_select3<3, -2, 5>(R, m1, m2, m3);
    for (int l = 0; l < 32; ++l) out[g * 32 + l] = bs::lane_value<true>(R, l);
  }
}

__global__ void alu_kernel(uint32_t seed, int iters, uint32_t* sink) {
  // 8 chains per thread; each step is a majority of the chain, its neighbour's previous value
  // and a constant, so no step can be folded into another and a round holds 8 independent
  // 3-input logic operations (one LOP3 each)
  uint32_t a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = threadIdx.x * (j + 1) + seed * 0x9E3779B9u + blockIdx.x;
  const uint32_t k0 = seed ^ 0x85EBCA6Bu, k1 = seed * 0xC2B2AE35u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      uint32_t b[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        // one LOP3 instruction with the majority truth table (0xE8)
        asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(b[j]) : "r"(a[j]), "r"(a[(j + 1) & 7]),
                     "r"((r & 1) ? k1 : k0));
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = b[j];
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= a[j];
  if (s == 0x12345678u) sink[0] = s;  // keeps the chains alive
}

}  // namespace

extern "C" int bitssa_test_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, int32_t which) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out)) || which < 0 || which > 1) return -1;
  if (n == 0) return 0;
  uint4 *dc = nullptr, *dout = nullptr;
  uint2* dk = nullptr;
  int rc = -4;
  if (cudaMalloc(&dc, sizeof(uint4) * n) == cudaSuccess && cudaMalloc(&dk, sizeof(uint2) * n) == cudaSuccess &&
      cudaMalloc(&dout, sizeof(uint4) * n) == cudaSuccess &&
      cudaMemcpy(dc, ctr, sizeof(uint4) * n, cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(dk, key, sizeof(uint2) * n, cudaMemcpyHostToDevice) == cudaSuccess) {
    philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(dc, dk, dout, n, which);
    if (cudaGetLastError() == cudaSuccess && cudaMemcpy(out, dout, sizeof(uint4) * n, cudaMemcpyDeviceToHost) == cudaSuccess)
      rc = 0;
  }
  cudaGetLastError();
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  return rc;
}

extern "C" int bitssa_test_bitslice(int32_t op, const int64_t* x, const int64_t* y, int64_t* out, int64_t n) {
  if (op < 0 || op > 4 || n < 0 || (n % 32) != 0 || (n > 0 && (!x || !y || !out))) return -1;
  for (int64_t i = 0; i < n; ++i)
    if (x[i] < 0 || x[i] > 255 || y[i] < 0 || y[i] > 255) return -1;
  if (n == 0) return 0;
  long long *dx = nullptr, *dy = nullptr, *dout = nullptr;
  int rc = -4;
  const size_t bytes = sizeof(long long) * (size_t)n;
  if (cudaMalloc(&dx, bytes) == cudaSuccess && cudaMalloc(&dy, bytes) == cudaSuccess &&
      cudaMalloc(&dout, bytes) == cudaSuccess && cudaMemcpy(dx, x, bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
      cudaMemcpy(dy, y, bytes, cudaMemcpyHostToDevice) == cudaSuccess) {
    const long long groups = n / 32;
    bitslice_kernel<<<(unsigned)((groups + 127) / 128), 128>>>(op, dx, dy, dout, n);
    if (cudaGetLastError() == cudaSuccess && cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost) == cudaSuccess) rc = 0;
  }
  cudaGetLastError();
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(dout);
  return rc;
}

extern "C" int bitssa_bench_alu(int32_t device, int32_t iters, double* ops_per_s, double* ms) {
  if (iters < 1 || !ops_per_s || !ms) return -1;
  int prev = -1;
  cudaGetDevice(&prev);
  if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return -4;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int block = 256;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, alu_kernel, block, 0);
  const int grid = sms * (occ > 0 ? occ : 1);
  uint32_t* sink = nullptr;
  cudaEvent_t e0, e1;
  int rc = -4;
  if (cudaMalloc(&sink, 16) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
      cudaEventCreate(&e1) == cudaSuccess) {
    alu_kernel<<<grid, block>>>(1u, iters / 10 + 1, sink);  // warm-up
    cudaEventRecord(e0);
    alu_kernel<<<grid, block>>>(2u, iters, sink);
    cudaEventRecord(e1);
    float t = 0.0f;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) {
      // one LOP3 per (iteration, round, chain, thread)
      const double ops = (double)grid * block * (double)iters * 16.0 * 8.0;
      *ms = t;
      *ops_per_s = ops / (t * 1e-3);
      rc = 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  cudaGetLastError();
  cudaFree(sink);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
