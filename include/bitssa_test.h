/*
 * bitssa_test.h -- test and measurement entry points of libbitssa.
 *
 * These expose single pieces of the hot path so that they can be checked on
 * their own; the simulation itself is reached only through bitssa.h.  All
 * arrays are HOST memory; each call copies its inputs to the current device,
 * runs one kernel, copies the result back and synchronises.  Return value: 0 on
 * success, SSA_EINVAL (-1) for bad arguments, SSA_ECUDA (-4) for CUDA errors.
 */
#ifndef BITSSA_TEST_H
#define BITSSA_TEST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Philox4x32-10 block function (Salmon et al., SC'11, the generator of every
 * random bit of the method's steps 1 and a) evaluated on the device for n
 * (counter, key) pairs.  ctr: uint32[n][4], key: uint32[n][2], out: uint32[n][4].
 * which = 0: libbitssa's own device function; 1: curand_Philox4x32_10 from the
 * CUDA toolkit (a reference implementation, for comparison only).
 */
int bitssa_test_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, int32_t which);

/*
 * Bit-sliced integer primitives of Sec. 4.1 run on 8-bit operands.  x, y:
 * int64[n] per-lane operands in [0, 255] (n a multiple of 32); lane j of the
 * device words holds x[j], y[j].  out: int64[n].
 *   op 0: x + y (ripple-carry add, 9-bit result)
 *   op 1: x - y (two's complement on 9 planes, read back as a signed value)
 *   op 2: [x < y] (borrow chain)
 *   op 3: x * y (schoolbook product, 16 planes)
 *   op 4: x + c with c = +3 where y % 4 == 1, -2 where y % 4 == 2, +5 where y % 4 == 3,
 *         else 0
 *         (the masked constant update of Eq. equation-v, on 10 signed planes)
 */
int bitssa_test_bitslice(int32_t op, const int64_t* x, const int64_t* y, int64_t* out, int64_t n);

/*
 * Integer-ALU issue microbenchmark: a grid that fills every SM runs
 * independent chains of 3-input logic operations (LOP3) for `iters` rounds.
 * Writes the 32-bit logic operations per second executed by all threads and the
 * kernel time.  device = -1: current device.
 */
int bitssa_bench_alu(int32_t device, int32_t iters, double* ops_per_s, double* ms);

#ifdef __cplusplus
}
#endif
#endif
