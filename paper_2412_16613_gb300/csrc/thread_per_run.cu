// thread_per_run.cu -- comparison baseline: one GPU thread per run, plain direct
// method (Sec. 3, steps 1-7) for Frank's model without ghost reactions.
//
// Each step: h1 = A L, h2 = A D, h3 = L D (Eq. equation-as); with equal rates
// the reaction index comes from an exact uniform integer in [0, H), H = sum h
// (Lemire's multiply-shift with rejection), otherwise from an fp64 uniform
// scaled by a0 = sum k_r h_r; tau = -log(u) / a0 (Eq. equation-tau with the
// state-dependent total rate).  Each run has its own Philox stream
// (tag 2): counter (run lo, run hi16 | attempt << 16 | 2 << 24, step lo, step hi).
// The clock follows the same precision modes as the bit-sliced kernel.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "philox.cuh"

namespace bitssa {

namespace {

__device__ __forceinline__ int tpr_ee_bin(int l, int d) {
  if (l + d == 0) return 64;
  const int b = (64 * l) / (l + d);
  return b > 63 ? 63 : b;
}

__device__ __forceinline__ uint4 run_counter(long long run, unsigned long long step, uint32_t attempt) {
  return make_uint4((uint32_t)run, ((uint32_t)(run >> 32) & 0xFFFFu) | (attempt << 16) | (2u << 24),
                    (uint32_t)step, (uint32_t)(step >> 32));
}

}  // namespace

// One run per thread at a time; the loop is warp-synchronous (every thread stays in it
// until the warp runs out of runs, and the warp reconverges after each step), so runs
// of different lengths and the rare branches do not leave the warp split.
__global__ void __launch_bounds__(256) thread_per_run_kernel(const __grid_constant__ ThreadLaunch p) {
  extern __shared__ unsigned int s_hist[];
  const int n_snap = p.n_snap;
  for (int i = threadIdx.x; i < n_snap * kHistBins; i += blockDim.x) s_hist[i] = 0u;
  __syncthreads();

  const Ensemble& e = p.ens;
  const PhiloxKey key{(uint32_t)e.seed, (uint32_t)(e.seed >> 32)};
  const double k1 = p.rates[0], k2 = p.rates[1], k3 = p.rates[2];
  const double kunit = k1;  // the common rate when unit_rates
  unsigned long long c_steps = 0, c_abs = 0;
  unsigned int errors = 0u;
  unsigned long long outc[4] = {0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;

  long long run = (long long)blockIdx.x * blockDim.x + threadIdx.x - stride;
  long long row = 0, grun = 0;
  int l = 0, d = 0, a = 0, snap = 0;
  long long h1 = 0, h2 = 0, h3 = 0;
  double t = 0.0, t_abs = 0.0;
  float t_f = 0.0f, c_f = 0.0f;
  unsigned long long step = 0;
  bool active = false, exhausted = false, done = false, absorbed = false;

  auto real_total = [&]() {
    return ((e.active & 1u) ? h1 : 0) + ((e.active & 2u) ? h2 : 0) + ((e.active & 4u) ? h3 : 0);
  };
  auto capture = [&](int s) {
    atomicAdd(&s_hist[s * kHistBins + tpr_ee_bin(l, d)], 1u);
    if (p.snap_counts) {
      int* o = p.snap_counts + ((long long)s * p.n_runs_total + row) * p.n_species;
      o[p.perm[0]] = l;
      o[p.perm[1]] = d;
      o[p.perm[2]] = a;
    }
  };

  for (;;) {
    if (!active && !exhausted) {
      run += stride;
      if (run >= e.n_runs) {
        exhausted = true;
      } else {
        row = e.run_offset + run;
        grun = e.group_base * 32 + run;  // run index inside the ensemble
        if (p.init_counts) {
          l = p.init_counts[row * 3 + 0];
          d = p.init_counts[row * 3 + 1];
          a = p.init_counts[row * 3 + 2];
        } else {
          l = e.init[0];
          d = e.init[1];
          a = e.init[2];
        }
        t = 0.0;
        t_f = c_f = 0.0f;
        snap = 0;
        step = 0;
        t_abs = __longlong_as_double(0x7FF0000000000000ll);
        h1 = (long long)a * l;
        h2 = (long long)a * d;
        h3 = (long long)l * d;
        absorbed = real_total() == 0;
        if (absorbed) t_abs = 0.0;
        done = absorbed;
        active = true;
      }
    }
    if (__all_sync(0xFFFFFFFFu, exhausted && !active)) break;
    if (active && !done) {
      if (p.step_budget > 0 && (long long)step >= p.step_budget) {
        errors |= kErrTimeout;
        done = true;
      } else {
        const uint4 w = philox4x32_10(run_counter(grun, step, 0u), key);
        int r;
        double a0;
        if (p.unit_rates) {
          // exact uniform integer in [0, H) (Lemire's method with rejection)
          const unsigned long long H = (unsigned long long)(h1 + h2 + h3);
          unsigned long long m = (unsigned long long)w.x * H;
          if ((uint32_t)m < (uint32_t)H) {
            const uint32_t thresh = (uint32_t)(0u - (uint32_t)H) % (uint32_t)H;
            uint32_t attempt = 0u;
            while ((uint32_t)m < thresh && attempt < 64u) {
              const uint32_t fresh = attempt == 0u ? w.y : philox4x32_10(run_counter(grun, step, attempt), key).x;
              ++attempt;
              m = (unsigned long long)fresh * H;
            }
            if ((uint32_t)m < thresh) errors |= kErrRedraw;
          }
          const long long n = (long long)(m >> 32);
          r = n < h1 ? 0 : (n < h1 + h2 ? 1 : 2);
          a0 = kunit * (double)H;
        } else {
          const double a1 = k1 * (double)h1, a2 = k2 * (double)h2, a3 = k3 * (double)h3;
          a0 = a1 + a2 + a3;
          const unsigned long long x = ((unsigned long long)w.y << 21) | (w.x >> 11);
          const double v = (double)x * 0x1p-53 * a0;
          r = v < a1 ? 0 : (v < a1 + a2 ? 1 : 2);
          if (r == 2 && a3 == 0.0) r = a2 > 0.0 ? 1 : 0;  // rounding at the top edge
        }
        // clock
        double t_new = t;
        float tf_new = t_f, cf_new = c_f;
        if (p.precision == kP64 || p.precision == kP64LogSum) {
          const unsigned long long x = ((unsigned long long)w.w << 21) | (w.z >> 11);
          const double u = (double)(x + 1ull) * 0x1p-53;
          t_new = t + (-log(u) / a0);
        } else {
          const float u = (float)((w.w >> 8) + 1u) * 0x1p-24f;
          const float tau = -logf(u) / (float)a0;
          if (p.precision == kP32Kahan) {
            const float y = tau - c_f;
            const float s = t_f + y;
            cf_new = (s - t_f) - y;
            tf_new = s;
            t_new = (double)s;
          } else if (p.precision == kP32Plain) {
            tf_new = t_f + tau;
            t_new = (double)tf_new;
          } else {
            t_new = t + (double)tau;
          }
        }
        while (snap < n_snap && (p.precision == kP32Kahan || p.precision == kP32Plain ? tf_new > p.thr[snap].t_f : t_new > p.thr[snap].t)) {
          capture(snap);
          ++snap;
        }
        if (p.precision == kP32Kahan || p.precision == kP32Plain ? tf_new > p.thr[n_snap].t_f : t_new > p.thr[n_snap].t) {
          done = true;
        } else {
          t = t_new;
          t_f = tf_new;
          c_f = cf_new;
          // the reaction (Eq. eq_nu)
          if (r == 0) {
            ++l;
            --a;
          } else if (r == 1) {
            ++d;
            --a;
          } else {
            --l;
            --d;
            a += 2;
          }
          ++step;
          h1 = (long long)a * l;
          h2 = (long long)a * d;
          h3 = (long long)l * d;
          if (real_total() == 0) {
            absorbed = true;
            done = true;
            t_abs = (p.precision == kP32Kahan || p.precision == kP32Plain) ? (double)t_f : t;
          }
        }
      }
    }
    if (active && done) {
      if (absorbed)
        for (; snap < n_snap; ++snap) capture(snap);
      int* o = p.final_counts + row * p.n_species;
      o[p.perm[0]] = l;
      o[p.perm[1]] = d;
      o[p.perm[2]] = a;
      p.t_abs[row] = t_abs;
      signed char oc = -1;
      if (absorbed) {
        const int nz = (l != 0) + (d != 0) + (a != 0);
        oc = nz == 1 ? (signed char)(l ? p.perm[0] : (d ? p.perm[1] : p.perm[2])) : (signed char)-2;
        ++c_abs;
      }
      p.outcome[row] = oc;
      outc[oc >= 0 ? oc : 3] += 1;
      c_steps += step;
      atomicMax(&p.counters[kMaxGroupSteps], step);
      active = false;
    }
    __syncwarp();
  }

  unsigned long long v[4] = {c_steps, c_steps, c_steps, c_abs};
  const int idx[4] = {kLaneSteps, kGroupSteps, kReactions, kAbsorbed};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&p.counters[idx[k]], x);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long x = outc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    if ((threadIdx.x & 31) == 0 && x && p.ens_absorbed) atomicAdd(&p.ens_absorbed[k], x);
  }
  const unsigned int err = __reduce_or_sync(0xFFFFFFFFu, errors);
  if ((threadIdx.x & 31) == 0 && err) atomicOr(p.status, err);
  __syncthreads();
  for (int i = threadIdx.x; i < n_snap * kHistBins; i += blockDim.x)
    if (s_hist[i]) atomicAdd(&p.hist[i], (unsigned long long)s_hist[i]);
}

int thread_per_run_launch(const ThreadLaunch& p, int grid, int block, int smem, void* stream) {
  thread_per_run_kernel<<<grid, block, smem, (cudaStream_t)stream>>>(p);
  return (int)cudaGetLastError();
}

int thread_per_run_max_active_blocks(int block, int smem, int* blocks) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, thread_per_run_kernel, block,
                                                            (size_t)smem);
}

}  // namespace bitssa
