// noalloc.cu -- ssa_run_frank_noalloc: a single-ensemble run of the bit-sliced
// kernel that allocates no device memory.
//
// Who needs it: callers that may not allocate device memory -- a plug-in hosted by
// a framework that owns every byte of device memory and hands out buffers from its
// own pool, or a latency-critical loop in which cudaMalloc (which can synchronise
// the device and has no bounded latency) is not allowed.  They hand in their own
// input and output buffers; the small scratch the kernel needs for itself (the
// work-queue counter, the run counters, the error word and the snapshot thresholds)
// lives in a fixed-size device array that is part of the library image.  The call
// uses the paper's bound (pad_pow2 = 0) and the group clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/bitssa.h"
#include "internal.h"

using namespace bitssa;

namespace {

// The scratch: run counters, the queue counter, the error word, and the crossing
// thresholds of up to kNoAllocMaxSnap snapshots plus t_end.
constexpr int kNoAllocMaxSnap = 64;
struct NoAllocScratch {
  unsigned long long counters[kCounters];
  unsigned long long queue;
  unsigned int status[4];
  Threshold thr[kNoAllocMaxSnap + 1];
};

// One copy per device that loads the library, kept until the process exits.
// Host code must not use this name as an address: it is a host-side stand-in for
// the device symbol; the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

int noalloc_fail(int code, const std::string& msg) {
  set_thread_error(msg);  // read back with ssa_last_error(NULL)
  return code;
}

// Device address of the scratch for the current device (looked up once per device,
// with that device current).
int scratch_for_current_device(NoAllocScratch** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(SSA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(SSA_EUNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(SSA_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = (NoAllocScratch*)g_scratch_addr[dev];
  return SSA_OK;
}


}  // namespace

extern "C" int ssa_run_frank_noalloc(const int64_t* N0, const double* rates, int64_t n_runs, uint64_t seed,
                                     int32_t thin_bits, double t_end, const double* snapshot_times,
                                     int32_t n_snap, int32_t precision, int32_t* final_counts, double* t_abs,
                                     int8_t* outcome, uint64_t* ee_hist, uint64_t* counters_out,
                                     void* cuda_stream) {
  // ---- arguments (all checked before any CUDA call)
  if (!N0 || !rates) return noalloc_fail(SSA_EINVAL, "N0 and rates are required");
  if (n_runs < 0) return noalloc_fail(SSA_EINVAL, "n_runs must be >= 0");
  if (n_runs > (1ll << 37)) return noalloc_fail(SSA_EINVAL, "n_runs beyond 2^37");
  if (n_snap < 0) return noalloc_fail(SSA_EINVAL, "n_snap must be >= 0");
  if (n_snap > kNoAllocMaxSnap)
    return noalloc_fail(SSA_EINVAL, "n_snap above 64, the size of the fixed scratch array");
  if (n_snap > 0 && !snapshot_times) return noalloc_fail(SSA_EINVAL, "snapshot_times is NULL");
  if (!(t_end >= 0.0)) return noalloc_fail(SSA_EINVAL, "t_end must be >= 0");
  for (int s = 0; s < n_snap; ++s) {
    if (!(snapshot_times[s] >= 0.0) || snapshot_times[s] > t_end)
      return noalloc_fail(SSA_EINVAL, "snapshot times must lie in [0, t_end]");
    if (s > 0 && snapshot_times[s] < snapshot_times[s - 1])
      return noalloc_fail(SSA_EINVAL, "snapshot times must be ascending");
  }
  if (precision < 0 || precision > 4) return noalloc_fail(SSA_EINVAL, "unknown precision mode");
  if (thin_bits < 1 || thin_bits > 64) return noalloc_fail(SSA_EINVAL, "thin_bits must be in [1, 64]");
  double kmax = 0.0;
  for (int r = 0; r < 3; ++r) {
    if (!(rates[r] >= 0.0) || std::isinf(rates[r])) return noalloc_fail(SSA_EINVAL, "rates must be finite and >= 0");
    kmax = std::max(kmax, rates[r]);
  }
  if (!(kmax > 0.0)) return noalloc_fail(SSA_EINVAL, "at least one rate must be > 0");
  long long n_tot = 0;
  for (int i = 0; i < 3; ++i) {
    if (N0[i] < 0) return noalloc_fail(SSA_EINVAL, "initial counts must be >= 0");
    n_tot += N0[i];
  }
  if (n_tot < 1) return noalloc_fail(SSA_EINVAL, "the total count must be >= 1");
  if (n_tot > 65536) return noalloc_fail(SSA_EUNSUPPORTED, "N_tot above 65536");
  if (n_runs > 0 && (!final_counts || !t_abs || !outcome))
    return noalloc_fail(SSA_EINVAL, "final_counts, t_abs and outcome are required");
  if (n_snap > 0 && !ee_hist) return noalloc_fail(SSA_EINVAL, "ee_hist is required when n_snap > 0");

  // ---- the ensemble (Frank's model in species order L, D, A)
  const int init[3] = {(int)N0[0], (int)N0[1], (int)N0[2]};
  const Ensemble en = make_ensemble(n_tot, init, rates, thin_bits, seed, n_runs, 0, 0, 0);
  Threshold thr[kNoAllocMaxSnap + 1];
  for (int s = 0; s < n_snap; ++s) thr[s] = make_threshold(snapshot_times[s], en.lambda);
  thr[n_snap] = make_threshold(t_end, en.lambda);

  // ---- scratch: the library's own device array
  NoAllocScratch* scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st != SSA_OK) return st;
  const cudaStream_t stream = (cudaStream_t)cuda_stream;
  cudaError_t e;
  if ((e = cudaMemsetAsync(scratch, 0, offsetof(NoAllocScratch, thr), stream)) != cudaSuccess)
    return noalloc_fail(SSA_ECUDA, std::string("clear scratch: ") + cudaGetErrorString(e));
  if ((e = cudaMemcpyAsync(scratch->thr, thr, sizeof(Threshold) * (n_snap + 1), cudaMemcpyHostToDevice, stream)) !=
      cudaSuccess)
    return noalloc_fail(SSA_ECUDA, std::string("upload thresholds: ") + cudaGetErrorString(e));
  if (n_snap > 0 &&
      (e = cudaMemsetAsync(ee_hist, 0, sizeof(uint64_t) * kHistBins * (size_t)n_snap, stream)) != cudaSuccess)
    return noalloc_fail(SSA_ECUDA, std::string("clear ee_hist: ") + cudaGetErrorString(e));

  // ---- the launch
  if (n_runs > 0) {
    FrankLaunch fl;
    std::memset(&fl, 0, sizeof fl);
    fl.ens = en;
    fl.thr = scratch->thr;
    fl.item_begin = 0;
    fl.item_end = (n_runs + 31) / 32;
    fl.n_snap = n_snap;
    fl.precision = precision;
    fl.perm[0] = 0;
    fl.perm[1] = 1;
    fl.perm[2] = 2;
    fl.n_species = 3;
    fl.final_counts = final_counts;
    fl.t_abs = t_abs;
    fl.outcome = (signed char*)outcome;
    fl.hist = (unsigned long long*)ee_hist;
    fl.n_runs_total = n_runs;
    fl.counters = scratch->counters;
    fl.status = scratch->status;
    fl.queue = &scratch->queue;
    fl.stage_offset = -1;
    const int K = std::max(1, en.K);
    const int block = 64, smem = n_snap * kHistBins * (int)sizeof(unsigned int);
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (frank_max_active_blocks(K, precision == SSA_P64 ? 2 : 0, block, smem, &occ) != 0 || occ < 1)
      return noalloc_fail(SSA_ECUDA, "occupancy query failed for the bit-sliced kernel");
    const long long need = (fl.item_end + block - 1) / block;
    const int grid = (int)std::max(1ll, std::min(need, (long long)sms * occ));
    if ((e = (cudaError_t)frank_launcher(K)(fl, grid, block, smem, (void*)stream)) != cudaSuccess)
      return noalloc_fail(SSA_ECUDA, std::string("bit-sliced kernel launch: ") + cudaGetErrorString(e));
  }
  unsigned long long host_counters[kCounters];
  unsigned int status = 0;
  if ((e = cudaMemcpyAsync(host_counters, scratch->counters, sizeof host_counters, cudaMemcpyDeviceToHost,
                           stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&status, scratch->status, sizeof status, cudaMemcpyDeviceToHost, stream)) != cudaSuccess)
    return noalloc_fail(SSA_ECUDA, std::string("read counters: ") + cudaGetErrorString(e));
  if ((e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return noalloc_fail(SSA_ECUDA, std::string("simulation: ") + cudaGetErrorString(e));
  host_counters[kErrorFlags] = status;
  host_counters[kLayoutUsed] = n_runs > 0 ? SSA_LAYOUT_THREAD : 0;
  if (counters_out) std::memcpy(counters_out, host_counters, sizeof host_counters);
  if (status & kErrRedraw) return noalloc_fail(SSA_EOVERFLOW, "64 redraws of n in a row");
  if (status & kErrRange) return noalloc_fail(SSA_EOVERFLOW, "internal range check failed");
  if (status & kErrTimeout) return noalloc_fail(SSA_ETIMEOUT, "a group reached the step budget");
  return SSA_OK;
}
