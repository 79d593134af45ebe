// lattice.cu -- host side of Frank's model on a periodic lattice: the ssa_lattice_* entry points
// of include/bitssa.h.  Validates and copies the inputs, derives the uniformisation constants
// (u = min(k_max, d), rho_r, rho_h, and for every cap m = 2^b the slots c(m), K and Lambda = M 2^K u),
// picks the instantiation whose count planes hold the caps the runs may reach, owns the device
// buffers, and launches the kernel of lattice_kernel.cuh.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bitssa.h"
#include "internal.h"
#include "lattice.h"

namespace bitssa {
void current_allocator(ssa_alloc_fn* alloc, ssa_free_fn* release, void** user);

int lattice_launch_p4(const LatticeLaunch&, int, int, int, void*);
int lattice_launch_p8(const LatticeLaunch&, int, int, int, void*);
int lattice_launch_p12(const LatticeLaunch&, int, int, int, void*);
int lattice_launch_p16(const LatticeLaunch&, int, int, int, void*);
int lattice_kw_p4();
int lattice_kw_p8();
int lattice_kw_p12();
int lattice_kw_p16();
int lattice_occupancy_p4(int, int, int*);
int lattice_occupancy_p8(int, int, int*);
int lattice_occupancy_p12(int, int, int*);
int lattice_occupancy_p16(int, int, int*);

int lattice_launch(int P, const LatticeLaunch& p, int grid, int block, int smem, void* stream) {
  switch (P) {
    case 4: return lattice_launch_p4(p, grid, block, smem, stream);
    case 8: return lattice_launch_p8(p, grid, block, smem, stream);
    case 12: return lattice_launch_p12(p, grid, block, smem, stream);
    case 16: return lattice_launch_p16(p, grid, block, smem, stream);
    default: return -1;
  }
}

int lattice_draw_planes(int P) {
  switch (P) {
    case 4: return lattice_kw_p4();
    case 8: return lattice_kw_p8();
    case 12: return lattice_kw_p12();
    case 16: return lattice_kw_p16();
    default: return -1;
  }
}

int lattice_max_active_blocks(int P, int block, int smem, int* blocks) {
  switch (P) {
    case 4: return lattice_occupancy_p4(block, smem, blocks);
    case 8: return lattice_occupancy_p8(block, smem, blocks);
    case 12: return lattice_occupancy_p12(block, smem, blocks);
    case 16: return lattice_occupancy_p16(block, smem, blocks);
    default: return -1;
  }
}

int lattice_smem_bytes(int M, int T) { return lat_smem_bytes(M, T); }

}  // namespace bitssa

using namespace bitssa;

struct ssa_lattice {
  int device = 0;
  cudaStream_t stream = nullptr;
  ssa_options opt{};
  ssa_alloc_fn alloc = nullptr;
  ssa_free_fn release = nullptr;
  void* user = nullptr;
  std::string err;
  int sm_count = 0;
  int P = 0;
  long long n_runs = 0, n_groups = 0;
  int M = 0;
  int n_snap = 0;
  bool ran = false;
  LatticeLaunch lp{};
  unsigned long long counters[kLatCounters] = {0};
  struct Buf {
    void* p;
    size_t bytes;
  };
  std::vector<Buf> bufs;
  int* d_init = nullptr;
  uint32_t* d_planes = nullptr;
  int* d_final = nullptr;
  double* d_th = nullptr;
  signed char* d_outcome = nullptr;
  long long* d_events = nullptr;
  long long* d_groups = nullptr;
  unsigned long long* d_counters = nullptr;
  double* d_snap = nullptr;
  long long* d_snap_tot = nullptr;
  int* d_snap_dom = nullptr;
  size_t snap_cap = 0;  // snapshots the snapshot buffers hold
};

namespace {

thread_local std::string t_lat_err;

int lfail(ssa_lattice* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else {
    t_lat_err = msg;
    set_thread_error(msg);
  }
  return code;
}

int lcuda(ssa_lattice* c, cudaError_t e, const char* what) {
  return lfail(c, SSA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct LatDeviceGuard {
  int prev = -1;
  explicit LatDeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~LatDeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

void* lalloc(ssa_lattice* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc) {
    p = c->alloc(bytes, c->device, (void*)c->stream, c->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->bufs.push_back({p, bytes});
  return p;
}

void lfree(ssa_lattice* c, void* p) {
  for (size_t i = 0; i < c->bufs.size(); ++i) {
    if (c->bufs[i].p == p) {
      if (c->release) c->release(p, c->bufs[i].bytes, c->device, (void*)c->stream, c->user);
      else cudaFree(p);
      c->bufs.erase(c->bufs.begin() + (long)i);
      return;
    }
  }
}

void lfree_all(ssa_lattice* c) {
  for (auto& b : c->bufs) {
    if (c->release) c->release(b.p, b.bytes, c->device, (void*)c->stream, c->user);
    else cudaFree(b.p);
  }
  c->bufs.clear();
}

int bitlen(unsigned long long v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

bool pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

// The smallest occupancy cap at or above v >= 1: 1 .. 8, then (4 + j) 2^e, j = 0 .. 3.
unsigned long long cap_at_or_above(unsigned long long v) {
  if (v <= 8) return v < 1 ? 1 : v;
  const unsigned long long unit = 1ull << (bitlen(v - 1) - 3);  // 4 unit < v <= 8 unit
  return (v + unit - 1) / unit * unit;
}

// The largest float at or below v (finite v >= 0).
float float_at_or_below(double v) {
  float f = (float)v;
  if ((double)f > v) f = std::nextafter(f, -INFINITY);
  return f;
}

size_t field_bytes(const ssa_lattice* c, int field) {
  const size_t nr = (size_t)c->n_runs, M = (size_t)c->M, ns = (size_t)c->n_snap;
  switch (field) {
    case SSA_LAT_FINAL_COUNTS: return nr * M * 3 * sizeof(int);
    case SSA_LAT_HOMOCHIRAL_TIME: return nr * sizeof(double);
    case SSA_LAT_OUTCOME: return nr;
    case SSA_LAT_EVENTS: return nr * 2 * sizeof(long long);
    case SSA_LAT_SNAP_TOTALS: return ns * nr * 3 * sizeof(long long);
    case SSA_LAT_SNAP_DOMAINS: return ns * nr * 2 * sizeof(int);
    case SSA_LAT_GROUPS: return (size_t)c->n_groups * 3 * sizeof(long long);
    case SSA_LAT_COUNTERS: return kLatCounters * sizeof(unsigned long long);
    default: return 0;
  }
}

}  // namespace

extern "C" {

int ssa_lattice_create(int32_t lx, int32_t ly, const double* rates, double hop, const int64_t* N0,
                       int32_t n0_per_run, int64_t n_runs, uint64_t seed, const ssa_options* opt,
                       int32_t cap_bits_max, ssa_lattice** out) {
  if (!out) return lfail(nullptr, SSA_EINVAL, "out is NULL");
  *out = nullptr;
  if (!pow2(lx) || !pow2(ly)) return lfail(nullptr, SSA_EINVAL, "lx and ly must be powers of two");
  const long long M = (long long)lx * ly;
  if (M > kLatMaxSites) return lfail(nullptr, SSA_EUNSUPPORTED, "lattices of more than 16384 sites are not supported");
  if (!rates) return lfail(nullptr, SSA_EINVAL, "rates is NULL");
  double k_max = 0.0;
  for (int r = 0; r < 3; ++r) {
    if (!(rates[r] >= 0.0) || !std::isfinite(rates[r])) return lfail(nullptr, SSA_EINVAL, "rates must be finite and >= 0");
    k_max = std::max(k_max, rates[r]);
  }
  if (!(k_max > 0.0)) return lfail(nullptr, SSA_EINVAL, "some rate must be positive");
  if (!(hop > 0.0) || !std::isfinite(hop)) return lfail(nullptr, SSA_EINVAL, "the hop rate d must be finite and > 0");
  if (n_runs < 0) return lfail(nullptr, SSA_EINVAL, "n_runs must be >= 0");
  if (n0_per_run != 0 && n0_per_run != 1) return lfail(nullptr, SSA_EINVAL, "n0_per_run must be 0 or 1");
  if (!N0) return lfail(nullptr, SSA_EINVAL, "N0 is NULL");
  if (cap_bits_max < 0 || cap_bits_max > 15) return lfail(nullptr, SSA_EINVAL, "cap_bits_max must be in [0, 15]");
  ssa_options o;
  ssa_default_options(&o);
  if (opt) o = *opt;
  int precision;
  switch (o.precision) {
    case SSA_P64:
    case SSA_P64_LOGSUM: precision = kP64LogSum; break;
    case SSA_P32_KAHAN: precision = kP32Kahan; break;
    case SSA_P32_D64ACC: precision = kP32D64Acc; break;
    case SSA_P32_PLAIN: precision = kP32Plain; break;
    default: return lfail(nullptr, SSA_EINVAL, "unknown precision");
  }
  if (o.thin_bits < 1 || o.thin_bits > 64) return lfail(nullptr, SSA_EINVAL, "thin_bits must be in [1, 64]");
  if (o.step_budget < 0) return lfail(nullptr, SSA_EINVAL, "step_budget must be >= 0");
  if (o.first_run < 0 || o.first_run % 32 != 0) return lfail(nullptr, SSA_EINVAL, "first_run must be a non-negative multiple of 32");
  if (o.block_size != 0 && (o.block_size < 32 || o.block_size > kLatMaxBlock || o.block_size % 32 != 0))
    return lfail(nullptr, SSA_EINVAL, "block_size must be a multiple of 32 in [32, 224]");
  if (o.blocks_per_sm < 0) return lfail(nullptr, SSA_EINVAL, "blocks_per_sm must be >= 0");
  if (o.engine != SSA_ENGINE_BITSLICED || o.layout != SSA_LAYOUT_AUTO || o.shared_n || o.pad_pow2 ||
      o.recompute || o.clock != SSA_CLOCK_GROUP || (o.word_width != 0 && o.word_width != 32) || o.tail_groups ||
      o.keep_snap_counts)
    return lfail(nullptr, SSA_EUNSUPPORTED, "the lattice runs the group clock on its own kernel; engine, layout, "
                                            "shared_n, pad_pow2, recompute, clock, word_width, tail_groups and "
                                            "keep_snap_counts must keep their defaults");
  // uniformisation constants (integers rho_r = k_max / u, rho_h = d / u, u = min(k_max, d))
  const double unit = std::min(k_max, hop);
  const double rr = k_max / unit, rh = hop / unit;
  const long long rho_r = std::llround(rr), rho_h = std::llround(rh);
  if (std::fabs(rr - (double)rho_r) > 1e-9 * rr || std::fabs(rh - (double)rho_h) > 1e-9 * rh)
    return lfail(nullptr, SSA_EINVAL, "max(k) / d or d / max(k) must be an integer");
  if (rho_r >= (1ll << kLatRhoBits)) return lfail(nullptr, SSA_EUNSUPPORTED, "max(k) / d must be below 65536");
  if (rho_h >= (1ll << 16)) return lfail(nullptr, SSA_EUNSUPPORTED, "d / max(k) must be below 65536");
  // initial counts and the initial cap
  const size_t rows = n0_per_run ? (size_t)n_runs * (size_t)M : (size_t)M;
  std::vector<int> init(rows * 3);
  long long n_max = 0;
  for (size_t i = 0; i < rows; ++i) {
    long long site = 0;
    for (int c = 0; c < 3; ++c) {
      const int64_t v = N0[i * 3 + c];
      if (v < 0 || v > 32768) return lfail(nullptr, SSA_EINVAL, "site counts must be in [0, 32768]");
      init[i * 3 + c] = (int)v;
      site += v;
    }
    n_max = std::max(n_max, site);
  }
  if (n_max > 32768) return lfail(nullptr, SSA_EUNSUPPORTED, "site totals above 32768 are not supported");
  // the caps 1 .. 8 and (4 + j) 2^e, with their slots c(m) = 4 rho_h 2^bh + rho_r m (m - 1) / 2 and K
  std::vector<LatCap> levels;
  for (unsigned long long m = 1; m <= 65536 && levels.size() < (size_t)kLatMaxLevels;) {
    LatCap cp{};
    cp.m = (unsigned)m;
    cp.bh = bitlen(m - 1);
    const unsigned long long hop_slots = 4ull * (unsigned long long)rho_h << cp.bh;
    const unsigned long long cm = hop_slots + (unsigned long long)rho_r * (m * (m - 1) / 2);
    cp.K = bitlen(cm - 1);
    cp.lambda = cp.K <= 32 ? (double)M * std::ldexp(unit, cp.K) : 0.0;
    cp.inv_lambda_f = cp.K <= 32 ? (float)(1.0 / cp.lambda) : 0.0f;
    cp.hop_slots = cp.K <= 32 ? (unsigned)hop_slots : 0u;
    levels.push_back(cp);
    m = cap_at_or_above(m + 1);  // the next cap above m
  }
  const int b0 = n_max > 1 ? bitlen((unsigned long long)(n_max - 1)) : 0;  // 2^b0 >= the first cap
  const int need = std::max(b0, (int)cap_bits_max);
  int P = 0;
  for (int cand : {4, 8, 12, 16}) {
    if (cand - 1 < need) continue;
    const int KW = lattice_draw_planes(cand);
    bool fits = true;
    for (const LatCap& cp : levels) {
      if (cp.m < (unsigned long long)std::max<long long>(n_max, 1) || cp.m > (1u << (cand - 1))) continue;
      if (cp.K > 32) break;  // the run stops there, as the definition does
      if (cp.K > KW || (KW < 32 && cp.K == KW)) fits = false;
    }
    if (fits) {
      P = cand;
      break;
    }
  }
  if (!P) return lfail(nullptr, SSA_EUNSUPPORTED, "the caps these counts and rates need exceed the kernel's planes");

  ssa_lattice* c = new ssa_lattice();
  c->opt = o;
  current_allocator(&c->alloc, &c->release, &c->user);
  c->P = P;
  c->M = (int)M;
  c->n_runs = n_runs;
  c->n_groups = (n_runs + 31) / 32;
  // device and stream
  {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
      cudaGetLastError();
      delete c;
      return lfail(nullptr, SSA_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    if (o.device >= n) {
      delete c;
      return lfail(nullptr, SSA_EINVAL, "device ordinal out of range");
    }
    if (o.device >= 0) c->device = o.device;
    else if ((e = cudaGetDevice(&c->device)) != cudaSuccess) {
      delete c;
      return lfail(nullptr, SSA_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    c->stream = (cudaStream_t)o.cuda_stream;
  }
  LatticeLaunch& lp = c->lp;
  lp.lx = lx;
  lp.ly = ly;
  lp.lx_log = bitlen((unsigned long long)lx) - 1;
  lp.M = (int)M;
  lp.rec = 3 * P;
  lp.n_runs = n_runs;
  lp.n_groups = c->n_groups;
  lp.group_base = o.first_run / 32;
  lp.seed = seed;
  lp.rho_r = (unsigned)rho_r;
  lp.rho_h = (unsigned)rho_h;
  lp.q = o.thin_bits;
  lp.thin = 0;
  lp.always = 0;
  for (int r = 0; r < 3; ++r) {
    if (rates[r] == k_max) {
      lp.always |= 1u << r;
      lp.thin_T[r] = 0;
    } else {
      lp.thin = 1;
      lp.thin_T[r] = (unsigned long long)std::floor(rates[r] / k_max * std::ldexp(1.0, o.thin_bits));
    }
  }
  lp.precision = precision;
  lp.step_budget = o.step_budget;
  lp.n_levels = (int)levels.size();
  for (size_t i = 0; i < levels.size(); ++i) lp.cap[i] = levels[i];
  lp.init_per_run = n0_per_run;
  {
    LatDeviceGuard guard(c->device);
    const size_t nr = (size_t)n_runs;
    c->d_init = (int*)lalloc(c, sizeof(int) * init.size());
    c->d_planes = (uint32_t*)lalloc(c, sizeof(uint32_t) * (size_t)c->n_groups * (size_t)M * (size_t)lp.rec);
    c->d_final = (int*)lalloc(c, sizeof(int) * nr * (size_t)M * 3);
    c->d_th = (double*)lalloc(c, sizeof(double) * nr);
    c->d_outcome = (signed char*)lalloc(c, nr);
    c->d_events = (long long*)lalloc(c, sizeof(long long) * 2 * nr);
    c->d_groups = (long long*)lalloc(c, sizeof(long long) * 3 * (size_t)c->n_groups);
    c->d_counters = (unsigned long long*)lalloc(c, sizeof(unsigned long long) * kLatCounters);
    if (!c->d_init || !c->d_planes || !c->d_final || !c->d_th || !c->d_outcome || !c->d_events || !c->d_groups ||
        !c->d_counters) {
      lfree_all(c);
      delete c;
      return lfail(nullptr, SSA_ENOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(c->d_init, init.data(), sizeof(int) * init.size(), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      lfree_all(c);
      delete c;
      return lfail(nullptr, SSA_ECUDA, std::string("upload initial counts: ") + cudaGetErrorString(e));
    }
  }
  lp.init = c->d_init;
  lp.planes = c->d_planes;
  lp.final_counts = c->d_final;
  lp.t_homochiral = c->d_th;
  lp.outcome = c->d_outcome;
  lp.events = c->d_events;
  lp.group_info = c->d_groups;
  lp.counters = c->d_counters;
  *out = c;
  return SSA_OK;
}

int ssa_lattice_run(ssa_lattice* c, double t_end, const double* snapshot_times, int32_t n_snap) {
  if (!c) return lfail(nullptr, SSA_EINVAL, "ctx is NULL");
  c->ran = false;
  if (!(t_end >= 0.0) || !std::isfinite(t_end)) return lfail(c, SSA_EINVAL, "t_end must be finite and >= 0");
  if (n_snap < 0 || n_snap > kLatMaxSnap) return lfail(c, SSA_EINVAL, "n_snap must be in [0, 64]");
  if (n_snap > 0 && !snapshot_times) return lfail(c, SSA_EINVAL, "snapshot_times is NULL");
  for (int s = 0; s < n_snap; ++s) {
    if (!(snapshot_times[s] >= 0.0) || !(snapshot_times[s] <= t_end))
      return lfail(c, SSA_EINVAL, "snapshot times must lie in [0, t_end]");
    if (s > 0 && !(snapshot_times[s] >= snapshot_times[s - 1]))
      return lfail(c, SSA_EINVAL, "snapshot times must be ascending");
  }
  nvtxRangePushA("ssa_lattice_run");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  LatDeviceGuard guard(c->device);
  cudaError_t e;
  if (n_snap > 0 && (size_t)n_snap > c->snap_cap) {
    if (c->d_snap) lfree(c, c->d_snap);
    if (c->d_snap_tot) lfree(c, c->d_snap_tot);
    if (c->d_snap_dom) lfree(c, c->d_snap_dom);
    c->snap_cap = 0;
    c->d_snap = (double*)lalloc(c, sizeof(double) * (size_t)n_snap);
    c->d_snap_tot = (long long*)lalloc(c, sizeof(long long) * 3 * (size_t)n_snap * (size_t)c->n_runs);
    c->d_snap_dom = (int*)lalloc(c, sizeof(int) * 2 * (size_t)n_snap * (size_t)c->n_runs);
    if (!c->d_snap || !c->d_snap_tot || !c->d_snap_dom) return lfail(c, SSA_ENOMEM, "device allocation failed");
    c->snap_cap = (size_t)n_snap;
  }
  c->n_snap = n_snap;
  if (n_snap > 0 &&
      (e = cudaMemcpyAsync(c->d_snap, snapshot_times, sizeof(double) * (size_t)n_snap, cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess)
    return lcuda(c, e, "upload snapshot times");
  if ((e = cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * kLatCounters, c->stream)) != cudaSuccess)
    return lcuda(c, e, "clear counters");
  LatticeLaunch lp = c->lp;
  lp.t_end = t_end;
  lp.t_end_f = float_at_or_below(t_end);
  for (int i = 0; i < n_snap; ++i) lp.snap_f[i] = float_at_or_below(snapshot_times[i]);
  lp.snap = n_snap > 0 ? c->d_snap : nullptr;
  lp.n_snap = n_snap;
  lp.snap_totals = n_snap > 0 ? c->d_snap_tot : nullptr;
  lp.snap_domains = n_snap > 0 ? c->d_snap_dom : nullptr;
  const int T = c->opt.block_size ? c->opt.block_size : kLatDefaultWindow;
  const int block = T + 32;  // T step threads and the service warp
  lp.block = T;
  if (c->n_groups > 0) {
    const int smem = lattice_smem_bytes(c->M, T);
    int per_sm = 0;
    if (lattice_max_active_blocks(c->P, block, smem, &per_sm) != 0 || per_sm < 1)
      return lfail(c, SSA_EUNSUPPORTED, "the lattice kernel does not fit an SM at this lattice and block size");
    if (c->opt.blocks_per_sm > 0) per_sm = std::min(per_sm, c->opt.blocks_per_sm);
    const long long grid = std::min<long long>(c->n_groups, (long long)per_sm * std::max(c->sm_count, 1));
    const int rc = lattice_launch(c->P, lp, (int)grid, block, smem, (void*)c->stream);
    if (rc != 0) return lcuda(c, (cudaError_t)rc, "lattice kernel launch");
  }
  if ((e = cudaMemcpyAsync(c->counters, c->d_counters, sizeof(unsigned long long) * kLatCounters,
                           cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return lcuda(c, e, "read counters");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return lcuda(c, e, "lattice run");
  c->ran = true;
  if (c->counters[kLatErrors] > 0) {
    std::vector<long long> info((size_t)c->n_groups * 3);
    if ((e = cudaMemcpy(info.data(), c->d_groups, sizeof(long long) * info.size(), cudaMemcpyDeviceToHost)) !=
        cudaSuccess)
      return lcuda(c, e, "read group status");
    for (long long g = 0; g < c->n_groups; ++g) {
      const long long st = info[(size_t)g * 3 + 2];
      const std::string where = "group " + std::to_string(g) + ": ";
      if (st == kLatTimeout) return lfail(c, SSA_ETIMEOUT, where + "step budget reached");
      if (st == kLatRange) return lfail(c, SSA_EOVERFLOW, where + "the occupancy cap needs more than 32 planes of n");
      if (st == kLatCapacity)
        return lfail(c, SSA_EOVERFLOW, where + "the occupancy cap outgrew this context's count planes "
                                               "(create it with a larger cap_bits_max)");
      if (st == kLatBadInit) return lfail(c, SSA_EOVERFLOW, where + "initial counts above the count planes");
    }
  }
  return SSA_OK;
}

int ssa_lattice_field_bytes(const ssa_lattice* c, int32_t field, size_t* bytes) {
  if (!c || !bytes) return lfail(const_cast<ssa_lattice*>(c), SSA_EINVAL, "null argument");
  *bytes = field_bytes(c, field);
  return SSA_OK;
}

int ssa_lattice_fetch(ssa_lattice* c, int32_t field, void* dst, size_t dst_bytes, int32_t dst_on_device) {
  if (!c) return lfail(nullptr, SSA_EINVAL, "ctx is NULL");
  if (!c->ran) return lfail(c, SSA_ESTATE, "ssa_lattice_fetch before ssa_lattice_run");
  if (field < SSA_LAT_FINAL_COUNTS || field > SSA_LAT_COUNTERS) return lfail(c, SSA_EINVAL, "unknown field");
  const size_t bytes = field_bytes(c, field);
  if (dst_bytes < bytes) return lfail(c, SSA_EINVAL, "destination too small");
  if (bytes == 0) return SSA_OK;
  if (!dst) return lfail(c, SSA_EINVAL, "dst is NULL");
  LatDeviceGuard guard(c->device);
  if (field == SSA_LAT_COUNTERS && !dst_on_device) {
    std::memcpy(dst, c->counters, bytes);
    return SSA_OK;
  }
  const void* src = nullptr;
  switch (field) {
    case SSA_LAT_FINAL_COUNTS: src = c->d_final; break;
    case SSA_LAT_HOMOCHIRAL_TIME: src = c->d_th; break;
    case SSA_LAT_OUTCOME: src = c->d_outcome; break;
    case SSA_LAT_EVENTS: src = c->d_events; break;
    case SSA_LAT_SNAP_TOTALS: src = c->d_snap_tot; break;
    case SSA_LAT_SNAP_DOMAINS: src = c->d_snap_dom; break;
    case SSA_LAT_GROUPS: src = c->d_groups; break;
    case SSA_LAT_COUNTERS: src = c->d_counters; break;
  }
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e != cudaSuccess) return lcuda(c, e, "fetch copy");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return lcuda(c, e, "fetch synchronize");
  return SSA_OK;
}

int ssa_lattice_destroy(ssa_lattice* c) {
  if (!c) return SSA_OK;
  {
    LatDeviceGuard guard(c->device);
    if (!c->bufs.empty()) cudaStreamSynchronize(c->stream);
    lfree_all(c);
  }
  delete c;
  return SSA_OK;
}

const char* ssa_lattice_last_error(const ssa_lattice* c) { return c ? c->err.c_str() : t_lat_err.c_str(); }

}  // extern "C"
