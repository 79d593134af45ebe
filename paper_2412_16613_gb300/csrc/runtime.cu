// runtime.cu -- host side of libbitssa: the C ABI declared in include/bitssa.h.
//
// Validates and copies the inputs, derives the per-ensemble constants of the
// method (lambda_int = N (N - 1) / 2 of Eq. equation-z, or its general form
// m_pair C(N, 2) + u_max N, or 2^K when padded; K; the thinning thresholds), owns
// the device buffers, and launches the bit-sliced kernel instantiation for each K:
// Frank's two layouts or the general-network kernel (or the one-thread-per-run
// baseline).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/bitssa.h"
#include "internal.h"

using namespace bitssa;

namespace bitssa {

namespace {
int bits_of(unsigned long long v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}
}  // namespace

// Per-ensemble constants from their definitions.
Ensemble make_ensemble(long long n_tot, const int init[3], const double k[3], int q, unsigned long long seed,
                       long long n_runs, long long run_offset, long long group_base, int pad_pow2) {
  Ensemble e;
  std::memset(&e, 0, sizeof e);
  e.seed = seed;
  e.n_runs = n_runs;
  e.run_offset = run_offset;
  e.group_base = group_base;
  e.n_tot = (int)n_tot;
  const unsigned long long z = (unsigned long long)n_tot * (unsigned long long)(n_tot - 1) / 2ull;
  e.K = bits_of(z);
  // padded: null events fill [z, 2^K), so that no K-bit draw is rejected
  const unsigned long long lam = pad_pow2 ? (1ull << e.K) : z;
  e.lambda_int = (unsigned int)lam;
  e.reject = pad_pow2 ? 0 : 1;
  set_precheck(e);
  const double kmax = std::max(k[0], std::max(k[1], k[2]));
  e.lambda = kmax * (double)lam;
  e.inv_lambda_f = (float)(1.0 / e.lambda);
  e.thin_bits = q;
  for (int r = 0; r < 3; ++r) {
    e.init[r] = init[r];
    if (k[r] > 0.0) e.active |= 1u << r;
    if (k[r] == kmax) {
      e.thin_always |= 1u << r;
      e.thin_T[r] = 0;
    } else {
      e.thin_T[r] = (long long)(unsigned long long)std::floor(std::ldexp(k[r] / kmax, q));
      e.thin = 1;
    }
  }
  return e;
}

// Per-ensemble constants of a general network.  lambda_int = m_pair C(N, 2) + u_max N bounds
// sum_r h_r over every state with N molecules: the pairs {i, j} (i < j) and {i, i} carry
// n_i n_j and C(n_i, 2), which sum to C(N, 2) (Eq. equation-z), and each carries at most m_pair
// reactions; each species carries at most u_max first-order reactions of propensity n_i <= N.
Ensemble make_general_ensemble(const Network& net, long long n_tot, const int* init, const double* k, int q,
                               unsigned long long seed, long long n_runs, long long run_offset,
                               long long group_base, int pad_pow2, unsigned long long* lambda_unpadded) {
  Ensemble e;
  std::memset(&e, 0, sizeof e);
  e.seed = seed;
  e.n_runs = n_runs;
  e.run_offset = run_offset;
  e.group_base = group_base;
  e.n_tot = (int)n_tot;
  int pair[kMaxSpecies][kMaxSpecies] = {{0}}, uni[kMaxSpecies] = {0};
  for (int r = 0; r < net.R; ++r) {
    if (net.order[r] == 2) ++pair[std::min(net.a[r], net.b[r])][std::max(net.a[r], net.b[r])];
    else ++uni[net.a[r]];
  }
  int m_pair = 0, u_max = 0;
  for (int i = 0; i < net.S; ++i) {
    u_max = std::max(u_max, uni[i]);
    for (int j = 0; j < net.S; ++j) m_pair = std::max(m_pair, pair[i][j]);
  }
  const unsigned long long N = (unsigned long long)n_tot;
  const unsigned long long z = (unsigned long long)m_pair * (N * (N - 1) / 2ull) + (unsigned long long)u_max * N;
  if (lambda_unpadded) *lambda_unpadded = z;
  e.K = bits_of(z);
  const unsigned long long lam = pad_pow2 ? (1ull << std::min(e.K, 31)) : z;
  e.lambda_int = (unsigned int)lam;
  e.reject = pad_pow2 ? 0 : 1;
  set_precheck(e);
  double kmax = 0.0;
  for (int r = 0; r < net.R; ++r) kmax = std::max(kmax, k[r]);
  e.lambda = kmax * (double)lam;
  e.inv_lambda_f = (float)(1.0 / e.lambda);
  e.thin_bits = q;
  for (int i = 0; i < net.S; ++i) e.init[i] = init ? init[i] : 0;
  for (int r = 0; r < net.R; ++r) {
    if (k[r] > 0.0) e.active |= 1u << r;
    if (k[r] == kmax) {
      e.thin_always |= 1u << r;
      e.thin_T[r] = 0;
    } else {
      e.thin_T[r] = (long long)(unsigned long long)std::floor(std::ldexp(k[r] / kmax, q));
      e.thin = 1;
    }
  }
  return e;
}

// The crossing threshold of time t for total rate lambda.
Threshold make_threshold(double t, double lambda) {
  Threshold h;
  std::memset(&h, 0, sizeof h);
  h.t = t;
  float f = (float)t;
  if ((double)f > t) f = std::nextafter(f, -INFINITY);
  h.t_f = f;
  if (std::isinf(t) || !(lambda > 0.0)) {
    h.E = LLONG_MIN;
    h.M = 1ull << 63;
    return h;
  }
  const double theta = -lambda * t;  // ln exp(-lambda t)
  long long E = (long long)std::floor(theta / M_LN2);
  double m = std::exp(theta - (double)E * M_LN2);
  while (m >= 2.0) {
    m *= 0.5;
    ++E;
  }
  while (m < 1.0) {
    m *= 2.0;
    --E;
  }
  h.E = E;
  h.M = (unsigned long long)std::ldexp(m, 63);  // m in [1, 2): exact
  return h;
}

}  // namespace bitssa

namespace {

// An NVTX range for the lifetime of a scope: named ranges around runs, launches and the tuner
// for profilers that follow NVTX (no cost without one attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct Allocator {
  ssa_alloc_fn alloc = nullptr;
  ssa_free_fn release = nullptr;
  void* user = nullptr;
};

std::mutex g_alloc_mu;
Allocator g_alloc;
thread_local std::string t_err;


}  // namespace

struct ssa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  ssa_options opt{};
  Allocator alloc;
  std::string err;
  int S = 3;
  int R = 3;
  int perm[3] = {0, 1, 2};  // canonical species (L, D, A) -> caller's species index
  bool general = false;     // the general-network kernel runs this context
  Network net{};            // the network, for the general kernel
  bool batch = false;
  int n_ens = 0;
  long long n_runs_total = 0;
  std::vector<Ensemble> ens;
  std::vector<double> rates;  // [n_ens][3]
  // batch work items, sorted by K (descending), and the K of each launch range
  std::vector<int> item_ens, item_group;
  std::vector<std::pair<int, std::pair<long long, long long>>> ranges;  // K -> [begin, end)
  struct Buf {
    void* p;
    size_t bytes;
  };
  std::vector<Buf> bufs;
  Ensemble* d_ens = nullptr;
  Threshold* d_thr = nullptr;
  size_t thr_cap = 0;
  int* d_item_ens = nullptr;
  int* d_item_group = nullptr;
  int* d_init = nullptr;
  int* d_final = nullptr;
  double* d_tabs = nullptr;
  signed char* d_outcome = nullptr;
  unsigned long long* d_hist = nullptr;
  size_t hist_cap = 0;
  unsigned long long* d_ens_abs = nullptr;
  int* d_snap = nullptr;
  size_t snap_cap = 0;
  unsigned long long* d_counters = nullptr;  // [kCounters] then the queues
  unsigned int* d_status = nullptr;
  int layout_used = 0;  // SSA_LAYOUT_* bits of the last run, 0 if none
  int tuned_layout = -1;  // ssa_tune's choice for SSA_LAYOUT_AUTO: -1 none, else an SSA_LAYOUT_*
  int tuned_block = 0;    // ssa_tune's block size for the one-thread layout, 0 none
  int tuned_products = -1;  // ssa_tune's mode for the general kernel: -1 none, 0 incremental, 1 products
  int tuned_tail = -1;      // ssa_tune's tail hand-off threshold: -1 none, 0 off, else groups per warp
  int n_queues = 0;
  bool ran = false;
  int n_snap = 0;
  unsigned long long counters[kCounters] = {0};
  int sm_count = 0;
  // batch: the K buckets run concurrently on side streams forked from `stream`
  std::vector<cudaStream_t> side;
  cudaGraphExec_t batch_graph = nullptr;     // the batch's fork / launches / join, captured once
  std::vector<unsigned char> batch_graph_key; // the launch plan it was captured from
  std::vector<cudaEvent_t> side_done;
  cudaEvent_t fork = nullptr;
};

namespace {

int fail(ssa_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else t_err = msg;
  return code;
}

int cuda_fail(ssa_ctx* c, cudaError_t e, const char* what) {
  return fail(c, SSA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (dev >= 0 && dev != prev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

void* dev_alloc(ssa_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc.alloc) {
    p = c->alloc.alloc(bytes, c->device, (void*)c->stream, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) c->bufs.push_back({p, bytes});
  return p;
}

void dev_free(ssa_ctx* c, void* p) {
  for (size_t i = 0; i < c->bufs.size(); ++i) {
    if (c->bufs[i].p == p) {
      if (c->alloc.release) c->alloc.release(p, c->bufs[i].bytes, c->device, (void*)c->stream, c->alloc.user);
      else cudaFree(p);
      c->bufs.erase(c->bufs.begin() + (long)i);
      return;
    }
  }
}

void dev_free_all(ssa_ctx* c) {
  for (auto& b : c->bufs) {
    if (c->alloc.release) c->alloc.release(b.p, b.bytes, c->device, (void*)c->stream, c->alloc.user);
    else cudaFree(b.p);
  }
  c->bufs.clear();
}

// ---------------------------------------------------------------------------
// Validation of the network: order 1 or 2, conservation of the total count
// (Sec. 2), at most 8 species and 8 reactions, and recognition of Frank's model
// (Eqs. 1-3) up to relabelling (every other network goes to the general kernel).
// ---------------------------------------------------------------------------
int check_network(const int32_t* reac, const int32_t* prod, int S, int R, int perm[3], bool* frank,
                  std::string* why) {
  *frank = false;
  if (!reac || !prod) return (*why = "null stoichiometry", SSA_EINVAL);
  if (S < 1 || R < 1 || S > 64 || R > 64) return (*why = "n_species / n_reactions out of range", SSA_EINVAL);
  for (int r = 0; r < R; ++r) {
    int order = 0, made = 0;
    for (int i = 0; i < S; ++i) {
      if (reac[r * S + i] < 0 || prod[r * S + i] < 0) return (*why = "negative stoichiometry", SSA_EINVAL);
      order += reac[r * S + i];
      made += prod[r * S + i];
    }
    if (order < 1 || order > 2)
      return (*why = "reaction " + std::to_string(r) + " has order " + std::to_string(order) +
                     " (orders 1 and 2 only)", SSA_EINVAL);
    if (made != order)
      return (*why = "reaction " + std::to_string(r) + " does not conserve the total count", SSA_EINVAL);
  }
  if (S > kMaxSpecies || R > kMaxReactions)
    return (*why = "at most 8 species and 8 reactions", SSA_EUNSUPPORTED);
  if (S != 3 || R != 3) return SSA_OK;  // a general network
  // reaction 2: X + Y -> 2A
  int A = -1;
  for (int i = 0; i < 3; ++i)
    if (prod[2 * 3 + i] == 2) A = i;
  auto is_auto = [&](int r, int& X) {  // A + X -> 2X
    X = -1;
    for (int i = 0; i < 3; ++i)
      if (i != A && reac[r * 3 + i] == 1 && prod[r * 3 + i] == 2) X = i;
    return X >= 0 && reac[r * 3 + A] == 1 && prod[r * 3 + A] == 0;
  };
  int X = -1, Y = -1;
  const bool ok = A >= 0 && is_auto(0, X) && is_auto(1, Y) && X != Y && reac[2 * 3 + X] == 1 &&
                  reac[2 * 3 + Y] == 1 && reac[2 * 3 + A] == 0 && prod[2 * 3 + X] == 0 && prod[2 * 3 + Y] == 0;
  if (!ok) return SSA_OK;  // a general network
  perm[0] = X;
  perm[1] = Y;
  perm[2] = A;
  *frank = true;
  return SSA_OK;
}

// The network in the form the general kernel reads.  The ee histogram bins Frank's X and Y when
// the network is Frank's model, else species 0 and 1.
Network make_network(const int32_t* reac, const int32_t* prod, int S, int R, bool frank, const int perm[3]) {
  Network net;
  std::memset(&net, 0, sizeof net);
  net.S = S;
  net.R = R;
  for (int r = 0; r < R; ++r) {
    int first = -1, second = -1, order = 0;
    for (int i = 0; i < S; ++i) {
      const int m = reac[r * S + i];
      order += m;
      if (m == 2) first = second = i;
      if (m == 1) {
        if (first < 0) first = i;
        else second = i;
      }
      net.nu[r][i] = prod[r * S + i] - m;
    }
    net.order[r] = order;
    net.a[r] = first;
    net.b[r] = order == 2 ? second : -1;
  }
  for (int r = 0; r < R; ++r)
    for (int i = 0; i < S; ++i) {
      const unsigned int v = (unsigned int)net.nu[r][i] & 7u;  // three-bit two's complement
      for (int b = 0; b < 3; ++b)
        if ((v >> b) & 1u) net.nu_bits[i][b] |= 1u << r;
      if (v) net.changes |= 1u << i;
    }
  net.hist_x = frank ? perm[0] : 0;
  net.hist_y = frank ? perm[1] : (S > 1 ? 1 : -1);
  return net;
}

int check_rates(const double* k, std::string* why, int R = 3) {
  double kmax = 0.0;
  for (int r = 0; r < R; ++r) {
    if (!(k[r] >= 0.0) || std::isinf(k[r])) return (*why = "rates must be finite and >= 0", SSA_EINVAL);
    kmax = std::max(kmax, k[r]);
  }
  if (!(kmax > 0.0)) return (*why = "at least one rate must be > 0", SSA_EINVAL);
  return SSA_OK;
}

int check_options(const ssa_options& o, std::string* why) {
  if (o.precision < 0 || o.precision > 4) return (*why = "unknown precision mode", SSA_EINVAL);
  if (o.engine < 0 || o.engine > 2) return (*why = "unknown engine", SSA_EINVAL);
  if (o.engine == SSA_ENGINE_GENERAL && o.layout == SSA_LAYOUT_WARPS)
    return (*why = "the general engine runs one thread per group", SSA_EUNSUPPORTED);
  if (o.layout < SSA_LAYOUT_AUTO || o.layout > SSA_LAYOUT_WARPS) return (*why = "unknown layout", SSA_EINVAL);
  if (o.shared_n != 0 && o.shared_n != 1) return (*why = "shared_n must be 0 or 1", SSA_EINVAL);
  if (o.shared_n && o.engine == SSA_ENGINE_THREAD_PER_RUN)
    return (*why = "shared_n is a mode of the bit-sliced engines", SSA_EUNSUPPORTED);
  if (o.pad_pow2 < 0 || o.pad_pow2 > 2) return (*why = "pad_pow2 must be 0, 1 or 2", SSA_EINVAL);
  if (o.pad_pow2 == 2 && (o.engine == SSA_ENGINE_GENERAL || o.layout == SSA_LAYOUT_WARPS || o.shared_n))
    return (*why = "the state-following bound (pad_pow2 = 2) runs Frank's model on one thread per group",
            SSA_EUNSUPPORTED);
  if (o.recompute < 0 || o.recompute > 3) return (*why = "recompute must be 0, 1, 2 or 3", SSA_EINVAL);
  if (o.pad_pow2 && o.engine == SSA_ENGINE_THREAD_PER_RUN)
    return (*why = "pad_pow2 is a mode of the bit-sliced engines", SSA_EUNSUPPORTED);
  if (o.thin_bits < 1 || o.thin_bits > 64) return (*why = "thin_bits must be in [1, 64]", SSA_EINVAL);
  if (o.block_size < 0 || o.block_size > 256 || (o.block_size % 32) != 0)
    return (*why = "block_size must be 0 or a multiple of 32 up to 256", SSA_EINVAL);
  if (o.blocks_per_sm < 0) return (*why = "blocks_per_sm must be >= 0", SSA_EINVAL);
  if (o.step_budget < 0) return (*why = "step_budget must be >= 0", SSA_EINVAL);
  if (o.first_run < 0 || (o.first_run % 32) != 0) return (*why = "first_run must be a multiple of 32", SSA_EINVAL);
  if (o.clock != SSA_CLOCK_GROUP && o.clock != SSA_CLOCK_LANE) return (*why = "unknown clock", SSA_EINVAL);
  if (o.clock == SSA_CLOCK_LANE &&
      (o.engine != SSA_ENGINE_BITSLICED || o.layout == SSA_LAYOUT_WARPS || o.shared_n || o.pad_pow2 == 2))
    return (*why = "the per-run clock (SSA_CLOCK_LANE) runs Frank's model on one thread per group, with the "
                   "paper's or the padded bound",
            SSA_EUNSUPPORTED);
  if (o.clock == SSA_CLOCK_LANE && o.block_size > 128)
    return (*why = "per-run clocks keep 544 bytes of shared memory per thread: blocks of at most 128 threads",
            SSA_EUNSUPPORTED);
  if (o.word_width != 0 && o.word_width != 32 && o.word_width != 64)
    return (*why = "word_width must be 0, 32 or 64", SSA_EINVAL);
  if (o.word_width == 64)
    return (*why = "64-lane words (two groups per thread) do not fit a thread's registers", SSA_EUNSUPPORTED);
  if (o.tail_groups < -1 || o.tail_groups > kTailSlots) return (*why = "tail_groups must be in [-1, 4]", SSA_EINVAL);
  return SSA_OK;
}


int grow(ssa_ctx* c, void** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return SSA_OK;
  if (*p) dev_free(c, *p);
  *p = dev_alloc(c, need);
  *cap = *p ? need : 0;
  return *p ? SSA_OK : fail(c, SSA_ENOMEM, "device allocation failed");
}

int setup_device(ssa_ctx* c) {
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    cudaGetLastError();
    return fail(c, SSA_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  if (c->opt.device >= n) return fail(c, SSA_EINVAL, "device ordinal out of range");
  if (c->opt.device >= 0) c->device = c->opt.device;
  else if ((e = cudaGetDevice(&c->device)) != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess)
    return cuda_fail(c, e, "cudaDeviceGetAttribute");
  c->stream = (cudaStream_t)c->opt.cuda_stream;
  return SSA_OK;
}

int allocate_common(ssa_ctx* c, const std::vector<int>& init_rows) {
  const long long nr = c->n_runs_total;
  const int S = c->S;
  c->d_ens = (Ensemble*)dev_alloc(c, sizeof(Ensemble) * (size_t)c->n_ens);
  c->d_final = (int*)dev_alloc(c, sizeof(int) * (size_t)nr * S);
  c->d_tabs = (double*)dev_alloc(c, sizeof(double) * (size_t)nr);
  c->d_outcome = (signed char*)dev_alloc(c, (size_t)nr);
  c->d_ens_abs = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * 4 * (size_t)c->n_ens);
  c->n_queues = 1 + (int)c->ranges.size();
  c->d_counters = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long) * (kCounters + c->n_queues));
  c->d_status = (unsigned int*)dev_alloc(c, sizeof(unsigned int) * 4);
  if (!c->d_ens || !c->d_final || !c->d_tabs || !c->d_outcome || !c->d_ens_abs || !c->d_counters || !c->d_status)
    return fail(c, SSA_ENOMEM, "device allocation failed");
  cudaError_t e;
  if ((e = cudaMemcpyAsync(c->d_ens, c->ens.data(), sizeof(Ensemble) * c->ens.size(), cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "upload ensembles");
  if (!init_rows.empty()) {
    c->d_init = (int*)dev_alloc(c, sizeof(int) * init_rows.size());
    if (!c->d_init) return fail(c, SSA_ENOMEM, "device allocation failed");
    if ((e = cudaMemcpyAsync(c->d_init, init_rows.data(), sizeof(int) * init_rows.size(), cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "upload initial counts");
  }
  if (!c->item_ens.empty()) {
    c->d_item_ens = (int*)dev_alloc(c, sizeof(int) * c->item_ens.size());
    c->d_item_group = (int*)dev_alloc(c, sizeof(int) * c->item_group.size());
    if (!c->d_item_ens || !c->d_item_group) return fail(c, SSA_ENOMEM, "device allocation failed");
    cudaMemcpyAsync(c->d_item_ens, c->item_ens.data(), sizeof(int) * c->item_ens.size(), cudaMemcpyHostToDevice,
                    c->stream);
    cudaMemcpyAsync(c->d_item_group, c->item_group.data(), sizeof(int) * c->item_group.size(),
                    cudaMemcpyHostToDevice, c->stream);
  }
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  return SSA_OK;
}

int create_common(const int32_t* reac, const int32_t* prod, int32_t S, int32_t R, const ssa_options* opt,
                  ssa_ctx** out, ssa_ctx** made, int perm[3]) {
  for (int i = 0; i < 3; ++i) perm[i] = i;
  if (!out) return fail(nullptr, SSA_EINVAL, "out is NULL");
  *out = nullptr;
  ssa_options o;
  ssa_default_options(&o);
  if (opt) o = *opt;
  std::string why;
  int st = check_options(o, &why);
  if (st != SSA_OK) return fail(nullptr, st, why);
  bool frank = false;
  st = check_network(reac, prod, S, R, perm, &frank, &why);
  if (st != SSA_OK) return fail(nullptr, st, why);
  const bool general = !frank || o.engine == SSA_ENGINE_GENERAL;
  if (general && o.engine == SSA_ENGINE_THREAD_PER_RUN)
    return fail(nullptr, SSA_EUNSUPPORTED, "the thread-per-run engine runs Frank's model (A+X->2X, A+Y->2Y, "
                                           "X+Y->2A in this order) only");
  if (frank && !general && o.shared_n && o.layout == SSA_LAYOUT_THREAD)
    return fail(nullptr, SSA_EUNSUPPORTED, "shared_n runs Frank's model on the three-warp layout");
  if (general && o.layout == SSA_LAYOUT_WARPS)
    return fail(nullptr, SSA_EUNSUPPORTED, "a general network runs one thread per group");
  if (general && o.pad_pow2 == 2)
    return fail(nullptr, SSA_EUNSUPPORTED, "the state-following bound (pad_pow2 = 2) runs Frank's model only");
  if (general && o.clock == SSA_CLOCK_LANE)
    return fail(nullptr, SSA_EUNSUPPORTED, "the per-run clock (SSA_CLOCK_LANE) runs Frank's model only");
  ssa_ctx* c = new ssa_ctx();
  c->opt = o;
  c->S = S;
  c->R = R;
  c->general = general;
  if (general) {
    c->net = make_network(reac, prod, S, R, frank, perm);
    c->net.incremental = o.recompute == 1 ? 0 : 1;
  }
  for (int i = 0; i < 3; ++i) c->perm[i] = perm[i];
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    c->alloc = g_alloc;
  }
  *made = c;
  return SSA_OK;
}

// One bucket's launch in a batch: everything that decides the kernel and its arguments.
struct BatchLaunch {
  int K, warps, grid, block, stream;
  int general, smem;  // the general-network kernel and its dynamic shared memory
  FrankLaunch fl;
};

// Fork the side streams from the context's stream, launch every bucket, join.
int issue_batch(ssa_ctx* c, const std::vector<BatchLaunch>& plan) {
  cudaError_t e;
  if ((e = cudaEventRecord(c->fork, c->stream)) != cudaSuccess) return cuda_fail(c, e, "fork event");
  for (cudaStream_t s : c->side)
    if ((e = cudaStreamWaitEvent(s, c->fork, 0)) != cudaSuccess) return cuda_fail(c, e, "fork wait");
  for (const BatchLaunch& b : plan) {
    void* s = (void*)c->side[b.stream];
    if (b.general) {
      if ((e = (cudaError_t)general_launcher(b.K)(b.fl, b.grid, b.block, b.smem, s)) != cudaSuccess)
        return cuda_fail(c, e, "general bit-sliced kernel launch");
    } else if (b.warps) {
      if ((e = (cudaError_t)frank_trio_launcher(b.K)(b.fl, b.grid, 0, s)) != cudaSuccess)
        return cuda_fail(c, e, "three-warp bit-sliced kernel launch");
    } else if ((e = (cudaError_t)frank_launcher(b.K)(b.fl, b.grid, b.block, 0, s)) != cudaSuccess) {
      return cuda_fail(c, e, "bit-sliced kernel launch");
    }
  }
  for (size_t i = 0; i < c->side.size(); ++i) {
    if ((e = cudaEventRecord(c->side_done[i], c->side[i])) != cudaSuccess) return cuda_fail(c, e, "join event");
    if ((e = cudaStreamWaitEvent(c->stream, c->side_done[i], 0)) != cudaSuccess) return cuda_fail(c, e, "join wait");
  }
  return SSA_OK;
}

// Issue a batch's launch plan: on a capturable stream it is recorded once as a CUDA graph and
// replayed while it stays the same, so a batch of any size is one graph launch.
int run_plan(ssa_ctx* c, const std::vector<BatchLaunch>& plan) {
  cudaError_t e;
  if (!c->stream) return issue_batch(c, plan);  // the legacy default stream cannot be captured
  std::vector<unsigned char> key(sizeof(BatchLaunch) * plan.size());
  std::memcpy(key.data(), plan.data(), key.size());
  if (!c->batch_graph || key != c->batch_graph_key) {
    if (c->batch_graph) cudaGraphExecDestroy(c->batch_graph);
    c->batch_graph = nullptr;
    c->batch_graph_key.clear();
    if ((e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
      return cuda_fail(c, e, "begin capture of the batch launch");
    const int st = issue_batch(c, plan);
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (st != SSA_OK || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return st != SSA_OK ? st : cuda_fail(c, ee, "end capture of the batch launch");
    }
    e = cudaGraphInstantiate(&c->batch_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->batch_graph = nullptr;
      return cuda_fail(c, e, "instantiate the batch graph");
    }
    c->batch_graph_key = key;
  }
  if ((e = cudaGraphLaunch(c->batch_graph, c->stream)) != cudaSuccess) return cuda_fail(c, e, "batch graph launch");
  return SSA_OK;
}

// The layout of the bit-sliced engine for one launch of `groups` groups.  The three-warp
// layout finishes a group's step sooner (its work is split over three schedulers) but holds a
// group in three times as many threads; SSA_LAYOUT_AUTO takes it while its blocks fit at most
// two to an SM, where a launch's time is its longest group's steps times the step latency, and
// the one-thread layout beyond that, where the three-warp blocks would no longer all be
// resident (measured on GB300 at N_tot = 1024: three warps ahead up to 2^18 runs, one thread
// ahead from 2^19).  A batch decides per K bucket: 4096 ensembles of 1024 runs with N_tot
// log-uniform in [16, 65536] take 19.7 s on three warps against 36.2 s on one thread.
bool use_warps_layout(const ssa_options& o, long long groups, int sm_count) {
  if (o.layout == SSA_LAYOUT_THREAD) return false;
  if (o.layout == SSA_LAYOUT_WARPS) return true;
  return groups <= 64ll * sm_count;
}

// The layout of one launch of a context: a fixed option wins, then the tuner's choice, then the
// rule above.
bool ctx_warps(const ssa_ctx* c, long long groups) {
  if (c->general) return false;      // the general kernel has one layout
  if (c->opt.clock == SSA_CLOCK_LANE) return false;  // per-run clocks are built into one thread only
  if (c->opt.pad_pow2 == 2) return false;  // the state-following bound is built into one thread only
  if (c->opt.shared_n) return true;  // Frank's kernels: the shared draw is built into three warps only
  if (c->opt.layout == SSA_LAYOUT_AUTO && c->tuned_layout == SSA_LAYOUT_THREAD) return false;
  if (c->opt.layout == SSA_LAYOUT_AUTO && c->tuned_layout == SSA_LAYOUT_WARPS) return true;
  return use_warps_layout(c->opt, groups, c->sm_count);
}

// Shared memory of the general kernel per block, histogram excluded: the count planes of every
// thread ([species][plane][thread] words; enough planes for the products at K), the scratch
// words, and in incremental mode the K planes of every propensity; none with the planes in
// registers.
int general_smem(const ssa_ctx* c, int K, int block, bool regs) {
  if (regs) return 0;
  const int BM = bit_length(frank_nmax(K));
  const int words = c->net.S * std::max(BM, c->net.B) + kGeneralScratch + (c->net.incremental ? c->net.R * K : 0);
  return words * block * (int)sizeof(uint32_t);
}

// Whether the general kernel's launch at K keeps its count planes and propensities in registers:
// incremental mode not fixed to shared memory (recompute = 3), at most kRegSpecies species and
// kRegReactions reactions, K at most kRegMaxK, and the counts of every ensemble at that K inside
// the planes the products read (always so with a reaction of order 2).
bool general_in_registers(const ssa_ctx* c, int K) {
  if (!c->net.incremental || c->opt.recompute == 3) return false;
  if (c->net.S > kRegSpecies || c->net.R > kRegReactions || K > kRegMaxK) return false;
  for (const Ensemble& e : c->ens)
    if (std::max(1, e.K) == K && bit_length(e.n_tot) > bit_length(frank_nmax(K))) return false;
  return true;
}

// Launches of the general-network kernel: one for a single ensemble, one per K bucket (on the
// caller's stream, one after another) for a batch.
int launch_general(ssa_ctx* c, FrankLaunch fl, int block, int clock_variant) {
  cudaError_t e;
  // the propensity mode: a fixed option wins, then the tuner's choice, then incremental
  c->net.incremental = c->opt.recompute == 1 ? 0 : (c->opt.recompute >= 2 ? 1 : (c->tuned_products == 1 ? 0 : 1));
  c->net.regs = 0;
  fl.net = c->net;
  const int hist_smem = c->batch ? 0 : c->n_snap * kHistBins * (int)sizeof(unsigned int);
  c->layout_used = SSA_LAYOUT_THREAD | (c->net.incremental ? kLayoutGeneralIncremental : kLayoutGeneralProducts);
  if (!c->batch) {
    const int K = std::max(1, c->ens[0].K);
    const bool regs = general_in_registers(c, K);
    fl.net.regs = regs ? 1 : 0;
    if (regs) c->layout_used |= kLayoutGeneralRegisters;
    const int smem = hist_smem + general_smem(c, K, block, regs);
    int occ = 0;
    if (general_max_active_blocks(K, clock_variant | (regs ? 4 : 0), block, smem, &occ) != 0 || occ < 1)
      return fail(c, SSA_ECUDA, "occupancy query failed for the general bit-sliced kernel (shared memory " +
                                    std::to_string(smem) + " bytes per block)");
    const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
    const long long groups = (c->ens[0].n_runs + 31) / 32;
    const int grid = (int)std::max(1ll, std::min((groups + block - 1) / block, (long long)c->sm_count * bpsm));
    fl.ens = c->ens[0];
    fl.ens_table = nullptr;
    fl.item_begin = 0;
    fl.item_end = groups;
    fl.queue = c->d_counters + kCounters;
    if ((e = (cudaError_t)general_launcher(K)(fl, grid, block, smem, (void*)c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "general bit-sliced kernel launch");
    return SSA_OK;
  }
  // a batch: one launch per K bucket on the side streams, recorded as one graph like Frank's
  fl.ens_table = c->d_ens;
  fl.item_ens = c->d_item_ens;
  fl.item_group = c->d_item_group;
  std::vector<BatchLaunch> plan(c->ranges.size());
  std::memset(plan.data(), 0, sizeof(BatchLaunch) * plan.size());
  for (size_t r = 0; r < c->ranges.size(); ++r) {
    BatchLaunch& b = plan[r];
    b.K = std::max(1, c->ranges[r].first);
    b.general = 1;
    b.block = block;
    const bool regs = general_in_registers(c, b.K);
    if (regs) c->layout_used |= kLayoutGeneralRegisters;
    b.smem = general_smem(c, b.K, block, regs);
    b.stream = (int)(r % c->side.size());
    b.fl = fl;
    b.fl.net.regs = regs ? 1 : 0;
    b.fl.item_begin = c->ranges[r].second.first;
    b.fl.item_end = c->ranges[r].second.second;
    b.fl.queue = c->d_counters + kCounters + 1 + r;
    int occ = 0;
    if (general_max_active_blocks(b.K, clock_variant | 1 | (regs ? 4 : 0), block, b.smem, &occ) != 0 || occ < 1)
      return fail(c, SSA_ECUDA, "occupancy query failed for the general bit-sliced kernel (shared memory " +
                                    std::to_string(b.smem) + " bytes per block)");
    const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
    const long long groups = b.fl.item_end - b.fl.item_begin;
    b.grid = (int)std::max(1ll, std::min((groups + block - 1) / block, (long long)c->sm_count * bpsm));
  }
  return run_plan(c, plan);
}

int launch_runs(ssa_ctx* c) {
  NvtxRange range(c->batch ? "bitssa batch launch" : "bitssa launch");
  const int n_snap = c->n_snap;
  cudaError_t e;
  FrankLaunch fl;
  std::memset(&fl, 0, sizeof fl);
  fl.thr = c->d_thr;
  fl.init_counts = c->d_init;
  fl.n_snap = n_snap;
  fl.precision = c->opt.precision;
  fl.step_budget = c->opt.step_budget;
  for (int i = 0; i < 3; ++i) fl.perm[i] = c->perm[i];
  fl.n_species = c->S;
  fl.final_counts = c->d_final;
  fl.t_abs = c->d_tabs;
  fl.outcome = c->d_outcome;
  fl.hist = c->d_hist;
  fl.ens_absorbed = c->d_ens_abs;
  fl.snap_counts = c->opt.keep_snap_counts ? c->d_snap : nullptr;
  fl.stage_offset = -1;
  fl.adapt = c->opt.pad_pow2 == 2 ? 1 : 0;
  // the tail hand-off of the one-thread kernel: a fixed option wins, then the tuner's choice
  fl.tail_groups = c->opt.tail_groups < 0 ? 0 : (c->opt.tail_groups > 0 ? c->opt.tail_groups
                                                 : (c->tuned_tail >= 0 ? c->tuned_tail : kDefaultTailGroups));
  // per-run clocks: the records follow the histogram and the staging rows (no tail hand-off)
  fl.lane_clock = c->opt.clock == SSA_CLOCK_LANE ? 1 : 0;
  if (fl.lane_clock) fl.tail_groups = 0;
  fl.n_runs_total = c->n_runs_total;
  fl.counters = c->d_counters;
  fl.status = c->d_status;
  const int block = c->opt.block_size ? c->opt.block_size : (c->tuned_block ? c->tuned_block : 64);

  c->layout_used = 0;
  if (c->opt.engine == SSA_ENGINE_THREAD_PER_RUN) {
    if (c->batch) return fail(c, SSA_EUNSUPPORTED, "the thread-per-run engine runs single-ensemble contexts");
    ThreadLaunch tl;
    std::memset(&tl, 0, sizeof tl);
    tl.ens = c->ens[0];
    tl.thr = c->d_thr;
    tl.init_counts = c->d_init;
    tl.n_snap = n_snap;
    tl.precision = c->opt.precision;
    tl.step_budget = c->opt.step_budget;
    for (int r = 0; r < 3; ++r) tl.rates[r] = c->rates[r];
    tl.unit_rates = c->rates[0] == c->rates[1] && c->rates[1] == c->rates[2];
    for (int i = 0; i < 3; ++i) tl.perm[i] = c->perm[i];
    tl.n_species = c->S;
    tl.final_counts = c->d_final;
    tl.t_abs = c->d_tabs;
    tl.outcome = c->d_outcome;
    tl.hist = c->d_hist;
    tl.ens_absorbed = c->d_ens_abs;
    tl.snap_counts = fl.snap_counts;
    tl.n_runs_total = c->n_runs_total;
    tl.counters = c->d_counters;
    tl.status = c->d_status;
    const int tblock = c->opt.block_size ? c->opt.block_size : 256;
    const int smem = n_snap * kHistBins * (int)sizeof(unsigned int);
    int occ = 0;
    if ((e = (cudaError_t)thread_per_run_max_active_blocks(tblock, smem, &occ)) != cudaSuccess || occ < 1)
      return fail(c, SSA_ECUDA, "occupancy query failed for the thread-per-run kernel");
    const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
    const long long need = (c->n_runs_total + tblock - 1) / tblock;
    const int grid = (int)std::max(1ll, std::min(need, (long long)c->sm_count * bpsm));
    if ((e = (cudaError_t)thread_per_run_launch(tl, grid, tblock, smem, (void*)c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "thread-per-run launch");
    return SSA_OK;
  }

  const int clock_variant = c->opt.precision == SSA_P64 ? 2 : 0;
  const int adapt_variant = fl.adapt ? 4 : 0;  // the one-thread Frank kernel's instantiation
  if (c->general) return launch_general(c, fl, block, clock_variant);
  if (!c->batch) {
    const Ensemble& en = c->ens[0];
    const long long groups = (en.n_runs + 31) / 32;
    const int K = std::max(1, en.K);
    fl.ens = en;
    fl.ens_table = nullptr;
    fl.item_begin = 0;
    fl.item_end = groups;
    fl.queue = c->d_counters + kCounters;
    const int smem = n_snap * kHistBins * (int)sizeof(unsigned int);
    int occ = 0;
    const bool warps = ctx_warps(c, groups);
    c->layout_used = warps ? SSA_LAYOUT_WARPS : SSA_LAYOUT_THREAD;
    if (warps) {
      if (frank_trio_max_active_blocks(K, clock_variant, smem, &occ) != 0 || occ < 1)
        return fail(c, SSA_ECUDA, "occupancy query failed for the three-warp bit-sliced kernel");
      const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
      const long long need = (groups + 31) / 32;
      const int grid = (int)std::max(1ll, std::min(need, (long long)c->sm_count * bpsm));
      if ((e = (cudaError_t)frank_trio_launcher(K)(fl, grid, smem, (void*)c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "three-warp bit-sliced kernel launch");
      return SSA_OK;
    }
    // with the dump on, each thread stages a group's rows after the histogram (16-byte aligned)
    int tsmem = smem;
    if (fl.snap_counts) {
      fl.stage_offset = ((smem / (int)sizeof(unsigned int)) + 3) & ~3;
      tsmem = (fl.stage_offset + block * kStageStride) * (int)sizeof(unsigned int);
    }
    int lane_variant = 0;
    if (fl.lane_clock) {  // 32 records of 16 bytes and 32 bytes of next time points per thread
      fl.lane_offset = ((tsmem / (int)sizeof(unsigned int)) + 3) & ~3;
      tsmem = (fl.lane_offset + block * 32 * 4 + block * 32 / 4) * (int)sizeof(unsigned int);
      lane_variant = 8;
    }
    if (frank_max_active_blocks(K, clock_variant | adapt_variant | lane_variant, block, tsmem, &occ) != 0 || occ < 1)
      return fail(c, SSA_ECUDA, "occupancy query failed for the bit-sliced kernel");
    const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
    const long long need = (groups + block - 1) / block;
    const int grid = (int)std::max(1ll, std::min(need, (long long)c->sm_count * bpsm));
    if ((e = (cudaError_t)frank_launcher(K)(fl, grid, block, tsmem, (void*)c->stream)) != cudaSuccess)
      return cuda_fail(c, e, "bit-sliced kernel launch");
    return SSA_OK;
  }

  fl.ens_table = c->d_ens;
  fl.item_ens = c->d_item_ens;
  fl.item_group = c->d_item_group;
  // one launch per K bucket (largest K first), spread over the side streams so that the
  // buckets run concurrently; the caller's stream waits for all of them.  The plan is fixed
  // first; on a capturable stream it is recorded once as a CUDA graph and replayed while it
  // stays the same, so a batch of any size is one graph launch.
  std::vector<BatchLaunch> plan(c->ranges.size());
  std::memset(plan.data(), 0, sizeof(BatchLaunch) * plan.size());
  for (size_t r = 0; r < c->ranges.size(); ++r) {
    BatchLaunch& b = plan[r];
    b.K = std::max(1, c->ranges[r].first);
    b.fl = fl;
    b.fl.item_begin = c->ranges[r].second.first;
    b.fl.item_end = c->ranges[r].second.second;
    b.fl.queue = c->d_counters + kCounters + 1 + r;
    b.stream = (int)(r % c->side.size());
    const long long groups = b.fl.item_end - b.fl.item_begin;
    b.warps = ctx_warps(c, groups) ? 1 : 0;
    c->layout_used |= b.warps ? SSA_LAYOUT_WARPS : SSA_LAYOUT_THREAD;
    int occ = 0;
    if (b.warps) {
      if (frank_trio_max_active_blocks(b.K, clock_variant | 1, 0, &occ) != 0 || occ < 1)
        return fail(c, SSA_ECUDA, "occupancy query failed for the three-warp bit-sliced kernel");
      b.block = kTrioBlock;
      const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
      b.grid = (int)std::max(1ll, std::min((groups + 31) / 32, (long long)c->sm_count * bpsm));
    } else {
      if (frank_max_active_blocks(b.K, clock_variant | adapt_variant | 1, block, 0, &occ) != 0 || occ < 1)
        return fail(c, SSA_ECUDA, "occupancy query failed for the bit-sliced kernel");
      b.block = block;
      const int bpsm = c->opt.blocks_per_sm ? std::min(c->opt.blocks_per_sm, occ) : occ;
      b.grid = (int)std::max(1ll, std::min((groups + block - 1) / block, (long long)c->sm_count * bpsm));
    }
  }
  return run_plan(c, plan);
}

size_t field_bytes(const ssa_ctx* c, int field) {
  const size_t nr = (size_t)c->n_runs_total, S = (size_t)c->S;
  switch (field) {
    case SSA_FIELD_FINAL_COUNTS: return nr * S * sizeof(int32_t);
    case SSA_FIELD_ABSORB_TIME: return nr * sizeof(double);
    case SSA_FIELD_ABSORB_OUTCOME: return nr;
    case SSA_FIELD_EE_HIST: return (size_t)c->n_ens * (size_t)c->n_snap * kHistBins * sizeof(uint64_t);
    case SSA_FIELD_SNAP_COUNTS: return c->opt.keep_snap_counts ? (size_t)c->n_snap * nr * S * sizeof(int32_t) : 0;
    case SSA_FIELD_COUNTERS: return kCounters * sizeof(uint64_t);
    case SSA_FIELD_ENS_ABSORBED: return (size_t)c->n_ens * 4 * sizeof(uint64_t);
    default: return 0;
  }
}

}  // namespace

namespace bitssa {
void set_thread_error(const std::string& msg) { t_err = msg; }
void current_allocator(ssa_alloc_fn* alloc, ssa_free_fn* release, void** user) {
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  *alloc = g_alloc.alloc;
  *release = g_alloc.release;
  *user = g_alloc.user;
}
}  // namespace bitssa

extern "C" {

void ssa_default_options(ssa_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof *opt);
  opt->precision = SSA_P64;
  opt->engine = SSA_ENGINE_BITSLICED;
  opt->thin_bits = 32;
  opt->device = -1;
}

int ssa_version(void) { return 200; }  // 0.2.0: general networks, padded bound, general modes

int ssa_create(const int32_t* reactants, const int32_t* products, int32_t n_species, int32_t n_reactions,
               const double* rates, const int64_t* N0, int32_t n0_per_run, int64_t n_runs, uint64_t seed,
               const ssa_options* opt, ssa_ctx** out) {
  ssa_ctx* c = nullptr;
  int perm[3];
  int st = create_common(reactants, products, n_species, n_reactions, opt, out, &c, perm);
  if (st != SSA_OK) return st;
  std::string why;
  auto bail = [&](int code, std::string msg) {  // by value: msg may live in *c
    delete c;
    return fail(nullptr, code, msg);
  };
  if (!rates) return bail(SSA_EINVAL, "rates is NULL");
  if ((st = check_rates(rates, &why, c->R)) != SSA_OK) return bail(st, why);
  if (!N0) return bail(SSA_EINVAL, "N0 is NULL");
  if (n_runs < 0) return bail(SSA_EINVAL, "n_runs must be >= 0");
  if (n0_per_run != 0 && n0_per_run != 1) return bail(SSA_EINVAL, "n0_per_run must be 0 or 1");
  if (c->opt.first_run + n_runs > (1ll << 37)) return bail(SSA_EINVAL, "run index beyond 2^37");
  if (c->general) {
    // counts in the caller's species order, one total for every run
    const int S = c->S;
    long long n_tot = -1;
    std::vector<int> rows;
    const long long nrows = n0_per_run ? n_runs : 1;
    if (n0_per_run) rows.resize((size_t)n_runs * S);
    int shared[kMaxSpecies] = {0};
    for (long long j = 0; j < nrows; ++j) {
      long long tot = 0;
      for (int i = 0; i < S; ++i) {
        const long long v = N0[j * S + i];
        if (v < 0) return bail(SSA_EINVAL, "initial counts must be >= 0");
        if (v > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
        tot += v;
        if (n0_per_run) rows[(size_t)j * S + i] = (int)v;
        else shared[i] = (int)v;
      }
      if (n_tot < 0) n_tot = tot;
      if (tot != n_tot) return bail(SSA_EINVAL, "every run must have the same total count");
    }
    if (nrows == 0) n_tot = 1;
    if (n_tot < 1) return bail(SSA_EINVAL, "the total count must be >= 1");
    if (n_tot > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
    c->rates.assign(rates, rates + c->R);
    c->n_ens = 1;
    c->n_runs_total = n_runs;
    unsigned long long lam = 0;
    c->ens.push_back(make_general_ensemble(c->net, n_tot, shared, rates, c->opt.thin_bits, seed, n_runs, 0,
                                           c->opt.first_run / 32, c->opt.pad_pow2, &lam));
    if (lam >= (1ull << 31))
      return bail(SSA_EUNSUPPORTED, "the uniformisation bound m_pair C(N,2) + u_max N must stay below 2^31");
    c->ens.back().shared_n = c->opt.shared_n;
    c->net.B = bits_of((unsigned long long)n_tot);
    DeviceGuard guard(c->opt.device);
    if ((st = setup_device(c)) != SSA_OK) return bail(st, c->err);
    if ((st = allocate_common(c, rows)) != SSA_OK) {
      std::string msg = c->err;
      dev_free_all(c);
      return bail(st, msg);
    }
    *out = c;
    return SSA_OK;
  }
  // total count, identical for every run (Sec. 4)
  long long n_tot = -1;
  std::vector<int> rows;
  const long long nrows = n0_per_run ? n_runs : 1;
  if (n0_per_run) rows.resize((size_t)n_runs * 3);
  int shared[3] = {0, 0, 0};
  for (long long j = 0; j < nrows; ++j) {
    long long tot = 0;
    int canon[3];
    for (int ci = 0; ci < 3; ++ci) {
      const long long v = N0[j * 3 + perm[ci]];
      if (v < 0) return bail(SSA_EINVAL, "initial counts must be >= 0");
      if (v > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
      canon[ci] = (int)v;
      tot += v;
    }
    if (n_tot < 0) n_tot = tot;
    if (tot != n_tot) return bail(SSA_EINVAL, "every run must have the same total count");
    if (n0_per_run) std::memcpy(&rows[(size_t)j * 3], canon, sizeof canon);
    else std::memcpy(shared, canon, sizeof canon);
  }
  if (nrows == 0) n_tot = 1;
  if (n_tot < 1) return bail(SSA_EINVAL, "the total count must be >= 1");
  if (n_tot > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536 (lambda_int must stay below 2^31)");
  const double canon_rates[3] = {rates[0], rates[1], rates[2]};
  c->rates.assign(canon_rates, canon_rates + 3);
  c->n_ens = 1;
  c->n_runs_total = n_runs;
  c->ens.push_back(make_ensemble(n_tot, shared, canon_rates, c->opt.thin_bits, seed, n_runs, 0,
                                 c->opt.first_run / 32, c->opt.pad_pow2));
  c->ens.back().shared_n = c->opt.shared_n;
  DeviceGuard guard(c->opt.device);
  if ((st = setup_device(c)) != SSA_OK) return bail(st, c->err);
  if ((st = allocate_common(c, rows)) != SSA_OK) {
    std::string msg = c->err;
    dev_free_all(c);
    return bail(st, msg);
  }
  *out = c;
  return SSA_OK;
}

int ssa_create_batch(const int32_t* reactants, const int32_t* products, int32_t n_species, int32_t n_reactions,
                     int32_t n_ens, const int64_t* N0_ens, const double* rates_ens, const int64_t* runs_ens,
                     const uint64_t* seed_ens, const ssa_options* opt, ssa_ctx** out) {
  ssa_ctx* c = nullptr;
  int perm[3];
  int st = create_common(reactants, products, n_species, n_reactions, opt, out, &c, perm);
  if (st != SSA_OK) return st;
  std::string why;
  auto bail = [&](int code, std::string msg) {  // by value: msg may live in *c
    delete c;
    return fail(nullptr, code, msg);
  };
  if (n_ens < 1) return bail(SSA_EINVAL, "n_ens must be >= 1");
  if (!N0_ens || !rates_ens || !runs_ens || !seed_ens) return bail(SSA_EINVAL, "null batch array");
  if (c->opt.first_run != 0) return bail(SSA_EINVAL, "first_run must be 0 for a batch");
  if (c->opt.engine == SSA_ENGINE_THREAD_PER_RUN) return bail(SSA_EUNSUPPORTED, "batches run on the bit-sliced engines");
  if (c->opt.clock == SSA_CLOCK_LANE) return bail(SSA_EUNSUPPORTED, "the per-run clock runs single ensembles");
  c->batch = true;
  c->n_ens = n_ens;
  long long offset = 0;
  std::vector<std::pair<int, int>> order;  // (K, e)
  for (int e = 0; e < n_ens; ++e) {
    if ((st = check_rates(rates_ens + (size_t)c->R * e, &why, c->R)) != SSA_OK) return bail(st, why);
    if (runs_ens[e] < 0) return bail(SSA_EINVAL, "runs_ens must be >= 0");
    if (c->general) {
      const int S = c->S;
      int init[kMaxSpecies] = {0};
      long long tot = 0;
      for (int i = 0; i < S; ++i) {
        const long long v = N0_ens[(size_t)e * S + i];
        if (v < 0) return bail(SSA_EINVAL, "initial counts must be >= 0");
        if (v > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
        init[i] = (int)v;
        tot += v;
      }
      if (tot < 1) return bail(SSA_EINVAL, "the total count must be >= 1");
      if (tot > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
      const double* k = rates_ens + (size_t)c->R * e;
      unsigned long long lam = 0;
      c->ens.push_back(make_general_ensemble(c->net, tot, init, k, c->opt.thin_bits, seed_ens[e], runs_ens[e],
                                             offset, 0, c->opt.pad_pow2, &lam));
      if (lam >= (1ull << 31))
        return bail(SSA_EUNSUPPORTED, "the uniformisation bound m_pair C(N,2) + u_max N must stay below 2^31");
      c->ens.back().shared_n = c->opt.shared_n;
      c->rates.insert(c->rates.end(), k, k + c->R);
      c->net.B = std::max(c->net.B, bits_of((unsigned long long)tot));
      offset += runs_ens[e];
      order.push_back({std::max(1, c->ens.back().K), e});
      continue;
    }
    int canon[3];
    long long tot = 0;
    for (int ci = 0; ci < 3; ++ci) {
      const long long v = N0_ens[e * 3 + perm[ci]];
      if (v < 0) return bail(SSA_EINVAL, "initial counts must be >= 0");
      if (v > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
      canon[ci] = (int)v;
      tot += v;
    }
    if (tot < 1) return bail(SSA_EINVAL, "the total count must be >= 1");
    if (tot > 65536) return bail(SSA_EUNSUPPORTED, "N_tot above 65536");
    const double* k = rates_ens + 3 * e;
    c->ens.push_back(
        make_ensemble(tot, canon, k, c->opt.thin_bits, seed_ens[e], runs_ens[e], offset, 0, c->opt.pad_pow2));
    c->ens.back().shared_n = c->opt.shared_n;
    c->rates.insert(c->rates.end(), k, k + 3);
    offset += runs_ens[e];
    order.push_back({std::max(1, c->ens.back().K), e});
  }
  c->n_runs_total = offset;
  // work items sorted by K, largest first (the longest runs start first)
  std::stable_sort(order.begin(), order.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
    return a.first > b.first;
  });
  for (size_t i = 0; i < order.size();) {
    const int K = order[i].first;
    const long long begin = (long long)c->item_ens.size();
    for (; i < order.size() && order[i].first == K; ++i) {
      const int e = order[i].second;
      const long long groups = (c->ens[e].n_runs + 31) / 32;
      for (long long g = 0; g < groups; ++g) {
        c->item_ens.push_back(e);
        c->item_group.push_back((int)g);
      }
    }
    const long long end = (long long)c->item_ens.size();
    if (end > begin) c->ranges.push_back({K, {begin, end}});
  }
  DeviceGuard guard(c->opt.device);
  if ((st = setup_device(c)) != SSA_OK) return bail(st, c->err);
  {
    const size_t n_side = std::min<size_t>(8, std::max<size_t>(1, c->ranges.size()));
    cudaError_t e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    for (size_t i = 0; e == cudaSuccess && i < n_side; ++i) {
      cudaStream_t s = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
      if (e == cudaSuccess) c->side.push_back(s);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) c->side_done.push_back(ev);
    }
    if (e != cudaSuccess) {
      std::string msg = std::string("side streams: ") + cudaGetErrorString(e);
      for (auto s : c->side) cudaStreamDestroy(s);
      for (auto ev : c->side_done) cudaEventDestroy(ev);
      if (c->fork) cudaEventDestroy(c->fork);
      return bail(SSA_ECUDA, msg);
    }
  }
  if ((st = allocate_common(c, {})) != SSA_OK) {
    std::string msg = c->err;
    dev_free_all(c);
    for (auto s : c->side) cudaStreamDestroy(s);
    for (auto ev : c->side_done) cudaEventDestroy(ev);
    if (c->fork) cudaEventDestroy(c->fork);
    return bail(st, msg);
  }
  *out = c;
  return SSA_OK;
}

int ssa_run(ssa_ctx* c, double t_end, const double* snapshot_times, int32_t n_snap) {
  NvtxRange range("ssa_run");
  if (!c) return fail(nullptr, SSA_EINVAL, "ctx is NULL");
  if (!(t_end >= 0.0)) return fail(c, SSA_EINVAL, "t_end must be >= 0");
  if (n_snap < 0 || n_snap > kMaxSnap) return fail(c, SSA_EINVAL, "n_snap must be in [0, 64]");
  if (n_snap > 0 && !snapshot_times) return fail(c, SSA_EINVAL, "snapshot_times is NULL");
  for (int s = 0; s < n_snap; ++s) {
    if (!(snapshot_times[s] >= 0.0) || snapshot_times[s] > t_end)
      return fail(c, SSA_EINVAL, "snapshot times must lie in [0, t_end]");
    if (s > 0 && snapshot_times[s] < snapshot_times[s - 1])
      return fail(c, SSA_EINVAL, "snapshot times must be ascending");
  }
  DeviceGuard guard(c->device);
  cudaError_t e;
  c->ran = false;
  c->n_snap = n_snap;
  // thresholds [n_ens][n_snap + 1], the last one t_end
  std::vector<Threshold> thr((size_t)c->n_ens * (n_snap + 1));
  for (int ei = 0; ei < c->n_ens; ++ei) {
    for (int s = 0; s < n_snap; ++s) thr[(size_t)ei * (n_snap + 1) + s] = make_threshold(snapshot_times[s], c->ens[ei].lambda);
    thr[(size_t)ei * (n_snap + 1) + n_snap] = make_threshold(t_end, c->ens[ei].lambda);
  }
  int st;
  if ((st = grow(c, (void**)&c->d_thr, &c->thr_cap, sizeof(Threshold) * thr.size())) != SSA_OK) return st;
  const size_t hist_bytes = std::max<size_t>(8, (size_t)c->n_ens * n_snap * kHistBins * sizeof(unsigned long long));
  if ((st = grow(c, (void**)&c->d_hist, &c->hist_cap, hist_bytes)) != SSA_OK) return st;
  if (c->opt.keep_snap_counts) {
    const size_t snap_bytes = std::max<size_t>(16, (size_t)n_snap * (size_t)c->n_runs_total * c->S * sizeof(int));
    if ((st = grow(c, (void**)&c->d_snap, &c->snap_cap, snap_bytes)) != SSA_OK) return st;
  }
  if ((e = cudaMemcpyAsync(c->d_thr, thr.data(), sizeof(Threshold) * thr.size(), cudaMemcpyHostToDevice,
                           c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "upload thresholds");
  cudaMemsetAsync(c->d_hist, 0, hist_bytes, c->stream);
  cudaMemsetAsync(c->d_ens_abs, 0, sizeof(unsigned long long) * 4 * c->n_ens, c->stream);
  cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * (kCounters + c->n_queues), c->stream);
  cudaMemsetAsync(c->d_status, 0, sizeof(unsigned int) * 4, c->stream);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "clear outputs");
  if (c->n_runs_total > 0 && (st = launch_runs(c)) != SSA_OK) return st;
  unsigned int status = 0;
  if ((e = cudaMemcpyAsync(c->counters, c->d_counters, sizeof(unsigned long long) * kCounters,
                           cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "read counters");
  if ((e = cudaMemcpyAsync(&status, c->d_status, sizeof status, cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess)
    return cuda_fail(c, e, "read status");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "simulation");
  c->counters[kErrorFlags] = status;
  c->counters[kLayoutUsed] = c->layout_used | (c->counters[kLayoutUsed] & kLayoutTail);
  c->ran = true;
  if (status & kErrRedraw) return fail(c, SSA_EOVERFLOW, "64 redraws of n in a row");
  if (status & kErrRange) return fail(c, SSA_EOVERFLOW, "internal range check failed");
  if (status & kErrTimeout) return fail(c, SSA_ETIMEOUT, "a group reached the step budget");
  return SSA_OK;
}

int ssa_tune(ssa_ctx* c, double t_end, const double* snapshot_times, int32_t n_snap, int64_t probe_steps,
             int32_t* choice) {
  NvtxRange range("ssa_tune");
  if (!c) return fail(nullptr, SSA_EINVAL, "ctx is NULL");
  if (probe_steps < 0) return fail(c, SSA_EINVAL, "probe_steps must be >= 0");
  if (c->opt.engine == SSA_ENGINE_THREAD_PER_RUN)
    return fail(c, SSA_EUNSUPPORTED, "the tuner chooses bit-sliced layouts");
  struct Candidate {
    int layout, block, products;
  };
  // Frank's model: the rule (per K bucket in a batch), one thread per group at three block
  // sizes, three warps.  A general network: one thread per group at three block sizes, with the
  // propensities incremented or recomputed by products (unless the options fix the mode).
  const Candidate frank_cands[] = {{SSA_LAYOUT_AUTO, 64, 0}, {SSA_LAYOUT_THREAD, 32, 0}, {SSA_LAYOUT_THREAD, 64, 0},
                                   {SSA_LAYOUT_THREAD, 128, 0}, {SSA_LAYOUT_WARPS, 64, 0}};
  const Candidate general_cands[] = {{SSA_LAYOUT_THREAD, 32, 0}, {SSA_LAYOUT_THREAD, 64, 0},
                                     {SSA_LAYOUT_THREAD, 128, 0}, {SSA_LAYOUT_THREAD, 32, 1},
                                     {SSA_LAYOUT_THREAD, 64, 1}, {SSA_LAYOUT_THREAD, 128, 1}};
  std::vector<Candidate> cands;
  if (!c->general) {
    for (const Candidate& f : frank_cands)
      if ((c->opt.pad_pow2 != 2 && c->opt.clock != SSA_CLOCK_LANE) || f.layout == SSA_LAYOUT_THREAD)
        cands.push_back(f);
  } else
    for (const Candidate& g : general_cands)
      if (c->opt.recompute == 0 || g.products == (c->opt.recompute == 1 ? 1 : 0)) cands.push_back(g);
  DeviceGuard guard(c->device);
  const long long budget = c->opt.step_budget;
  const int old_layout = c->tuned_layout, old_block = c->tuned_block, old_products = c->tuned_products;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e;
  if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess) {
    if (ev[0]) cudaEventDestroy(ev[0]);
    return cuda_fail(c, e, "tuner events");
  }
  int st = SSA_OK;
  float best = -1.0f;
  Candidate win = cands[0];
  c->opt.step_budget = probe_steps;
  for (const Candidate& cand : cands) {
    c->tuned_layout = cand.layout;
    c->tuned_block = cand.block;
    c->tuned_products = cand.products;
    float ms = -1.0f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run also loads the kernel and records graphs
      cudaEventRecord(ev[0], c->stream);
      st = ssa_run(c, t_end, snapshot_times, n_snap);
      cudaEventRecord(ev[1], c->stream);
      if (st != SSA_OK && st != SSA_ETIMEOUT) break;
      st = SSA_OK;
      float t = 0.0f;
      if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess || (e = cudaEventElapsedTime(&t, ev[0], ev[1])) != cudaSuccess) {
        st = cuda_fail(c, e, "tuner timing");
        break;
      }
      if (ms < 0.0f || t < ms) ms = t;
    }
    if (st != SSA_OK) break;
    if (best < 0.0f || ms < best) {
      best = ms;
      win = cand;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  c->opt.step_budget = budget;
  c->ran = false;  // the probes' outputs are not a run of the caller's
  if (st != SSA_OK) {
    c->tuned_layout = old_layout;
    c->tuned_block = old_block;
    c->tuned_products = old_products;
    return st;
  }
  c->tuned_layout = win.layout;
  c->tuned_block = win.block;
  c->tuned_products = c->general ? win.products : -1;
  // Frank's model on one thread per group: the tail hand-off threshold, on the chosen layout
  if (!c->general && c->opt.tail_groups == 0 && c->opt.clock != SSA_CLOCK_LANE &&
      !ctx_warps(c, c->n_runs_total / 32)) {
    const int old_tail = c->tuned_tail;
    int best_tail = kDefaultTailGroups;
    float best_ms = -1.0f;
    c->opt.step_budget = probe_steps;
    const int tails[] = {0, 1, 2, kTailSlots};  // 0: off
    ev[0] = ev[1] = nullptr;
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess)
      st = cuda_fail(c, e, "tuner events");
    for (int ti = 0; st == SSA_OK && ti < 4; ++ti) {
      c->tuned_tail = tails[ti];
      float ms = -1.0f;
      for (int rep = 0; rep < 2 && st == SSA_OK; ++rep) {
        cudaEventRecord(ev[0], c->stream);
        st = ssa_run(c, t_end, snapshot_times, n_snap);
        cudaEventRecord(ev[1], c->stream);
        if (st == SSA_ETIMEOUT) st = SSA_OK;
        float t = 0.0f;
        if (st == SSA_OK && ((e = cudaEventSynchronize(ev[1])) != cudaSuccess ||
                             (e = cudaEventElapsedTime(&t, ev[0], ev[1])) != cudaSuccess))
          st = cuda_fail(c, e, "tuner timing");
        if (ms < 0.0f || t < ms) ms = t;
      }
      if (st == SSA_OK && (best_ms < 0.0f || ms < best_ms)) {
        best_ms = ms;
        best_tail = tails[ti];
      }
    }
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    c->opt.step_budget = budget;
    c->ran = false;
    c->tuned_tail = st == SSA_OK ? best_tail : old_tail;
    if (st != SSA_OK) return st;
  }
  if (choice) {
    choice[0] = win.layout;
    choice[1] = win.block;
  }
  return SSA_OK;
}

int ssa_field_bytes(const ssa_ctx* c, int32_t field, size_t* bytes) {
  if (!c || !bytes) return fail(const_cast<ssa_ctx*>(c), SSA_EINVAL, "null argument");
  *bytes = field_bytes(c, field);
  return SSA_OK;
}

int ssa_fetch(ssa_ctx* c, int32_t field, void* dst, size_t dst_bytes, int32_t dst_on_device) {
  if (!c) return fail(nullptr, SSA_EINVAL, "ctx is NULL");
  if (!c->ran) return fail(c, SSA_ESTATE, "ssa_fetch before a successful ssa_run");
  if (field < 0 || field > SSA_FIELD_ENS_ABSORBED) return fail(c, SSA_EINVAL, "unknown field");
  const size_t bytes = field_bytes(c, field);
  if (field == SSA_FIELD_SNAP_COUNTS && !c->opt.keep_snap_counts)
    return fail(c, SSA_ESTATE, "snapshot counts were not kept (keep_snap_counts = 0)");
  if (dst_bytes < bytes) return fail(c, SSA_EINVAL, "destination too small");
  if (bytes == 0) return SSA_OK;
  if (!dst) return fail(c, SSA_EINVAL, "dst is NULL");
  DeviceGuard guard(c->device);
  const void* src = nullptr;
  switch (field) {
    case SSA_FIELD_FINAL_COUNTS: src = c->d_final; break;
    case SSA_FIELD_ABSORB_TIME: src = c->d_tabs; break;
    case SSA_FIELD_ABSORB_OUTCOME: src = c->d_outcome; break;
    case SSA_FIELD_EE_HIST: src = c->d_hist; break;
    case SSA_FIELD_SNAP_COUNTS: src = c->d_snap; break;
    case SSA_FIELD_ENS_ABSORBED: src = c->d_ens_abs; break;
    case SSA_FIELD_COUNTERS:
      if (!dst_on_device) {
        std::memcpy(dst, c->counters, bytes);
        return SSA_OK;
      }
      src = nullptr;
      break;
  }
  cudaError_t e;
  if (field == SSA_FIELD_COUNTERS)
    e = cudaMemcpyAsync(dst, c->counters, bytes, cudaMemcpyHostToDevice, c->stream);
  else
    e = cudaMemcpyAsync(dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fetch copy");
  if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "fetch synchronize");
  return SSA_OK;
}

int ssa_destroy(ssa_ctx* c) {
  if (!c) return SSA_OK;
  {
    DeviceGuard guard(c->device);
    if (c->stream || !c->bufs.empty()) cudaStreamSynchronize(c->stream);
    if (c->batch_graph) cudaGraphExecDestroy(c->batch_graph);
    for (auto s : c->side) cudaStreamDestroy(s);
    for (auto ev : c->side_done) cudaEventDestroy(ev);
    if (c->fork) cudaEventDestroy(c->fork);
    dev_free_all(c);
  }
  delete c;
  return SSA_OK;
}

const char* ssa_last_error(const ssa_ctx* c) { return c ? c->err.c_str() : t_err.c_str(); }

int ssa_set_allocator(ssa_alloc_fn alloc, ssa_free_fn release, void* user) {
  if ((alloc == nullptr) != (release == nullptr)) return fail(nullptr, SSA_EINVAL, "alloc and release go together");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc.alloc = alloc;
  g_alloc.release = release;
  g_alloc.user = user;
  return SSA_OK;
}

}  // extern "C"
