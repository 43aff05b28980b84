// api.cu -- host side of the C ABI declared in include/snn.h.
//
// Host work is limited to what the paper does on the host before launching its
// construction kernels: validating the rule and synapse dictionaries, computing the
// integer CDF tables and the FP64 propagators, planning the batched generation work
// list (every projection x every logical rank), and reading results back.  Every
// per-synapse and per-neuron step runs in the CUDA kernels of build.cu / maps.cu /
// sim.cu.  There is no CPU fallback: without a usable GPU every call that needs one
// returns SNN_ECUDA.
#include <algorithm>
#include <cfenv>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/snn.h"
#include "maps_internal.cuh"
#include "sim_internal.cuh"
#include "snn_internal.cuh"

using namespace snn;

namespace {

struct PopSpec {
  uint32_t first, n;
  snn_iaf_psc_exp_params p;
};
struct ProjSpec {
  uint32_t src_first, n_src, src_stride, tgt_first, n_tgt, tgt_stride;
  snn_rule rule;
  snn_dist w, d;
  uint64_t seed;
  // derived at calibrate
  uint32_t d_smin = 0;
  std::vector<uint32_t> d_thr;
  std::vector<uint32_t> g_thr;   // gap table (pairwise Bernoulli by geometric gaps)
};
struct DriveSpec {
  uint32_t first, n;
  double rate, weight;
  uint64_t seed;
};

// Expected connections per source that a projection creates on a rank holding n_on of
// its targets, compared with the threshold xi of the all-sources images (Methods,
// "Remote connections": K_in N_target / N_source for fixed in-degree, N_target the
// targets on the target process).
double per_source(const ProjSpec& s, uint64_t n_on) {
  if (s.rule.kind == SNN_RULE_ONE_TO_ONE || s.rule.kind == SNN_RULE_ALL_TO_ALL) return 0.0;   // no decision
  if (s.rule.kind == SNN_RULE_FIXED_INDEGREE) return s.rule.param * (double)n_on / s.n_src;
  if (s.rule.kind == SNN_RULE_FIXED_TOTAL) return s.rule.param * (double)n_on / ((double)s.n_tgt * s.n_src);
  return s.rule.param * (double)n_on;                 // pairwise Bernoulli (both variants)
}

uint64_t gcd_u64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// Targets of a projection per rank: the residues of tgt_first + j tgt_stride (mod R)
// repeat with period q = R / gcd(tgt_stride, R), each once per period.
void targets_per_rank(const ProjSpec& s, uint32_t R, std::vector<uint64_t>* n_on) {
  n_on->assign(R, 0);
  const uint64_t q = R / gcd_u64(s.tgt_stride % R, R);
  const uint64_t a = s.n_tgt / q, b = s.n_tgt % q;
  for (uint64_t j = 0; j < std::min<uint64_t>(s.n_tgt, q); ++j)
    (*n_on)[(s.tgt_first + j * s.tgt_stride) % R] += a + (j < b ? 1 : 0);
}

uint32_t bits_for(uint64_t v) {  // bits to hold values 0..v
  uint32_t b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

}  // namespace

struct snn_ctx {
  snn_config cfg{};
  snn_allocator alloc{};
  cudaStream_t st = nullptr;
  int num_sms = 0;
  std::string err;
  std::vector<PopSpec> pops;
  std::vector<ProjSpec> projs;
  std::vector<DriveSpec> drives;
  uint32_t N = 0;
  bool calibrated = false;
  std::map<void*, size_t> live;
  uint64_t cur_bytes = 0, peak_bytes = 0;
  snn_stats_t stats{};

  // construction results
  Geom g{};
  uint64_t E = 0;
  std::vector<uint64_t> seg_start;        // [R+1]
  std::vector<uint32_t> M, rank_off;      // rank sizes / first neuron position
  std::vector<uint64_t> cbase;
  uint64_t* d_seg_start = nullptr;
  uint32_t* d_tgt = nullptr;
  void* d_w = nullptr;
  uint8_t* d_d = nullptr;
  uint64_t* d_dense = nullptr;           // [R][N+1]
  uint32_t* d_dense_off = nullptr;       // [R][R]
  float* d_scale_src = nullptr;          // fp16 per source gid
  float* d_row_scale = nullptr;          // fp16 per row (one rank)
  uint32_t* d_err = nullptr;
  MapsState maps{};
  uint32_t wbytes = 4;

  // simulation
  SimArgs sim{};
  uint32_t ring_slots = 0;
  cudaGraphExec_t graph = nullptr;
  uint32_t graph_steps = 0;
  bool capturing = false;
  // overlapped steps (one rank): neuron work on st, deliveries on st2 / st3, lists modulo 3
  bool overlap = false;
  SimArgs ov{};
  cudaStream_t st2 = nullptr, st3 = nullptr;   // deliveries of even and odd steps
  cudaEvent_t ev_u = nullptr, ev_dk[2] = {nullptr, nullptr};
  std::vector<uint32_t> host_gid_of;      // position -> gid
  std::vector<uint32_t> host_pos_of;      // gid -> position
};

namespace {

int fail(snn_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  if (code == SNN_ECUDA) (void)cudaGetLastError();   // a non-sticky error must not leak into later calls
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e__ = (call);                                                           \
    if (e__ != cudaSuccess)                                                             \
      return fail(c, SNN_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__));   \
  } while (0)

void* dalloc(snn_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->alloc.alloc) {
    p = c->alloc.alloc(c->alloc.user, bytes, (void*)c->st);
    if (p && ((uintptr_t)p & 15u)) {          // vector accesses need 16-byte alignment
      if (c->alloc.free) c->alloc.free(c->alloc.user, p, bytes, (void*)c->st);
      p = nullptr;
    }
  } else if (cudaMallocAsync(&p, bytes, c->st) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    c->live[p] = bytes;
    c->cur_bytes += bytes;
    c->peak_bytes = std::max(c->peak_bytes, c->cur_bytes);
  }
  return p;
}

void dfree(snn_ctx* c, void* p) {
  if (!p) return;
  auto it = c->live.find(p);
  if (it == c->live.end()) return;
  if (c->alloc.free) c->alloc.free(c->alloc.user, p, it->second, (void*)c->st);
  else cudaFreeAsync(p, c->st);
  c->cur_bytes -= it->second;
  c->live.erase(it);
}

template <typename T>
int alloc_into(snn_ctx* c, T** out, size_t count, const char* what) {
  *out = (T*)dalloc(c, count * sizeof(T));
  if (!*out) return fail(c, SNN_ENOMEM, std::string("allocation failed: ") + what);
  return SNN_OK;
}

#define AL(ptr, count, what)                                   \
  do {                                                         \
    int r__ = alloc_into(c, &(ptr), (size_t)(count), what);    \
    if (r__ != SNN_OK) return r__;                             \
  } while (0)

template <typename T>
int upload(snn_ctx* c, T** out, const std::vector<T>& v, const char* what) {
  AL(*out, std::max<size_t>(v.size(), 1), what);
  if (!v.empty()) CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->st));
  c->stats.h2d_bytes += v.size() * sizeof(T);
  return SNN_OK;
}

#define UP(ptr, vec, what)                         \
  do {                                             \
    int r__ = upload(c, &(ptr), vec, what);        \
    if (r__ != SNN_OK) return r__;                 \
  } while (0)

int check_dist_w(const snn_dist* w) {
  if (!w) return SNN_EINVAL;
  if (w->kind == SNN_W_CONST) return std::isfinite(w->mean) ? SNN_OK : SNN_EINVAL;
  if (w->kind == SNN_W_NORMAL_SIGN)
    return (std::isfinite(w->mean) && std::isfinite(w->sd) && w->sd >= 0) ? SNN_OK : SNN_EINVAL;
  return SNN_EINVAL;
}

int check_dist_d(const snn_dist* d) {
  if (!d) return SNN_EINVAL;
  if (d->kind == SNN_D_CONST) return (std::isfinite(d->mean) && d->mean >= 0) ? SNN_OK : SNN_EINVAL;
  if (d->kind == SNN_D_NORMAL_MIN)
    return (std::isfinite(d->mean) && d->sd > 0 && d->lo >= 0) ? SNN_OK : SNN_EINVAL;
  return SNN_EINVAL;
}

// Integer CDF table of the quantised normal delay: P(step <= s) =
// Phi(((s + 1/2) h - mean) / sd) for s >= s_min = max(1, round(lo / h)),
// thr_s = floor(P 2^32 + 1/2), stopping at the first s whose threshold reaches 2^32.
int delay_table(double mean, double sd, double lo, double dt, uint32_t* s_min,
                std::vector<uint32_t>* thr) {
  std::fesetround(FE_TONEAREST);
  thr->clear();
  // delays are stored in u8: the smallest step itself must fit before any threshold is
  // looked at (the clipped mass below lo lands on it)
  if (!(lo / dt < 255.5)) return SNN_EINVAL;
  const int smin = std::max(1, (int)std::nearbyint(lo / dt));
  if (smin > 255) return SNN_EINVAL;
  int s = smin;
  while (true) {
    const double x = ((s + 0.5) * dt - mean) / sd;
    const double phi = 0.5 * std::erfc(-x / std::sqrt(2.0));
    const double cth = std::floor(phi * 4294967296.0 + 0.5);
    if (cth >= 4294967296.0) break;
    thr->push_back((uint32_t)cth);
    ++s;
    if (s > 255) return SNN_EINVAL;
  }
  *s_min = (uint32_t)smin;
  return SNN_OK;
}

uint32_t const_delay_steps(double d, double dt) {
  std::fesetround(FE_TONEAREST);
  // clamped below the u32 range before the conversion; callers reject anything above 255
  return (uint32_t)std::min(65535.0, std::max(1.0, std::nearbyint(d / dt)));
}

// Integer CDF table of Poisson(rate * h / 1000).
std::vector<uint32_t> poisson_table(double rate_hz, double dt) {
  const double lam = rate_hz * dt / 1000.0;
  double pmf = std::exp(-lam), cdf = pmf;
  std::vector<uint32_t> thr;
  int i = 0;
  while (true) {
    const double cth = std::floor(cdf * 4294967296.0 + 0.5);
    if (cth >= 4294967296.0 || i >= 255) break;
    thr.push_back((uint32_t)cth);
    ++i;
    pmf = pmf * lam / i;
    cdf = cdf + pmf;
  }
  return thr;
}

// FP64 exact-integration propagators of iaf_psc_exp, stored fp32.
DevPop propagators(const snn_iaf_psc_exp_params& p, double h) {
  DevPop o{};
  const double P22 = std::exp(-h / p.tau_m);
  o.P22 = (float)P22;
  o.P20 = (float)(-(p.tau_m / p.C_m) * std::expm1(-h / p.tau_m));
  const double ts[2] = {p.tau_syn_ex, p.tau_syn_in};
  double P11[2], P21[2];
  for (int x = 0; x < 2; ++x) {
    P11[x] = std::exp(-h / ts[x]);
    const double delta = 1.0 / ts[x] - 1.0 / p.tau_m;
    const double frac = delta == 0.0 ? h : -std::expm1(-h * delta) / delta;
    P21[x] = (1.0 / p.C_m) * P22 * frac;
  }
  o.P11ex = (float)P11[0];
  o.P11in = (float)P11[1];
  o.P21ex = (float)P21[0];
  o.P21in = (float)P21[1];
  o.Ie = (float)p.I_e;
  o.Vth = (float)p.V_th;
  o.Vreset = (float)p.V_reset;
  std::fesetround(FE_TONEAREST);
  o.ref_steps = (uint32_t)std::nearbyint(p.t_ref / h);
  return o;
}

// Integer CDF table of the gap G >= 0 between kept pairs (pairwise Bernoulli by
// geometric gaps): thr_g = floor(P(G <= g) 2^32 + 1/2), P(G <= g) = 1 - (1 - p)^(g + 1)
// with the power accumulated by repeated fp64 multiplication; the table stops at the
// first threshold reaching 2^32 and holds at most 2^22 entries.
int gap_table(double p, std::vector<uint32_t>* thr) {
  thr->clear();
  const double q = 1.0 - p;
  double qq = q;
  while (true) {
    const double v = std::floor((1.0 - qq) * 4294967296.0 + 0.5);
    if (v >= 4294967296.0) break;
    thr->push_back((uint32_t)v);
    if (thr->size() > (size_t)1 << 22) return SNN_EINVAL;
    qq = qq * q;
  }
  return SNN_OK;
}

// rules generated in the fixed in-degree shape (K records per target, counter i_t K + k)
bool fixed_indegree_shape(const ProjSpec& p) {
  return p.rule.kind == SNN_RULE_FIXED_INDEGREE || p.rule.kind == SNN_RULE_ONE_TO_ONE ||
         p.rule.kind == SNN_RULE_ALL_TO_ALL;
}
uint64_t indegree_of(const ProjSpec& p) {
  if (p.rule.kind == SNN_RULE_ONE_TO_ONE) return 1;
  if (p.rule.kind == SNN_RULE_ALL_TO_ALL) return p.n_src;
  return (uint64_t)p.rule.param;
}

uint64_t counter_space(const ProjSpec& p) {
  if (fixed_indegree_shape(p)) return indegree_of(p) * p.n_tgt;
  if (p.rule.kind == SNN_RULE_FIXED_TOTAL) return (uint64_t)p.rule.param;
  return (uint64_t)p.n_tgt * p.n_src;
}

}  // namespace

// ============================================================================
extern "C" {

int snn_create(const snn_config* config, const snn_allocator* alloc, void* cuda_stream,
               snn_ctx** out) {
  if (!config || !out) return SNN_EINVAL;
  *out = nullptr;
  if (!(config->dt_ms > 0) || config->n_ranks < 1 || config->weight_format < 0 ||
      config->weight_format > 2 || (config->exchange != 0 && config->exchange != 1))
    return SNN_EINVAL;
  {
    const uint32_t rb = config->radix_bits ? (uint32_t)config->radix_bits : 8u;
    const uint32_t it = config->sort_items ? (uint32_t)config->sort_items : 16u;
    if (!sort_config_supported(rb, it)) return SNN_EINVAL;
    if (config->deliver_ctas_per_sm < 0 || config->deliver_ctas_per_sm > 32) return SNN_EINVAL;
    if (config->dry_run != 0 && (config->dry_run != 1 || config->n_ranks < 2 ||
                                 config->dry_run_rank >= config->n_ranks))
      return SNN_EINVAL;
    if (!(config->xi == config->xi)) return SNN_EINVAL;    // NaN threshold
    if (config->profile_kernels < 0 || config->profile_kernels > 2) return SNN_EINVAL;
    if (config->deliver_mode < 0 || config->deliver_mode > 1) return SNN_EINVAL;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || config->device < 0 || config->device >= ndev) {
    cudaGetLastError();
    return SNN_ECUDA;
  }
  if (cudaSetDevice(config->device) != cudaSuccess) return SNN_ECUDA;
  snn_ctx* c = new snn_ctx();
  c->cfg = *config;
  if (c->cfg.radix_bits == 0) c->cfg.radix_bits = 10;
  if (c->cfg.sort_items == 0) c->cfg.sort_items = 16;
  if (c->cfg.deliver_ctas_per_sm == 0) c->cfg.deliver_ctas_per_sm = 8;
  if (alloc) c->alloc = *alloc;
  c->st = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, config->device);
  c->wbytes = config->weight_format == SNN_WEIGHT_F32 ? 4 : 2;
  *out = c;
  return SNN_OK;
}

const char* snn_last_error(snn_ctx* c) { return c ? c->err.c_str() : "null context"; }

int snn_create_population(snn_ctx* c, uint32_t n, const snn_iaf_psc_exp_params* p,
                          uint32_t* first_gid) {
  if (!c) return SNN_EINVAL;
  if (c->calibrated) return fail(c, SNN_ESTATE, "create_population after calibrate");
  if (!p || n == 0) return fail(c, SNN_EINVAL, "population needs n > 0 and parameters");
  if (!(p->tau_m > 0 && p->C_m > 0 && p->tau_syn_ex > 0 && p->tau_syn_in > 0 && p->t_ref >= 0))
    return fail(c, SNN_EINVAL, "iaf_psc_exp time constants and C_m must be positive");
  if ((uint64_t)c->N + n > 0xFFFFFFF0ull) return fail(c, SNN_EINVAL, "too many neurons");
  if (c->pops.size() >= 65535) return fail(c, SNN_EINVAL, "too many populations");
  c->pops.push_back({c->N, n, *p});
  if (first_gid) *first_gid = c->N;
  c->N += n;
  return SNN_OK;
}

static int add_projection(snn_ctx* c, uint32_t src_first, uint32_t n_src, uint32_t src_stride,
                          uint32_t tgt_first, uint32_t n_tgt, uint32_t tgt_stride,
                          const snn_rule* rule, const snn_dist* weight, const snn_dist* delay,
                          uint64_t seed, uint32_t* proj_id) {
  if (c->calibrated) return fail(c, SNN_ESTATE, "connect after calibrate");
  if (!rule || n_src == 0 || n_tgt == 0) return fail(c, SNN_EINVAL, "empty projection or no rule");
  const uint64_t last_s = (uint64_t)src_first + (uint64_t)(n_src - 1) * src_stride;
  const uint64_t last_t = (uint64_t)tgt_first + (uint64_t)(n_tgt - 1) * tgt_stride;
  if (last_s >= c->N || last_t >= c->N) return fail(c, SNN_EINVAL, "projection range beyond created neurons");
  if (check_dist_w(weight) != SNN_OK) return fail(c, SNN_EINVAL, "bad weight distribution");
  if (check_dist_d(delay) != SNN_OK) return fail(c, SNN_EINVAL, "bad delay distribution");
  ProjSpec p{};
  p.src_first = src_first; p.n_src = n_src; p.src_stride = src_stride;
  p.tgt_first = tgt_first; p.n_tgt = n_tgt; p.tgt_stride = tgt_stride;
  p.rule = *rule; p.w = *weight; p.d = *delay; p.seed = seed;
  switch (rule->kind) {
    case SNN_RULE_FIXED_INDEGREE:
      if (!(rule->param >= 1) || rule->param != std::floor(rule->param) || rule->param > 4294967295.0)
        return fail(c, SNN_EINVAL, "fixed in-degree needs an integer K >= 1");
      break;
    case SNN_RULE_FIXED_TOTAL:
      if (!(rule->param >= 1) || rule->param != std::floor(rule->param) || rule->param > 1e15)
        return fail(c, SNN_EINVAL, "fixed total number needs an integer N >= 1");
      break;
    case SNN_RULE_PAIRWISE_BERNOULLI:
      if (!(rule->param >= 0 && rule->param <= 1)) return fail(c, SNN_EINVAL, "Bernoulli p outside [0, 1]");
      break;
    case SNN_RULE_PAIRWISE_BERNOULLI_GEOMETRIC:
      if (!(rule->param >= 0 && rule->param <= 1)) return fail(c, SNN_EINVAL, "Bernoulli p outside [0, 1]");
      if (rule->param > 0 && gap_table(rule->param, &p.g_thr) != SNN_OK)
        return fail(c, SNN_EINVAL, "connection probability too small for the gap table");
      break;
    case SNN_RULE_ONE_TO_ONE:
      if (n_src != n_tgt) return fail(c, SNN_EINVAL, "one-to-one needs as many sources as targets");
      break;
    case SNN_RULE_ALL_TO_ALL:
      if ((uint64_t)n_src * n_tgt >= (1ull << 50)) return fail(c, SNN_EINVAL, "all-to-all too large");
      break;
    default:
      return fail(c, SNN_EINVAL, "unknown rule");
  }
  if (delay->kind == SNN_D_NORMAL_MIN) {
    if (delay_table(delay->mean, delay->sd, delay->lo, c->cfg.dt_ms, &p.d_smin, &p.d_thr) != SNN_OK)
      return fail(c, SNN_EINVAL, "delay distribution has mass above 255 steps");
  } else {
    p.d_smin = const_delay_steps(delay->mean, c->cfg.dt_ms);
    if (p.d_smin > 255) return fail(c, SNN_EINVAL, "delay above 255 steps");
  }
  if (proj_id) *proj_id = (uint32_t)c->projs.size();
  c->projs.push_back(std::move(p));
  return SNN_OK;
}

int snn_connect(snn_ctx* c, uint32_t src_first, uint32_t n_src, uint32_t tgt_first, uint32_t n_tgt,
                const snn_rule* rule, const snn_dist* weight, const snn_dist* delay, uint64_t seed,
                uint32_t* proj_id) {
  if (!c) return SNN_EINVAL;
  return add_projection(c, src_first, n_src, 1, tgt_first, n_tgt, 1, rule, weight, delay, seed, proj_id);
}

int snn_remote_connect(snn_ctx* c, uint32_t sigma, uint32_t s_first, uint32_t n_s, uint32_t tau,
                       uint32_t t_first, uint32_t n_t, uint32_t port, const snn_rule* rule,
                       const snn_dist* weight, const snn_dist* delay, int32_t group, uint64_t seed,
                       uint32_t* proj_id) {
  if (!c) return SNN_EINVAL;
  const uint32_t R = c->cfg.n_ranks;
  if (sigma >= R || tau >= R || port != 0 || (group != -1 && group != 0))
    return fail(c, SNN_EINVAL, "remote_connect: rank, port or group out of range");
  const uint64_t sf = (uint64_t)s_first * R + sigma, tf = (uint64_t)t_first * R + tau;
  if (sf > 0xFFFFFFFFull || tf > 0xFFFFFFFFull) return fail(c, SNN_EINVAL, "remote_connect: range beyond neurons");
  return add_projection(c, (uint32_t)sf, n_s, R, (uint32_t)tf, n_t, R, rule, weight, delay, seed, proj_id);
}

int snn_set_poisson_drive(snn_ctx* c, uint32_t first, uint32_t n, double rate_hz, double weight_pA,
                          uint64_t seed) {
  if (!c) return SNN_EINVAL;
  if (c->calibrated) return fail(c, SNN_ESTATE, "drive after calibrate");
  if (n == 0 || (uint64_t)first + n > c->N || !(rate_hz >= 0) || !std::isfinite(weight_pA))
    return fail(c, SNN_EINVAL, "bad Poisson drive");
  c->drives.push_back({first, n, rate_hz, weight_pA, seed});
  return SNN_OK;
}

// ---------------------------------------------------------------------------
int snn_calibrate(snn_ctx* c) {
  if (!c) return SNN_EINVAL;
  if (c->calibrated) return fail(c, SNN_ESTATE, "calibrate called twice");
  if (c->N == 0) return fail(c, SNN_EINVAL, "no neurons");
  CK(cudaSetDevice(c->cfg.device));
  const uint32_t R = c->cfg.n_ranks;
  const uint32_t N = c->N;
  const double dt = c->cfg.dt_ms;
  if (R > N) return fail(c, SNN_EINVAL, "more ranks than neurons");
  cudaEvent_t ev[6];
  for (auto& e : ev) CK(cudaEventCreate(&e));
  CK(cudaEventRecord(ev[0], c->st));

  // ---- partition (round-robin) ----
  c->M.assign(R, 0);
  c->rank_off.assign(R + 1, 0);
  for (uint32_t t = 0; t < R; ++t) c->M[t] = (N - t + R - 1) / R;
  for (uint32_t t = 0; t < R; ++t) c->rank_off[t + 1] = c->rank_off[t] + c->M[t];
  if (!c->cfg.dry_run) {           // per-neuron maps serve the simulation state only
    c->host_gid_of.resize(N);
    c->host_pos_of.resize(N);
    for (uint32_t gid = 0; gid < N; ++gid) {
      const uint32_t pos = c->rank_off[gid % R] + gid / R;
      c->host_gid_of[pos] = gid;
      c->host_pos_of[gid] = pos;
    }
  }

  // ---- projections, counters, delay tables ----
  const uint32_t P = (uint32_t)c->projs.size();
  std::vector<DevProj> dp(P);
  std::vector<uint32_t> dtab;
  c->cbase.assign(P, 0);
  uint64_t ctot = 0;
  uint32_t dmax = 1;
  for (uint32_t i = 0; i < P; ++i) {
    const ProjSpec& s = c->projs[i];
    DevProj& d = dp[i];
    d.src_first = s.src_first; d.n_src = s.n_src; d.src_stride = s.src_stride;
    d.tgt_first = s.tgt_first; d.n_tgt = s.n_tgt; d.tgt_stride = s.tgt_stride;
    d.rule = fixed_indegree_shape(s) ? kRuleFixedIndegree : (uint32_t)s.rule.kind;
    d.src_mode = s.rule.kind == SNN_RULE_ALL_TO_ALL ? kSrcAll : (s.rule.kind == SNN_RULE_ONE_TO_ONE ? kSrcOneToOne : 0u);
    d.proj_id = i; d.seed = s.seed;
    d.K = fixed_indegree_shape(s) ? indegree_of(s) : 0;
    d.N = s.rule.kind == SNN_RULE_FIXED_TOTAL ? (uint64_t)s.rule.param : 0;
    d.pb_thr = (s.rule.kind == SNN_RULE_PAIRWISE_BERNOULLI || s.rule.kind == SNN_RULE_PAIRWISE_BERNOULLI_GEOMETRIC)
                   ? (uint64_t)std::floor(s.rule.param * 4294967296.0) : 0;
    d.cbase = ctot; d.csize = counter_space(s);
    c->cbase[i] = ctot;
    if (d.csize > ~0ull - ctot) return fail(c, SNN_EINVAL, "counter space of the projections exceeds 64 bits");
    ctot += d.csize;
    d.magic_div = fixed_indegree_shape(s) ? magic_for(d.K) : magic_for(d.n_src);
    d.w_kind = s.w.kind == SNN_W_CONST ? 0 : 1;
    d.w_mean = (float)s.w.mean; d.w_sd = (float)s.w.sd;
    d.d_kind = s.d.kind == SNN_D_CONST ? 0 : 1;
    d.d_const = s.d_smin;
    d.d_tbl_off = (uint32_t)dtab.size(); d.d_tbl_len = (uint32_t)s.d_thr.size();
    dtab.insert(dtab.end(), s.d_thr.begin(), s.d_thr.end());
    d.g_tbl_off = (uint32_t)dtab.size(); d.g_tbl_len = (uint32_t)s.g_thr.size();
    dtab.insert(dtab.end(), s.g_thr.begin(), s.g_thr.end());
    dmax = std::max(dmax, s.d_smin + (uint32_t)s.d_thr.size());
  }
  uint32_t maxM = 0;
  for (auto m : c->M) maxM = std::max(maxM, m);
  Geom& g = c->g;
  g.R = R; g.N = N;
  g.rb = R > 1 ? bits_for(R - 1) : 0;
  g.sb = bits_for(maxM - 1);
  g.db = bits_for(dmax);
  g.key_bits = g.rb + g.sb + g.db;
  g.cbits = std::max(1u, bits_for(ctot ? ctot - 1 : 0));
  g.magic_R = magic_for(R);
  if (g.key_bits + g.cbits > 64 && !c->cfg.dry_run)
    return fail(c, SNN_EINVAL, "network too large for 64-bit sort records");
  // pass plan: as few passes as digits of at most radix_bits allow; digits are 8 bits
  // wherever possible and widen one bit at a time (9, then 10) as the key requires, the
  // widest ones last (a wider pass costs more than an 8-bit one)
  const uint32_t RB = (uint32_t)c->cfg.radix_bits;
  const uint32_t BINS = kHistStride;
  const uint32_t passes = std::max(1u, (g.key_bits + RB - 1) / RB);
  if (passes > 6) return fail(c, SNN_EINVAL, "sort key too wide");
  uint8_t pass_bits[8] = {0}, pass_shift[8] = {0};
  {
    uint32_t w[8];
    for (uint32_t p = 0; p < passes; ++p) w[p] = 8;
    int extra = (int)g.key_bits - 8 * (int)passes;        // bits beyond 8 per digit
    for (uint32_t round = 0; round < 2 && extra > 0; ++round)
      for (int p = (int)passes - 1; p >= 0 && extra > 0; --p)
        if (w[p] < RB) { ++w[p]; --extra; }
    uint32_t left = g.key_bits, sh = 0;
    for (uint32_t p = 0; p < passes; ++p) {
      const uint32_t b = std::min(w[p], left);
      pass_bits[p] = (uint8_t)b;
      pass_shift[p] = (uint8_t)sh;
      sh += b;
      left -= b;
    }
  }

  // ---- counted projections: fixed total over several ranks, pairwise Bernoulli ----
  DevProj* d_projs;
  UP(d_projs, dp, "projections");
  uint32_t* d_dtab;
  UP(d_dtab, dtab, "delay and gap tables");
  std::vector<uint32_t> ft_proj, pb_proj;
  std::vector<uint64_t> ft_tile_first(1, 0), pb_t_first(1, 0);
  for (uint32_t i = 0; i < P; ++i) {
    const ProjSpec& s = c->projs[i];
    if (s.rule.kind == SNN_RULE_FIXED_TOTAL && R > 1) {
      ft_proj.push_back(i);
      ft_tile_first.push_back(ft_tile_first.back() + ((uint64_t)s.rule.param + kCountTile - 1) / kCountTile);
    } else if (s.rule.kind == SNN_RULE_PAIRWISE_BERNOULLI || s.rule.kind == SNN_RULE_PAIRWISE_BERNOULLI_GEOMETRIC) {
      pb_proj.push_back(i);
      pb_t_first.push_back(pb_t_first.back() + s.n_tgt);
    }
  }
  const bool counted = !ft_proj.empty() || !pb_proj.empty();
  const bool dry = c->cfg.dry_run != 0;
  const uint32_t dr = dry ? c->cfg.dry_run_rank : 0;
  if (dry && counted)
    return fail(c, SNN_EINVAL, "a dry run supports fixed in-degree, one-to-one and all-to-all only (the other "
                               "rules are placed by counting draws over every rank)");
  CountedArgs ca{};
  std::vector<uint64_t> ft_tot_h, pb_tot_h;
  std::vector<void*> counted_bufs;
  if (counted) {
    if (R > kMaxCountedRanks) return fail(c, SNN_EINVAL, "fixed total / Bernoulli support at most 1024 ranks");
    uint32_t *d_ftp, *d_pbp;
    uint64_t *d_ftf, *d_pbf;
    UP(d_ftp, ft_proj, "fixed-total list");
    UP(d_pbp, pb_proj, "Bernoulli list");
    UP(d_ftf, ft_tile_first, "fixed-total tiles");
    UP(d_pbf, pb_t_first, "Bernoulli targets");
    ca.projs = d_projs; ca.R = R; ca.magic_R = magic_for(R); ca.tables = d_dtab;
    ca.ft_proj = d_ftp; ca.ft_tile_first = d_ftf; ca.n_ft = (uint32_t)ft_proj.size();
    ca.n_ft_tiles = ft_tile_first.back();
    ca.pb_proj = d_pbp; ca.pb_t_first = d_pbf; ca.n_pb = (uint32_t)pb_proj.size();
    ca.n_pb_targets = pb_t_first.back();
    AL(ca.ft_tile_cnt, std::max<uint64_t>(ca.n_ft_tiles * R, 1), "fixed-total tile counts");
    AL(ca.ft_tile_off, std::max<uint64_t>(ca.n_ft_tiles * R, 1), "fixed-total tile offsets");
    AL(ca.ft_tot, std::max<uint64_t>((uint64_t)ca.n_ft * R, 1), "fixed-total block sizes");
    AL(ca.pb_cnt, std::max<uint64_t>(ca.n_pb_targets, 1), "Bernoulli counts");
    AL(ca.pb_off, std::max<uint64_t>(ca.n_pb_targets, 1), "Bernoulli offsets");
    AL(ca.pb_tot, std::max<uint64_t>((uint64_t)ca.n_pb * R, 1), "Bernoulli block sizes");
    counted_bufs = {d_ftp, d_pbp, d_ftf, d_pbf, ca.ft_tile_cnt, ca.ft_tile_off, ca.ft_tot, ca.pb_cnt, ca.pb_off,
                    ca.pb_tot};
    CK(launch_counted_count(ca, c->st, c->num_sms));
    c->stats.kernel_launches += (ca.n_ft_tiles ? 2 : 0) + (ca.n_pb_targets ? 2 : 0);
    ft_tot_h.resize((size_t)ca.n_ft * R);
    pb_tot_h.resize((size_t)ca.n_pb * R);
    if (!ft_tot_h.empty())
      CK(cudaMemcpyAsync(ft_tot_h.data(), ca.ft_tot, ft_tot_h.size() * 8, cudaMemcpyDeviceToHost, c->st));
    if (!pb_tot_h.empty())
      CK(cudaMemcpyAsync(pb_tot_h.data(), ca.pb_tot, pb_tot_h.size() * 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->stats.d2h_bytes += (ft_tot_h.size() + pb_tot_h.size()) * 8;
  }

  // ---- generation blocks: rank-major, then projection order ----
  std::vector<DevBlock> blocks;
  std::vector<uint64_t> block_base(counted ? (size_t)P * R : 0, 0);
  c->seg_start.assign(R + 1, 0);
  const uint64_t GEN_TILE = 4096;
  uint64_t pos = 0, tiles = 0;
  for (uint32_t t = 0; t < R; ++t) {
    c->seg_start[t] = pos;
    if (dry && t != dr) continue;               // a dry run generates only its rank's targets
    uint32_t kft = 0, kpb = 0;
    for (uint32_t i = 0; i < P; ++i) {
      const ProjSpec& s = c->projs[i];
      const bool is_ft_counted = s.rule.kind == SNN_RULE_FIXED_TOTAL && R > 1;
      const bool is_pb = s.rule.kind == SNN_RULE_PAIRWISE_BERNOULLI ||
                         s.rule.kind == SNN_RULE_PAIRWISE_BERNOULLI_GEOMETRIC;
      if (counted) block_base[(size_t)i * R + t] = pos;
      if (is_ft_counted || is_pb) {
        const uint32_t q = is_pb ? kpb++ : kft++;
        pos += is_pb ? pb_tot_h[(size_t)q * R + t] : ft_tot_h[(size_t)q * R + t];
        continue;
      }
      DevBlock b{};
      b.rank = t; b.proj = i;
      // targets tgt_first + ti * stride living on rank t: one residue class of ti
      const uint32_t st = s.tgt_stride % R;
      const uint32_t period = st == 0 ? 1 : R / std::__gcd(st, R);
      int64_t ti0 = -1;
      for (uint32_t r = 0; r < period && r < s.n_tgt; ++r) {
        if ((uint32_t)(((uint64_t)s.tgt_first + (uint64_t)r * s.tgt_stride) % R) == t) { ti0 = r; break; }
      }
      if (ti0 < 0) continue;
      b.ti0 = (uint32_t)ti0; b.tstep = period;
      b.n_t = (uint32_t)((s.n_tgt - 1 - (uint32_t)ti0) / period + 1);
      b.count = fixed_indegree_shape(s) ? (uint64_t)b.n_t * indegree_of(s)
                                                     : (uint64_t)s.rule.param;
      if (b.count == 0) continue;
      b.out_base = pos;
      b.tile_first = tiles;
      pos += b.count;
      tiles += (b.count + GEN_TILE - 1) / GEN_TILE;
      blocks.push_back(b);
    }
  }
  c->seg_start[R] = pos;
  const uint64_t E = pos;
  c->E = E;
  if (dry) {
    // records carry their generation position within the one built rank
    g.cbits = std::max(1u, bits_for(E ? E - 1 : 0));
    if (g.key_bits + g.cbits > 64) return fail(c, SNN_EINVAL, "rank share too large for 64-bit sort records");
  }
  const uint64_t SORT_TILE = sort_tile_items((uint32_t)c->cfg.sort_items);
  std::vector<uint64_t> seg_tile0(R + 1, 0);
  for (uint32_t t = 0; t < R; ++t)
    seg_tile0[t + 1] = seg_tile0[t] + (c->seg_start[t + 1] - c->seg_start[t] + SORT_TILE - 1) / SORT_TILE;
  const uint64_t n_sort_tiles = seg_tile0[R];

  // dense row offsets: rows of rank t in (slot, s) order
  std::vector<uint32_t> dense_off((size_t)R * R);
  for (uint32_t t = 0; t < R; ++t) {
    uint32_t acc = 0;
    for (uint32_t slot = 0; slot < R; ++slot) {
      const uint32_t sig = slot == 0 ? t : (slot <= t ? slot - 1 : slot);
      dense_off[(size_t)t * R + slot] = acc;
      acc += c->M[sig];
    }
  }

  // ---- device buffers for the build ----
  BuildArgs a{};
  DevBlock* d_blocks; uint64_t* d_seg_tile0; uint64_t* d_cbase;
  UP(d_blocks, blocks, "blocks");
  if (counted) {
    uint64_t* d_bb;
    UP(d_bb, block_base, "block bases");
    ca.block_base = d_bb;
    counted_bufs.push_back(d_bb);
  }
  UP(c->d_seg_start, c->seg_start, "segments");
  UP(d_seg_tile0, seg_tile0, "sort tiles");
  UP(d_cbase, c->cbase, "counter bases");
  UP(c->d_dense_off, dense_off, "dense offsets");
  AL(c->d_err, 4, "error word");
  CK(cudaMemsetAsync(c->d_err, 0, 4, c->st));
  uint64_t *rec_a = nullptr, *rec_b = nullptr, *hist = nullptr, *bin_base = nullptr, *status = nullptr;
  uint32_t* counters = nullptr;
  AL(rec_a, std::max<uint64_t>(E, 1), "records A");
  if (passes > 0) AL(rec_b, std::max<uint64_t>(E, 1), "records B");
  AL(hist, (uint64_t)R * std::max(passes, 1u) * BINS, "histograms");
  AL(bin_base, (uint64_t)R * std::max(passes, 1u) * BINS, "bin bases");
  AL(status, std::max<uint64_t>(n_sort_tiles, 1) * BINS, "look-back status");
  AL(counters, 8, "tile counters");
  CK(cudaMemsetAsync(hist, 0, (size_t)R * std::max(passes, 1u) * BINS * 8, c->st));
  CK(cudaMemsetAsync(status, 0, (size_t)std::max<uint64_t>(n_sort_tiles, 1) * BINS * 8, c->st));
  CK(cudaMemsetAsync(counters, 0, 32, c->st));

  a.blocks = d_blocks; a.nblocks = (uint32_t)blocks.size();
  a.n_gen_tiles = tiles;
  a.projs = d_projs; a.nproj = P; a.dtables = d_dtab; a.g = g;
  a.rec_a = rec_a; a.rec_b = rec_b; a.hist = hist; a.bin_base = bin_base;
  a.seg_start = c->d_seg_start; a.seg_tile0 = d_seg_tile0; a.status = status;
  a.counters = counters; a.err = c->d_err; a.passes = passes; a.radix_bits = RB;
  a.n_sort_tiles = n_sort_tiles; a.cbase_sorted = d_cbase; a.num_sms = c->num_sms;
  a.dense_off = c->d_dense_off;
  a.fuse_hist = counted ? 0u : 1u;
  a.pos_counters = dry ? 1u : 0u;
  a.sort_items = (uint32_t)c->cfg.sort_items;
  for (int p = 0; p < 8; ++p) { a.pass_bits[p] = pass_bits[p]; a.pass_shift[p] = pass_shift[p]; }

  CK(launch_generate(a, c->st));
  c->stats.kernel_launches += tiles ? 1 : 0;
  if (counted) {
    CK(launch_counted_place(ca, a, c->st));
    CK(launch_histogram(a, c->st));
    c->stats.kernel_launches += (ca.n_ft_tiles ? 1 : 0) + (ca.n_pb_targets ? 1 : 0) + 1;
  }
  CK(cudaEventRecord(ev[1], c->st));
  CK(launch_bin_scan(a, c->st));
  c->stats.kernel_launches += passes ? 1 : 0;
  cudaEvent_t evp;
  CK(cudaEventCreate(&evp));
  CK(cudaEventRecord(evp, c->st));
  uint64_t* cur = rec_a;
  uint64_t* oth = rec_b;
  for (uint32_t p = 0; p < passes; ++p) {
    CK(launch_sort_pass(a, p, cur, oth, p + 1, c->st));
    c->stats.kernel_launches += n_sort_tiles ? 1 : 0;
    std::swap(cur, oth);
  }
  CK(cudaEventRecord(ev[2], c->st));
  dfree(c, oth);
  dfree(c, status);
  dfree(c, hist);
  dfree(c, bin_base);

  // ---- final layout ----
  // the arrays hold 16 elements beyond the last synapse: the staged delivery copies
  // whole 16-element groups (its chunk ends round up), and reads but ignores the rest
  AL(c->d_tgt, E + 16, "targets");
  c->d_w = dalloc(c, (E + 16) * c->wbytes);
  if (!c->d_w) return fail(c, SNN_ENOMEM, "allocation failed: weights");
  AL(c->d_d, E + 16, "delays");
  AL(c->d_dense, (uint64_t)(dry ? 1 : R) * (N + 1), "row starts");
  if (c->cfg.weight_format == SNN_WEIGHT_F16) {
    // per source gid: power-of-two scale of the largest |mean| among its projections
    std::vector<float> sc(N, 1.0f);
    std::vector<int> ex(N, -1000);
    for (const auto& s : c->projs) {
      const double m = std::fabs(s.w.mean) + 4 * std::fabs(s.w.kind == SNN_W_CONST ? 0 : s.w.sd);
      if (m <= 0) continue;
      const int e = (int)std::nearbyint(std::log2(m));
      for (uint32_t k = 0; k < s.n_src; ++k) {
        const uint32_t gid = s.src_first + k * s.src_stride;
        ex[gid] = std::max(ex[gid], e);
      }
    }
    for (uint32_t gid = 0; gid < N; ++gid) sc[gid] = ex[gid] == -1000 ? 1.0f : std::ldexp(1.0f, ex[gid]);
    UP(c->d_scale_src, sc, "fp16 scales");
    if (R == 1) c->d_row_scale = c->d_scale_src;
  }
  a.tgt = c->d_tgt; a.w = c->d_w; a.d = c->d_d; a.w_format = (uint32_t)c->cfg.weight_format;
  a.dense = c->d_dense; a.row_scale_src = c->d_scale_src;
  a.dense_seg0 = dry ? dr : 0; a.dense_nseg = dry ? 1 : R;
  CK(launch_finalize(a, cur, E, c->st));
  c->stats.kernel_launches += E ? 2 : 1;
  CK(cudaEventRecord(ev[3], c->st));
  dfree(c, cur);
  dfree(c, d_blocks);
  dfree(c, counters);
  for (void* p : counted_bufs) dfree(c, p);

  // ---- image neurons and communication maps (logical ranks) ----
  if (R > 1) {
    // all_src[p][tau]: projection p gives all its sources images on tau
    std::vector<uint8_t> all_src((size_t)P * R, 0);
    if (c->cfg.xi > 0) {
      std::vector<uint64_t> n_on;
      for (uint32_t i = 0; i < P; ++i) {
        targets_per_rank(c->projs[i], R, &n_on);
        for (uint32_t t = 0; t < R; ++t)
          all_src[(size_t)i * R + t] = n_on[t] > 0 && per_source(c->projs[i], n_on[t]) >= c->cfg.xi;
      }
    }
    int rc = dry ? build_maps_dry(c, dr, dp, all_src) : build_maps(c, dp, d_projs, d_cbase, d_dtab, all_src);
    if (rc != SNN_OK) return rc;
  }
  CK(cudaEventRecord(ev[4], c->st));

  // ---- simulation state (a dry run builds connections only) ----
  // ring slots: delays 1 .. dmax ahead of the slot being read, so dmax + 1 slots
  const uint32_t D = dmax + 1;
  c->ring_slots = D;
  float* d_v0 = nullptr;
  if (!dry) {
  SimArgs& s = c->sim;
  s.N = N; s.R = R;
  s.err = c->d_err;
  AL(s.V, N, "V"); AL(s.Iex, N, "Iex"); AL(s.Iin, N, "Iin"); AL(s.refr, N, "refr");
  std::vector<uint16_t> pop_of(N);
  std::vector<DevPop> dpops;
  std::vector<float> v0(N);
  for (size_t pi = 0; pi < c->pops.size(); ++pi) {
    const PopSpec& ps = c->pops[pi];
    dpops.push_back(propagators(ps.p, dt));
    for (uint32_t k = 0; k < ps.n; ++k) {
      const uint32_t gid = ps.first + k;
      const uint32_t ppos = c->host_pos_of[gid];
      pop_of[ppos] = (uint16_t)pi;
      double v = ps.p.V_init_lo;
      if (ps.p.V_init_hi > ps.p.V_init_lo) {
        const uint4 b = philox_stream(gid, (uint32_t)pi, kPurposeVinit, ps.p.v_init_seed);
        const double u = ((double)(b.x >> 9) + 0.5) * 0x1p-23;
        v = ps.p.V_init_lo + (ps.p.V_init_hi - ps.p.V_init_lo) * u;
      }
      v0[ppos] = (float)v;
    }
  }
  uint16_t* d_pop_of; DevPop* d_pops;
  UP(d_pop_of, pop_of, "population index");
  UP(d_pops, dpops, "populations");
  UP(d_v0, v0, "V0");
  s.pop_of = d_pop_of; s.pops = d_pops; s.npops = (uint32_t)dpops.size();
  if (R > 1) {
    uint32_t* d_gid_of;
    UP(d_gid_of, c->host_gid_of, "gid of position");
    s.gid_of = d_gid_of;
  }
  std::vector<DevDrive> ddr;
  std::vector<uint32_t> ptab;
  for (size_t k = 0; k < c->drives.size(); ++k) {
    const DriveSpec& dr = c->drives[k];
    auto t = poisson_table(dr.rate, dt);
    DevDrive x{};
    x.first = dr.first; x.n = dr.n; x.weight = (float)dr.weight; x.idx = (uint32_t)k; x.seed = dr.seed;
    x.tbl_off = (uint32_t)ptab.size(); x.tbl_len = (uint32_t)t.size();
    ptab.insert(ptab.end(), t.begin(), t.end());
    ddr.push_back(x);
  }
  if (ptab.size() > 256) return fail(c, SNN_EINVAL, "Poisson tables exceed 256 entries in total");
  DevDrive* d_dr; uint32_t* d_ptab;
  UP(d_dr, ddr, "drives");
  UP(d_ptab, ptab, "Poisson tables");
  s.drives = d_dr; s.ndrives = (uint32_t)ddr.size();
  s.poisson_tbl = d_ptab; s.poisson_tbl_len = (uint32_t)ptab.size();
  bool merged = true;
  for (const auto& ps : c->pops) merged = merged && ps.p.tau_syn_ex == ps.p.tau_syn_in;
  s.n_rec = merged ? 1 : 2;
  s.ring_stride = (N + 3u) & ~3u;
  AL(s.ring, (uint64_t)D * s.n_rec * s.ring_stride, "ring buffers");
  CK(cudaMemsetAsync(s.ring, 0, (size_t)D * s.n_rec * s.ring_stride * 4, c->st));
  s.ring_slots = D;
  AL(s.step, 1, "step");
  AL(s.n_spk, 2, "spike counts");
  AL(s.spk, (uint64_t)2 * N, "spike lists");
  s.work = s.spk; s.n_work = s.n_spk; s.work_stride = N;      // one rank: rows = neurons
  AL(s.n_logged, 1, "log count");
  AL(s.n_events, 1, "event count");
  AL(s.n_spikes_total, 1, "spike count");
  CK(cudaMemsetAsync(s.step, 0, 4, c->st));
  CK(cudaMemsetAsync(s.n_spk, 0, 8, c->st));
  CK(cudaMemsetAsync(s.n_logged, 0, 8, c->st));
  CK(cudaMemsetAsync(s.n_events, 0, 8, c->st));
  CK(cudaMemsetAsync(s.n_spikes_total, 0, 8, c->st));
  s.log_cap = c->cfg.spike_log_capacity;
  if (s.log_cap) AL(s.log, s.log_cap, "spike log");
  s.rows = c->d_dense;
  s.tgt = c->d_tgt; s.w = c->d_w; s.d = c->d_d; s.w_format = (uint32_t)c->cfg.weight_format;
  s.row_scale = c->d_row_scale;
  // rows split into slices of about 1,024 events so that every CTA gets work
  {
    const double avg = E ? (double)E / std::max<uint64_t>(1, (uint64_t)N) : 0.0;
    s.slices = (uint32_t)std::min(64.0, std::max(1.0, std::ceil(avg / 1024.0)));
  }
  s.deliver_grid = (uint32_t)c->num_sms * (uint32_t)c->cfg.deliver_ctas_per_sm;
  s.update_grid = (uint32_t)c->num_sms * 8;
  s.lists = 2;
  // staged delivery of long rows: bulk copies need 16-byte aligned array bases; its grid
  // is at most what stays resident (CTAs take their items in a fixed order)
  const bool aligned = (((uintptr_t)c->d_tgt | (uintptr_t)c->d_w | (uintptr_t)c->d_d) & 15u) == 0;
  const int staged_per_sm = staged_deliver_ctas_per_sm((uint32_t)c->cfg.weight_format);
  const bool staged = aligned && c->cfg.deliver_mode == 0 && staged_per_sm > 0;
  s.staged_grid = (uint32_t)c->num_sms * (uint32_t)std::max(1, std::min(staged_per_sm, c->cfg.deliver_ctas_per_sm));
  if (R > 1) {
    int rc = setup_routing(c);
    if (rc != SNN_OK) return rc;
    s.staged = staged && s.item_lanes == 0;
  } else {
    s.staged = staged;
    // one rank: the neuron work of a step overlaps its delivery (two streams, lists
    // modulo 3); a small neuron grid leaves the delivery most of every SM
    c->ov = s;
    c->ov.lists = 3;
    c->ov.update_grid = (uint32_t)c->num_sms * 2;
    AL(c->ov.n_work, 3, "overlapped spike counts");
    AL(c->ov.work, (uint64_t)3 * N, "overlapped spike lists");
    c->ov.work_stride = N;
    CK(cudaMemsetAsync(c->ov.n_work, 0, 12, c->st));
    if (!c->st2) CK(cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking));
    if (!c->st3) CK(cudaStreamCreateWithFlags(&c->st3, cudaStreamNonBlocking));
    if (!c->ev_u) CK(cudaEventCreateWithFlags(&c->ev_u, cudaEventDisableTiming));
    for (auto& e : c->ev_dk)
      if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->overlap = true;
  }
  CK(launch_init_state(s, d_v0, c->st));
  c->stats.kernel_launches += 1;
  }
  CK(cudaEventRecord(ev[5], c->st));
  CK(cudaStreamSynchronize(c->st));
  if (d_v0) dfree(c, d_v0);
  uint32_t herr = 0;
  CK(cudaMemcpy(&herr, c->d_err, 4, cudaMemcpyDeviceToHost));
  c->stats.d2h_bytes += 4;
  float ms[5], ms_pass = 0;
  for (int k = 0; k < 5; ++k) CK(cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]));
  CK(cudaEventElapsedTime(&ms_pass, evp, ev[2]));
  for (auto& e : ev) cudaEventDestroy(e);
  cudaEventDestroy(evp);
  c->stats.t_sort_pass_ms = ms_pass;
  c->stats.t_generate_ms = ms[0];
  c->stats.t_sort_ms = ms[1];
  c->stats.t_finalize_ms = ms[2];
  c->stats.t_maps_ms = ms[3];
  c->stats.t_calibrate_ms = ms[0] + ms[1] + ms[2] + ms[3] + ms[4];
  c->stats.sort_passes = passes;
  c->stats.radix_bits = RB;
  c->stats.key_bits = g.key_bits;
  c->stats.ring_slots = D;
  c->stats.n_blocks = blocks.size();
  c->stats.gen_kernel_launches = tiles ? 1 : 0;
  c->stats.sort_kernel_launches = passes;
  c->calibrated = true;
  if (herr & kErrTimeout) return fail(c, SNN_ETIMEOUT, "a bounded device wait gave up during construction");
  if (herr) return fail(c, SNN_ECUDA, "device-side bounds check failed during construction");
  return SNN_OK;
}

// ---------------------------------------------------------------------------
// Kernels one batch of `steps` steps launches.
static uint64_t launches_per_batch(snn_ctx* c, uint32_t steps) {
  if (c->overlap && c->cfg.profile_kernels != 2) return 2ull * steps + 2;
  return (uint64_t)steps * (2 + (c->cfg.n_ranks > 1 ? route_kernels_per_step(c) : 0)) + 1;
}

// One rank, overlapped: step_update(PRE) decides the spikes of the first step; then
// per step k the delivery of step k (after the neuron work that listed its spikes) runs
// beside step_update(k) (stream st, after the delivery of step k - 1, whose slots it
// reads).  The last step_update takes the input only.  The delivery of step k needs only
// its list: it writes slots k + d with d >= 1 by commutative reductions, and no later
// kernel before step_update(k + 1) reads them.  So the deliveries of consecutive steps
// alternate between two streams and may run at the same time; step_update(k + 1) waits
// for the delivery of step k.
// With profile_kernels the same schedule runs (no graph) with a pair of timing events
// around every launch on its own stream, so each kernel is timed beside the others as
// in the graph-captured steps.
static int run_steps_overlapped(snn_ctx* c, uint32_t steps) {
  SimArgs& o = c->ov;
  cudaStream_t A = c->st;
  cudaStream_t B[2] = {c->st2, c->st3};
  const bool profile = c->cfg.profile_kernels && !c->capturing;
  std::vector<cudaEvent_t> evs;
  if (profile) {
    evs.resize(4 * (size_t)steps + 2);
    for (auto& e : evs) CK(cudaEventCreate(&e));
  }
  if (profile) CK(cudaEventRecord(evs[4 * (size_t)steps], A));
  CK(launch_step_update(o, 0, kStepPre, A));
  if (profile) CK(cudaEventRecord(evs[4 * (size_t)steps + 1], A));
  CK(cudaEventRecord(c->ev_u, A));
  for (uint32_t k = 0; k < steps; ++k) {
    cudaStream_t Bk = B[k & 1];
    if (k > 0) CK(cudaStreamWaitEvent(A, c->ev_dk[(k - 1) & 1], 0));
    CK(cudaStreamWaitEvent(Bk, c->ev_u, 0));
    if (profile) CK(cudaEventRecord(evs[4 * (size_t)k], Bk));
    CK(launch_deliver(o, k, Bk, false));
    if (profile) CK(cudaEventRecord(evs[4 * (size_t)k + 1], Bk));
    CK(cudaEventRecord(c->ev_dk[k & 1], Bk));
    if (profile) CK(cudaEventRecord(evs[4 * (size_t)k + 2], A));
    CK(launch_step_update(o, k, kStepPost | (k + 1 < steps ? kStepPre : 0u), A));
    if (profile) CK(cudaEventRecord(evs[4 * (size_t)k + 3], A));
    CK(cudaEventRecord(c->ev_u, A));
  }
  // join both delivery streams (the last step's delivery, and the one before it)
  CK(cudaStreamWaitEvent(A, c->ev_dk[(steps - 1) & 1], 0));
  if (steps > 1) CK(cudaStreamWaitEvent(A, c->ev_dk[steps & 1], 0));
  CK(launch_advance(o, steps, A));
  if (profile) {
    CK(cudaStreamSynchronize(A));
    float u = 0, d = 0;
    CK(cudaEventElapsedTime(&u, evs[4 * (size_t)steps], evs[4 * (size_t)steps + 1]));
    c->stats.t_update_ms += u;
    for (uint32_t k = 0; k < steps; ++k) {
      CK(cudaEventElapsedTime(&d, evs[4 * (size_t)k], evs[4 * (size_t)k + 1]));
      c->stats.t_deliver_ms += d;
      CK(cudaEventElapsedTime(&u, evs[4 * (size_t)k + 2], evs[4 * (size_t)k + 3]));
      c->stats.t_update_ms += u;
    }
    for (auto& e : evs) cudaEventDestroy(e);
    c->stats.update_launches += steps + 1;
    c->stats.deliver_launches += steps;
  }
  if (!c->capturing) c->stats.kernel_launches += launches_per_batch(c, steps);
  return SNN_OK;
}

static int run_steps(snn_ctx* c, uint32_t steps) {
  SimArgs& s = c->sim;
  if (steps == 0) return SNN_OK;
  if (c->overlap && c->cfg.profile_kernels != 2) return run_steps_overlapped(c, steps);
  const bool routed = c->cfg.n_ranks > 1;
  const bool profile = c->cfg.profile_kernels && !c->capturing;
  std::vector<cudaEvent_t> evs;
  if (profile) {
    evs.resize(3 * (size_t)steps);
    for (auto& e : evs) CK(cudaEventCreate(&e));
  }
  // programmatic dependent launches chain the kernels of a batch (not when each kernel
  // is timed): every kernel but the batch's first update starts while its predecessor
  // drains; the advance kernel after the batch is a normal launch
  const bool pdl = !profile;
  for (uint32_t k = 0; k < steps; ++k) {
    if (profile) CK(cudaEventRecord(evs[3 * k], c->st));
    CK(launch_update(s, k, c->st, pdl && k > 0));
    if (routed) CK(launch_route(c, k, pdl));
    if (profile) CK(cudaEventRecord(evs[3 * k + 1], c->st));
    CK(launch_deliver(s, k, c->st, pdl));
    if (profile) CK(cudaEventRecord(evs[3 * k + 2], c->st));
  }
  CK(launch_advance(s, steps, c->st));
  if (profile) {
    CK(cudaStreamSynchronize(c->st));
    for (uint32_t k = 0; k < steps; ++k) {
      float u = 0, d = 0;
      CK(cudaEventElapsedTime(&u, evs[3 * k], evs[3 * k + 1]));
      CK(cudaEventElapsedTime(&d, evs[3 * k + 1], evs[3 * k + 2]));
      c->stats.t_update_ms += u;
      c->stats.t_deliver_ms += d;
    }
    for (auto& e : evs) cudaEventDestroy(e);
    c->stats.update_launches += steps;
    c->stats.deliver_launches += steps;
  }
  if (!c->capturing) c->stats.kernel_launches += launches_per_batch(c, steps);
  return SNN_OK;
}

static int build_graph(snn_ctx* c, uint32_t steps) {
  cudaStream_t cap;
  CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t keep = c->st;
  c->st = cap;
  CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  c->capturing = true;
  int rc = run_steps(c, steps);
  c->capturing = false;
  cudaGraph_t gr;
  cudaError_t e = cudaStreamEndCapture(cap, &gr);
  c->st = keep;
  if (rc != SNN_OK) { cudaStreamDestroy(cap); return rc; }
  CK(e);
  CK(cudaGraphInstantiate(&c->graph, gr, 0));
  cudaGraphDestroy(gr);
  cudaStreamDestroy(cap);
  c->graph_steps = steps;
  return SNN_OK;
}

int snn_simulate(snn_ctx* c, uint32_t steps) {
  if (!c) return SNN_EINVAL;
  if (!c->calibrated) return fail(c, SNN_ESTATE, "simulate before calibrate");
  if (c->cfg.dry_run) return fail(c, SNN_ESTATE, "a dry run builds connections only");
  CK(cudaSetDevice(c->cfg.device));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, c->st));
  uint32_t left = steps;
  if (c->cfg.use_graph && !c->cfg.profile_kernels) {
    const uint32_t G = 10;
    if (!c->graph && steps >= G) {
      int rc = build_graph(c, G);
      if (rc != SNN_OK) return rc;
    }
    while (c->graph && left >= c->graph_steps) {
      CK(cudaGraphLaunch(c->graph, c->st));
      left -= c->graph_steps;
      c->stats.kernel_launches += launches_per_batch(c, c->graph_steps);
    }
  }
  int rc = run_steps(c, left);
  if (rc != SNN_OK) return rc;
  CK(cudaEventRecord(e1, c->st));
  CK(cudaStreamSynchronize(c->st));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->stats.t_simulate_ms += ms;
  c->stats.steps_done += steps;
  uint32_t herr = 0;
  CK(cudaMemcpy(&herr, c->d_err, 4, cudaMemcpyDeviceToHost));
  c->stats.d2h_bytes += 4;
  if (herr & kErrTimeout) return fail(c, SNN_ETIMEOUT, "a bounded device wait gave up during simulation");
  if (herr) return fail(c, SNN_ECUDA, "device-side bounds check failed during simulation");
  return SNN_OK;
}

int snn_get_spikes(snn_ctx* c, uint32_t* host_step, uint32_t* host_gid, uint64_t cap, uint64_t* n_out) {
  if (!c) return SNN_EINVAL;
  if (!c->calibrated) return fail(c, SNN_ESTATE, "no simulation");
  if (c->cfg.dry_run) return fail(c, SNN_ESTATE, "a dry run builds connections only");
  unsigned long long n = 0;
  CK(cudaMemcpyAsync(&n, c->sim.n_logged, 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  const uint64_t kept = std::min<uint64_t>(n, c->sim.log_cap);
  if (n_out) *n_out = kept;
  c->stats.spike_log_overflow = n - kept;
  if (!host_step && !host_gid) return SNN_OK;
  std::vector<uint2> buf(kept);
  if (kept) CK(cudaMemcpy(buf.data(), c->sim.log, kept * sizeof(uint2), cudaMemcpyDeviceToHost));
  std::sort(buf.begin(), buf.end(), [](const uint2& x, const uint2& y) {
    return x.x != y.x ? x.x < y.x : x.y < y.y;
  });
  const uint64_t m = std::min<uint64_t>(kept, cap);
  for (uint64_t i = 0; i < m; ++i) {
    if (host_step) host_step[i] = buf[i].x;
    if (host_gid) host_gid[i] = buf[i].y;
  }
  if (kept > cap) return fail(c, SNN_EOVERFLOW, "spike buffer too small");
  if (n > kept) return fail(c, SNN_EOVERFLOW, "spike log overflowed");
  return SNN_OK;
}

int snn_get_state(snn_ctx* c, uint32_t first, uint32_t n, float* V, float* Iex, float* Iin) {
  if (!c) return SNN_EINVAL;
  if (!c->calibrated) return fail(c, SNN_ESTATE, "no state before calibrate");
  if (c->cfg.dry_run) return fail(c, SNN_ESTATE, "a dry run builds connections only");
  if ((uint64_t)first + n > c->N) return fail(c, SNN_EINVAL, "range beyond neurons");
  const uint32_t N = c->N;
  float* src[3] = {c->sim.V, c->sim.Iex, c->sim.Iin};
  float* dst[3] = {V, Iex, Iin};
  std::vector<float> all(N);
  for (int k = 0; k < 3; ++k) {
    if (!dst[k]) continue;
    if (c->cfg.n_ranks == 1) {
      CK(cudaMemcpy(dst[k], src[k] + first, (size_t)n * 4, cudaMemcpyDeviceToHost));
    } else {
      CK(cudaMemcpy(all.data(), src[k], (size_t)N * 4, cudaMemcpyDeviceToHost));
      for (uint32_t i = 0; i < n; ++i) dst[k][i] = all[c->host_pos_of[first + i]];
    }
  }
  return SNN_OK;
}

static void decode_weights(snn_ctx* c, const std::vector<uint8_t>& raw, uint64_t n, float* out,
                           const std::vector<float>* scale_of_syn) {
  for (uint64_t i = 0; i < n; ++i) {
    float v;
    if (c->cfg.weight_format == SNN_WEIGHT_F32) {
      std::memcpy(&v, &raw[i * 4], 4);
    } else if (c->cfg.weight_format == SNN_WEIGHT_BF16) {
      uint16_t h;
      std::memcpy(&h, &raw[i * 2], 2);
      uint32_t u = (uint32_t)h << 16;
      std::memcpy(&v, &u, 4);
    } else {
      __half h;
      std::memcpy(&h, &raw[i * 2], 2);
      v = __half2float(h) * (scale_of_syn ? (*scale_of_syn)[i] : 1.0f);
    }
    out[i] = v;
  }
}

int snn_get_connections(snn_ctx* c, uint32_t rank, uint64_t* row_ptr, uint64_t row_cap, uint32_t* tgt,
                        float* w, uint8_t* d, uint64_t syn_cap, uint64_t* n_rows, uint64_t* n_syn) {
  if (!c) return SNN_EINVAL;
  if (!c->calibrated) return fail(c, SNN_ESTATE, "no connections before calibrate");
  if (rank >= c->cfg.n_ranks) return fail(c, SNN_EINVAL, "rank out of range");
  std::vector<uint64_t> rp;
  int rc = rank_row_ptr(c, rank, &rp);
  if (rc != SNN_OK) return rc;
  const uint64_t a = c->seg_start[rank], b = c->seg_start[rank + 1];
  if (n_rows) *n_rows = rp.size() - 1;
  if (n_syn) *n_syn = b - a;
  if (row_ptr) {
    if (row_cap < rp.size()) return fail(c, SNN_EOVERFLOW, "row_ptr buffer too small");
    for (size_t i = 0; i < rp.size(); ++i) row_ptr[i] = rp[i] - a;
  }
  const uint64_t n = b - a;
  if ((tgt || w || d) && syn_cap < n) return fail(c, SNN_EOVERFLOW, "synapse buffers too small");
  if (tgt && n) CK(cudaMemcpy(tgt, c->d_tgt + a, n * 4, cudaMemcpyDeviceToHost));
  if (d && n) CK(cudaMemcpy(d, c->d_d + a, n, cudaMemcpyDeviceToHost));
  if (w && n) {
    std::vector<uint8_t> raw(n * c->wbytes);
    CK(cudaMemcpy(raw.data(), (uint8_t*)c->d_w + a * c->wbytes, n * c->wbytes, cudaMemcpyDeviceToHost));
    std::vector<float> sc;
    if (c->cfg.weight_format == SNN_WEIGHT_F16) {
      std::vector<float> rs;
      rc = rank_row_scales(c, rank, &rs);
      if (rc != SNN_OK) return rc;
      sc.resize(n);
      for (size_t r = 0; r + 1 < rp.size(); ++r)
        for (uint64_t e = rp[r]; e < rp[r + 1]; ++e) sc[e - a] = rs[r];
    }
    decode_weights(c, raw, n, w, sc.empty() ? nullptr : &sc);
  }
  return SNN_OK;
}

int snn_get_row(snn_ctx* c, uint32_t rank, uint64_t row, uint32_t* tgt, float* w, uint8_t* d, uint64_t cap,
                uint64_t* n_out) {
  if (!c) return SNN_EINVAL;
  if (!c->calibrated) return fail(c, SNN_ESTATE, "no connections before calibrate");
  if (rank >= c->cfg.n_ranks) return fail(c, SNN_EINVAL, "rank out of range");
  uint64_t ab[2];
  float scale = 1.0f;
  int rc = rank_row_bounds(c, rank, row, ab, &scale);
  if (rc != SNN_OK) return rc;
  const uint64_t n = ab[1] - ab[0];
  if (n_out) *n_out = n;
  if ((tgt || w || d) && cap < n) return fail(c, SNN_EOVERFLOW, "row buffers too small");
  if (tgt && n) CK(cudaMemcpy(tgt, c->d_tgt + ab[0], n * 4, cudaMemcpyDeviceToHost));
  if (d && n) CK(cudaMemcpy(d, c->d_d + ab[0], n, cudaMemcpyDeviceToHost));
  if (w && n) {
    std::vector<uint8_t> raw(n * c->wbytes);
    CK(cudaMemcpy(raw.data(), (uint8_t*)c->d_w + ab[0] * c->wbytes, n * c->wbytes, cudaMemcpyDeviceToHost));
    std::vector<float> sc(n, scale);
    decode_weights(c, raw, n, w, &sc);
  }
  return SNN_OK;
}

int snn_get_delay_table(snn_ctx* c, uint32_t proj_id, uint32_t* thr, uint64_t cap, uint64_t* n_out,
                        uint32_t* s_min) {
  if (!c) return SNN_EINVAL;
  if (proj_id >= c->projs.size()) return fail(c, SNN_EINVAL, "no such projection");
  const ProjSpec& p = c->projs[proj_id];
  if (n_out) *n_out = p.d_thr.size();
  if (s_min) *s_min = p.d_smin;
  if (thr) {
    if (cap < p.d_thr.size()) return fail(c, SNN_EOVERFLOW, "table buffer too small");
    std::copy(p.d_thr.begin(), p.d_thr.end(), thr);
  }
  return SNN_OK;
}

int snn_stats(snn_ctx* c, snn_stats_t* out) {
  if (!c || !out) return SNN_EINVAL;
  snn_stats_t s = c->stats;
  s.n_neurons = c->N;
  s.n_synapses = c->E;
  s.n_projections = c->projs.size();
  s.device_bytes = c->cur_bytes;
  s.peak_device_bytes = c->peak_bytes;
  s.n_images = c->maps.n_images_total;
  if (c->calibrated && !c->cfg.dry_run) {
    unsigned long long v[2] = {0, 0};
    CK(cudaMemcpy(&v[0], c->sim.n_spikes_total, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&v[1], c->sim.n_events, 8, cudaMemcpyDeviceToHost));
    c->stats.d2h_bytes += 16;
    s.n_spikes = v[0];
    s.n_events = v[1];
  }
  *out = s;
  return SNN_OK;
}

int snn_selftest_bounded_wait(void* cuda_stream) {
  cudaStream_t st = (cudaStream_t)cuda_stream;
  uint64_t* status = nullptr;
  uint32_t* err = nullptr;
  if (cudaMalloc(&status, 2 * 256 * sizeof(uint64_t)) != cudaSuccess) return SNN_ENOMEM;
  if (cudaMalloc(&err, 4) != cudaSuccess) { cudaFree(status); return SNN_ENOMEM; }
  int rc = SNN_ECUDA;
  uint32_t h = 0;
  if (cudaMemsetAsync(status, 0, 2 * 256 * sizeof(uint64_t), st) == cudaSuccess &&
      cudaMemsetAsync(err, 0, 4, st) == cudaSuccess && launch_bounded_wait_selftest(status, err, st) == cudaSuccess &&
      cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, st) == cudaSuccess &&
      cudaStreamSynchronize(st) == cudaSuccess)
    rc = (h & kErrTimeout) ? SNN_ETIMEOUT : SNN_OK;
  cudaFree(status);
  cudaFree(err);
  return rc;
}

int snn_ring_reduction_probe(snn_ctx* c, int32_t mode, uint64_t n_events, uint32_t reps, double* ms_per_launch) {
  if (!c || !ms_per_launch) return SNN_EINVAL;
  if (!c->calibrated || c->cfg.dry_run) return fail(c, SNN_ESTATE, "the probe needs a calibrated network");
  if (c->cfg.n_ranks != 1) return fail(c, SNN_EINVAL, "the probe runs on one logical rank");
  if (mode != 0 && mode != 1) return fail(c, SNN_EINVAL, "probe mode is 0 or 1");
  if (n_events == 0 || n_events > c->E || reps == 0) return fail(c, SNN_EINVAL, "need 0 < n_events <= synapses, reps > 0");
  CK(cudaSetDevice(c->cfg.device));
  const unsigned grid = c->sim.deliver_grid ? c->sim.deliver_grid : (unsigned)c->num_sms * 4u;
  cudaEvent_t e[2] = {nullptr, nullptr};
  CK(cudaEventCreate(&e[0]));
  if (cudaEventCreate(&e[1]) != cudaSuccess) {
    cudaEventDestroy(e[0]);
    return fail(c, SNN_ECUDA, "cudaEventCreate");
  }
  cudaError_t err = cudaEventRecord(e[0], c->st);
  for (uint32_t r = 0; r < reps && err == cudaSuccess; ++r) {
    const uint64_t e0 = ((uint64_t)r * n_events) % (c->E - n_events + 1);
    err = launch_ring_probe(c->sim, e0, n_events, r % c->ring_slots, (uint32_t)mode, grid, c->st);
  }
  if (err == cudaSuccess) err = cudaEventRecord(e[1], c->st);
  if (err == cudaSuccess) err = cudaEventSynchronize(e[1]);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e[0], e[1]);
  cudaEventDestroy(e[0]);
  cudaEventDestroy(e[1]);
  if (err != cudaSuccess) return fail(c, SNN_ECUDA, std::string("ring reduction probe: ") + cudaGetErrorString(err));
  c->stats.kernel_launches += reps;
  *ms_per_launch = (double)ms / reps;
  return SNN_OK;
}

void snn_destroy(snn_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->cfg.device);
  if (c->graph) cudaGraphExecDestroy(c->graph);
  cudaStreamSynchronize(c->st);
  if (c->st2) cudaStreamDestroy(c->st2);
  if (c->st3) cudaStreamDestroy(c->st3);
  if (c->ev_u) cudaEventDestroy(c->ev_u);
  for (auto e : c->ev_dk)
    if (e) cudaEventDestroy(e);
  std::vector<void*> ptrs;
  for (auto& kv : c->live) ptrs.push_back(kv.first);
  for (void* p : ptrs) dfree(c, p);
  cudaStreamSynchronize(c->st);
  delete c;
}

}  // extern "C"

// ---- helpers shared with maps.cu and noalloc.cu (C++ linkage) ----
namespace snn {
int host_delay_table(double mean, double sd, double lo, double dt, uint32_t* s_min,
                     std::vector<uint32_t>* thr) {
  return delay_table(mean, sd, lo, dt, s_min, thr);
}
uint32_t host_const_delay_steps(double d, double dt) { return const_delay_steps(d, dt); }
void* ctx_alloc(snn_ctx* c, size_t bytes) { return dalloc(c, bytes); }
void ctx_free(snn_ctx* c, void* p) { dfree(c, p); }
int ctx_fail(snn_ctx* c, int code, const char* msg) { return fail(c, code, msg); }
cudaStream_t ctx_stream(snn_ctx* c) { return c->st; }
MapsState& ctx_maps(snn_ctx* c) { return c->maps; }
SimArgs& ctx_sim(snn_ctx* c) { return c->sim; }
const Geom& ctx_geom(snn_ctx* c) { return c->g; }
uint64_t ctx_geom_synapses(snn_ctx* c) { return c->E; }
const std::vector<uint64_t>& ctx_seg_start(snn_ctx* c) { return c->seg_start; }
const std::vector<uint32_t>& ctx_rank_sizes(snn_ctx* c) { return c->M; }
const std::vector<uint32_t>& ctx_rank_off(snn_ctx* c) { return c->rank_off; }
uint64_t* ctx_dense(snn_ctx* c) { return c->d_dense; }
const uint32_t* ctx_dense_off(snn_ctx* c) { return c->d_dense_off; }
const uint64_t* ctx_dseg_start(snn_ctx* c) { return c->d_seg_start; }
const float* ctx_scale_src(snn_ctx* c) { return c->d_scale_src; }
int ctx_num_sms(snn_ctx* c) { return c->num_sms; }
uint32_t* ctx_err(snn_ctx* c) { return c->d_err; }
int ctx_exchange(snn_ctx* c) { return c->cfg.exchange; }
uint32_t ctx_N(snn_ctx* c) { return c->N; }
}  // namespace snn
