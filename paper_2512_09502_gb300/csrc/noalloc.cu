// noalloc.cu -- one projection's source-sorted connections built into caller-owned
// device buffers without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns every byte of
// device memory under a fixed budget (a simulator embedding this library as a
// plugin, a real-time loop that must never reach the allocator), or code that keeps
// allocator state untouched between its own set-up and tear-down.  For them this
// file provides snn_connect_sorted_noalloc, which runs the same generation, radix
// sort and finalize kernels as snn_calibrate on a single logical rank, with every
// intermediate buffer (the 64-bit sort records, the look-back status words, the
// digit histograms) taken from one file-scope __device__ scratch array of fixed size.
// The caller passes only its input description and its output buffers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/snn.h"
#include "snn_internal.cuh"

namespace snn {

int host_delay_table(double mean, double sd, double lo, double dt, uint32_t* s_min,
                     std::vector<uint32_t>* thr);
uint32_t host_const_delay_steps(double d, double dt);

namespace {

constexpr uint64_t kMaxSynapses = SNN_NOALLOC_MAX_SYNAPSES;
constexpr uint32_t kBins = 256;            // radix 8 (the only sort width built)
constexpr uint32_t kMaxPasses = 6;
constexpr uint64_t kTile = 4096;           // records per sort tile the scratch is sized for
constexpr uint64_t kMaxTiles = (kMaxSynapses + kTile - 1) / kTile;

struct Scratch {
  uint64_t rec_a[kMaxSynapses];
  uint64_t rec_b[kMaxSynapses];
  uint64_t status[kMaxTiles * kBins];
  uint64_t hist[kMaxPasses * kHistStride];
  uint64_t bin_base[kMaxPasses * kHistStride];
  uint64_t seg_start[2];
  uint64_t seg_tile0[2];
  uint64_t cbase[1];
  DevBlock block;
  DevProj proj;
  uint32_t dtab[256];
  uint32_t counters[8];
  uint32_t err[4];
  uint32_t dense_off[4];
};

// Shared by every call on a device; held by every GPU that loads the library until
// the process exits.
static __device__ __align__(256) Scratch g_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
Scratch* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up once per device; the
// host-side symbol is only a stand-in and must never reach a kernel).
int scratch_address(Scratch** out, char* msg, size_t msg_len) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    std::snprintf(msg, msg_len, "no current CUDA device");
    return SNN_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      std::snprintf(msg, msg_len, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return SNN_ECUDA;
    }
    g_addr[dev] = (Scratch*)p;
  }
  *out = g_addr[dev];
  return SNN_OK;
}

}  // namespace
}  // namespace snn

using namespace snn;

extern "C" int snn_connect_sorted_noalloc(uint32_t n_neurons, uint32_t src_first, uint32_t n_src,
                                          uint32_t tgt_first, uint32_t n_tgt, const snn_rule* rule,
                                          const snn_dist* weight, const snn_dist* delay, uint64_t seed,
                                          double dt_ms, uint64_t* dev_row_ptr, uint32_t* dev_tgt,
                                          float* dev_w, uint8_t* dev_d, uint64_t syn_cap,
                                          uint64_t* n_syn, void* cuda_stream, char* host_errmsg,
                                          size_t errmsg_len) {
  char local_msg[160];
  char* msg = host_errmsg && errmsg_len ? host_errmsg : local_msg;
  const size_t mlen = host_errmsg && errmsg_len ? errmsg_len : sizeof(local_msg);
  msg[0] = 0;
  cudaStream_t st = (cudaStream_t)cuda_stream;
#define NA_FAIL(code, ...)                      \
  do {                                          \
    std::snprintf(msg, mlen, __VA_ARGS__);      \
    return code;                                \
  } while (0)
  // Once work is queued on the stream, a failing call first waits for that work: the
  // queued kernels use the shared scratch, and the next call (perhaps on another
  // stream) would otherwise clear it under them.
  bool enqueued = false;
#define NA_CK(call)                                                      \
  do {                                                                   \
    const cudaError_t e__ = (call);                                      \
    if (e__ != cudaSuccess) {                                            \
      if (enqueued) (void)cudaStreamSynchronize(st);                     \
      NA_FAIL(SNN_ECUDA, "%s: %s", #call, cudaGetErrorString(e__));      \
    }                                                                    \
    enqueued = true;                                                     \
  } while (0)

  if (!rule || !weight || !delay || !dev_row_ptr || !(dt_ms > 0) || n_neurons == 0 || n_src == 0 ||
      n_tgt == 0)
    NA_FAIL(SNN_EINVAL, "missing argument");
  if ((uint64_t)src_first + n_src > n_neurons || (uint64_t)tgt_first + n_tgt > n_neurons)
    NA_FAIL(SNN_EINVAL, "projection range beyond n_neurons");
  uint64_t E = 0;
  if (rule->kind == SNN_RULE_FIXED_INDEGREE || rule->kind == SNN_RULE_FIXED_TOTAL) {
    if (!(rule->param >= 1) || rule->param != std::floor(rule->param))
      NA_FAIL(SNN_EINVAL, "%s needs an integer parameter >= 1",
              rule->kind == SNN_RULE_FIXED_INDEGREE ? "fixed in-degree" : "fixed total number");
    // bounded before the integer conversion and the product, so that neither wraps
    const uint64_t per_tgt_cap = rule->kind == SNN_RULE_FIXED_INDEGREE ? kMaxSynapses / n_tgt : kMaxSynapses;
    if (rule->param > (double)per_tgt_cap)
      NA_FAIL(SNN_EINVAL, "more synapses than the allocation-free limit of %llu", (unsigned long long)kMaxSynapses);
    E = rule->kind == SNN_RULE_FIXED_INDEGREE ? (uint64_t)rule->param * n_tgt : (uint64_t)rule->param;
  } else {
    NA_FAIL(SNN_EINVAL, "only fixed in-degree and fixed total number are supported here");
  }
  if (E > kMaxSynapses)
    NA_FAIL(SNN_EINVAL, "%llu synapses exceed the allocation-free limit of %llu",
            (unsigned long long)E, (unsigned long long)kMaxSynapses);
  if (n_syn) *n_syn = E;
  if (syn_cap < E || !dev_tgt || !dev_w || !dev_d)
    NA_FAIL(SNN_EOVERFLOW, "output buffers hold %llu synapses, %llu needed", (unsigned long long)syn_cap,
            (unsigned long long)E);
  if (weight->kind != SNN_W_CONST && weight->kind != SNN_W_NORMAL_SIGN) NA_FAIL(SNN_EINVAL, "bad weight distribution");

  // delay table (same host computation as snn_connect)
  uint32_t d_smin = 0;
  std::vector<uint32_t> thr;
  if (delay->kind == SNN_D_NORMAL_MIN) {
    if (!(delay->sd > 0) || host_delay_table(delay->mean, delay->sd, delay->lo, dt_ms, &d_smin, &thr) != SNN_OK)
      NA_FAIL(SNN_EINVAL, "bad delay distribution or mass above 255 steps");
  } else if (delay->kind == SNN_D_CONST) {
    d_smin = host_const_delay_steps(delay->mean, dt_ms);
    if (d_smin > 255) NA_FAIL(SNN_EINVAL, "delay above 255 steps");
  } else {
    NA_FAIL(SNN_EINVAL, "bad delay distribution");
  }
  const uint32_t dmax = d_smin + (uint32_t)thr.size();

  Scratch* sc = nullptr;
  int rc = scratch_address(&sc, msg, mlen);
  if (rc != SNN_OK) return rc;
  int dev = 0, num_sms = 0;
  NA_CK(cudaGetDevice(&dev));
  NA_CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));

  // geometry of a single rank: key = (source << db) | delay
  auto bits_for = [](uint64_t v) { uint32_t b = 0; while (b < 64 && (v >> b) != 0) ++b; return b; };
  Geom g{};
  g.R = 1; g.N = n_neurons; g.rb = 0;
  g.sb = bits_for(n_neurons - 1);
  g.db = bits_for(dmax);
  g.key_bits = g.sb + g.db;
  g.cbits = std::max(1u, bits_for(E - 1));
  g.magic_R = magic_for(1);
  const uint32_t passes = (g.key_bits + 7) / 8;
  if (passes > kMaxPasses || g.key_bits + g.cbits > 64) NA_FAIL(SNN_EINVAL, "network too large");
  uint8_t pass_bits[8] = {0}, pass_shift[8] = {0};
  for (uint32_t p = 0, sh = 0; p < passes; ++p) {     // 8-bit digits, the last one narrower
    pass_bits[p] = (uint8_t)std::min(8u, g.key_bits - sh);
    pass_shift[p] = (uint8_t)sh;
    sh += pass_bits[p];
  }

  DevProj P{};
  P.src_first = src_first; P.n_src = n_src; P.src_stride = 1;
  P.tgt_first = tgt_first; P.n_tgt = n_tgt; P.tgt_stride = 1;
  P.rule = (uint32_t)rule->kind; P.proj_id = 0; P.seed = seed;
  P.K = rule->kind == SNN_RULE_FIXED_INDEGREE ? (uint64_t)rule->param : 0;
  P.N = rule->kind == SNN_RULE_FIXED_TOTAL ? (uint64_t)rule->param : 0;
  P.cbase = 0; P.csize = E;
  P.magic_div = rule->kind == SNN_RULE_FIXED_INDEGREE ? magic_for(P.K) : magic_for(n_src);
  P.w_kind = weight->kind == SNN_W_CONST ? 0 : 1;
  P.w_mean = (float)weight->mean; P.w_sd = (float)weight->sd;
  P.d_kind = delay->kind == SNN_D_CONST ? 0 : 1;
  P.d_const = d_smin; P.d_tbl_off = 0; P.d_tbl_len = (uint32_t)thr.size();
  DevBlock B{};
  B.out_base = 0; B.count = E; B.tile_first = 0; B.rank = 0; B.proj = 0;
  B.ti0 = 0; B.tstep = 1; B.n_t = n_tgt;
  const uint64_t n_gen_tiles = (E + 4095) / 4096;
  const uint64_t n_sort_tiles = (E + kTile - 1) / kTile;
  const uint64_t seg_start[2] = {0, E};
  const uint64_t seg_tile0[2] = {0, n_sort_tiles};
  const uint64_t cbase[1] = {0};
  const uint32_t dense_off[4] = {0, 0, 0, 0};

  // inputs into the scratch; everything that must start at zero is cleared
  NA_CK(cudaMemcpyAsync(&sc->proj, &P, sizeof(P), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(&sc->block, &B, sizeof(B), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(sc->seg_start, seg_start, sizeof(seg_start), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(sc->seg_tile0, seg_tile0, sizeof(seg_tile0), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(sc->cbase, cbase, sizeof(cbase), cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(sc->dense_off, dense_off, sizeof(dense_off), cudaMemcpyHostToDevice, st));
  if (!thr.empty())
    NA_CK(cudaMemcpyAsync(sc->dtab, thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemsetAsync(sc->hist, 0, sizeof(sc->hist), st));
  NA_CK(cudaMemsetAsync(sc->status, 0, n_sort_tiles * kBins * sizeof(uint64_t), st));
  NA_CK(cudaMemsetAsync(sc->counters, 0, sizeof(sc->counters), st));
  NA_CK(cudaMemsetAsync(sc->err, 0, sizeof(sc->err), st));

  BuildArgs a{};
  a.blocks = &sc->block; a.nblocks = 1; a.n_gen_tiles = n_gen_tiles;
  a.projs = &sc->proj; a.nproj = 1; a.dtables = sc->dtab; a.g = g;
  a.rec_a = sc->rec_a; a.rec_b = sc->rec_b; a.hist = sc->hist; a.bin_base = sc->bin_base;
  a.seg_start = sc->seg_start; a.seg_tile0 = sc->seg_tile0; a.status = sc->status;
  a.counters = sc->counters; a.err = sc->err; a.passes = passes; a.radix_bits = 8;
  a.n_sort_tiles = n_sort_tiles; a.cbase_sorted = sc->cbase; a.num_sms = num_sms;
  a.dense_off = sc->dense_off;
  a.tgt = dev_tgt; a.w = dev_w; a.d = dev_d; a.w_format = 0;
  a.dense = dev_row_ptr; a.row_scale_src = nullptr;
  a.dense_seg0 = 0; a.dense_nseg = 1;
  a.fuse_hist = 1;
  a.sort_items = 0;                        // records per thread giving kTile-record tiles
  for (uint32_t it : {8u, 12u, 16u})
    if (sort_tile_items(it) == kTile) a.sort_items = it;
  if (a.sort_items == 0) NA_FAIL(SNN_ECUDA, "no sort tile shape of %llu records", (unsigned long long)kTile);
  for (int p = 0; p < 8; ++p) { a.pass_bits[p] = pass_bits[p]; a.pass_shift[p] = pass_shift[p]; }

  NA_CK(launch_generate(a, st));
  NA_CK(launch_bin_scan(a, st));
  uint64_t* cur = sc->rec_a;
  uint64_t* oth = sc->rec_b;
  for (uint32_t p = 0; p < passes; ++p) {
    NA_CK(launch_sort_pass(a, p, cur, oth, p + 1, st));
    std::swap(cur, oth);
  }
  NA_CK(launch_finalize(a, cur, E, st));
  uint32_t herr = 0;
  NA_CK(cudaMemcpyAsync(&herr, sc->err, 4, cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if (herr & kErrTimeout) NA_FAIL(SNN_ETIMEOUT, "a bounded device wait gave up");
  if (herr) NA_FAIL(SNN_ECUDA, "device-side bounds check failed");
  return SNN_OK;
#undef NA_CK
#undef NA_FAIL
}
