// snn_internal.cuh -- internal declarations shared by the library's translation units.
//
// Record layout of the construction sort (one uint64 per synapse):
//     record = key << cbits | cidx
//     key    = (slot << (sb + db)) | (s << db) | d
// slot is the source rank seen from the target rank (0 = local, then the other ranks
// in ascending order), s the source's rank-local index, d the delay in steps and
// cidx the synapse's global generation counter (projection counter base + projection-
// local counter).  Sorting by the key with a stable LSD radix sort over records that
// were written in generation order reproduces "sorted by source as first key, then
// delay, ties in generation order" (paper, Methods, "GPU memory levels": one source's
// connections are (first index, count)), and cidx lets the last stage regenerate the
// target and weight of every synapse from the counter-based generator.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace snn {

constexpr uint32_t kPurposeSynapse = 0;
constexpr uint32_t kPurposeFtTarget = 1;
constexpr uint32_t kPurposePbTest = 2;
constexpr uint32_t kPurposePoisson = 3;
constexpr uint32_t kPurposeVinit = 4;
constexpr uint32_t kPurposePbGap = 5;
constexpr uint32_t kPurposeProbe = 6;     // targets of the ring-reduction probe (no step of the method)

constexpr uint32_t kRuleFixedIndegree = 0;
constexpr uint32_t kRuleFixedTotal = 1;
constexpr uint32_t kRulePairwiseBernoulli = 2;
constexpr uint32_t kRuleBernoulliGeometric = 3;   // pairwise Bernoulli by geometric gaps
// all-to-all and one-to-one run as fixed in-degree (K = n_src, K = 1) with a fixed source
constexpr uint32_t kSrcAll = 1, kSrcOneToOne = 2;

// device error word bits
constexpr uint32_t kErrTimeout = 1u;
constexpr uint32_t kErrBounds = 2u;

// Philox-4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 bijection with the
// published multipliers and Weyl key increments.  On the device each 32 x 32 product's
// high and low words come from two 32-bit multiplies: the same integers, and they issue
// faster than one widening multiply (generation of the 5.625G-synapse network 36.1 ->
// 32.2 ms on a GB300).
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
    const uint32_t h0 = __umulhi(0xD2511F53u, c.x), l0 = 0xD2511F53u * c.x;
    const uint32_t h1 = __umulhi(0xCD9E8D57u, c.z), l1 = 0xCD9E8D57u * c.z;
    c = make_uint4(h1 ^ c.y ^ k.x, l1, h0 ^ c.w ^ k.y, l0);
#else
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
#endif
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__host__ __device__ __forceinline__ uint4 philox_stream(uint64_t counter, uint32_t word2,
                                                        uint32_t purpose, uint64_t seed) {
  return philox4x32_10(make_uint4((uint32_t)counter, (uint32_t)(counter >> 32), word2, purpose),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// integer in [0, n): high word of w * n
__device__ __forceinline__ uint32_t uniform_index(uint32_t w, uint32_t n) { return __umulhi(w, n); }

// uniform in (0, 1): ((w >> 9) + 0.5) * 2^-23, exact in fp32
__device__ __forceinline__ float u01(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-07f;
}

// floor(n / d) for 64-bit n with m = floor(2^64 / d) (2^64 - 1 for d = 1)
__host__ __device__ __forceinline__ uint64_t div_magic(uint64_t n, uint64_t d, uint64_t m) {
#ifdef __CUDA_ARCH__
  uint64_t q = __umul64hi(n, m);
#else
  uint64_t q = (uint64_t)(((unsigned __int128)n * m) >> 64);
#endif
  if (n - q * d >= d) ++q;
  return q;
}

inline uint64_t magic_for(uint64_t d) {
  return d <= 1 ? ~0ull : (uint64_t)(((unsigned __int128)1 << 64) / d);
}

struct DevProj {
  uint32_t src_first, n_src, src_stride;
  uint32_t tgt_first, n_tgt, tgt_stride;
  uint32_t rule, proj_id;
  uint32_t src_mode;        // fixed in-degree shape: 0 random source, kSrcAll (source = k),
  uint32_t src_pad;         // kSrcOneToOne (source = target index)
  uint64_t K, N;            // fixed in-degree K / fixed total N
  uint64_t pb_thr;          // Bernoulli threshold (<= 2^32)
  uint64_t cbase, csize;    // global counter base and size
  uint64_t seed;
  uint64_t magic_div;       // floor(2^64 / K) (FI) or floor(2^64 / n_src) (PB)
  uint32_t w_kind;          // 0 const, 1 normal_sign
  float w_mean, w_sd;
  uint32_t d_kind;          // 0 const, 1 table
  uint32_t d_const;         // constant steps, or s_min of the table
  uint32_t d_tbl_off, d_tbl_len;
  uint32_t g_tbl_off, g_tbl_len;   // gap table of pairwise Bernoulli by geometric gaps
};

// one generation block: the records of projection `proj` whose targets live on `rank`
struct DevBlock {
  uint64_t out_base;   // absolute position of the block's first record
  uint64_t count;      // records in the block
  uint64_t tile_first; // first generation tile
  uint32_t rank, proj;
  uint32_t ti0, tstep; // targets i = ti0 + m * tstep (projection-local index)
  uint32_t n_t, pad;
};

struct Geom {
  uint32_t R, rb, sb, db, key_bits, cbits;
  uint32_t N;               // neurons
  uint32_t pad;
  uint64_t magic_R;         // floor(2^64 / R)
};

struct DevPop {
  float P22, P20, P11ex, P11in, P21ex, P21in, Ie, Vth, Vreset;
  uint32_t ref_steps;
};

struct DevDrive {
  uint32_t first, n;
  float weight;
  uint32_t idx;
  uint64_t seed;
  uint32_t tbl_off, tbl_len;
};

__device__ __forceinline__ uint32_t upper_bound_u32(const uint32_t* a, uint32_t n, uint32_t v) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint32_t upper_bound_u64(const uint64_t* a, uint32_t n, uint64_t v) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ---- launchers (build.cu) ----
struct BuildArgs {
  const DevBlock* blocks; uint32_t nblocks; uint64_t n_gen_tiles;
  const DevProj* projs; uint32_t nproj;
  const uint32_t* dtables;
  Geom g;
  uint64_t* rec_a; uint64_t* rec_b;
  uint64_t* hist;           // [R][passes][bins]
  uint64_t* bin_base;       // [R][passes][bins]
  const uint64_t* seg_start;  // [R+1]
  const uint64_t* seg_tile0;  // [R+1] sort tiles
  uint64_t* status;
  uint32_t* counters;       // [passes] tile counters
  uint32_t* err;
  uint32_t passes, radix_bits;
  uint64_t n_sort_tiles;
  const uint64_t* cbase_sorted;   // [nproj] cbase of projections in id order
  uint32_t* tgt; void* w; uint8_t* d; uint32_t w_format;
  uint64_t* dense;          // [dense_nseg][N+1] row starts (absolute) of segments dense_seg0 ..
  uint32_t dense_seg0, dense_nseg;   // all ranks: 0, R; a dry run: its one rank
  const uint32_t* dense_off;  // [R][R]
  const float* row_scale_src; // per source gid (fp16 format) or null
  int num_sms;
  uint32_t fuse_hist;         // generation accumulates the sort histograms itself
  uint32_t pos_counters;      // records carry their generation position, not the counter
                              // (one uncounted block per projection: a dry run)
  uint32_t sort_items;        // records per thread of a sort tile (tile = 256 x items)
  // pass plan: digit p is (key >> pass_shift[p]) & ((1 << pass_bits[p]) - 1); histogram
  // and bin arrays use kHistStride bins per pass
  uint8_t pass_shift[8], pass_bits[8];
};
constexpr uint32_t kHistStride = 1024;     // bins of the widest (10-bit) digit

// counted generation (fixed total over several ranks; pairwise Bernoulli): the
// records of such a projection land in (rank, projection) blocks whose sizes are
// counted first, so their placement needs a count / scan / place sequence.
struct CountedArgs {
  const DevProj* projs;
  uint32_t R; uint64_t magic_R;
  // fixed total over several ranks: tiles of kCountTile draws
  const uint32_t* ft_proj;        // [n_ft] projection ids
  const uint64_t* ft_tile_first;  // [n_ft + 1]
  uint32_t n_ft; uint64_t n_ft_tiles;
  uint32_t* ft_tile_cnt;          // [n_ft_tiles][R]
  uint64_t* ft_tile_off;          // [n_ft_tiles][R]
  uint64_t* ft_tot;               // [n_ft][R]
  // pairwise Bernoulli: one counter per target
  const uint32_t* pb_proj;        // [n_pb]
  const uint64_t* pb_t_first;     // [n_pb + 1] first target slot of each projection
  uint32_t n_pb; uint64_t n_pb_targets;
  uint32_t* pb_cnt;               // [n_pb_targets] by projection-local target index
  uint64_t* pb_off;               // [n_pb_targets] offset of the target within its block
  uint64_t* pb_tot;               // [n_pb][R]
  const uint64_t* block_base;     // [nproj][R] absolute first record of block (p, rank)
  const uint32_t* tables;         // delay and gap tables (BuildArgs::dtables)
};
constexpr uint32_t kCountTile = 4096;
constexpr uint32_t kMaxCountedRanks = 1024;

cudaError_t launch_counted_count(const CountedArgs& c, cudaStream_t st, int num_sms);
cudaError_t launch_counted_place(const CountedArgs& c, const BuildArgs& a, cudaStream_t st);
cudaError_t launch_histogram(const BuildArgs& a, cudaStream_t st);
cudaError_t launch_bounded_wait_selftest(uint64_t* status, uint32_t* err, cudaStream_t st);

cudaError_t launch_generate(const BuildArgs& a, cudaStream_t st);
cudaError_t launch_bin_scan(const BuildArgs& a, cudaStream_t st);
cudaError_t launch_sort_pass(const BuildArgs& a, uint32_t pass, const uint64_t* in, uint64_t* out,
                             uint32_t epoch, cudaStream_t st);
cudaError_t launch_finalize(const BuildArgs& a, const uint64_t* rec, uint64_t E, cudaStream_t st);
uint32_t sort_tile_items(uint32_t items);
bool sort_config_supported(uint32_t radix_bits, uint32_t items);

}  // namespace snn
