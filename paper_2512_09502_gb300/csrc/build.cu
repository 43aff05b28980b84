// build.cu -- on-device network construction: connection generation, the
// source/delay radix sort, and the final per-rank CSR layout.
//
// Paper: Methods, "Creation of the remote connection structures for point-to-point
// MPI communication" (connections generated in GPU memory from the rule dictionary,
// sorted by source), "GPU memory levels" (sorted by source as first key so that one
// source's connections are (first index, count)).  The per-rank structure (targets on
// their rank, remote sources as image rows) follows "Remote connections".
//
// Pipeline (one launch each, every projection and every logical rank batched):
//   gen_kernel       counter-based generation of all records, written in generation
//                    order into their rank segment, with the digit histograms of every
//                    sort pass accumulated on the fly (no extra read of the records);
//   bin_scan_kernel  exclusive scan of the histograms -> global bin bases;
//   onesweep_pass    one stable LSD pass per 8- to 10-bit digit over 8,192-record tiles:
//                    warp ranking from digit-bit ballots, shared-memory staging so that each
//                    digit run is written contiguously, then a decoupled look-back over
//                    the segment's earlier tiles (bounded spin) for the global offsets;
//   finalize_kernel  decodes the sorted records: rank-local target, weight
//                    (regenerated from the counter), delay; writes the SoA arrays and
//                    the dense row starts (the CSR) from record boundaries.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "snn_internal.cuh"

namespace snn {

constexpr int GEN_BLOCK = 256;
constexpr int GEN_TILE = 4096;
constexpr int SORT_BLOCK = 512;
constexpr int SORT_MIN_CTAS = 2;       // resident sort CTAs per SM (64 registers: 32 warps)
constexpr int MAX_PASSES = 6;
constexpr uint32_t SPIN_LIMIT = 1u << 22;


// ---------------------------------------------------------------------------
// generation
// ---------------------------------------------------------------------------
// Inverse of an integer CDF table: #{i : thr[i] <= w}.  The guide table (Chen & Asau's
// indexed search) holds the count at the start of each 2^24-wide window of w, so the
// search starts there and needs at most a few compares; the result equals a plain
// binary search.
constexpr int GUIDE_BITS = 12;      // guide cells: the top 12 bits of the uniform word

__device__ __forceinline__ uint32_t guided_count(const uint32_t* thr, uint32_t len, const uint8_t* guide,
                                                 uint32_t w) {
  uint32_t c = guide[w >> (32 - GUIDE_BITS)];
  while (c < len && thr[c] <= w) ++c;
  return c;
}

// Generation modes of a block: fixed in-degree with a random source (word x of the
// synapse's Philox block), all-to-all (source = k), one-to-one (source = the target's
// index), and fixed total number on one rank (draw index = counter, random source).
constexpr int GenRandom = 0, GenAll = 1, GenOneToOne = 2, GenFixedTotal = 3;

// The items of one generation tile: records e0 .. e0 + n - 1 of block blk.  ONE32: one
// rank, counters as record ids and a key of at most 32 bits with its digit histograms
// fused (the common case): no source-rank slot, 32-bit digit extraction.
struct DigitPlan {
  uint32_t sh[MAX_PASSES], mk[MAX_PASSES];   // digit p = (key >> sh[p]) & mk[p]; mk = 0: no pass
};

template <int MODE, bool DTAB, bool ONE32>
__device__ __forceinline__ void gen_items(const BuildArgs& a, const DevBlock& blk, const DevProj& P,
                                          const uint32_t* s_tbl, const uint8_t* s_guide,
                                          uint32_t (*s_hist)[kHistStride], uint64_t e0, uint32_t n,
                                          const DigitPlan& dp, bool fuse_hist) {
  const Geom g = a.g;
  const int tid = threadIdx.x;
  const uint64_t cmask = g.cbits >= 64 ? ~0ull : ((1ull << g.cbits) - 1);
  const uint2 key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
  constexpr bool FI = MODE != GenFixedTotal;
  // fixed in-degree: (target m, k) of this thread's first item, then incremental
  uint64_t m = 0;
  uint32_t k = 0;
  if (FI) {
    const uint64_t e = e0 + tid;
    m = div_magic(e, P.K, P.magic_div);
    k = (uint32_t)(e - m * P.K);
  }
  const uint64_t cstep = (uint64_t)blk.tstep * P.K;
  uint64_t cm = ((uint64_t)blk.ti0 + m * blk.tstep) * P.K;   // counter of (target m, k = 0)
  const uint32_t Kk = (uint32_t)P.K;
  const uint64_t obase = blk.out_base;
  const uint64_t cbase = P.cbase;
  // the projection's fields in registers: the loop's shared-memory histogram increments
  // would otherwise make the compiler reload them from the shared copy every item
  const uint32_t proj_id = P.proj_id, n_src = P.n_src, src_first = P.src_first, src_stride = P.src_stride;
  const uint32_t d_const = P.d_const, d_len = P.d_tbl_len;
  for (uint32_t i = tid; i < n; i += GEN_BLOCK) {
    const uint64_t e = e0 + i;
    const uint64_t c = FI ? cm + k : e;
    const uint4 b = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), proj_id, kPurposeSynapse), key);
    const uint32_t si = MODE == GenAll ? k : (MODE == GenOneToOne ? (uint32_t)c : uniform_index(b.x, n_src));
    const uint32_t src = src_first + si * src_stride;
    uint32_t d = d_const;
    if (DTAB) d += guided_count(s_tbl, d_len, s_guide, b.y);
    if (ONE32) {
      const uint32_t k32 = (src << g.db) | d;
      a.rec_a[obase + e] = ((uint64_t)k32 << g.cbits) | ((cbase + c) & cmask);
#pragma unroll
      for (int p = 0; p < MAX_PASSES; ++p)
        if (dp.mk[p]) atomicAdd(&s_hist[p][(k32 >> dp.sh[p]) & dp.mk[p]], 1u);
    } else {
      uint32_t sig = 0, s = src;
      if (g.R > 1) {
        s = (uint32_t)div_magic(src, g.R, g.magic_R);
        sig = src - s * g.R;
      }
      const uint32_t slot = sig == blk.rank ? 0u : (sig < blk.rank ? sig + 1 : sig);
      const uint64_t kk = ((uint64_t)slot << (g.sb + g.db)) | ((uint64_t)s << g.db) | d;
      const uint64_t cid = a.pos_counters ? obase + e : cbase + c;
      a.rec_a[obase + e] = (kk << g.cbits) | (cid & cmask);
      if (fuse_hist) {
        if (g.key_bits <= 32) {
          const uint32_t k32 = (uint32_t)kk;
#pragma unroll
          for (int p = 0; p < MAX_PASSES; ++p)
            if (dp.mk[p]) atomicAdd(&s_hist[p][(k32 >> dp.sh[p]) & dp.mk[p]], 1u);
        } else {
#pragma unroll
          for (int p = 0; p < MAX_PASSES; ++p)
            if (dp.mk[p]) atomicAdd(&s_hist[p][(uint32_t)(kk >> dp.sh[p]) & dp.mk[p]], 1u);
        }
      }
    }
    if (FI) {                     // advance to item i + GEN_BLOCK
      k += GEN_BLOCK;
      while (k >= Kk) {
        k -= Kk;
        cm += cstep;
      }
    }
  }
}

__global__ void __launch_bounds__(GEN_BLOCK) gen_kernel(BuildArgs a) {
  constexpr int BINS = kHistStride;
  __shared__ uint32_t s_hist[MAX_PASSES][BINS];
  __shared__ uint32_t s_tbl[256];
  __shared__ uint8_t s_guide[1 << GUIDE_BITS];
  __shared__ DevBlock s_blk;
  __shared__ DevProj s_proj;
  const int tid = threadIdx.x;
  const Geom g = a.g;
  const uint32_t passes = a.passes;
  for (int i = tid; i < MAX_PASSES * BINS; i += GEN_BLOCK) (&s_hist[0][0])[i] = 0;
  // per-pass digit extraction of the sort key
  DigitPlan dp;
#pragma unroll
  for (int p = 0; p < MAX_PASSES; ++p) {
    dp.sh[p] = a.pass_shift[p];
    dp.mk[p] = p < (int)passes ? (1u << a.pass_bits[p]) - 1 : 0u;
  }
  const bool hist = a.fuse_hist && g.key_bits <= 32;

  const uint64_t per = (a.n_gen_tiles + gridDim.x - 1) / gridDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * per;
  const uint64_t t1 = min(t0 + per, a.n_gen_tiles);
  int cur_rank = -1;

  uint32_t cur_tbl = 0xFFFFFFFFu;      // delay table staged in s_tbl / s_guide
  for (uint64_t tile = t0; tile < t1; ++tile) {
    __syncthreads();
    if (tid == 0) {
      uint32_t lo = 0, hi = a.nblocks;   // last block with tile_first <= tile
      while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (a.blocks[mid].tile_first <= tile) lo = mid + 1; else hi = mid;
      }
      s_blk = a.blocks[lo - 1];
      s_proj = a.projs[s_blk.proj];
    }
    __syncthreads();
    const DevBlock blk = s_blk;
    const DevProj& P = s_proj;
    if ((int)blk.rank != cur_rank) {          // flush the previous segment's histogram
      if (cur_rank >= 0) {
        for (int i = tid; i < (int)passes * BINS; i += GEN_BLOCK) {
          const uint32_t v = (&s_hist[0][0])[i];
          if (v) atomicAdd((unsigned long long*)&a.hist[((uint64_t)cur_rank * passes) * BINS + i], v);
          (&s_hist[0][0])[i] = 0;
        }
      }
      cur_rank = blk.rank;
    }
    if (P.d_kind == 1 && P.d_tbl_off != cur_tbl) {   // block-uniform: P is shared
      // stage the delay table and its guide only when the projection's table changes
      for (uint32_t i = tid; i < P.d_tbl_len; i += GEN_BLOCK) s_tbl[i] = a.dtables[P.d_tbl_off + i];
      __syncthreads();
      for (uint32_t cell = tid; cell < (1u << GUIDE_BITS); cell += GEN_BLOCK)
        s_guide[cell] = (uint8_t)upper_bound_u32(s_tbl, P.d_tbl_len, cell << (32 - GUIDE_BITS));
      __syncthreads();
      cur_tbl = P.d_tbl_off;
    }

    const uint64_t e0 = (tile - blk.tile_first) * (uint64_t)GEN_TILE;
    const uint32_t n = (uint32_t)min((uint64_t)GEN_TILE, blk.count - e0);
    // the item loop, specialised per source mode, delay kind and key form (block-uniform
    // choices taken once per tile instead of once per synapse)
    const bool fi = P.rule == kRuleFixedIndegree;
    const int mode = !fi ? GenFixedTotal : (P.src_mode == kSrcAll ? GenAll
                                          : (P.src_mode == kSrcOneToOne ? GenOneToOne : GenRandom));
    const bool one32 = g.R == 1 && hist && !a.pos_counters;
    const bool dtab = P.d_kind == 1;
#define SNN_GEN_CASE(M_, D_, O_) \
    if (mode == M_ && dtab == D_ && one32 == O_) gen_items<M_, D_, O_>(a, blk, P, s_tbl, s_guide, s_hist, e0, n, dp, a.fuse_hist);
    SNN_GEN_CASE(GenRandom, true, true) SNN_GEN_CASE(GenRandom, true, false)
    SNN_GEN_CASE(GenRandom, false, true) SNN_GEN_CASE(GenRandom, false, false)
    SNN_GEN_CASE(GenAll, true, true) SNN_GEN_CASE(GenAll, true, false)
    SNN_GEN_CASE(GenAll, false, true) SNN_GEN_CASE(GenAll, false, false)
    SNN_GEN_CASE(GenOneToOne, true, true) SNN_GEN_CASE(GenOneToOne, true, false)
    SNN_GEN_CASE(GenOneToOne, false, true) SNN_GEN_CASE(GenOneToOne, false, false)
    SNN_GEN_CASE(GenFixedTotal, true, true) SNN_GEN_CASE(GenFixedTotal, true, false)
    SNN_GEN_CASE(GenFixedTotal, false, true) SNN_GEN_CASE(GenFixedTotal, false, false)
#undef SNN_GEN_CASE
  }
  __syncthreads();
  if (cur_rank >= 0) {
    for (int i = tid; i < (int)passes * BINS; i += GEN_BLOCK) {
      const uint32_t v = (&s_hist[0][0])[i];
      if (v) atomicAdd((unsigned long long*)&a.hist[((uint64_t)cur_rank * passes) * BINS + i], v);
    }
  }
}

cudaError_t launch_generate(const BuildArgs& a, cudaStream_t st) {
  if (a.n_gen_tiles == 0) return cudaSuccess;
  const uint64_t grid = std::min<uint64_t>(a.n_gen_tiles, (uint64_t)a.num_sms * 8);
  gen_kernel<<<(unsigned)grid, GEN_BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// histogram scan -> bin bases (absolute positions)
// ---------------------------------------------------------------------------
__global__ void bin_scan_kernel(BuildArgs a) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.g.R * a.passes) return;
  const uint32_t r = i / a.passes, p = i - r * a.passes;
  const uint32_t bins = 1u << a.pass_bits[p];
  uint64_t acc = a.seg_start[r];
  for (uint32_t b = 0; b < bins; ++b) {
    a.bin_base[(uint64_t)i * kHistStride + b] = acc;
    acc += a.hist[(uint64_t)i * kHistStride + b];
  }
}

cudaError_t launch_bin_scan(const BuildArgs& a, cudaStream_t st) {
  const uint32_t n = a.g.R * a.passes;
  if (n == 0) return cudaSuccess;
  bin_scan_kernel<<<(n + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// one stable LSD pass (onesweep: Adinets & Merrill 2022)
// ---------------------------------------------------------------------------
constexpr uint64_t ST_AGG = 1ull << 62;
constexpr uint64_t ST_INC = 2ull << 62;
constexpr uint64_t ST_VAL = (1ull << 46) - 1;

__device__ __forceinline__ uint64_t ld_status(const uint64_t* p) {
  return *(const volatile unsigned long long*)p;
}
__device__ __forceinline__ void st_status(uint64_t* p, uint64_t v) {
  *(volatile unsigned long long*)p = v;
}

// Per-warp digit counts are 32-bit for 8- and 9-bit digits and 16-bit for 10-bit ones
// (a warp's running counts, then their exclusive scan over warps, stay below the
// 8,192-record tile), so that two 10-bit tiles of 16 records per thread still fit an SM.
template <int RB>
using WarpCount = typename std::conditional<(RB >= 10), uint16_t, uint32_t>::type;

template <int RB, int ITEMS>
struct SortSmem {
  static constexpr int BINS = 1 << RB;
  static constexpr int NW = SORT_BLOCK / 32;
  uint64_t stage[SORT_BLOCK * ITEMS];
  uint64_t gbase[BINS];
  WarpCount<RB> whist[NW][BINS];
  uint32_t binstart[BINS];
  uint32_t wsum[NW];
  uint32_t tile;
};

// Exclusive prefix of bin b over the predecessor tiles of this segment: sum the
// aggregates of earlier tiles until one carries an inclusive prefix.  Four status
// words are requested per round trip; a word that is not ready yet is polled with a
// bounded wait (a global error flag short-cuts every other wait once one gave up).
__device__ __forceinline__ uint64_t look_back(const BuildArgs& a, uint64_t tile, uint64_t first_tile,
                                              uint32_t b, uint32_t bins, uint32_t epoch) {
  constexpr int W = 4;
  const uint64_t ep = (uint64_t)(epoch & 0xFFFF) << 46;
  uint64_t excl = 0;
  uint64_t k = tile - 1;                    // tile > first_tile here
  while (true) {
    uint64_t st[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
      st[w] = (k >= first_tile + w) ? ld_status(a.status + (k - w) * bins + b) : 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      uint64_t s = st[w];
      const uint64_t* sp = a.status + (k - w) * bins + b;
      uint32_t spins = 0;
      while (((s >> 62) == 0) || (((s >> 46) & 0xFFFF) != (epoch & 0xFFFF))) {
        if (++spins > SPIN_LIMIT || (*(volatile uint32_t*)a.err & kErrTimeout)) {
          atomicOr(a.err, kErrTimeout);
          s = ST_INC | ep;
          break;
        }
        __nanosleep(32);
        s = ld_status(sp);
      }
      excl += s & ST_VAL;
      if ((s >> 62) == 2) return excl;      // the segment's first tile is always inclusive
    }
    k -= W;
  }
}

// Two adjacent status words (bins b and b + 1, b even: one 16-byte access)
__device__ __forceinline__ ulonglong2 ld_status2(const uint64_t* p) {
  ulonglong2 v;
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_status2(uint64_t* p, uint64_t v0, uint64_t v1) {
  asm volatile("st.volatile.global.v2.u64 [%0], {%1, %2};" :: "l"(p), "l"(v0), "l"(v1) : "memory");
}
__device__ __forceinline__ bool status_ready(uint64_t s, uint32_t epoch) {
  return (s >> 62) != 0 && ((s >> 46) & 0xFFFF) == (epoch & 0xFFFF);
}

// look_back for the bins b0 and b0 + 1 of one thread (10-bit digits: two bins per
// thread) in one walk: each predecessor's pair of status words is one 16-byte load, and
// the walk ends when both bins have met an inclusive prefix.  The same bounded wait.
__device__ __forceinline__ void look_back2(const BuildArgs& a, uint64_t tile, uint64_t first_tile, uint32_t b0,
                                           uint32_t bins, uint32_t epoch, uint64_t& ex0, uint64_t& ex1) {
  constexpr int W = 4;
  ex0 = 0;
  ex1 = 0;
  bool done0 = false, done1 = false;
  uint64_t k = tile - 1;                    // tile > first_tile here
  while (true) {
    ulonglong2 st[W];
#pragma unroll
    for (int w = 0; w < W; ++w)
      st[w] = (k >= first_tile + w) ? ld_status2(a.status + (k - w) * bins + b0) : make_ulonglong2(0, 0);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      ulonglong2 s = st[w];
      const uint64_t* sp = a.status + (k - w) * bins + b0;
      uint32_t spins = 0;
      while ((!done0 && !status_ready(s.x, epoch)) || (!done1 && !status_ready(s.y, epoch))) {
        if (++spins > SPIN_LIMIT || (*(volatile uint32_t*)a.err & kErrTimeout)) {
          atomicOr(a.err, kErrTimeout);
          return;
        }
        __nanosleep(32);
        s = ld_status2(sp);
      }
      if (!done0) {
        ex0 += s.x & ST_VAL;
        done0 = (s.x >> 62) == 2;
      }
      if (!done1) {
        ex1 += s.y & ST_VAL;
        done1 = (s.y >> 62) == 2;
      }
      if (done0 && done1) return;           // the segment's first tile is always inclusive
    }
    k -= W;
  }
}

// Self-test of the bounded wait: tile 1 looks back at tile 0, whose status is never
// published, so every bin's wait must give up and flag kErrTimeout.
__global__ void bounded_wait_selftest(BuildArgs a, uint32_t bins) {
  if (threadIdx.x < bins) (void)look_back(a, 1, 0, threadIdx.x, bins, 1);
}

cudaError_t launch_bounded_wait_selftest(uint64_t* status, uint32_t* err, cudaStream_t st) {
  BuildArgs a{};
  a.status = status;
  a.err = err;
  bounded_wait_selftest<<<1, 256, 0, st>>>(a, 256);
  return cudaGetLastError();
}

template <int RB, int ITEMS, bool HI>
__global__ void __launch_bounds__(SORT_BLOCK, SORT_MIN_CTAS) onesweep_pass(BuildArgs a, uint32_t pass,
                                                             const uint64_t* __restrict__ in,
                                                             uint64_t* __restrict__ out,
                                                             uint32_t epoch) {
  constexpr int BINS = 1 << RB;
  constexpr int NW = SORT_BLOCK / 32;
  constexpr int BPT = (BINS + SORT_BLOCK - 1) / SORT_BLOCK;   // bins per thread
  static_assert(BPT == 1 || BINS == 2 * SORT_BLOCK, "two bins per thread only for 10-bit digits");
  constexpr int TILE = SORT_BLOCK * ITEMS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem<RB, ITEMS>& sm = *reinterpret_cast<SortSmem<RB, ITEMS>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) sm.tile = atomicAdd(&a.counters[pass], 1u);
  for (int i = tid; i < NW * BINS; i += SORT_BLOCK) (&sm.whist[0][0])[i] = 0;
  __syncthreads();
  const uint64_t tile = sm.tile;
  if (tile >= a.n_sort_tiles) return;

  const uint32_t seg = upper_bound_u64(a.seg_tile0, a.g.R, tile) - 1;
  const uint64_t first_tile = a.seg_tile0[seg];
  const uint64_t base = a.seg_start[seg] + (tile - first_tile) * TILE;
  const uint64_t seg_end = a.seg_start[seg + 1];
  const uint32_t n = (uint32_t)min((uint64_t)TILE, seg_end - base);
  const uint32_t shift = a.g.cbits + a.pass_shift[pass];
  const uint64_t dmask = (1ull << a.pass_bits[pass]) - 1;
  // HI: the digit lies in the record's high word (shift >= 32), so a 32-bit shift of that
  // word extracts it (the key and counter fit 64 bits); otherwise the 64-bit shift
  const uint32_t shift_hi = shift - 32;
  auto digit = [&](uint64_t r) -> uint32_t {
    return HI ? (((uint32_t)(r >> 32)) >> shift_hi) & (uint32_t)dmask : (uint32_t)((r >> shift) & dmask);
  };

  uint64_t rec[ITEMS];
  uint32_t rnk[ITEMS];
  const uint32_t wbase = warp * 32 * ITEMS;
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    rec[j] = idx < n ? in[base + idx] : ~0ull;
  }
  // Stable warp-level ranking: item j's peers (lanes holding the same digit) come from
  // one ballot per digit bit, plus one for the out-of-range marker in a partial tile
  // (or from match.any for every fourth item); the leader of each peer group advances
  // the warp's running count of that digit.
  const uint32_t lt = (1u << lane) - 1;
  const int nbits = n == (uint32_t)TILE ? RB : RB + 1;   // the marker bit only in a partial tile
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    const uint32_t d = idx < n ? digit(rec[j]) : (uint32_t)BINS;
    uint32_t peers = 0xffffffffu;
    if ((j & 3) == 3) {
      // every fourth item on the match unit, the rest on ballots: the ballot loop keeps
      // the ALU pipe busy, and match.any runs beside it
      peers = __match_any_sync(0xffffffffu, d);
    } else {
#pragma unroll
      for (int bit = 0; bit <= RB; ++bit) {
        if (bit == RB && nbits == RB) break;
        const uint32_t m = 0u - ((d >> bit) & 1u);
        const uint32_t bl = __ballot_sync(0xffffffffu, m != 0u);
        peers &= ~(bl ^ m);
      }
    }
    const int leader = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == leader && d < BINS) {
      old = sm.whist[warp][d];
      sm.whist[warp][d] = (WarpCount<RB>)(old + __popc(peers));
    }
    old = __shfl_sync(0xffffffffu, old, leader);
    rnk[j] = old + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();

  uint32_t tot[BPT];
  uint32_t tsum = 0;
#pragma unroll
  for (int q = 0; q < BPT; ++q) {
    const int b = tid * BPT + q;
    uint32_t t = 0;
    if (b < BINS) {
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        const uint32_t c = sm.whist[w][b];
        sm.whist[w][b] = (WarpCount<RB>)t;
        t += c;
      }
    }
    tot[q] = t;
    tsum += t;
  }
  const bool first = tile == first_tile;
  const uint64_t ep = (uint64_t)(epoch & 0xFFFF) << 46;
  uint64_t* strow = a.status + tile * BINS;
  if constexpr (BPT == 2) {
    st_status2(strow + tid * 2, (first ? ST_INC : ST_AGG) | ep | tot[0], (first ? ST_INC : ST_AGG) | ep | tot[1]);
  } else {
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int b = tid * BPT + q;
      if (b < BINS) st_status(strow + b, (first ? ST_INC : ST_AGG) | ep | tot[q]);
    }
  }

  // tile-local exclusive scan of the bin counts (thread-contiguous bins)
  uint32_t incl = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) sm.wsum[warp] = incl;
  __syncthreads();
  uint32_t woff = 0;
  for (int w = 0; w < warp; ++w) woff += sm.wsum[w];
  uint32_t bstart[BPT];
  uint32_t run = woff + incl - tsum;
#pragma unroll
  for (int q = 0; q < BPT; ++q) {
    const int b = tid * BPT + q;
    bstart[q] = run;
    if (b < BINS) sm.binstart[b] = run;
    run += tot[q];
  }
  __syncthreads();

  // staging in shared memory needs only tile-local offsets, so it runs before the
  // look-back: the predecessors get that much longer to publish inclusive prefixes
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    if (idx < n) {
      const uint32_t d = digit(rec[j]);
      sm.stage[sm.binstart[d] + sm.whist[warp][d] + rnk[j]] = rec[j];
    }
  }
  const uint64_t* bbase = a.bin_base + ((uint64_t)seg * a.passes + pass) * kHistStride;
  if constexpr (BPT == 2) {        // 10-bit digits: bins 2 tid and 2 tid + 1, one walk
    const uint32_t b0 = (uint32_t)tid * 2;
    uint64_t e0 = 0, e1 = 0;
    if (!first) {
      look_back2(a, tile, first_tile, b0, BINS, epoch, e0, e1);
      st_status2(strow + b0, ST_INC | ep | ((e0 + tot[0]) & ST_VAL), ST_INC | ep | ((e1 + tot[1]) & ST_VAL));
    }
    sm.gbase[b0] = bbase[b0] + e0 - bstart[0];
    sm.gbase[b0 + 1] = bbase[b0 + 1] + e1 - bstart[1];
  } else {
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
      const int b = tid * BPT + q;
      if (b >= BINS) continue;
      uint64_t excl = 0;
      if (!first) {
        excl = look_back(a, tile, first_tile, (uint32_t)b, BINS, epoch);
        st_status(strow + b, ST_INC | ep | ((excl + tot[q]) & ST_VAL));
      }
      // global position of staged element k of bin b = gbase[b] + k
      sm.gbase[b] = bbase[b] + excl - bstart[q];
    }
  }
  __syncthreads();
  for (uint32_t k = tid; k < n; k += SORT_BLOCK) {
    const uint64_t r = sm.stage[k];
    const uint32_t d = digit(r);
    const uint64_t gpos = sm.gbase[d] + k;
    if (gpos < seg_end) out[gpos] = r; else atomicOr(a.err, kErrBounds);
  }
}

template <int RB, int ITEMS, bool HI>
static cudaError_t sort_pass_hi(const BuildArgs& a, uint32_t pass, const uint64_t* in, uint64_t* out,
                                uint32_t epoch, cudaStream_t st) {
  const size_t smem = sizeof(SortSmem<RB, ITEMS>);
  cudaError_t e = cudaFuncSetAttribute(onesweep_pass<RB, ITEMS, HI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  onesweep_pass<RB, ITEMS, HI><<<(unsigned)a.n_sort_tiles, SORT_BLOCK, smem, st>>>(a, pass, in, out, epoch);
  return cudaGetLastError();
}

template <int RB, int ITEMS>
static cudaError_t sort_pass_rb(const BuildArgs& a, uint32_t pass, const uint64_t* in, uint64_t* out,
                                uint32_t epoch, cudaStream_t st) {
  if (a.g.cbits + a.pass_shift[pass] >= 32) return sort_pass_hi<RB, ITEMS, true>(a, pass, in, out, epoch, st);
  return sort_pass_hi<RB, ITEMS, false>(a, pass, in, out, epoch, st);
}

bool sort_config_supported(uint32_t radix_bits, uint32_t items) {
  return radix_bits >= 8 && radix_bits <= 10 && (items == 8 || items == 12 || items == 16);
}

uint32_t sort_tile_items(uint32_t items) { return SORT_BLOCK * items; }

cudaError_t launch_sort_pass(const BuildArgs& a, uint32_t pass, const uint64_t* in, uint64_t* out,
                             uint32_t epoch, cudaStream_t st) {
  if (a.n_sort_tiles == 0) return cudaSuccess;
  // kernel width for this pass's digit
  const uint32_t rb = a.pass_bits[pass] <= 8 ? 8u : (a.pass_bits[pass] <= 9 ? 9u : 10u);
#define SNN_SORT_CASE(RB_, IT_) \
  if (rb == RB_ && a.sort_items == IT_) return sort_pass_rb<RB_, IT_>(a, pass, in, out, epoch, st);
  SNN_SORT_CASE(8, 8) SNN_SORT_CASE(8, 12) SNN_SORT_CASE(8, 16)
  SNN_SORT_CASE(9, 8) SNN_SORT_CASE(9, 12) SNN_SORT_CASE(9, 16)
  SNN_SORT_CASE(10, 8) SNN_SORT_CASE(10, 12) SNN_SORT_CASE(10, 16)
#undef SNN_SORT_CASE
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// counted generation: fixed total over several ranks, pairwise Bernoulli
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rank_of(uint32_t g, uint32_t R, uint64_t magic_R) {
  return g - (uint32_t)div_magic(g, R, magic_R) * R;
}

// record of one synapse (source src, delay from w1) on target rank `rank`
__device__ __forceinline__ uint64_t make_record(const DevProj& P, const Geom& g, uint32_t rank, uint64_t c,
                                                uint32_t src, uint32_t w1, const uint32_t* tbl) {
  uint32_t sig = 0, s = src;
  if (g.R > 1) {
    s = (uint32_t)div_magic(src, g.R, g.magic_R);
    sig = src - s * g.R;
  }
  const uint32_t slot = sig == rank ? 0u : (sig < rank ? sig + 1 : sig);
  uint32_t d = P.d_const;
  if (P.d_kind == 1) d += upper_bound_u32(tbl, P.d_tbl_len, w1);
  const uint64_t kk = ((uint64_t)slot << (g.sb + g.db)) | ((uint64_t)s << g.db) | d;
  const uint64_t cmask = g.cbits >= 64 ? ~0ull : ((1ull << g.cbits) - 1);
  return (kk << g.cbits) | ((P.cbase + c) & cmask);
}

__device__ __forceinline__ uint32_t pb_word(const DevProj& P, uint64_t q) {
  const uint4 tb = philox_stream(q >> 2, P.proj_id, kPurposePbTest, P.seed);
  const uint32_t lane = (uint32_t)(q & 3);
  return lane == 0 ? tb.x : lane == 1 ? tb.y : lane == 2 ? tb.z : tb.w;
}

__global__ void __launch_bounds__(256) ft_count_kernel(CountedArgs c) {
  __shared__ uint32_t s_cnt[kMaxCountedRanks];
  for (uint64_t tile = blockIdx.x; tile < c.n_ft_tiles; tile += gridDim.x) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < c.R; i += blockDim.x) s_cnt[i] = 0;
    const uint32_t q = upper_bound_u64(c.ft_tile_first, c.n_ft, tile) - 1;
    const DevProj& P = c.projs[c.ft_proj[q]];
    __syncthreads();
    const uint64_t j0 = (tile - c.ft_tile_first[q]) * kCountTile;
    const uint32_t n = (uint32_t)min((uint64_t)kCountTile, P.N - j0);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint4 bt = philox_stream(j0 + i, P.proj_id, kPurposeFtTarget, P.seed);
      const uint32_t t = P.tgt_first + uniform_index(bt.x, P.n_tgt) * P.tgt_stride;
      atomicAdd(&s_cnt[rank_of(t, c.R, c.magic_R)], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < c.R; i += blockDim.x) c.ft_tile_cnt[tile * c.R + i] = s_cnt[i];
  }
}

// one thread per (projection, rank): running offsets over the projection's tiles
__global__ void ft_scan_kernel(CountedArgs c) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (uint64_t)c.n_ft * c.R) return;
  const uint32_t q = (uint32_t)(k / c.R), r = (uint32_t)(k - (uint64_t)q * c.R);
  uint64_t acc = 0;
  for (uint64_t t = c.ft_tile_first[q]; t < c.ft_tile_first[q + 1]; ++t) {
    c.ft_tile_off[t * c.R + r] = acc;
    acc += c.ft_tile_cnt[t * c.R + r];
  }
  c.ft_tot[k] = acc;
}

// one warp per target of a Bernoulli projection: pairs kept
// Pairwise Bernoulli by geometric gaps, one warp per target ti: lane l of a round draws
// gap j = j0 + l (word x of the PB_GAP block at counter ti * n_src + j, inverted through
// the gap table) and the warp's prefix sum of (gap + 1) gives the kept sources s_j in
// ascending order; the walk ends with the first round that passes n_src.  Every lane
// calls round(s, kept, mask, rank): kept lanes form a prefix of the warp, mask is the
// ballot of kept lanes and rank the lane's position among them.
template <typename Fn>
__device__ __forceinline__ void geometric_walk(const DevProj& P, const uint32_t* tbl, uint64_t ti, Fn round) {
  const uint32_t lane = threadIdx.x & 31;
  int64_t base = -1;                          // last kept source before this round
  for (uint64_t j0 = 0;; j0 += 32) {
    const uint4 b = philox_stream(ti * P.n_src + j0 + lane, P.proj_id, kPurposePbGap, P.seed);
    const uint64_t step = (uint64_t)upper_bound_u32(tbl, P.g_tbl_len, b.x) + 1;
    uint64_t incl = step;                     // inclusive warp prefix sum of the steps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += v;
    }
    const int64_t s = base + (int64_t)incl;
    const bool keep = s < (int64_t)P.n_src;
    const uint32_t m = __ballot_sync(0xffffffffu, keep);
    round(keep ? (uint32_t)s : 0u, keep, m, (uint32_t)__popc(m & ((1u << lane) - 1)));
    if (m != 0xffffffffu) break;              // a source passed n_src: the walk is done
    base += (int64_t)__shfl_sync(0xffffffffu, incl, 31);
  }
}

__global__ void pb_count_kernel(CountedArgs c) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < c.n_pb_targets; x += nwarps) {
    const uint32_t q = upper_bound_u64(c.pb_t_first, c.n_pb, x) - 1;
    const DevProj& P = c.projs[c.pb_proj[q]];
    const uint64_t ti = x - c.pb_t_first[q];
    uint32_t cnt = 0;
    if (P.rule == kRuleBernoulliGeometric) {
      if (P.pb_thr)
        geometric_walk(P, c.tables + P.g_tbl_off, ti,
                       [&](uint32_t, bool, uint32_t m, uint32_t) { cnt += __popc(m); });
    } else {
      for (uint32_t s0 = 0; s0 < P.n_src; s0 += 32) {
        const uint32_t s = s0 + lane;
        const bool keep = s < P.n_src && (uint64_t)pb_word(P, ti * P.n_src + s) < P.pb_thr;
        cnt += __popc(__ballot_sync(0xffffffffu, keep));
      }
    }
    if (lane == 0) c.pb_cnt[x] = cnt;
  }
}

// one thread per (projection, rank): offsets of the rank's targets (ascending)
__global__ void pb_scan_kernel(CountedArgs c) {
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (uint64_t)c.n_pb * c.R) return;
  const uint32_t q = (uint32_t)(k / c.R), r = (uint32_t)(k - (uint64_t)q * c.R);
  const DevProj& P = c.projs[c.pb_proj[q]];
  uint64_t acc = 0;
  for (uint32_t ti = 0; ti < P.n_tgt; ++ti) {
    const uint32_t t = P.tgt_first + ti * P.tgt_stride;
    if (rank_of(t, c.R, c.magic_R) != r) continue;
    c.pb_off[c.pb_t_first[q] + ti] = acc;
    acc += c.pb_cnt[c.pb_t_first[q] + ti];
  }
  c.pb_tot[k] = acc;
}

// fixed total over several ranks: regenerate each tile's draws and place them, in draw
// order within each (rank, projection) block
__global__ void __launch_bounds__(256) ft_place_kernel(CountedArgs c, BuildArgs a) {
  constexpr int NW = 8, ITEMS = kCountTile / 256;
  __shared__ uint32_t s_w[NW][kMaxCountedRanks / 4 * 4];
  __shared__ uint32_t s_tbl[256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t lt = (1u << lane) - 1;
  const uint32_t nb = 32 - __clz(c.R);        // bits of the values 0 .. R
  for (uint64_t tile = blockIdx.x; tile < c.n_ft_tiles; tile += gridDim.x) {
    __syncthreads();
    for (uint32_t i = tid; i < NW * c.R; i += 256) s_w[i / c.R][i % c.R] = 0;
    const uint32_t q = upper_bound_u64(c.ft_tile_first, c.n_ft, tile) - 1;
    const uint32_t pid = c.ft_proj[q];
    const DevProj& P = c.projs[pid];
    if (P.d_kind == 1)
      for (uint32_t i = tid; i < P.d_tbl_len; i += 256) s_tbl[i] = a.dtables[P.d_tbl_off + i];
    __syncthreads();
    const uint64_t j0 = (tile - c.ft_tile_first[q]) * kCountTile;
    const uint32_t n = (uint32_t)min((uint64_t)kCountTile, P.N - j0);
    uint64_t rec[ITEMS];
    uint32_t rk[ITEMS], rnk[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      const uint32_t idx = warp * 32 * ITEMS + j * 32 + lane;
      rk[j] = 0xFFFFFFFFu;
      if (idx < n) {
        const uint64_t cc = j0 + idx;
        const uint4 b = philox_stream(cc, P.proj_id, kPurposeSynapse, P.seed);
        const uint4 bt = philox_stream(cc, P.proj_id, kPurposeFtTarget, P.seed);
        const uint32_t t = P.tgt_first + uniform_index(bt.x, P.n_tgt) * P.tgt_stride;
        rk[j] = rank_of(t, c.R, c.magic_R);
        const uint32_t src = P.src_first + uniform_index(b.x, P.n_src) * P.src_stride;
        rec[j] = make_record(P, a.g, rk[j], cc, src, b.y, s_tbl);
      }
      // peers (same target rank) from one ballot per bit of the rank (R marks no draw)
      const uint32_t key = rk[j] == 0xFFFFFFFFu ? c.R : rk[j];
      uint32_t peers = 0xffffffffu;
      for (uint32_t bit = 0; bit < nb; ++bit) {
        const uint32_t m = 0u - ((key >> bit) & 1u);
        const uint32_t bl = __ballot_sync(0xffffffffu, m != 0u);
        peers &= ~(bl ^ m);
      }
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (lane == leader && rk[j] != 0xFFFFFFFFu) {
        old = s_w[warp][rk[j]];
        s_w[warp][rk[j]] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      rnk[j] = old + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    for (uint32_t r = tid; r < c.R; r += 256) {          // exclusive prefix over warps
      uint32_t acc = 0;
      for (int w = 0; w < NW; ++w) {
        const uint32_t v = s_w[w][r];
        s_w[w][r] = acc;
        acc += v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
      if (rk[j] == 0xFFFFFFFFu) continue;
      const uint64_t pos = c.block_base[(uint64_t)pid * c.R + rk[j]] + c.ft_tile_off[tile * c.R + rk[j]] +
                           s_w[warp][rk[j]] + rnk[j];
      if (pos < a.seg_start[rk[j] + 1]) a.rec_a[pos] = rec[j]; else atomicOr(a.err, kErrBounds);
    }
  }
}

// pairwise Bernoulli: one warp per target, kept pairs in source order
__global__ void __launch_bounds__(256) pb_place_kernel(CountedArgs c, BuildArgs a) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < c.n_pb_targets; x += nwarps) {
    const uint32_t q = upper_bound_u64(c.pb_t_first, c.n_pb, x) - 1;
    const uint32_t pid = c.pb_proj[q];
    const DevProj& P = c.projs[pid];
    const uint64_t ti = x - c.pb_t_first[q];
    const uint32_t t = P.tgt_first + (uint32_t)ti * P.tgt_stride;
    const uint32_t rank = rank_of(t, c.R, c.magic_R);
    uint64_t pos = c.block_base[(uint64_t)pid * c.R + rank] + c.pb_off[x];
    const uint64_t end = a.seg_start[rank + 1];
    if (P.rule == kRuleBernoulliGeometric) {
      if (P.pb_thr)
        geometric_walk(P, c.tables + P.g_tbl_off, ti, [&](uint32_t s, bool keep, uint32_t m, uint32_t r) {
          if (keep) {
            const uint64_t qq = ti * P.n_src + s;
            const uint4 b = philox_stream(qq, P.proj_id, kPurposeSynapse, P.seed);
            const uint32_t src = P.src_first + s * P.src_stride;
            const uint64_t at = pos + r;
            const uint64_t rr = make_record(P, a.g, rank, qq, src, b.y, a.dtables + P.d_tbl_off);
            if (at < end) a.rec_a[at] = rr; else atomicOr(a.err, kErrBounds);
          }
          pos += __popc(m);
        });
      continue;
    }
    for (uint32_t s0 = 0; s0 < P.n_src; s0 += 32) {
      const uint32_t s = s0 + lane;
      const uint64_t qq = ti * P.n_src + s;
      const bool keep = s < P.n_src && (uint64_t)pb_word(P, qq) < P.pb_thr;
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const uint4 b = philox_stream(qq, P.proj_id, kPurposeSynapse, P.seed);
        const uint32_t src = P.src_first + s * P.src_stride;
        const uint64_t at = pos + __popc(m & ((1u << lane) - 1));
        const uint64_t r = make_record(P, a.g, rank, qq, src, b.y, a.dtables + P.d_tbl_off);
        if (at < end) a.rec_a[at] = r; else atomicOr(a.err, kErrBounds);
      }
      pos += __popc(m);
    }
  }
}

cudaError_t launch_counted_count(const CountedArgs& c, cudaStream_t st, int num_sms) {
  if (c.R > kMaxCountedRanks) return cudaErrorInvalidValue;
  if (c.n_ft_tiles) {
    ft_count_kernel<<<(unsigned)std::min<uint64_t>(c.n_ft_tiles, (uint64_t)num_sms * 8), 256, 0, st>>>(c);
    ft_scan_kernel<<<(unsigned)(((uint64_t)c.n_ft * c.R + 255) / 256), 256, 0, st>>>(c);
  }
  if (c.n_pb_targets) {
    pb_count_kernel<<<(unsigned)std::min<uint64_t>((c.n_pb_targets * 32 + 255) / 256, (uint64_t)num_sms * 16),
                      256, 0, st>>>(c);
    pb_scan_kernel<<<(unsigned)(((uint64_t)c.n_pb * c.R + 255) / 256), 256, 0, st>>>(c);
  }
  return cudaGetLastError();
}

cudaError_t launch_counted_place(const CountedArgs& c, const BuildArgs& a, cudaStream_t st) {
  if (c.n_ft_tiles)
    ft_place_kernel<<<(unsigned)std::min<uint64_t>(c.n_ft_tiles, (uint64_t)a.num_sms * 8), 256, 0, st>>>(c, a);
  if (c.n_pb_targets)
    pb_place_kernel<<<(unsigned)std::min<uint64_t>((c.n_pb_targets * 32 + 255) / 256, (uint64_t)a.num_sms * 16),
                      256, 0, st>>>(c, a);
  return cudaGetLastError();
}

// per-segment digit histograms of all records (when generation could not fuse them)
__global__ void __launch_bounds__(256) hist_kernel(BuildArgs a) {
  constexpr int BINS = kHistStride;
  __shared__ uint32_t s_hist[MAX_PASSES][BINS];
  const uint32_t passes = a.passes;
  for (int i = threadIdx.x; i < MAX_PASSES * BINS; i += 256) (&s_hist[0][0])[i] = 0;
  const uint64_t per = (a.n_sort_tiles + gridDim.x - 1) / gridDim.x;
  const uint64_t t0 = (uint64_t)blockIdx.x * per, t1 = min(t0 + per, a.n_sort_tiles);
  int cur = -1;
  for (uint64_t tile = t0; tile < t1; ++tile) {
    const uint32_t seg = upper_bound_u64(a.seg_tile0, a.g.R, tile) - 1;
    __syncthreads();
    if ((int)seg != cur) {
      if (cur >= 0)
        for (int i = threadIdx.x; i < (int)passes * BINS; i += 256) {
          const uint32_t v = (&s_hist[0][0])[i];
          if (v) atomicAdd((unsigned long long*)&a.hist[((uint64_t)cur * passes) * BINS + i], v);
          (&s_hist[0][0])[i] = 0;
        }
      cur = seg;
    }
    __syncthreads();
    const uint64_t tile_n = (uint64_t)SORT_BLOCK * a.sort_items;
    const uint64_t base = a.seg_start[seg] + (tile - a.seg_tile0[seg]) * tile_n;
    const uint64_t end = min(base + tile_n, a.seg_start[seg + 1]);
    for (uint64_t i = base + threadIdx.x; i < end; i += 256) {
      const uint64_t kk = a.rec_a[i] >> a.g.cbits;
#pragma unroll
      for (int p = 0; p < MAX_PASSES; ++p)
        if (p < (int)passes) atomicAdd(&s_hist[p][(kk >> a.pass_shift[p]) & ((1u << a.pass_bits[p]) - 1)], 1u);
    }
  }
  __syncthreads();
  if (cur >= 0)
    for (int i = threadIdx.x; i < (int)passes * BINS; i += 256) {
      const uint32_t v = (&s_hist[0][0])[i];
      if (v) atomicAdd((unsigned long long*)&a.hist[((uint64_t)cur * passes) * BINS + i], v);
    }
}

cudaError_t launch_histogram(const BuildArgs& a, cudaStream_t st) {
  if (a.n_sort_tiles == 0 || a.passes == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<uint64_t>(a.n_sort_tiles, (uint64_t)a.num_sms * 8);
  hist_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// finalize: SoA arrays + dense row starts
// ---------------------------------------------------------------------------
__device__ __forceinline__ float draw_weight(const DevProj& P, uint32_t w2, uint32_t w3) {
  if (P.w_kind == 0) return P.w_mean;
  const float u1 = u01(w2), u2 = u01(w3);
  const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
  float w = fmaf(P.w_sd, z, P.w_mean);
  return P.w_mean >= 0.f ? fmaxf(w, 0.f) : fminf(w, 0.f);
}

constexpr int FIN_Q = 4;   // consecutive records per thread of the finalize kernel

// Target of draw c of a fixed-total projection.  Out of line: the finalize loop is
// unrolled over its records and would otherwise hold eight copies of this Philox block
// in its instruction footprint, for a path that fixed in-degree records never take.
__device__ __noinline__ uint32_t fixed_total_target(const DevProj& Q, uint64_t c) {
  const uint4 bt = philox_stream(c, Q.proj_id, kPurposeFtTarget, Q.seed);
  return Q.tgt_first + uniform_index(bt.x, Q.n_tgt) * Q.tgt_stride;
}

// Each thread decodes FIN_Q consecutive sorted records: one pair of 16-byte loads, the
// projection lookup reused while the counters stay in one projection, and one vector
// store per output array.  Row starts: a record whose row differs from its
// predecessor's writes the starts of the rows in between.
__global__ void __launch_bounds__(256) finalize_kernel(BuildArgs a, const uint64_t* __restrict__ rec,
                                                      uint64_t E, uint32_t vec) {
  const Geom g = a.g;
  const uint64_t cmask = g.cbits >= 64 ? ~0ull : ((1ull << g.cbits) - 1);
  const uint64_t smask = (1ull << g.sb) - 1;
  const uint64_t dmask = (1ull << g.db) - 1;
  const uint64_t nq = (E + FIN_Q - 1) / FIN_Q;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += stride) {
    const uint64_t i0 = q * FIN_Q;
    const bool full = vec && i0 + FIN_Q <= E;
    uint64_t r[FIN_Q];
    if (full) {
      const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(rec + i0);
      const ulonglong2 y = *reinterpret_cast<const ulonglong2*>(rec + i0 + 2);
      r[0] = x.x; r[1] = x.y; r[2] = y.x; r[3] = y.y;
    } else {
#pragma unroll
      for (int j = 0; j < FIN_Q; ++j) r[j] = i0 + j < E ? rec[i0 + j] : 0ull;
    }
    uint32_t seg = g.R == 1 ? 0u : upper_bound_u64(a.seg_start + 1, g.R, i0);
    uint64_t seg_hi = a.seg_start[seg + 1];
    const uint32_t* doff = a.dense_off + (uint64_t)seg * g.R;
    uint64_t* dn = a.dense + (uint64_t)(seg - a.dense_seg0) * ((uint64_t)g.N + 1);
    int64_t prow = -1;
    if (i0 > a.seg_start[seg]) {
      const uint64_t kp = rec[i0 - 1] >> g.cbits;
      const uint32_t ps = (uint32_t)(kp >> (g.db + g.sb));
      prow = ps < g.R ? (int64_t)((uint64_t)doff[ps] + ((kp >> g.db) & smask)) : (int64_t)g.N;
    }
    uint32_t p = 0, blk_i = 0;
    uint64_t p_lo = 0, p_hi = 0;   // counters [p_lo, p_hi) of the cached projection p (none yet)
    uint32_t tl[FIN_Q], wb[FIN_Q], dd[FIN_Q];
    bool ok[FIN_Q];
#pragma unroll
    for (int j = 0; j < FIN_Q; ++j) {
      const uint64_t i = i0 + j;
      ok[j] = false;
      tl[j] = 0; wb[j] = 0; dd[j] = 0;
      if (i >= E) continue;
      while (i >= seg_hi) {          // first record of a later segment
        ++seg;
        seg_hi = a.seg_start[seg + 1];
        doff = a.dense_off + (uint64_t)seg * g.R;
        dn = a.dense + (uint64_t)(seg - a.dense_seg0) * ((uint64_t)g.N + 1);
        prow = -1;
      }
      const uint64_t key = r[j] >> g.cbits;
      const uint64_t cidx = r[j] & cmask;
      const uint32_t d = (uint32_t)(key & dmask);
      const uint32_t s = (uint32_t)((key >> g.db) & smask);
      const uint32_t slot = (uint32_t)(key >> (g.db + g.sb));
      const uint64_t row = slot < g.R ? (uint64_t)doff[slot] + s : (uint64_t)g.N;
      if (row >= g.N) {              // corrupt record: flag it, write nothing for it
        atomicOr(a.err, kErrBounds);
        prow = (int64_t)g.N;
        continue;
      }
      for (int64_t x = prow + 1; x <= (int64_t)row; ++x) dn[x] = i;
      if (i == seg_hi - 1)
        for (uint64_t x = row + 1; x <= g.N; ++x) dn[x] = seg_hi;
      prow = (int64_t)row;

      // projection of the counter, then target and weight regenerated from it
      uint64_t c;
      uint32_t t;
      if (a.pos_counters) {
        // generation position: its block gives projection, first target and target step
        if (cidx - p_lo >= p_hi - p_lo) {
          uint32_t lo = 0, hi = a.nblocks;
          while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.blocks[mid].out_base <= cidx) lo = mid + 1; else hi = mid;
          }
          blk_i = lo - 1;
          p_lo = a.blocks[blk_i].out_base;
          p_hi = p_lo + a.blocks[blk_i].count;
          p = a.blocks[blk_i].proj;
        }
        const DevBlock& B = a.blocks[blk_i];
        const DevProj& Q = a.projs[p];
        const uint64_t l = cidx - B.out_base;
        if (Q.rule == kRuleFixedIndegree) {
          const uint64_t m = div_magic(l, Q.K, Q.magic_div);
          const uint64_t ti = B.ti0 + m * B.tstep;
          c = ti * Q.K + (l - m * Q.K);
          t = Q.tgt_first + (uint32_t)ti * Q.tgt_stride;
        } else {                       // fixed total on one rank: the draw index
          c = l;
          t = fixed_total_target(Q, c);
        }
      } else {
        if (cidx - p_lo >= p_hi - p_lo) {
          p = upper_bound_u64(a.cbase_sorted, a.nproj, cidx) - 1;
          p_lo = a.cbase_sorted[p];
          p_hi = p + 1 < a.nproj ? a.cbase_sorted[p + 1] : ~0ull;
        }
        const DevProj& Q = a.projs[p];
        c = cidx - Q.cbase;
        if (Q.rule == kRuleFixedIndegree) {
          t = Q.tgt_first + (uint32_t)div_magic(c, Q.K, Q.magic_div) * Q.tgt_stride;
        } else if (Q.rule == kRuleFixedTotal) {
          t = fixed_total_target(Q, c);
        } else {
          t = Q.tgt_first + (uint32_t)div_magic(c, Q.n_src, Q.magic_div) * Q.tgt_stride;
        }
      }
      const DevProj& P = a.projs[p];
      tl[j] = g.R == 1 ? t : (uint32_t)div_magic(t, g.R, g.magic_R);
      dd[j] = d;
      const uint4 b = philox_stream(c, P.proj_id, kPurposeSynapse, P.seed);
      const float w = draw_weight(P, b.z, b.w);
      if (a.w_format == 0) {
        wb[j] = __float_as_uint(w);
      } else if (a.w_format == 1) {
        wb[j] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
      } else {
        const uint32_t sig = slot != 0 ? (slot <= seg ? slot - 1 : slot) : seg;
        const uint64_t src_gid = (uint64_t)s * g.R + sig;
        const float sc = a.row_scale_src ? a.row_scale_src[src_gid] : 1.0f;
        wb[j] = __half_as_ushort(__float2half_rn(w / sc));
      }
      ok[j] = true;
    }
    if (full && ok[0] && ok[1] && ok[2] && ok[3]) {
      *reinterpret_cast<uint4*>(a.tgt + i0) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
      *reinterpret_cast<uint32_t*>(a.d + i0) = dd[0] | (dd[1] << 8) | (dd[2] << 16) | (dd[3] << 24);
      if (a.w_format == 0)
        *reinterpret_cast<uint4*>((uint32_t*)a.w + i0) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
      else
        *reinterpret_cast<uint2*>((uint16_t*)a.w + i0) = make_uint2(wb[0] | (wb[1] << 16), wb[2] | (wb[3] << 16));
    } else {
#pragma unroll
      for (int j = 0; j < FIN_Q; ++j) {
        if (!ok[j]) continue;
        const uint64_t i = i0 + j;
        a.tgt[i] = tl[j];
        a.d[i] = (uint8_t)dd[j];
        if (a.w_format == 0) ((uint32_t*)a.w)[i] = wb[j];
        else ((uint16_t*)a.w)[i] = (uint16_t)wb[j];
      }
    }
  }
}

// The projection a run of counters belongs to, held in registers while the counters of
// consecutive records stay inside it (one-rank finalize).
struct ProjRegs {
  uint64_t lo, hi;          // counters [lo, hi) of the projection
  uint64_t K, magic;        // fixed in-degree K (or n_src for Bernoulli) and its divisor magic
  uint2 key;                // Philox key (the projection seed)
  uint32_t rule, proj_id, tgt_first, tgt_stride, w_kind, idx;
  float w_mean, w_sd;
};

__device__ __forceinline__ void load_proj_regs(const BuildArgs& a, uint64_t cidx, ProjRegs& q) {
  const uint32_t p = upper_bound_u64(a.cbase_sorted, a.nproj, cidx) - 1;
  const DevProj& P = a.projs[p];
  q.lo = a.cbase_sorted[p];
  q.hi = p + 1 < a.nproj ? a.cbase_sorted[p + 1] : ~0ull;
  q.rule = P.rule;
  q.K = P.rule == kRuleFixedIndegree ? P.K : (uint64_t)P.n_src;
  q.magic = P.magic_div;
  q.key = make_uint2((uint32_t)P.seed, (uint32_t)(P.seed >> 32));
  q.proj_id = P.proj_id;
  q.tgt_first = P.tgt_first;
  q.tgt_stride = P.tgt_stride;
  q.w_kind = P.w_kind;
  q.w_mean = P.w_mean;
  q.w_sd = P.w_sd;
  q.idx = p;
}

// Finalize on one rank (no rank slots, counters as record ids): the same outputs as
// finalize_kernel with the per-record work cut to the decode itself.  The row of a
// record is its source; each projection's fields stay in registers while consecutive
// records keep to its counters.  WF: weight format (0 fp32, 1 bf16, 2 fp16 with a
// per-source scale).
template <int WF>
__global__ void __launch_bounds__(256) finalize_one_rank_kernel(BuildArgs a, const uint64_t* __restrict__ rec,
                                                                uint64_t E, uint32_t vec) {
  const Geom g = a.g;
  const uint32_t cbits = g.cbits, db = g.db;
  const uint64_t cmask = cbits >= 64 ? ~0ull : ((1ull << cbits) - 1);
  const uint32_t smask = (uint32_t)((1ull << g.sb) - 1);
  const uint32_t dmask = (1u << db) - 1;
  const uint32_t N = g.N;
  uint64_t* __restrict__ dn = a.dense;
  const uint64_t nq = (E + FIN_Q - 1) / FIN_Q;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  ProjRegs q;
  q.lo = 0;
  q.hi = 0;                       // an empty range: the first record loads its projection
  for (uint64_t qi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; qi < nq; qi += stride) {
    const uint64_t i0 = qi * FIN_Q;
    const bool full = vec && i0 + FIN_Q <= E;
    uint64_t r[FIN_Q];
    if (full) {
      const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(rec + i0);
      const ulonglong2 y = *reinterpret_cast<const ulonglong2*>(rec + i0 + 2);
      r[0] = x.x; r[1] = x.y; r[2] = y.x; r[3] = y.y;
    } else {
#pragma unroll
      for (int j = 0; j < FIN_Q; ++j) r[j] = i0 + j < E ? rec[i0 + j] : 0ull;
    }
    int64_t prow = i0 > 0 ? (int64_t)((uint32_t)(rec[i0 - 1] >> (cbits + db)) & smask) : -1;
    uint32_t tl[FIN_Q], wb[FIN_Q], dd[FIN_Q];
    bool ok[FIN_Q];
#pragma unroll
    for (int j = 0; j < FIN_Q; ++j) {
      const uint64_t i = i0 + j;
      ok[j] = false;
      tl[j] = 0; wb[j] = 0; dd[j] = 0;
      if (i >= E) continue;
      const uint64_t key = r[j] >> cbits;
      const uint64_t cidx = r[j] & cmask;
      const uint32_t row = (uint32_t)(key >> db) & smask;
      if ((key >> db) > smask || row >= N) {     // corrupt record: flag it, write nothing for it
        atomicOr(a.err, kErrBounds);
        prow = (int64_t)N;
        continue;
      }
      for (int64_t x = prow + 1; x <= (int64_t)row; ++x) dn[x] = i;
      if (i == E - 1)
        for (uint64_t x = (uint64_t)row + 1; x <= N; ++x) dn[x] = E;
      prow = row;
      if (cidx - q.lo >= q.hi - q.lo) load_proj_regs(a, cidx, q);
      const uint64_t c = cidx - q.lo;
      uint32_t t;
      if (q.rule == kRuleFixedTotal) t = fixed_total_target(a.projs[q.idx], c);
      else t = q.tgt_first + (uint32_t)div_magic(c, q.K, q.magic) * q.tgt_stride;
      tl[j] = t;
      dd[j] = (uint32_t)key & dmask;
      const uint4 b = philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), q.proj_id, kPurposeSynapse), q.key);
      float w = q.w_mean;
      if (q.w_kind != 0) {
        const float u1 = u01(b.z), u2 = u01(b.w);
        const float z = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
        w = fmaf(q.w_sd, z, q.w_mean);
        w = q.w_mean >= 0.f ? fmaxf(w, 0.f) : fminf(w, 0.f);
      }
      if (WF == 0) {
        wb[j] = __float_as_uint(w);
      } else if (WF == 1) {
        wb[j] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
      } else {
        const float sc = a.row_scale_src ? a.row_scale_src[row] : 1.0f;
        wb[j] = __half_as_ushort(__float2half_rn(w / sc));
      }
      ok[j] = true;
    }
    if (full && ok[0] && ok[1] && ok[2] && ok[3]) {
      *reinterpret_cast<uint4*>(a.tgt + i0) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
      *reinterpret_cast<uint32_t*>(a.d + i0) = dd[0] | (dd[1] << 8) | (dd[2] << 16) | (dd[3] << 24);
      if (WF == 0)
        *reinterpret_cast<uint4*>((uint32_t*)a.w + i0) = make_uint4(wb[0], wb[1], wb[2], wb[3]);
      else
        *reinterpret_cast<uint2*>((uint16_t*)a.w + i0) = make_uint2(wb[0] | (wb[1] << 16), wb[2] | (wb[3] << 16));
    } else {
#pragma unroll
      for (int j = 0; j < FIN_Q; ++j) {
        if (!ok[j]) continue;
        const uint64_t i = i0 + j;
        a.tgt[i] = tl[j];
        a.d[i] = (uint8_t)dd[j];
        if (WF == 0) ((uint32_t*)a.w)[i] = wb[j];
        else ((uint16_t*)a.w)[i] = (uint16_t)wb[j];
      }
    }
  }
}

__global__ void fill_empty_segments(uint64_t* dense, const uint64_t* seg_start, uint32_t seg0, uint32_t nseg,
                                    uint32_t N) {
  const uint64_t total = (uint64_t)nseg * (N + 1);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t seg = seg0 + (uint32_t)(i / (N + 1));
    if (seg_start[seg] == seg_start[seg + 1]) dense[i] = seg_start[seg];
  }
}

cudaError_t launch_finalize(const BuildArgs& a, const uint64_t* rec, uint64_t E, cudaStream_t st) {
  const uint64_t total = (uint64_t)a.dense_nseg * (a.g.N + 1);
  if (total)
    fill_empty_segments<<<(unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)a.num_sms * 16), 256, 0,
                          st>>>(a.dense, a.seg_start, a.dense_seg0, a.dense_nseg, a.g.N);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || E == 0) return e;
  const uint64_t nq = (E + FIN_Q - 1) / FIN_Q;
  const uint64_t grid = std::min<uint64_t>((nq + 255) / 256, (uint64_t)a.num_sms * 16);
  // vector loads and stores need 16-byte aligned bases (quad starts are multiples of 4)
  const uint32_t vec = (((uintptr_t)rec | (uintptr_t)a.tgt | (uintptr_t)a.w | (uintptr_t)a.d) & 15u) == 0;
  if (a.g.R == 1 && !a.pos_counters && a.dense_seg0 == 0 && a.dense_nseg == 1) {
    if (a.w_format == 0) finalize_one_rank_kernel<0><<<(unsigned)grid, 256, 0, st>>>(a, rec, E, vec);
    else if (a.w_format == 1) finalize_one_rank_kernel<1><<<(unsigned)grid, 256, 0, st>>>(a, rec, E, vec);
    else finalize_one_rank_kernel<2><<<(unsigned)grid, 256, 0, st>>>(a, rec, E, vec);
  } else {
    finalize_kernel<<<(unsigned)grid, 256, 0, st>>>(a, rec, E, vec);
  }
  return cudaGetLastError();
}

}  // namespace snn
