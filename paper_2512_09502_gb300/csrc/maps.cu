// maps.cu -- image neurons, the point-to-point and collective communication maps of
// the logical ranks, spike routing, and the row accessors of the inspection calls.
//
// Paper, Methods, "Remote connections":
//  * rank tau represents a remote source (sigma, s) by an image neuron with local
//    index >= M_tau; (R_{tau,sigma}, L_{tau,sigma}) map remote source -> image, sorted
//    by source (Eq. sortedmaps);
//  * the source rank keeps S_{tau,sigma} built from regenerated sources, aligned with
//    R (Eq. mapalign), and T_{sigma,s} / P_{sigma,s}: target ranks of s and its
//    positions in their maps (simulation preparation);
//  * collective: H_{0,sigma} (sorted sources of sigma with remote images),
//    I_{0,sigma,tau} (image of H[j] on tau, or -1), G / Q (group, position in H).
// Here every map is derived in one batched pass from the sorted layout (target side)
// and from one regeneration of every synapse's source (source side), instead of the
// paper's incremental per-RemoteConnect updates; the resulting maps are those the
// incremental algorithm produces when RemoteConnect is called once per source rank in
// ascending order.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "maps_internal.cuh"

namespace snn {

namespace {

constexpr int MB = 256;   // block size of the map kernels

// ---- generic device exclusive scan of uint32 counts into uint64 offsets ----
__global__ void scan_block_sums(const uint32_t* in, uint64_t n, uint64_t* block_sum) {
  __shared__ uint64_t s[MB];
  const uint64_t base = (uint64_t)blockIdx.x * MB * 4;
  uint64_t acc = 0;
  for (int k = 0; k < 4; ++k) {
    const uint64_t i = base + (uint64_t)k * MB + threadIdx.x;
    if (i < n) acc += in[i];
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = MB / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sum[blockIdx.x] = s[0];
}

__global__ void scan_sums_serial(uint64_t* block_sum, uint64_t nb, uint64_t* total) {
  // one CTA: chunked exclusive scan of the block sums
  __shared__ uint64_t s[MB];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint64_t c0 = 0; c0 < nb; c0 += MB) {
    const uint64_t i = c0 + threadIdx.x;
    const uint64_t v = i < nb ? block_sum[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < MB; o <<= 1) {
      const uint64_t t = (int)threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < nb) block_sum[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == MB - 1) carry += s[MB - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_apply(const uint32_t* in, uint64_t n, const uint64_t* block_off, uint64_t* out) {
  __shared__ uint64_t s[MB * 4];
  const uint64_t base = (uint64_t)blockIdx.x * MB * 4;
  for (int k = 0; k < 4; ++k) {
    const uint64_t i = base + (uint64_t)k * MB + threadIdx.x;
    s[k * MB + threadIdx.x] = i < n ? in[i] : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {   // serial over 1024 entries: simple and cheap at these sizes
    uint64_t acc = block_off[blockIdx.x];
    for (int k = 0; k < MB * 4; ++k) {
      const uint64_t v = s[k];
      s[k] = acc;
      acc += v;
    }
  }
  __syncthreads();
  for (int k = 0; k < 4; ++k) {
    const uint64_t i = base + (uint64_t)k * MB + threadIdx.x;
    if (i < n) out[i] = s[k * MB + threadIdx.x];
  }
}

// out[i] = sum_{j<i} in[j]; out[n] = total (out has n + 1 entries)
cudaError_t exclusive_scan(snn_ctx* c, const uint32_t* in, uint64_t n, uint64_t* out) {
  cudaStream_t st = ctx_stream(c);
  const uint64_t nb = std::max<uint64_t>(1, (n + MB * 4 - 1) / (MB * 4));
  uint64_t* bs = (uint64_t*)ctx_alloc(c, nb * 8);
  if (!bs) return cudaErrorMemoryAllocation;
  scan_block_sums<<<(unsigned)nb, MB, 0, st>>>(in, n, bs);
  scan_sums_serial<<<1, MB, 0, st>>>(bs, nb, out + n);
  scan_apply<<<(unsigned)nb, MB, 0, st>>>(in, n, bs, out);
  const cudaError_t e = cudaGetLastError();
  ctx_free(c, bs);
  return e;
}

// ---- target side: image rows ----
// Target-side kernels work on a window of ranks tau = t0 + tl, tl < nt, whose dense row
// starts are dense[tl][N + 1] (the whole network: t0 = 0, nt = R; a dry run: one rank).
// used[tl][r] for the dense rows r >= M_tau (image candidates): row has connections
__global__ void image_flags(const uint64_t* dense, uint32_t N, uint32_t t0, uint32_t nt, const uint32_t* M,
                            uint32_t* flag /*[nt][N]*/) {
  const uint64_t total = (uint64_t)nt * N;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t tl = (uint32_t)(i / N), r = (uint32_t)(i - (uint64_t)tl * N);
    const uint64_t* dn = dense + (uint64_t)tl * (N + 1);
    flag[i] = (r >= M[t0 + tl] && dn[r + 1] > dn[r]) ? 1u : 0u;
  }
}

// rows of every rank of the window: local rows, then images; image source (sigma, s)
__global__ void image_fill(const uint64_t* dense, uint32_t N, uint32_t R, uint32_t t0, uint32_t nt,
                           const uint32_t* M, const uint32_t* flag, const uint64_t* img_pos /*[nt*N+1]*/,
                           const uint64_t* rows_off /*[nt+1]*/, const uint32_t* dense_off,
                           const uint64_t* seg_start, uint64_t* rows, uint32_t* img_gid) {
  const uint64_t total = (uint64_t)nt * N;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t tl = (uint32_t)(i / N), r = (uint32_t)(i - (uint64_t)tl * N);
    const uint32_t tau = t0 + tl;
    const uint64_t* dn = dense + (uint64_t)tl * (N + 1);
    const uint64_t img_first = img_pos[(uint64_t)tl * N];          // images before rank tau
    const uint64_t rbase = rows_off[tl];
    if (r < M[tau]) {
      rows[rbase + r] = dn[r];
    } else if (flag[i]) {
      const uint64_t k = img_pos[i] - img_first;                    // image index within tau
      rows[rbase + M[tau] + k] = dn[r];
      // (slot, s) of dense row r: last slot with dense_off <= r
      const uint32_t* doff = dense_off + (uint64_t)tau * R;
      uint32_t lo = 0, hi = R;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (doff[mid] <= r) lo = mid + 1; else hi = mid;
      }
      const uint32_t slot = lo - 1;
      const uint32_t sig = slot == 0 ? tau : (slot <= tau ? slot - 1 : slot);
      img_gid[img_pos[i]] = (r - doff[slot]) * R + sig;
    }
    if (r == N - 1) rows[rows_off[tl + 1] - 1] = seg_start[tau + 1];   // terminal entry
  }
}

// ---- all-sources images (threshold xi) ----
// One (projection, target rank tau) pair: every source of the projection that lives
// on another rank gets an image on tau.
struct AllSrcPair {
  uint32_t src_first, n_src, src_stride, tau;
};
constexpr uint32_t kAllSrcChunk = 4096;   // sources per block of all_sources_flags

// The x-th source of a pair.  Contiguous sources (stride 1) are visited rank by rank,
// by local index within a rank -- x = off(k) + j for the gid src_first + k + j R, where
// the first n_src mod R residues k hold one source more -- so consecutive threads mark
// consecutive image rows; RemoteConnect sources (stride R) are in that order already.
__device__ __forceinline__ uint32_t pair_source(const AllSrcPair& P, uint32_t R, uint32_t x) {
  if (P.src_stride != 1) return P.src_first + x * P.src_stride;
  const uint32_t q = P.n_src / R, rem = P.n_src - q * R, head = rem * (q + 1);
  uint32_t k, j;
  if (x < head) {
    k = x / (q + 1);
    j = x - k * (q + 1);
  } else {                                  // q > 0 here: x < n_src = head + (R - rem) q
    const uint32_t y = x - head;
    k = rem + y / q;
    j = y - (k - rem) * q;
  }
  return P.src_first + k + j * R;
}

// Marks the target-side image flag of dense row (slot of sigma, s) on tau (window
// t0 .. t0 + nt - 1; tflag [nt][N]) and/or the source-side flag of S_{tau,sigma}
// (sflag [sigma][tau][Mmax]).  Block b takes chunk b - chunk_first[k] of pair k (at
// most kAllSrcChunk sources).  Every write stores 1, so overlapping pairs need no atomics.
__global__ void all_sources_flags(const AllSrcPair* pairs, const uint32_t* chunk_first /*[np + 1]*/,
                                  uint32_t np, uint32_t R, uint64_t magic_R, uint32_t N, uint32_t t0,
                                  const uint32_t* dense_off, uint32_t* tflag, uint8_t* sflag, uint32_t Mmax) {
  __shared__ uint32_t s_k;
  if (threadIdx.x == 0) {
    uint32_t lo = 0, hi = np;             // last k with chunk_first[k] <= blockIdx.x
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (chunk_first[mid] <= blockIdx.x) lo = mid; else hi = mid;
    }
    s_k = lo;
  }
  __syncthreads();
  const AllSrcPair P = pairs[s_k];
  const uint32_t x0 = (blockIdx.x - chunk_first[s_k]) * kAllSrcChunk;
  const uint32_t x1 = min(P.n_src, x0 + kAllSrcChunk);
  for (uint32_t x = x0 + threadIdx.x; x < x1; x += blockDim.x) {
    const uint32_t gid = pair_source(P, R, x);
    const uint32_t s = (uint32_t)div_magic(gid, R, magic_R), sig = gid - s * R;
    if (sig == P.tau) continue;
    if (tflag) {
      const uint32_t slot = sig < P.tau ? sig + 1 : sig;
      tflag[(uint64_t)(P.tau - t0) * N + dense_off[(uint64_t)P.tau * R + slot] + s] = 1u;
    }
    if (sflag) sflag[((uint64_t)sig * R + P.tau) * Mmax + s] = 1;
  }
}

// ---- source side: regenerate every synapse's source and target rank ----
// (skip[p]: projection p has all-sources images on every rank holding its targets;
// its flags are set by all_sources_flags)
__global__ void source_flags(const DevProj* projs, uint32_t nproj, const uint64_t* cbase,
                             uint64_t ctot, uint32_t R, uint64_t magic_R, uint32_t Mmax,
                             const uint32_t* tables, const uint8_t* skip, uint8_t* flag /*[sigma][tau][Mmax]*/) {
  __shared__ uint64_t s_cb[1024];
  const uint32_t ncache = nproj < 1024 ? nproj : 1024;
  for (uint32_t k = threadIdx.x; k < ncache; k += blockDim.x) s_cb[k] = cbase[k];
  __syncthreads();
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < ctot;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t p = (nproj <= 1024 ? upper_bound_u64(s_cb, nproj, x) : upper_bound_u64(cbase, nproj, x)) - 1;
    if (skip[p]) continue;
    const DevProj& P = projs[p];
    const uint64_t c = x - P.cbase;
    uint32_t src, tgt;
    if (P.rule == kRuleFixedIndegree) {
      const uint64_t ti = div_magic(c, P.K, P.magic_div);
      if (P.src_mode == 0) {
        const uint4 b = philox_stream(c, P.proj_id, kPurposeSynapse, P.seed);
        src = P.src_first + uniform_index(b.x, P.n_src) * P.src_stride;
      } else {                     // all-to-all: source k = c - ti K; one-to-one: source ti
        src = P.src_first + (uint32_t)(P.src_mode == kSrcAll ? c - ti * P.K : ti) * P.src_stride;
      }
      tgt = P.tgt_first + (uint32_t)ti * P.tgt_stride;
    } else if (P.rule == kRuleFixedTotal) {
      const uint4 b = philox_stream(c, P.proj_id, kPurposeSynapse, P.seed);
      const uint4 bt = philox_stream(c, P.proj_id, kPurposeFtTarget, P.seed);
      src = P.src_first + uniform_index(b.x, P.n_src) * P.src_stride;
      tgt = P.tgt_first + uniform_index(bt.x, P.n_tgt) * P.tgt_stride;
    } else if (P.rule == kRuleBernoulliGeometric) {
      // the thread of a target's first counter walks that target's gaps
      if (!P.pb_thr) continue;
      const uint64_t ti = div_magic(c, P.n_src, P.magic_div);
      if (c != ti * P.n_src) continue;
      tgt = P.tgt_first + (uint32_t)ti * P.tgt_stride;
      const uint32_t tau = tgt - (uint32_t)div_magic(tgt, R, magic_R) * R;
      const uint32_t* tbl = tables + P.g_tbl_off;
      int64_t s_i = -1;
      for (uint64_t j = 0;; ++j) {
        const uint4 b = philox_stream(ti * P.n_src + j, P.proj_id, kPurposePbGap, P.seed);
        s_i += (int64_t)upper_bound_u32(tbl, P.g_tbl_len, b.x) + 1;
        if (s_i >= (int64_t)P.n_src) break;
        src = P.src_first + (uint32_t)s_i * P.src_stride;
        const uint32_t s = (uint32_t)div_magic(src, R, magic_R), sig = src - s * R;
        if (sig != tau) flag[((uint64_t)sig * R + tau) * Mmax + s] = 1;
      }
      continue;
    } else {
      const uint4 tb = philox_stream(c >> 2, P.proj_id, kPurposePbTest, P.seed);
      const uint32_t lane = (uint32_t)(c & 3);
      const uint32_t w = lane == 0 ? tb.x : lane == 1 ? tb.y : lane == 2 ? tb.z : tb.w;
      if ((uint64_t)w >= P.pb_thr) continue;
      const uint64_t ti = div_magic(c, P.n_src, P.magic_div);
      src = P.src_first + (uint32_t)(c - ti * P.n_src) * P.src_stride;
      tgt = P.tgt_first + (uint32_t)ti * P.tgt_stride;
    }
    const uint32_t s = (uint32_t)div_magic(src, R, magic_R), sig = src - s * R;
    const uint32_t tau = tgt - (uint32_t)div_magic(tgt, R, magic_R) * R;
    if (sig != tau) flag[((uint64_t)sig * R + tau) * Mmax + s] = 1;
  }
}

// dst[k] = src[k * stride] (stride > 0) or src[idx[k]] (idx given): boundary values of a
// scan gathered on the device so that the host reads them in one copy
__global__ void gather_u64(const uint64_t* src, uint64_t stride, const uint32_t* idx, uint64_t count,
                           uint64_t* dst) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (uint64_t)gridDim.x * blockDim.x)
    dst[k] = src[idx ? (uint64_t)idx[k] : k * stride];
}

// *out = max over i < n of ptr[i + 1] - ptr[i] (out starts at 0)
__global__ void max_gap(const uint64_t* ptr, uint64_t n, unsigned long long* out) {
  unsigned long long m = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const unsigned long long g = ptr[i + 1] - ptr[i];
    m = g > m ? g : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void u8_to_u32(const uint8_t* in, uint64_t n, uint32_t* out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// S values and T/P counts per source; H flags
__global__ void s_fill(const uint8_t* flag, const uint64_t* pos, uint64_t n, uint32_t Mmax,
                       uint32_t* S_vals) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    if (flag[i]) S_vals[pos[i]] = (uint32_t)(i % Mmax);
}

__global__ void tp_count(const uint8_t* flag, uint32_t R, uint32_t Mmax, const uint32_t* M,
                         const uint32_t* rank_off, uint32_t N, uint32_t* cnt /*[N] by position*/,
                         uint32_t* in_h) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = R;                 // rank of position i
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (rank_off[mid] <= i) lo = mid + 1; else hi = mid;
    }
    const uint32_t sig = lo - 1, s = (uint32_t)i - rank_off[sig];
    uint32_t k = 0;
    for (uint32_t tau = 0; tau < R; ++tau) k += flag[((uint64_t)sig * R + tau) * Mmax + s];
    cnt[i] = k;
    in_h[i] = k ? 1u : 0u;
    (void)M;
  }
}

__global__ void tp_fill(const uint8_t* flag, const uint64_t* spos /*S positions, global*/,
                        const uint64_t* S_off /*[R*R+1]*/, uint32_t R, uint32_t Mmax,
                        const uint32_t* rank_off, uint32_t N, const uint64_t* tp_ptr,
                        uint32_t* T, uint32_t* Pv) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = R;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (rank_off[mid] <= i) lo = mid + 1; else hi = mid;
    }
    const uint32_t sig = lo - 1, s = (uint32_t)i - rank_off[sig];
    uint64_t o = tp_ptr[i];
    for (uint32_t tau = 0; tau < R; ++tau) {
      const uint64_t f = ((uint64_t)sig * R + tau) * Mmax + s;
      if (flag[f]) {
        T[o] = tau;
        Pv[o] = (uint32_t)(spos[f] - S_off[(uint64_t)sig * R + tau]);
        ++o;
      }
    }
  }
}

__global__ void h_fill(const uint32_t* in_h, const uint64_t* hpos, const uint32_t* rank_off, uint32_t R,
                       uint32_t N, uint32_t* H) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (!in_h[i]) continue;
    uint32_t lo = 0, hi = R;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (rank_off[mid] <= i) lo = mid + 1; else hi = mid;
    }
    H[hpos[i]] = (uint32_t)i - rank_off[lo - 1];
  }
}

// I_{0,sigma,tau}[j]: search H_{0,sigma}[j] in R_{tau,sigma} (tau's image list)
__global__ void i_fill(const uint32_t* H, const uint64_t* h_off /*[R+1]*/, uint32_t R, const uint32_t* M,
                       const uint32_t* img_s, const uint64_t* img_off /*[R][R+1] by slot*/,
                       const uint64_t* img_first /*[R]*/, int32_t* I /*[sum_sigma |H| * R]*/) {
  const uint64_t nh = h_off[R];
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nh * R;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t j = x / R;
    const uint32_t tau = (uint32_t)(x - j * R);
    uint32_t lo = 0, hi = R;                 // sigma of H entry j
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (h_off[mid] <= j) lo = mid + 1; else hi = mid;
    }
    const uint32_t sig = lo - 1;
    int32_t out = -1;
    if (tau != sig) {
      const uint32_t slot = sig < tau ? sig + 1 : sig;
      const uint64_t a0 = img_off[(uint64_t)tau * (R + 1) + slot], a1 = img_off[(uint64_t)tau * (R + 1) + slot + 1];
      const uint32_t* Rm = img_s + img_first[tau];
      const uint32_t h = H[j];
      uint64_t l = a0, r = a1;
      while (l < r) {
        const uint64_t m = (l + r) >> 1;
        if (Rm[m] < h) l = m + 1; else r = m;
      }
      if (l < a1 && Rm[l] == h) out = (int32_t)(M[tau] + l);
    }
    I[j * R + tau] = out;
  }
}

__global__ void img_s_of_gid(const uint32_t* img_gid, uint64_t n, uint32_t R, uint64_t magic_R,
                             uint32_t* img_s) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    img_s[i] = (uint32_t)div_magic(img_gid[i], R, magic_R);
}

// image counts per (tau, slot) of the window from the image prefix positions
__global__ void img_slot_offsets(const uint64_t* img_pos, uint32_t N, uint32_t R, uint32_t t0, uint32_t nt,
                                 const uint32_t* dense_off, const uint64_t* img_first,
                                 uint64_t* img_off /*[nt][R+1]*/) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt * (R + 1)) return;
  const uint32_t tl = k / (R + 1), slot = k - tl * (R + 1);
  const uint64_t r = slot < R ? dense_off[(uint64_t)(t0 + tl) * R + slot] : N;
  img_off[k] = img_pos[(uint64_t)tl * N + r] - img_first[tl];
}

unsigned grid_for(snn_ctx* c, uint64_t n) {
  return (unsigned)std::min<uint64_t>((n + MB - 1) / MB, (uint64_t)ctx_num_sms(c) * 32);
}

}  // namespace

#define MCK(call)                                                                     \
  do {                                                                                \
    const cudaError_t e__ = (call);                                                   \
    if (e__ != cudaSuccess) return ctx_fail(c, SNN_ECUDA, cudaGetErrorString(e__));   \
  } while (0)

template <typename T>
static T* alloc_n(snn_ctx* c, uint64_t n) {
  return (T*)ctx_alloc(c, std::max<uint64_t>(n, 1) * sizeof(T));
}

// host copy of src[k * stride] (or src[idx[k]]) for k < count, one device gather and one copy
static int read_boundaries(snn_ctx* c, const uint64_t* src, uint64_t stride, const uint32_t* idx, uint64_t count,
                           uint64_t* host) {
  cudaStream_t st = ctx_stream(c);
  uint64_t* tmp = alloc_n<uint64_t>(c, count);
  if (!tmp) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  gather_u64<<<grid_for(c, count), MB, 0, st>>>(src, stride, idx, count, tmp);
  MCK(cudaGetLastError());
  MCK(cudaMemcpyAsync(host, tmp, count * 8, cudaMemcpyDeviceToHost, st));
  MCK(cudaStreamSynchronize(st));
  ctx_free(c, tmp);
  return SNN_OK;
}

// rank sizes and first positions on the device (both builds)
static int maps_ranks(snn_ctx* c) {
  MapsState& m = ctx_maps(c);
  cudaStream_t st = ctx_stream(c);
  const Geom& g = ctx_geom(c);
  const uint32_t R = g.R, N = g.N;
  const auto& Mh = ctx_rank_sizes(c);
  const auto& roff = ctx_rank_off(c);
  uint32_t Mmax = 0;
  for (auto x : Mh) Mmax = std::max(Mmax, x);
  m.R = R; m.N = N; m.Mmax = Mmax;
  m.M.assign(Mh.begin(), Mh.end());
  m.rank_off.assign(roff.begin(), roff.end());
  m.d_M = alloc_n<uint32_t>(c, R);
  m.d_rank_off = alloc_n<uint32_t>(c, R + 1);
  if (!m.d_M || !m.d_rank_off) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  MCK(cudaMemcpyAsync(m.d_M, Mh.data(), R * 4, cudaMemcpyHostToDevice, st));
  MCK(cudaMemcpyAsync(m.d_rank_off, roff.data(), (R + 1) * 4, cudaMemcpyHostToDevice, st));
  return SNN_OK;
}

// Marks the all-sources images of the pairs (p, tau) with all_src[p * R + tau] on the
// target ranks t0 .. t0 + nt - 1 (tflag, target side) or on every rank (sflag, source
// side).
static int mark_all_sources(snn_ctx* c, const std::vector<DevProj>& projs, const std::vector<uint8_t>& all_src,
                            uint32_t t0, uint32_t nt, uint32_t* tflag, uint8_t* sflag) {
  const Geom& g = ctx_geom(c);
  const uint32_t R = g.R;
  std::vector<AllSrcPair> pairs;
  std::vector<uint32_t> chunk_first(1, 0);
  for (size_t p = 0; p < projs.size(); ++p) {
    const DevProj& P = projs[p];
    if (P.n_src == 0) continue;
    for (uint32_t tau = t0; tau < t0 + nt; ++tau) {
      if (!all_src[p * R + tau]) continue;
      const uint64_t nb = (uint64_t)chunk_first.back() + (P.n_src + kAllSrcChunk - 1) / kAllSrcChunk;
      if (nb > 0x7FFFFFFFull) return ctx_fail(c, SNN_EINVAL, "maps: too many all-sources images");
      pairs.push_back({P.src_first, P.n_src, P.src_stride, tau});
      chunk_first.push_back((uint32_t)nb);
    }
  }
  if (pairs.empty()) return SNN_OK;
  cudaStream_t st = ctx_stream(c);
  AllSrcPair* d_pairs = alloc_n<AllSrcPair>(c, pairs.size());
  uint32_t* d_chunk = alloc_n<uint32_t>(c, chunk_first.size());
  if (!d_pairs || !d_chunk) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  MCK(cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(AllSrcPair), cudaMemcpyHostToDevice, st));
  MCK(cudaMemcpyAsync(d_chunk, chunk_first.data(), chunk_first.size() * 4, cudaMemcpyHostToDevice, st));
  all_sources_flags<<<chunk_first.back(), MB, 0, st>>>(d_pairs, d_chunk, (uint32_t)pairs.size(), R, g.magic_R,
                                                       g.N, t0, ctx_dense_off(c), tflag, sflag, ctx_maps(c).Mmax);
  MCK(cudaGetLastError());
  MCK(cudaStreamSynchronize(st));       // the host vectors above must outlive the copies
  ctx_free(c, d_pairs);
  ctx_free(c, d_chunk);
  return SNN_OK;
}

// Target side for the ranks t0 .. t0 + nt - 1 (dense row starts [nt][N + 1]): images,
// per-rank compacted rows (local rows, then images), R/L offsets per (rank, slot).
static int maps_target(snn_ctx* c, uint32_t t0, uint32_t nt, const std::vector<DevProj>& projs,
                       const std::vector<uint8_t>& all_src) {
  MapsState& m = ctx_maps(c);
  cudaStream_t st = ctx_stream(c);
  const Geom& g = ctx_geom(c);
  const uint32_t R = g.R, N = g.N;
  const uint64_t RN = (uint64_t)nt * N;
  uint32_t* flag = alloc_n<uint32_t>(c, RN);
  uint64_t* img_pos = alloc_n<uint64_t>(c, RN + 1);
  if (!flag || !img_pos) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  image_flags<<<grid_for(c, RN), MB, 0, st>>>(ctx_dense(c), N, t0, nt, m.d_M, flag);
  MCK(cudaGetLastError());
  {
    const int rc = mark_all_sources(c, projs, all_src, t0, nt, flag, nullptr);
    if (rc != SNN_OK) return rc;
  }
  MCK(exclusive_scan(c, flag, RN, img_pos));
  // images per rank: img_pos at rank boundaries
  std::vector<uint64_t> bounds(nt + 1);
  {
    const int rc = read_boundaries(c, img_pos, N, nullptr, nt + 1, bounds.data());
    if (rc != SNN_OK) return rc;
  }
  m.t0 = t0;
  m.nt = nt;
  m.n_img.assign(nt, 0);
  m.img_first.assign(nt + 1, 0);
  m.rows_off.assign(nt + 1, 0);
  for (uint32_t t = 0; t < nt; ++t) {
    m.n_img[t] = bounds[t + 1] - bounds[t];
    m.img_first[t + 1] = m.img_first[t] + m.n_img[t];
    m.rows_off[t + 1] = m.rows_off[t] + m.M[t0 + t] + m.n_img[t] + 1;
  }
  m.n_images_total = m.img_first[nt];
  m.d_rows_off = alloc_n<uint64_t>(c, nt + 1);
  m.d_img_first = alloc_n<uint64_t>(c, nt + 1);
  m.rows = alloc_n<uint64_t>(c, m.rows_off[nt]);
  m.img_gid = alloc_n<uint32_t>(c, m.n_images_total);
  m.img_s = alloc_n<uint32_t>(c, m.n_images_total);
  m.d_img_off = alloc_n<uint64_t>(c, (uint64_t)nt * (R + 1));
  if (!m.d_rows_off || !m.d_img_first || !m.rows || !m.img_gid || !m.img_s || !m.d_img_off)
    return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  MCK(cudaMemcpyAsync(m.d_rows_off, m.rows_off.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, st));
  MCK(cudaMemcpyAsync(m.d_img_first, m.img_first.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, st));
  image_fill<<<grid_for(c, RN), MB, 0, st>>>(ctx_dense(c), N, R, t0, nt, m.d_M, flag, img_pos, m.d_rows_off,
                                            ctx_dense_off(c), ctx_dseg_start(c), m.rows, m.img_gid);
  MCK(cudaGetLastError());
  if (m.n_images_total)
    img_s_of_gid<<<grid_for(c, m.n_images_total), MB, 0, st>>>(m.img_gid, m.n_images_total, R, g.magic_R, m.img_s);
  MCK(cudaGetLastError());
  img_slot_offsets<<<(nt * (R + 1) + MB - 1) / MB, MB, 0, st>>>(img_pos, N, R, t0, nt, ctx_dense_off(c),
                                                               m.d_img_first, m.d_img_off);
  MCK(cudaGetLastError());
  m.img_off.resize((size_t)nt * (R + 1));
  MCK(cudaMemcpyAsync(m.img_off.data(), m.d_img_off, (size_t)nt * (R + 1) * 8, cudaMemcpyDeviceToHost, st));
  ctx_free(c, flag);
  ctx_free(c, img_pos);

  return SNN_OK;
}

int build_maps(snn_ctx* c, const std::vector<DevProj>& projs, const DevProj* d_projs, const uint64_t* d_cbase,
               const uint32_t* d_tables, const std::vector<uint8_t>& all_src) {
  MapsState& m = ctx_maps(c);
  cudaStream_t st = ctx_stream(c);
  const Geom& g = ctx_geom(c);
  const uint32_t R = g.R, N = g.N;
  const auto& roff = ctx_rank_off(c);
  int rc = maps_ranks(c);
  if (rc != SNN_OK) return rc;
  const uint32_t Mmax = m.Mmax;
  rc = maps_target(c, 0, R, projs, all_src);
  if (rc != SNN_OK) return rc;

  // ---- source side: regenerated sources -> S, T/P, H, I, G/Q ----
  const uint64_t nf = (uint64_t)R * R * Mmax;
  uint8_t* sflag = alloc_n<uint8_t>(c, nf);
  if (!sflag) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  MCK(cudaMemsetAsync(sflag, 0, nf, st));
  // a projection forced on every rank holding its targets needs no regeneration: its
  // connections only reach (sigma, s, tau) that the marking below sets anyway
  std::vector<uint8_t> skip(projs.size(), 1);
  uint64_t ctot = 0;
  for (size_t p = 0; p < projs.size(); ++p) {
    const DevProj& P = projs[p];
    for (uint32_t j = 0; j < std::min(P.n_tgt, R) && skip[p]; ++j)
      skip[p] = all_src[p * R + (P.tgt_first + (uint64_t)j * P.tgt_stride) % R];
    if (!skip[p]) ctot = std::max(ctot, P.cbase + P.csize);
  }
  if (ctot) {
    uint8_t* d_skip = alloc_n<uint8_t>(c, projs.size());
    if (!d_skip) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
    MCK(cudaMemcpyAsync(d_skip, skip.data(), projs.size(), cudaMemcpyHostToDevice, st));
    source_flags<<<grid_for(c, ctot), MB, 0, st>>>(d_projs, (uint32_t)projs.size(), d_cbase, ctot, R, g.magic_R,
                                                  Mmax, d_tables, d_skip, sflag);
    MCK(cudaGetLastError());
    MCK(cudaStreamSynchronize(st));       // skip must outlive the copy
    ctx_free(c, d_skip);
  }
  rc = mark_all_sources(c, projs, all_src, 0, R, nullptr, sflag);
  if (rc != SNN_OK) return rc;
  uint32_t* f32v = alloc_n<uint32_t>(c, nf);
  m.spos = alloc_n<uint64_t>(c, nf + 1);
  if (!f32v || !m.spos) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  u8_to_u32<<<grid_for(c, nf), MB, 0, st>>>(sflag, nf, f32v);
  MCK(cudaGetLastError());
  MCK(exclusive_scan(c, f32v, nf, m.spos));
  ctx_free(c, f32v);
  // S offsets per (sigma, tau): positions at plane boundaries
  m.S_off.assign((size_t)R * R + 1, 0);
  {
    const int rc = read_boundaries(c, m.spos, Mmax, nullptr, (uint64_t)R * R + 1, m.S_off.data());
    if (rc != SNN_OK) return rc;
  }
  m.d_S_off = alloc_n<uint64_t>(c, (uint64_t)R * R + 1);
  m.S_vals = alloc_n<uint32_t>(c, m.S_off[(size_t)R * R]);
  if (!m.d_S_off || !m.S_vals) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  MCK(cudaMemcpyAsync(m.d_S_off, m.S_off.data(), ((size_t)R * R + 1) * 8, cudaMemcpyHostToDevice, st));
  s_fill<<<grid_for(c, nf), MB, 0, st>>>(sflag, m.spos, nf, Mmax, m.S_vals);
  MCK(cudaGetLastError());
  // T/P per source position, H membership
  uint32_t* tpc = alloc_n<uint32_t>(c, N);
  uint32_t* inh = alloc_n<uint32_t>(c, N);
  m.tp_ptr = alloc_n<uint64_t>(c, N + 1);
  m.h_pos = alloc_n<uint64_t>(c, N + 1);
  if (!tpc || !inh || !m.tp_ptr || !m.h_pos) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  tp_count<<<grid_for(c, N), MB, 0, st>>>(sflag, R, Mmax, m.d_M, m.d_rank_off, N, tpc, inh);
  MCK(cudaGetLastError());
  MCK(exclusive_scan(c, tpc, N, m.tp_ptr));
  MCK(exclusive_scan(c, inh, N, m.h_pos));
  uint64_t ntp = 0, nh = 0;
  MCK(cudaMemcpyAsync(&ntp, m.tp_ptr + N, 8, cudaMemcpyDeviceToHost, st));
  MCK(cudaMemcpyAsync(&nh, m.h_pos + N, 8, cudaMemcpyDeviceToHost, st));
  m.h_off.assign(R + 1, 0);
  {
    const int rc = read_boundaries(c, m.h_pos, 0, m.d_rank_off, R + 1, m.h_off.data());
    if (rc != SNN_OK) return rc;
  }
  m.n_tp = ntp;
  m.n_h = nh;
  m.T = alloc_n<uint32_t>(c, ntp);
  m.P = alloc_n<uint32_t>(c, ntp);
  m.H = alloc_n<uint32_t>(c, nh);
  m.I = alloc_n<int32_t>(c, nh * R);
  m.d_h_off = alloc_n<uint64_t>(c, R + 1);
  if (!m.T || !m.P || !m.H || !m.I || !m.d_h_off) return ctx_fail(c, SNN_ENOMEM, "maps: allocation failed");
  MCK(cudaMemcpyAsync(m.d_h_off, m.h_off.data(), (R + 1) * 8, cudaMemcpyHostToDevice, st));
  tp_fill<<<grid_for(c, N), MB, 0, st>>>(sflag, m.spos, m.d_S_off, R, Mmax, m.d_rank_off, N, m.tp_ptr, m.T, m.P);
  MCK(cudaGetLastError());
  h_fill<<<grid_for(c, N), MB, 0, st>>>(inh, m.h_pos, m.d_rank_off, R, N, m.H);
  MCK(cudaGetLastError());
  if (nh)
    i_fill<<<grid_for(c, nh * R), MB, 0, st>>>(m.H, m.d_h_off, R, m.d_M, m.img_s, m.d_img_off, m.d_img_first, m.I);
  MCK(cudaGetLastError());
  ctx_free(c, tpc);
  ctx_free(c, inh);
  ctx_free(c, sflag);
  MCK(cudaStreamSynchronize(st));
  return SNN_OK;
}

// Dry run (one rank's share of the network): the target side of that rank only; the
// source-side maps would need every rank's connections.
int build_maps_dry(snn_ctx* c, uint32_t rank, const std::vector<DevProj>& projs,
                   const std::vector<uint8_t>& all_src) {
  int rc = maps_ranks(c);
  if (rc != SNN_OK) return rc;
  rc = maps_target(c, rank, 1, projs, all_src);
  if (rc != SNN_OK) return rc;
  ctx_maps(c).dry = true;
  MCK(cudaStreamSynchronize(ctx_stream(c)));
  return SNN_OK;
}

// ---- routing: spikes -> delivery work items (global rows) ----
namespace {
// One warp per spike: the warp reserves the spike's rows in the work list with one
// atomic, then its lanes fill them in parallel, each row with the rank it belongs to.
__global__ void route_kernel(RouteArgs r, uint32_t k_step) {
  pdl_wait();                      // the update's spike list is complete
  pdl_trigger();
  const uint32_t n = __ldcg(r.step) + k_step;
  const uint32_t nspk = __ldcg(r.n_spk + (n & 1));
  const uint32_t* spk = r.spk + (uint64_t)(n & 1) * r.N;
  if (blockIdx.x == 0 && threadIdx.x == 0) r.n_work[(n + 1) & 1] = 0;
  uint32_t* work = r.work + (uint64_t)(n & 1) * r.work_cap;
  uint32_t* wtau = r.work_tau + (uint64_t)(n & 1) * r.work_cap;
  const uint32_t lane = threadIdx.x & 31, lt = (1u << lane) - 1;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t k = gw; k < nspk; k += nw) {
    const uint32_t i = __ldcg(spk + k);                      // neuron position
    uint32_t lo = 0, hi = r.R;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (r.rank_off[mid] <= i) lo = mid + 1; else hi = mid;
    }
    const uint32_t sig = lo - 1, s = i - r.rank_off[sig];
    // rows: the local row on the source's own rank, then one image row per other rank
    uint64_t o0, o1;
    uint32_t cnt = 1;
    if (r.exchange == 0) {
      o0 = r.tp_ptr[i];
      o1 = r.tp_ptr[i + 1];
      cnt += (uint32_t)(o1 - o0);
    } else {
      o0 = r.h_pos[i];
      o1 = r.h_pos[i + 1];
      if (o1 > o0)
        for (uint32_t t0 = 0; t0 < r.R; t0 += 32) {
          const uint32_t tau = t0 + lane;
          const bool has = tau < r.R && tau != sig && r.I[o0 * r.R + tau] >= 0;
          cnt += __popc(__ballot_sync(0xffffffffu, has));
        }
    }
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&r.n_work[n & 1], cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((uint64_t)base + cnt > r.work_cap) {
      if (lane == 0) atomicOr(r.err, kErrBounds);
      continue;
    }
    if (lane == 0) {
      work[base] = (uint32_t)(r.rows_off[sig] + s);
      wtau[base] = sig;
    }
    if (r.exchange == 0) {
      // point-to-point: packets of positions P to ranks T, received through L
      for (uint64_t j = o0 + lane; j < o1; j += 32) {
        const uint32_t tau = r.T[j];
        const uint32_t slot = sig < tau ? sig + 1 : sig;
        const uint64_t img = r.img_off[(uint64_t)tau * (r.R + 1) + slot] + r.P[j];   // L - M_tau
        const uint64_t wpos = base + 1 + (j - o0);
        work[wpos] = (uint32_t)(r.rows_off[tau] + r.M[tau] + img);
        wtau[wpos] = tau;
      }
    } else if (o1 > o0) {
      // collective: position q in H_{0,sigma}, every other rank looks up I
      const uint64_t q = o0;
      uint32_t w = base + 1;
      for (uint32_t t0 = 0; t0 < r.R; t0 += 32) {
        const uint32_t tau = t0 + lane;
        const int32_t L = (tau < r.R && tau != sig) ? r.I[q * r.R + tau] : -1;
        const uint32_t m = __ballot_sync(0xffffffffu, L >= 0);
        if (L >= 0) {
          const uint32_t wpos = w + __popc(m & lt);
          work[wpos] = (uint32_t)(r.rows_off[tau] + (uint32_t)L);
          wtau[wpos] = tau;
        }
        w += __popc(m);
      }
    }
  }
}
}  // namespace

namespace {
// fp16 weights are stored as w / scale with a power-of-two scale per source neuron;
// delivery multiplies by the scale of the row's source: for rank tau's local row s the
// neuron s R + tau, for an image row the image's gid.  One entry per row start of the
// concatenated per-rank rows (the sentinel after each rank's rows gets 1).
__global__ void row_scale_fill(const uint64_t* rows_off, uint32_t R, const uint32_t* M, const uint64_t* img_first,
                               const uint32_t* img_gid, const float* scale_src, float* out, uint64_t total) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t w = upper_bound_u64(rows_off, R + 1, x) - 1;
    const uint64_t r = x - rows_off[w];
    const uint64_t n_img = rows_off[w + 1] - rows_off[w] - 1 - M[w];
    float v = 1.0f;
    if (r < M[w]) v = scale_src[r * R + w];
    else if (r - M[w] < n_img) v = scale_src[img_gid[img_first[w] + (r - M[w])]];
    out[x] = v;
  }
}
}  // namespace

int setup_routing(snn_ctx* c) {
  MapsState& m = ctx_maps(c);
  SimArgs& s = ctx_sim(c);
  RouteArgs& r = m.route;
  r.R = m.R; r.N = m.N;
  r.rank_off = m.d_rank_off; r.M = m.d_M; r.rows_off = m.d_rows_off;
  r.tp_ptr = m.tp_ptr; r.T = m.T; r.P = m.P; r.img_off = m.d_img_off;
  r.h_pos = m.h_pos; r.I = m.I;
  r.exchange = (uint32_t)ctx_exchange(c);
  r.step = s.step; r.err = ctx_err(c);
  r.spk = s.spk; r.n_spk = s.n_spk;
  // capacity: every neuron spiking once with all its images
  uint64_t maxfan = 1 + (r.exchange == 0 ? 0 : (uint64_t)m.R - 1);
  if (r.exchange == 0) {
    // the largest T list
    unsigned long long* d_mx = alloc_n<unsigned long long>(c, 1);
    if (!d_mx) return ctx_fail(c, SNN_ENOMEM, "routing: allocation failed");
    cudaStream_t st = ctx_stream(c);
    MCK(cudaMemsetAsync(d_mx, 0, 8, st));
    max_gap<<<grid_for(c, m.N), MB, 0, st>>>(m.tp_ptr, m.N, d_mx);
    MCK(cudaGetLastError());
    unsigned long long mx = 0;
    MCK(cudaMemcpyAsync(&mx, d_mx, 8, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    ctx_free(c, d_mx);
    maxfan = 1 + mx;
  }
  r.work_cap = std::min<uint64_t>((uint64_t)m.N * maxfan, 0xFFFFFFFFull);
  r.work = alloc_n<uint32_t>(c, 2 * r.work_cap);
  r.work_tau = alloc_n<uint32_t>(c, 2 * r.work_cap);
  r.n_work = alloc_n<uint32_t>(c, 2);
  if (!r.work || !r.work_tau || !r.n_work) return ctx_fail(c, SNN_ENOMEM, "routing: allocation failed");
  MCK(cudaMemsetAsync(r.n_work, 0, 8, ctx_stream(c)));
  s.work = r.work; s.n_work = r.n_work; s.work_stride = r.work_cap; s.work_rank = r.work_tau;
  s.rows = m.rows; s.rows_off = m.d_rows_off; s.rank_off = m.d_rank_off;
  if (ctx_scale_src(c)) {
    const uint64_t total = m.rows_off.back();
    float* rs = alloc_n<float>(c, std::max<uint64_t>(total, 1));
    if (!rs) return ctx_fail(c, SNN_ENOMEM, "routing: allocation failed");
    row_scale_fill<<<grid_for(c, total), MB, 0, ctx_stream(c)>>>(m.d_rows_off, m.R, m.d_M, m.d_img_first, m.img_gid,
                                                                 ctx_scale_src(c), rs, total);
    MCK(cudaGetLastError());
    s.row_scale = rs;
  }
  // rows average E / (local rows + images); short rows are delivered by lane groups
  const uint64_t n_rows = m.rows_off.empty() ? 0 : m.rows_off.back();
  const double avg = n_rows ? (double)ctx_geom_synapses(c) / (double)n_rows : 0.0;
  s.item_lanes = 0;
  if (avg < 256.0) {
    uint32_t L = 4;
    while (L < 32 && L * 4 < avg) L *= 2;     // about four events per lane
    s.item_lanes = L;
  }
  return SNN_OK;
}

cudaError_t launch_route(snn_ctx* c, uint32_t k_step, bool pdl) {
  MapsState& m = ctx_maps(c);
  return launch_pdl(route_kernel, dim3((unsigned)std::max(1, ctx_num_sms(c) * 2)), dim3(256), ctx_stream(c), pdl,
                    m.route, k_step);
}

uint32_t route_kernels_per_step(snn_ctx* c) { return ctx_geom(c).R > 1 ? 1 : 0; }

// ---- inspection ----
// index of `rank` in the target-side arrays, or -1 (with the error set) when a dry run
// did not build it
static int64_t window_of(snn_ctx* c, uint32_t rank) {
  const MapsState& m = ctx_maps(c);
  if (rank < m.t0 || rank >= m.t0 + m.nt) {
    ctx_fail(c, SNN_ESTATE, ("a dry run built only rank " + std::to_string(m.t0)).c_str());
    return -1;
  }
  return (int64_t)(rank - m.t0);
}

int rank_row_ptr(snn_ctx* c, uint32_t rank, std::vector<uint64_t>* rp) {
  const Geom& g = ctx_geom(c);
  if (g.R == 1) {
    rp->resize((size_t)g.N + 1);
    MCK(cudaMemcpy(rp->data(), ctx_dense(c), ((size_t)g.N + 1) * 8, cudaMemcpyDeviceToHost));
    return SNN_OK;
  }
  MapsState& m = ctx_maps(c);
  const int64_t w = window_of(c, rank);
  if (w < 0) return SNN_ESTATE;
  const uint64_t a = m.rows_off[w], b = m.rows_off[w + 1];
  rp->resize(b - a);
  MCK(cudaMemcpy(rp->data(), m.rows + a, (b - a) * 8, cudaMemcpyDeviceToHost));
  return SNN_OK;
}

int rank_row_scales(snn_ctx* c, uint32_t rank, std::vector<float>* scales) {
  const Geom& g = ctx_geom(c);
  std::vector<float> src(g.N, 1.0f);
  if (ctx_scale_src(c)) MCK(cudaMemcpy(src.data(), ctx_scale_src(c), (size_t)g.N * 4, cudaMemcpyDeviceToHost));
  if (g.R == 1) {
    *scales = src;
    return SNN_OK;
  }
  MapsState& m = ctx_maps(c);
  const int64_t w = window_of(c, rank);
  if (w < 0) return SNN_ESTATE;
  const uint32_t M = m.M[rank];
  std::vector<uint32_t> gids(m.n_img[w]);
  if (!gids.empty())
    MCK(cudaMemcpy(gids.data(), m.img_gid + m.img_first[w], gids.size() * 4, cudaMemcpyDeviceToHost));
  scales->assign(M + gids.size(), 1.0f);
  for (uint32_t s = 0; s < M; ++s) (*scales)[s] = src[(uint64_t)s * g.R + rank];
  for (size_t k = 0; k < gids.size(); ++k) (*scales)[M + k] = src[gids[k]];
  return SNN_OK;
}

int rank_row_bounds(snn_ctx* c, uint32_t rank, uint64_t row, uint64_t ab[2], float* scale) {
  const Geom& g = ctx_geom(c);
  std::vector<float> sc;
  if (g.R == 1) {
    if (row >= g.N) return ctx_fail(c, SNN_EINVAL, "row out of range");
    MCK(cudaMemcpy(ab, ctx_dense(c) + row, 16, cudaMemcpyDeviceToHost));
    *scale = 1.0f;
    if (ctx_scale_src(c)) MCK(cudaMemcpy(scale, ctx_scale_src(c) + row, 4, cudaMemcpyDeviceToHost));
    return SNN_OK;
  }
  MapsState& m = ctx_maps(c);
  const int64_t w = window_of(c, rank);
  if (w < 0) return SNN_ESTATE;
  const uint64_t nrows = m.rows_off[w + 1] - m.rows_off[w] - 1;
  if (row >= nrows) return ctx_fail(c, SNN_EINVAL, "row out of range");
  MCK(cudaMemcpy(ab, m.rows + m.rows_off[w] + row, 16, cudaMemcpyDeviceToHost));
  *scale = 1.0f;
  if (ctx_scale_src(c)) {
    uint32_t gid;
    if (row < m.M[rank]) gid = (uint32_t)(row * g.R + rank);
    else MCK(cudaMemcpy(&gid, m.img_gid + m.img_first[w] + (row - m.M[rank]), 4, cudaMemcpyDeviceToHost));
    MCK(cudaMemcpy(scale, ctx_scale_src(c) + gid, 4, cudaMemcpyDeviceToHost));
  }
  return SNN_OK;
}

}  // namespace snn

using namespace snn;

extern "C" int snn_get_maps(snn_ctx* c, uint32_t tau, uint32_t sigma, int32_t which, int64_t* host_buf,
                            uint64_t cap, uint64_t* n_out) {
  if (!c) return SNN_EINVAL;
  if (n_out) *n_out = 0;
  const Geom& g = ctx_geom(c);
  if (g.R <= 1) return ctx_fail(c, SNN_EINVAL, "maps exist only with more than one logical rank");
  MapsState& m = ctx_maps(c);
  if (!m.rows) return ctx_fail(c, SNN_ESTATE, "no maps before calibrate");
  const uint32_t R = g.R;
  if (tau >= R || sigma >= R) return ctx_fail(c, SNN_EINVAL, "rank out of range");
  if (m.dry && which != SNN_MAP_R && which != SNN_MAP_L)
    return ctx_fail(c, SNN_ESTATE, "a dry run builds no source-side maps");
  std::vector<int64_t> out;
  auto fetch_u32 = [&](const uint32_t* p, uint64_t a, uint64_t b) -> int {
    std::vector<uint32_t> t(b - a);
    if (b > a) MCK(cudaMemcpy(t.data(), p + a, (b - a) * 4, cudaMemcpyDeviceToHost));
    out.assign(t.begin(), t.end());
    return SNN_OK;
  };
  int rc = SNN_OK;
  switch (which) {
    case SNN_MAP_R:
    case SNN_MAP_L: {
      if (tau == sigma) break;
      const int64_t w = window_of(c, tau);
      if (w < 0) return SNN_ESTATE;
      const uint32_t slot = sigma < tau ? sigma + 1 : sigma;
      const uint64_t a = m.img_off[(size_t)w * (R + 1) + slot], b = m.img_off[(size_t)w * (R + 1) + slot + 1];
      if (which == SNN_MAP_R) {
        rc = fetch_u32(m.img_s, m.img_first[w] + a, m.img_first[w] + b);
      } else {
        out.resize(b - a);
        for (uint64_t k = a; k < b; ++k) out[k - a] = (int64_t)m.M[tau] + (int64_t)k;
      }
      break;
    }
    case SNN_MAP_S: {
      if (tau == sigma) break;
      const uint64_t k = (uint64_t)sigma * R + tau;
      rc = fetch_u32(m.S_vals, m.S_off[k], m.S_off[k + 1]);
      break;
    }
    case SNN_MAP_T:
    case SNN_MAP_P:
    case SNN_MAP_TP_PTR: {
      const uint32_t a = m.rank_off[sigma], b = m.rank_off[sigma + 1];
      std::vector<uint64_t> ptr(b - a + 1);
      MCK(cudaMemcpy(ptr.data(), m.tp_ptr + a, ptr.size() * 8, cudaMemcpyDeviceToHost));
      if (which == SNN_MAP_TP_PTR) {
        out.resize(ptr.size());
        for (size_t k = 0; k < ptr.size(); ++k) out[k] = (int64_t)(ptr[k] - ptr[0]);
      } else {
        rc = fetch_u32(which == SNN_MAP_T ? m.T : m.P, ptr.front(), ptr.back());
      }
      break;
    }
    case SNN_MAP_H:
      rc = fetch_u32(m.H, m.h_off[sigma], m.h_off[sigma + 1]);
      break;
    case SNN_MAP_I: {
      const uint64_t a = m.h_off[sigma], b = m.h_off[sigma + 1];
      std::vector<int32_t> t((b - a) * R);
      if (b > a) MCK(cudaMemcpy(t.data(), m.I + a * R, t.size() * 4, cudaMemcpyDeviceToHost));
      out.resize(b - a);
      for (uint64_t j = 0; j < b - a; ++j) out[j] = t[j * R + tau];
      break;
    }
    case SNN_MAP_Q:
    case SNN_MAP_GQ_PTR: {
      const uint32_t a = m.rank_off[sigma], b = m.rank_off[sigma + 1];
      std::vector<uint64_t> hp(b - a + 1);
      MCK(cudaMemcpy(hp.data(), m.h_pos + a, hp.size() * 8, cudaMemcpyDeviceToHost));
      if (which == SNN_MAP_GQ_PTR) {
        out.resize(hp.size());
        for (size_t k = 0; k < hp.size(); ++k) out[k] = (int64_t)(hp[k] - hp[0]);
      } else {
        out.resize(hp.back() - hp.front());
        for (size_t k = 0; k < out.size(); ++k) out[k] = (int64_t)k;
      }
      break;
    }
    default:
      return ctx_fail(c, SNN_EINVAL, "unknown map selector");
  }
  if (rc != SNN_OK) return rc;
  if (n_out) *n_out = out.size();
  if (host_buf) {
    if (cap < out.size()) return ctx_fail(c, SNN_EOVERFLOW, "map buffer too small");
    std::copy(out.begin(), out.end(), host_buf);
  }
  return SNN_OK;
}
