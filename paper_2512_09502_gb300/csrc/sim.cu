// sim.cu -- state propagation: iaf_psc_exp exact-integration update and ring-buffer
// spike delivery through the source-sorted connection rows.
//
// Delivery follows the paper's Appendix (point-to-point example, delivery figure):
// a spike reaches the targets through the outgoing connections of its row (a local
// neuron, or an image neuron on the target rank), and each target's circular buffer
// slot shifted by the connection delay accumulates multiplicity x weight.  The neuron
// model (not stated in the paper) is the exactly integrated iaf_psc_exp of Rotter &
// Diesmann (1999) with propagators computed in FP64 at calibrate.
//
// When every population has tau_syn_ex == tau_syn_in the two receptors obey the same
// linear dynamics, so one ring and one current (I_ex, holding the sum) give the same
// membrane potential with half the ring footprint; I_in then stays 0.
//
// One step = update_kernel (reads and clears ring slot n, integrates, appends spikes
// to the per-step delivery list) then deliver_kernel (walks the rows of every listed
// spike and red.add's the weights into slots n + d; a CTA per row slice for the long
// rows of one rank, deliver_rows_kernel's lane groups for the short image rows of many
// ranks).  The step needs no host involvement
// and is captured as a CUDA graph.  The step index of a launch is *step + k, with k baked
// into the launch (or graph node); one advance kernel after a batch of steps adds the
// batch length, so no per-step completion handshake is needed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sim_internal.cuh"

namespace snn {

constexpr int UPD_BLOCK = 256;
constexpr int UPD_Q = 4;          // consecutive neurons per thread
constexpr int DEL_BLOCK = 256;
constexpr int DEL_ILP = 4;        // events per thread per iteration
constexpr uint32_t MAX_SMEM_DRIVES = 16;

// #{i < len : thr[i] <= w}; thresholds are ascending
__device__ __forceinline__ uint32_t table_count(const uint32_t* thr, uint32_t len, uint32_t w) {
  if (len <= 32) {           // short tables (Poisson counts): independent compares
    uint32_t c = 0;
    for (uint32_t i = 0; i < len; ++i) c += thr[i] <= w ? 1u : 0u;
    return c;
  }
  return upper_bound_u32(thr, len, w);
}

// Poisson counts of the four neurons of one thread for drive dr at step n, from word
// (g mod 4) of the block with counter (g div 4, n) (one block when the four are
// consecutive gids on one rank); in[k]: neuron k is driven by dr.
__device__ __forceinline__ void poisson_counts4(const SimArgs& a, const DevDrive& dr, const uint32_t* s_tbl,
                                                uint32_t q, uint32_t n, bool full, const bool* live,
                                                const uint32_t* gid, uint32_t* cnt, bool* in) {
  uint32_t wd[UPD_Q];
  if (a.R == 1 && full) {
    const uint4 b = philox_stream((uint64_t)q | ((uint64_t)n << 32), dr.idx, kPurposePoisson, dr.seed);
    wd[0] = b.x; wd[1] = b.y; wd[2] = b.z; wd[3] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) {
      wd[k] = 0u;
      if (live[k]) {
        const uint4 b = philox_stream((uint64_t)(gid[k] >> 2) | ((uint64_t)n << 32), dr.idx,
                                      kPurposePoisson, dr.seed);
        const uint32_t lo = (gid[k] & 1u) ? b.y : b.x, hi = (gid[k] & 1u) ? b.w : b.z;
        wd[k] = (gid[k] & 2u) ? hi : lo;
      }
    }
  }
  uint32_t wmax = 0;
#pragma unroll
  for (int k = 0; k < UPD_Q; ++k) {
    in[k] = live[k] && gid[k] - dr.first < dr.n;
    cnt[k] = 0;
    if (in[k]) wmax = wd[k] > wmax ? wd[k] : wmax;
  }
  const uint32_t* tb = s_tbl + dr.tbl_off;
  if (dr.tbl_len <= 32) {          // one pass over the ascending thresholds serves all four
    for (uint32_t j = 0; j < dr.tbl_len; ++j) {
      const uint32_t t = tb[j];
      if (t > wmax) break;
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) cnt[k] += t <= wd[k] ? 1u : 0u;
    }
  } else {
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) cnt[k] = upper_bound_u32(tb, dr.tbl_len, wd[k]);
  }
}

// One thread updates UPD_Q = 4 consecutive neuron positions: 16-byte loads and stores
// of the state and ring slot (the host guarantees 16-byte aligned arrays and a ring
// stride that is a multiple of 4) and, on one rank, a single Philox block for the four
// Poisson counts (neuron g draws word g mod 4 of the block with counter (g div 4, n)).
//
// The spike decision of step n needs V, the currents and refractoriness of step n - 1
// only: the ring input of step n enters the currents.  So everything up to the spike
// append -- state loads, V propagation, the Poisson counts of up to EARLY_DRIVES drives,
// the threshold, the V / refr stores and the append to list n & 1 -- precedes pdl_wait
// and overlaps the previous step's delivery.  After the wait come the ring slot (read
// and cleared), I <- P11 I + ring, the drives in drive order (the order of the method's
// step), and the reset of list (n + 1) & 1, which the previous delivery reads.
constexpr uint32_t EARLY_DRIVES = 2;
__global__ void __launch_bounds__(UPD_BLOCK, 4) update_kernel(SimArgs a, uint32_t k_step) {
  __shared__ uint32_t s_tbl[256];
  __shared__ DevPop s_pop[64];
  __shared__ DevDrive s_dr[MAX_SMEM_DRIVES];
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31;
  const uint32_t n = __ldcg(a.step) + k_step;   // written only by the advance kernel
  for (uint32_t i = tid; i < a.poisson_tbl_len && i < 256; i += UPD_BLOCK) s_tbl[i] = a.poisson_tbl[i];
  for (uint32_t i = tid; i < a.npops && i < 64; i += UPD_BLOCK) s_pop[i] = a.pops[i];
  for (uint32_t i = tid; i < a.ndrives && i < MAX_SMEM_DRIVES; i += UPD_BLOCK) s_dr[i] = a.drives[i];
  const uint32_t slot = n % a.ring_slots;
  float* rex = a.ring + ((uint64_t)slot * a.n_rec) * a.ring_stride;
  float* rin = rex + a.ring_stride;
  const bool two = a.n_rec == 2;
  const bool early = a.ndrives <= EARLY_DRIVES;
  const uint32_t nq = (a.N + UPD_Q - 1) / UPD_Q;
  bool staged = false;             // the shared tables are published by the first iteration's barrier
  for (uint32_t qb = blockIdx.x * UPD_BLOCK; qb < nq; qb += gridDim.x * UPD_BLOCK) {
    const uint32_t q = qb + tid;
    const uint32_t i0 = q * UPD_Q;
    const bool full = q < nq && i0 + UPD_Q <= a.N;
    float V[UPD_Q], Iex[UPD_Q], Iin[UPD_Q];
    uint32_t refr[UPD_Q], pi[UPD_Q], gid[UPD_Q];
    bool live[UPD_Q], spike[UPD_Q];
    // phase 1: the state loads of the four neurons (I_in is identically 0 with a merged ring)
    if (full) {
      // state written by the previous update: L2 loads (no L1 line may outlive a step)
      const float4 v = __ldcg(reinterpret_cast<const float4*>(a.V) + q);
      const float4 e = __ldcg(reinterpret_cast<const float4*>(a.Iex) + q);
      const uint2 r = __ldcg(reinterpret_cast<const uint2*>(a.refr) + q);
      const uint2 p = reinterpret_cast<const uint2*>(a.pop_of)[q];
      V[0] = v.x; V[1] = v.y; V[2] = v.z; V[3] = v.w;
      Iex[0] = e.x; Iex[1] = e.y; Iex[2] = e.z; Iex[3] = e.w;
      refr[0] = r.x & 0xFFFFu; refr[1] = r.x >> 16; refr[2] = r.y & 0xFFFFu; refr[3] = r.y >> 16;
      pi[0] = p.x & 0xFFFFu; pi[1] = p.x >> 16; pi[2] = p.y & 0xFFFFu; pi[3] = p.y >> 16;
      if (two) {
        const float4 ii = __ldcg(reinterpret_cast<const float4*>(a.Iin) + q);
        Iin[0] = ii.x; Iin[1] = ii.y; Iin[2] = ii.z; Iin[3] = ii.w;
      } else {
#pragma unroll
        for (int k = 0; k < UPD_Q; ++k) Iin[k] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) live[k] = true;
    } else {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        const uint32_t i = i0 + k;
        live[k] = q < nq && i < a.N;
        V[k] = Iex[k] = Iin[k] = 0.f;
        refr[k] = pi[k] = 0;
        if (live[k]) {
          V[k] = __ldcg(a.V + i); Iex[k] = __ldcg(a.Iex + i);
          refr[k] = __ldcg(a.refr + i); pi[k] = a.pop_of[i];
          if (two) Iin[k] = __ldcg(a.Iin + i);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) gid[k] = a.R == 1 ? i0 + k : (live[k] ? a.gid_of[i0 + k] : 0u);
    if (!staged) {                 // block-uniform: the state loads above are already in flight
      __syncthreads();
      staged = true;
    }
    // phase 2: membrane potential (from the currents of step n - 1) and the spike decision
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) {
      spike[k] = false;
      if (live[k]) {
        const DevPop& P = pi[k] < 64 ? s_pop[pi[k]] : a.pops[pi[k]];
        float v = V[k];
        uint32_t rf = refr[k];
        if (rf == 0) v = P.P22 * v + P.P21ex * Iex[k] + P.P21in * Iin[k] + P.P20 * P.Ie;
        else --rf;
        if (v >= P.Vth) {
          v = P.Vreset;
          rf = P.ref_steps;
          spike[k] = true;
        }
        V[k] = v; refr[k] = rf;
      }
    }
    uint32_t cnt_e[EARLY_DRIVES][UPD_Q];
    bool in_e[EARLY_DRIVES][UPD_Q];
    if (early) {
#pragma unroll
      for (uint32_t dq = 0; dq < EARLY_DRIVES; ++dq)
        if (dq < a.ndrives) poisson_counts4(a, s_dr[dq], s_tbl, q, n, full, live, gid, cnt_e[dq], in_e[dq]);
    }
    if (full) {
      reinterpret_cast<float4*>(a.V)[q] = make_float4(V[0], V[1], V[2], V[3]);
      reinterpret_cast<uint2*>(a.refr)[q] = make_uint2(refr[0] | (refr[1] << 16), refr[2] | (refr[3] << 16));
    } else {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        if (!live[k]) continue;
        a.V[i0 + k] = V[k];
        a.refr[i0 + k] = (uint16_t)refr[k];
      }
    }
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) {
      // warp-aggregated append of the step's spiking positions (on one rank these are
      // directly the rows to deliver; with several ranks the router expands them)
      const uint32_t mask = __ballot_sync(0xffffffffu, spike[k]);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        uint32_t sbase = 0;
        if ((int)lane == leader) {
          sbase = atomicAdd(&a.n_spk[n & 1], __popc(mask));
          atomicAdd(a.n_spikes_total, (unsigned long long)__popc(mask));
        }
        sbase = __shfl_sync(0xffffffffu, sbase, leader);
        const uint32_t off = __popc(mask & ((1u << lane) - 1));
        if (spike[k]) {
          a.spk[(uint64_t)(n & 1) * a.N + sbase + off] = i0 + k;
          if (a.log_cap) {
            unsigned long long lb = 0;
            if ((int)lane == leader) lb = atomicAdd(a.n_logged, (unsigned long long)__popc(mask));
            lb = __shfl_sync(mask, lb, leader);
            const unsigned long long ls = lb + off;
            if (ls < a.log_cap) a.log[ls] = make_uint2(n, gid[k]);
          }
        }
      }
    }
    // phase 3: after the previous delivery -- synaptic input of step n, drives, ring cleared
    pdl_wait();
    if (qb == blockIdx.x * UPD_BLOCK) {
      if (blockIdx.x == 0 && tid == 0) a.n_spk[(n + 1) & 1] = 0;   // next step's list
      pdl_trigger();
    }
    float in_ex[UPD_Q], in_in[UPD_Q];
    if (full) {
      const float4 x = __ldcg(reinterpret_cast<const float4*>(rex) + q);
      in_ex[0] = x.x; in_ex[1] = x.y; in_ex[2] = x.z; in_ex[3] = x.w;
      if (two) {
        const float4 y = __ldcg(reinterpret_cast<const float4*>(rin) + q);
        in_in[0] = y.x; in_in[1] = y.y; in_in[2] = y.z; in_in[3] = y.w;
      } else {
#pragma unroll
        for (int k = 0; k < UPD_Q; ++k) in_in[k] = 0.f;
      }
    } else {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        in_ex[k] = in_in[k] = 0.f;
        if (live[k]) {
          in_ex[k] = __ldcg(rex + i0 + k);
          if (two) in_in[k] = __ldcg(rin + i0 + k);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) {
      if (!live[k]) continue;
      const DevPop& P = pi[k] < 64 ? s_pop[pi[k]] : a.pops[pi[k]];
      Iex[k] = P.P11ex * Iex[k] + in_ex[k];
      Iin[k] = P.P11in * Iin[k] + in_in[k];
    }
    for (uint32_t dq = 0; dq < a.ndrives; ++dq) {
      const DevDrive dr = dq < MAX_SMEM_DRIVES ? s_dr[dq] : a.drives[dq];
      uint32_t cnt[UPD_Q];
      bool in[UPD_Q];
      if (early) {
#pragma unroll
        for (int k = 0; k < UPD_Q; ++k) {
          cnt[k] = dq == 0 ? cnt_e[0][k] : cnt_e[1][k];
          in[k] = dq == 0 ? in_e[0][k] : in_e[1][k];
        }
      } else {
        poisson_counts4(a, dr, s_tbl, q, n, full, live, gid, cnt, in);
      }
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        if (!in[k]) continue;
        if (dr.weight >= 0.f || !two) Iex[k] += (float)cnt[k] * dr.weight;
        else Iin[k] += (float)cnt[k] * dr.weight;
      }
    }
    if (full) {
      reinterpret_cast<float4*>(a.Iex)[q] = make_float4(Iex[0], Iex[1], Iex[2], Iex[3]);
      reinterpret_cast<float4*>(rex)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (two) {
        reinterpret_cast<float4*>(a.Iin)[q] = make_float4(Iin[0], Iin[1], Iin[2], Iin[3]);
        reinterpret_cast<float4*>(rin)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        if (!live[k]) continue;
        a.Iex[i0 + k] = Iex[k];
        rex[i0 + k] = 0.f;
        if (two) { a.Iin[i0 + k] = Iin[k]; rin[i0 + k] = 0.f; }
      }
    }
  }
  if (blockIdx.x * UPD_BLOCK >= nq) {   // a CTA without neurons still keeps the protocol
    pdl_wait();
    if (blockIdx.x == 0 && tid == 0) a.n_spk[(n + 1) & 1] = 0;
  }
}

// Neuron work of an overlapped step n (one rank): POST takes ring slot n (read and
// cleared), I <- P11 I + ring, then the drives of step n in drive order; PRE decides the
// spikes of step m (m = n + 1 after POST, m = n alone) from V, I and refractoriness of
// step m - 1 and appends them to list m mod 3.  The delivery of step n runs meanwhile:
// it reads list n mod 3 and adds into slots n + d, d >= 1, never into slot n.  The kernel
// with POST resets list (n + 2) mod 3, which the delivery of step n - 1 (complete)
// read and step_update(n + 1) fills.
__global__ void __launch_bounds__(UPD_BLOCK, 4) step_update_kernel(SimArgs a, uint32_t k_step, uint32_t mode) {
  __shared__ uint32_t s_tbl[256];
  __shared__ DevPop s_pop[64];
  __shared__ DevDrive s_dr[MAX_SMEM_DRIVES];
  const int tid = threadIdx.x;
  const uint32_t lane = tid & 31;
  const uint32_t n = __ldcg(a.step) + k_step;
  const bool post = mode & kStepPost, pre = mode & kStepPre;
  const uint32_t m = post ? n + 1 : n;
  const uint32_t lm = m % 3;
  for (uint32_t i = tid; i < a.poisson_tbl_len && i < 256; i += UPD_BLOCK) s_tbl[i] = a.poisson_tbl[i];
  for (uint32_t i = tid; i < a.npops && i < 64; i += UPD_BLOCK) s_pop[i] = a.pops[i];
  for (uint32_t i = tid; i < a.ndrives && i < MAX_SMEM_DRIVES; i += UPD_BLOCK) s_dr[i] = a.drives[i];
  if (post && blockIdx.x == 0 && tid == 0) a.n_work[(n + 2) % 3] = 0;
  float* rex = a.ring + ((uint64_t)(n % a.ring_slots) * a.n_rec) * a.ring_stride;
  float* rin = rex + a.ring_stride;
  const bool two = a.n_rec == 2;
  const uint32_t nq = (a.N + UPD_Q - 1) / UPD_Q;
  bool staged = false;
  for (uint32_t qb = blockIdx.x * UPD_BLOCK; qb < nq; qb += gridDim.x * UPD_BLOCK) {
    const uint32_t q = qb + tid;
    const uint32_t i0 = q * UPD_Q;
    const bool full = q < nq && i0 + UPD_Q <= a.N;
    float V[UPD_Q], Iex[UPD_Q], Iin[UPD_Q], in_ex[UPD_Q], in_in[UPD_Q];
    uint32_t refr[UPD_Q], pi[UPD_Q], gid[UPD_Q];
    bool live[UPD_Q], spike[UPD_Q];
    if (full) {
      const float4 v = __ldcg(reinterpret_cast<const float4*>(a.V) + q);
      const float4 e = __ldcg(reinterpret_cast<const float4*>(a.Iex) + q);
      const uint2 r = __ldcg(reinterpret_cast<const uint2*>(a.refr) + q);
      const uint2 p = reinterpret_cast<const uint2*>(a.pop_of)[q];
      V[0] = v.x; V[1] = v.y; V[2] = v.z; V[3] = v.w;
      Iex[0] = e.x; Iex[1] = e.y; Iex[2] = e.z; Iex[3] = e.w;
      refr[0] = r.x & 0xFFFFu; refr[1] = r.x >> 16; refr[2] = r.y & 0xFFFFu; refr[3] = r.y >> 16;
      pi[0] = p.x & 0xFFFFu; pi[1] = p.x >> 16; pi[2] = p.y & 0xFFFFu; pi[3] = p.y >> 16;
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) in_ex[k] = in_in[k] = Iin[k] = 0.f;
      if (post) {
        const float4 x = __ldcg(reinterpret_cast<const float4*>(rex) + q);
        in_ex[0] = x.x; in_ex[1] = x.y; in_ex[2] = x.z; in_ex[3] = x.w;
      }
      if (two) {
        const float4 ii = __ldcg(reinterpret_cast<const float4*>(a.Iin) + q);
        Iin[0] = ii.x; Iin[1] = ii.y; Iin[2] = ii.z; Iin[3] = ii.w;
        if (post) {
          const float4 y = __ldcg(reinterpret_cast<const float4*>(rin) + q);
          in_in[0] = y.x; in_in[1] = y.y; in_in[2] = y.z; in_in[3] = y.w;
        }
      }
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) live[k] = true;
    } else {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        const uint32_t i = i0 + k;
        live[k] = q < nq && i < a.N;
        V[k] = Iex[k] = Iin[k] = in_ex[k] = in_in[k] = 0.f;
        refr[k] = pi[k] = 0;
        if (live[k]) {
          V[k] = __ldcg(a.V + i); Iex[k] = __ldcg(a.Iex + i);
          refr[k] = __ldcg(a.refr + i); pi[k] = a.pop_of[i];
          if (post) in_ex[k] = __ldcg(rex + i);
          if (two) {
            Iin[k] = __ldcg(a.Iin + i);
            if (post) in_in[k] = __ldcg(rin + i);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) gid[k] = live[k] ? i0 + k : 0u;   // one rank: position = gid
    if (!staged) {
      __syncthreads();
      staged = true;
    }
    if (post) {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        if (!live[k]) continue;
        const DevPop& P = pi[k] < 64 ? s_pop[pi[k]] : a.pops[pi[k]];
        Iex[k] = P.P11ex * Iex[k] + in_ex[k];
        Iin[k] = P.P11in * Iin[k] + in_in[k];
      }
      for (uint32_t dq = 0; dq < a.ndrives; ++dq) {
        const DevDrive dr = dq < MAX_SMEM_DRIVES ? s_dr[dq] : a.drives[dq];
        uint32_t cnt[UPD_Q];
        bool in[UPD_Q];
        poisson_counts4(a, dr, s_tbl, q, n, full, live, gid, cnt, in);
#pragma unroll
        for (int k = 0; k < UPD_Q; ++k) {
          if (!in[k]) continue;
          if (dr.weight >= 0.f || !two) Iex[k] += (float)cnt[k] * dr.weight;
          else Iin[k] += (float)cnt[k] * dr.weight;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) {
      spike[k] = false;
      if (pre && live[k]) {
        const DevPop& P = pi[k] < 64 ? s_pop[pi[k]] : a.pops[pi[k]];
        float v = V[k];
        uint32_t rf = refr[k];
        if (rf == 0) v = P.P22 * v + P.P21ex * Iex[k] + P.P21in * Iin[k] + P.P20 * P.Ie;
        else --rf;
        if (v >= P.Vth) {
          v = P.Vreset;
          rf = P.ref_steps;
          spike[k] = true;
        }
        V[k] = v; refr[k] = rf;
      }
    }
    if (full) {
      if (pre) {
        reinterpret_cast<float4*>(a.V)[q] = make_float4(V[0], V[1], V[2], V[3]);
        reinterpret_cast<uint2*>(a.refr)[q] = make_uint2(refr[0] | (refr[1] << 16), refr[2] | (refr[3] << 16));
      }
      if (post) {
        reinterpret_cast<float4*>(a.Iex)[q] = make_float4(Iex[0], Iex[1], Iex[2], Iex[3]);
        reinterpret_cast<float4*>(rex)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (two) {
          reinterpret_cast<float4*>(a.Iin)[q] = make_float4(Iin[0], Iin[1], Iin[2], Iin[3]);
          reinterpret_cast<float4*>(rin)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < UPD_Q; ++k) {
        if (!live[k]) continue;
        const uint32_t i = i0 + k;
        if (pre) { a.V[i] = V[k]; a.refr[i] = (uint16_t)refr[k]; }
        if (post) {
          a.Iex[i] = Iex[k];
          rex[i] = 0.f;
          if (two) { a.Iin[i] = Iin[k]; rin[i] = 0.f; }
        }
      }
    }
    if (!pre) continue;
#pragma unroll
    for (int k = 0; k < UPD_Q; ++k) {
      const uint32_t mask = __ballot_sync(0xffffffffu, spike[k]);
      if (mask) {
        const int leader = __ffs(mask) - 1;
        uint32_t sbase = 0;
        if ((int)lane == leader) {
          sbase = atomicAdd(&a.n_work[lm], __popc(mask));
          atomicAdd(a.n_spikes_total, (unsigned long long)__popc(mask));
        }
        sbase = __shfl_sync(0xffffffffu, sbase, leader);
        const uint32_t off = __popc(mask & ((1u << lane) - 1));
        if (spike[k]) {
          a.work[(uint64_t)lm * a.work_stride + sbase + off] = i0 + k;
          if (a.log_cap) {
            unsigned long long lb = 0;
            if ((int)lane == leader) lb = atomicAdd(a.n_logged, (unsigned long long)__popc(mask));
            lb = __shfl_sync(mask, lb, leader);
            const unsigned long long ls = lb + off;
            if (ls < a.log_cap) a.log[ls] = make_uint2(m, gid[k]);
          }
        }
      }
    }
  }
}

// Streaming loads of the connection arrays with an L2 evict-first policy, and ring
// reductions with evict-last: each connection is read once per spike, while the ring's
// active slots are reused by every step, so the ring should keep the L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_stream_u32(const void* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_stream_u16(const void* p, uint64_t pol) {
  unsigned short v;
  asm volatile("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_stream_u8(const void* p, uint64_t pol) {
  unsigned short v;
  asm volatile("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=h"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void red_add_keep(float* p, float v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" :: "l"(p), "f"(v), "l"(pol) : "memory");
}

template <typename WT>
__device__ __forceinline__ float load_w(const WT* w, uint64_t e, uint64_t pol);
template <>
__device__ __forceinline__ float load_w<float>(const float* w, uint64_t e, uint64_t pol) {
  return __uint_as_float(ld_stream_u32(w + e, pol));
}
template <>
__device__ __forceinline__ float load_w<__nv_bfloat16>(const __nv_bfloat16* w, uint64_t e, uint64_t pol) {
  return __uint_as_float(ld_stream_u16(w + e, pol) << 16);
}
template <>
__device__ __forceinline__ float load_w<__half>(const __half* w, uint64_t e, uint64_t pol) {
  return __half2float(__ushort_as_half((unsigned short)ld_stream_u16(w + e, pol)));
}

// Events lo + first, lo + first + stride, ... < hi of one row: DEL_ILP events per thread
// are loaded before their reductions are issued.  nb = step mod D: an event of delay d
// (1 <= d < D) lands in slot nb + d, less D when that passes the ring's end.
template <typename WT, int STRIDE>
__device__ __forceinline__ void deliver_span(const SimArgs& a, const WT* __restrict__ w, uint32_t nb,
                                             uint64_t lo, uint64_t hi, uint32_t first, uint32_t stride,
                                             uint32_t toff, float sc, uint64_t pol_stream, uint64_t pol_ring) {
  float* __restrict__ ring = a.ring;
  const uint32_t st = STRIDE ? (uint32_t)STRIDE : stride;
  for (uint64_t e0 = lo + first; e0 < hi; e0 += (uint64_t)DEL_ILP * st) {
    float ww[DEL_ILP];
    uint32_t tt[DEL_ILP], dd[DEL_ILP];
#pragma unroll
    for (int k = 0; k < DEL_ILP; ++k) {
      const uint64_t e = e0 + (uint64_t)k * st;
      if (e < hi) {
        ww[k] = load_w<WT>(w, e, pol_stream) * sc;
        tt[k] = ld_stream_u32(a.tgt + e, pol_stream) + toff;
        dd[k] = ld_stream_u8(a.d + e, pol_stream);
      }
    }
#pragma unroll
    for (int k = 0; k < DEL_ILP; ++k) {
      const uint64_t e = e0 + (uint64_t)k * st;
      if (e < hi) {
        if (tt[k] < a.N) {
          uint32_t slot = nb + dd[k];
          if (slot >= a.ring_slots) slot -= a.ring_slots;
          const uint32_t rec = (a.n_rec == 2 && ww[k] < 0.f) ? 1u : 0u;
          red_add_keep(ring + ((uint64_t)slot * a.n_rec + rec) * a.ring_stride + tt[k], ww[k], pol_ring);
        } else {
          atomicOr(a.err, kErrBounds);    // corrupt connection: flagged, never written
        }
      }
    }
  }
}

__device__ __forceinline__ void add_events(const SimArgs& a, unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.n_events, v);
}

// Long rows (one rank: full out-degrees): each (row, slice) item is one CTA's work.
template <typename WT>
__global__ void __launch_bounds__(DEL_BLOCK) deliver_kernel(SimArgs a, const WT* __restrict__ w,
                                                            uint32_t k_step) {
  pdl_wait();                      // the step's list is complete
  pdl_trigger();
  const uint32_t n = __ldcg(a.step) + k_step;
  const uint32_t nb = n % a.ring_slots;
  const uint32_t li = a.lists == 3 ? n % 3 : n & 1;
  const uint32_t nitems = __ldcg(a.n_work + li);
  const uint32_t* items = a.work + (uint64_t)li * a.work_stride;
  const uint32_t* taus = a.work_rank ? a.work_rank + (uint64_t)li * a.work_stride : nullptr;
  const uint32_t slices = a.slices;
  const uint64_t total = (uint64_t)nitems * slices;
  const uint64_t pol_stream = policy_evict_first(), pol_ring = policy_evict_last();
  for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
    const uint32_t si = (uint32_t)(it / slices), sl = (uint32_t)(it - (uint64_t)si * slices);
    const uint32_t row = __ldcg(items + si);
    const uint64_t ra = a.rows[row], rb = a.rows[row + 1];
    const uint64_t len = rb - ra;
    const uint64_t lo = ra + len * sl / slices, hi = ra + len * (sl + 1) / slices;
    const float sc = a.row_scale ? a.row_scale[row] : 1.0f;
    const uint32_t toff = taus ? a.rank_off[__ldcg(taus + si)] : 0u;   // first neuron position of the row's rank
    deliver_span<WT, DEL_BLOCK>(a, w, nb, lo, hi, threadIdx.x, DEL_BLOCK, toff, sc, pol_stream, pol_ring);
    if (sl == 0 && threadIdx.x == 0) atomicAdd(a.n_events, (unsigned long long)len);   // a few per CTA
  }
}

// Short rows (many logical ranks: a spike's connections are split into one image row
// per rank): a group of item_lanes lanes per row, 32 / item_lanes rows per warp in flight.
template <typename WT>
__global__ void __launch_bounds__(DEL_BLOCK) deliver_rows_kernel(SimArgs a, const WT* __restrict__ w,
                                                                 uint32_t k_step) {
  pdl_wait();                      // the step's list is complete
  pdl_trigger();
  const uint32_t n = __ldcg(a.step) + k_step;
  const uint32_t nb = n % a.ring_slots;
  const uint32_t li = a.lists == 3 ? n % 3 : n & 1;
  const uint32_t nitems = __ldcg(a.n_work + li);
  const uint32_t* items = a.work + (uint64_t)li * a.work_stride;
  const uint32_t* taus = a.work_rank ? a.work_rank + (uint64_t)li * a.work_stride : nullptr;
  const uint32_t L = a.item_lanes;                     // 4, 8, 16 or 32
  const uint32_t lane = threadIdx.x & 31, sub = lane / L, sl = lane % L, per_warp = 32 / L;
  const uint64_t gw = ((uint64_t)blockIdx.x * DEL_BLOCK + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * DEL_BLOCK) >> 5;
  const uint64_t pol_stream = policy_evict_first(), pol_ring = policy_evict_last();
  unsigned long long events = 0;
  for (uint64_t b = gw * per_warp; b < nitems; b += nw * per_warp) {
    const uint64_t it = b + sub;
    uint64_t lo = 0, hi = 0;
    uint32_t toff = 0;
    float sc = 1.0f;
    if (it < nitems) {
      const uint32_t row = __ldcg(items + it);
      lo = a.rows[row];
      hi = a.rows[row + 1];
      toff = taus ? a.rank_off[__ldcg(taus + it)] : 0u;
      if (a.row_scale) sc = a.row_scale[row];
      if (sl == 0) events += hi - lo;
    }
    deliver_span<WT, 0>(a, w, nb, lo, hi, sl, L, toff, sc, pol_stream, pol_ring);
  }
  add_events(a, events);
}

// ---------------------------------------------------------------------------
// Delivery with staged rows: bulk asynchronous copies (cp.async.bulk, completed on an
// mbarrier) move each chunk of a row's targets, weights and delays into shared memory
// while the chunks before it are being delivered.  Warp 0 is the producer: lane 0 walks
// the CTA's (row, slice) items, splits each slice into chunks of up to TD_CHUNK events,
// and issues three copies per chunk into the next free stage.  Warps 1-7 consume the
// stages in order and issue the reductions.  Every wait is bounded: a wait that gives up
// sets kErrTimeout and ends its thread's loop; the producer then waits (bounded again)
// for the copies it issued before it returns.
constexpr int TD_STAGES = 4;
constexpr int TD_CHUNK = 1024;                // events per staged chunk
constexpr int TD_CAP = TD_CHUNK + 32;         // chunk start rounded down, end up, to 16 events
constexpr int TD_BLOCK = 256;
constexpr int TD_CONSUMER_WARPS = TD_BLOCK / 32 - 1;
constexpr uint32_t TD_CONSUMERS = TD_BLOCK - 32;    // consumer threads
constexpr int TD_ILP = 4;                           // events per consumer thread in flight
constexpr uint32_t TD_SPIN = 1u << 22;

template <typename WT>
struct __align__(128) TdStage {
  uint32_t tgt[TD_CAP];
  WT w[TD_CAP];
  uint8_t d[TD_CAP];
};
struct TdMeta {
  uint32_t off, n, toff, done;   // first event's index in the stage, events, rank offset, end marker
  float sc;                      // weight scale of the row (fp16 format)
};
template <typename WT>
struct TdSmem {
  TdStage<WT> st[TD_STAGES];
  TdMeta meta[TD_STAGES];
  unsigned long long full[TD_STAGES], empty[TD_STAGES];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_test_parity(unsigned long long* b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait for the phase of parity `parity` to complete; false when it gave up (or
// another wait of the grid already did).
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, uint32_t parity, uint32_t* err) {
  for (uint32_t spins = 0; !mbar_test_parity(b, parity); ++spins) {
    if (spins > TD_SPIN || (*(volatile uint32_t*)err & kErrTimeout)) {
      atomicOr(err, kErrTimeout);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar,
                                          uint64_t pol) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
               :: "r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol) : "memory");
}

template <typename WT>
__device__ __forceinline__ float stage_w(const WT* w, uint32_t i);
template <>
__device__ __forceinline__ float stage_w<float>(const float* w, uint32_t i) { return w[i]; }
template <>
__device__ __forceinline__ float stage_w<__nv_bfloat16>(const __nv_bfloat16* w, uint32_t i) {
  return __bfloat162float(w[i]);
}
template <>
__device__ __forceinline__ float stage_w<__half>(const __half* w, uint32_t i) { return __half2float(w[i]); }

template <typename WT>
__global__ void __launch_bounds__(TD_BLOCK) deliver_staged_kernel(SimArgs a, const WT* __restrict__ w,
                                                                  uint32_t k_step) {
  __shared__ TdSmem<WT> sm;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < TD_STAGES; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], TD_CONSUMER_WARPS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();                      // the step's list is complete
  pdl_trigger();
  const uint32_t n = __ldcg(a.step) + k_step;
  const uint32_t nb = n % a.ring_slots;
  const uint32_t li = a.lists == 3 ? n % 3 : n & 1;

  if (warp == 0) {
    // ---- producer ----
    const uint32_t nitems = __ldcg(a.n_work + li);
    const uint32_t* items = a.work + (uint64_t)li * a.work_stride;
    const uint32_t* taus = a.work_rank ? a.work_rank + (uint64_t)li * a.work_stride : nullptr;
    const uint32_t slices = a.slices;
    const uint64_t total = (uint64_t)nitems * slices;
    const uint64_t pol = policy_evict_first();
    const uint64_t G = gridDim.x;
    uint32_t k = 0;
    bool ok = true;
    for (uint64_t it0 = blockIdx.x; ok && it0 < total; it0 += 32 * G) {
      // the bounds of the CTA's next 32 items, one per lane, loaded at once; lane 0 then
      // issues their chunks in item order
      const uint64_t it = it0 + (uint64_t)lane * G;
      uint64_t lo = 0, hi = 0;
      uint32_t toff = 0;
      float sc = 1.0f;
      if (it < total) {
        const uint32_t si = (uint32_t)(it / slices), sl = (uint32_t)(it - (uint64_t)si * slices);
        const uint32_t row = __ldcg(items + si);
        const uint64_t ra = a.rows[row], rb = a.rows[row + 1];
        const uint64_t len = rb - ra;
        lo = ra + len * sl / slices;
        hi = ra + len * (sl + 1) / slices;
        if (a.row_scale) sc = a.row_scale[row];
        if (taus) toff = a.rank_off[__ldcg(taus + si)];
        if (sl == 0) atomicAdd(a.n_events, (unsigned long long)len);
      }
      for (int l = 0; l < 32; ++l) {
        const uint64_t lo_l = __shfl_sync(0xffffffffu, lo, l), hi_l = __shfl_sync(0xffffffffu, hi, l);
        const uint32_t toff_l = __shfl_sync(0xffffffffu, toff, l);
        const float sc_l = __shfl_sync(0xffffffffu, sc, l);
        if (lane == 0 && ok) {
          for (uint64_t c0 = lo_l; c0 < hi_l; c0 += TD_CHUNK) {
            const uint64_t c1 = min(c0 + (uint64_t)TD_CHUNK, hi_l);
            const uint32_t s = k % TD_STAGES, r = k / TD_STAGES;
            if (r > 0 && !mbar_wait(&sm.empty[s], (r - 1) & 1, a.err)) { ok = false; break; }
            const uint64_t base = c0 & ~15ull, end = (c1 + 15) & ~15ull;
            const uint32_t nn = (uint32_t)(end - base);
            sm.meta[s] = TdMeta{(uint32_t)(c0 - base), (uint32_t)(c1 - c0), toff_l, 0u, sc_l};
            mbar_arrive_expect_tx(&sm.full[s], nn * (4u + (uint32_t)sizeof(WT) + 1u));
            bulk_load(sm.st[s].tgt, a.tgt + base, nn * 4u, &sm.full[s], pol);
            bulk_load(sm.st[s].w, w + base, nn * (uint32_t)sizeof(WT), &sm.full[s], pol);
            bulk_load(sm.st[s].d, a.d + base, nn, &sm.full[s], pol);
            ++k;
          }
        }
        __syncwarp();
      }
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
    }
    if (lane != 0) return;
    if (ok) {                      // end marker: a stage without copies
      const uint32_t s = k % TD_STAGES, r = k / TD_STAGES;
      if (r == 0 || mbar_wait(&sm.empty[s], (r - 1) & 1, a.err)) {
        sm.meta[s] = TdMeta{0u, 0u, 0u, 1u, 1.0f};
        mbar_arrive(&sm.full[s]);
        return;
      }
    }
    // gave up: wait for every copy still in flight before the CTA's shared memory goes
    for (uint32_t q = k > TD_STAGES ? k - TD_STAGES : 0; q < k; ++q) {
      uint32_t spins = 0;
      while (!mbar_test_parity(&sm.full[q % TD_STAGES], (q / TD_STAGES) & 1) && ++spins < TD_SPIN) __nanosleep(32);
    }
    return;
  }
  // ---- consumers ----
  const uint64_t pol_ring = policy_evict_last();
  const uint32_t ctid = tid - 32;
  float* __restrict__ ring = a.ring;
  for (uint32_t k = 0;; ++k) {
    const uint32_t s = k % TD_STAGES;
    if (!mbar_wait(&sm.full[s], (k / TD_STAGES) & 1, a.err)) return;
    const TdMeta m = sm.meta[s];
    if (m.done) return;
    const TdStage<WT>& st = sm.st[s];
    // TD_ILP events per thread read from the stage before their reductions are issued
    for (uint32_t j0 = ctid; j0 < m.n; j0 += TD_ILP * TD_CONSUMERS) {
      uint32_t tt[TD_ILP], dd[TD_ILP];
      float ww[TD_ILP];
#pragma unroll
      for (int q = 0; q < TD_ILP; ++q) {
        const uint32_t j = j0 + q * TD_CONSUMERS;
        tt[q] = 0;
        dd[q] = 0;
        ww[q] = 0.f;
        if (j < m.n) {
          const uint32_t i = m.off + j;
          tt[q] = st.tgt[i] + m.toff;
          ww[q] = stage_w<WT>(st.w, i) * m.sc;
          dd[q] = st.d[i];
        }
      }
#pragma unroll
      for (int q = 0; q < TD_ILP; ++q) {
        if (j0 + q * TD_CONSUMERS >= m.n) continue;
        if (tt[q] < a.N) {
          uint32_t slot = nb + dd[q];
          if (slot >= a.ring_slots) slot -= a.ring_slots;
          const uint32_t rec = (a.n_rec == 2 && ww[q] < 0.f) ? 1u : 0u;
          red_add_keep(ring + ((uint64_t)slot * a.n_rec + rec) * a.ring_stride + tt[q], ww[q], pol_ring);
        } else {
          atomicOr(a.err, kErrBounds);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&sm.empty[s]);
  }
}

// ---------------------------------------------------------------------------
// Ceiling probe of the delivery's ring reductions.  It measures the GPU and is no step of
// the method: every reduction adds a zero (x + 0 = x and x + (-0) = x for every float x), so
// the ring keeps its values.  Each CTA takes chunks of PROBE_CHUNK consecutive synapses of
// [e0, e0 + n).  mode 0: deliver_span over the chunk, the direct delivery's loop with the
// weights multiplied by zero (targets, weights and delays streamed, slot = nb + d).  mode 1:
// the delay of the first synapse of each run of 256, and a target drawn uniformly by
// Philox-4x32-10 from the synapse index: nothing but the reductions moves through memory.
constexpr uint32_t PROBE_CHUNK = 8192;

template <typename WT>
__global__ void __launch_bounds__(DEL_BLOCK) ring_probe_kernel(SimArgs a, const WT* __restrict__ w, uint64_t e0,
                                                               uint64_t n, uint32_t nb, uint32_t mode) {
  const uint64_t pol_stream = policy_evict_first(), pol_ring = policy_evict_last();
  const uint64_t nchunks = (n + PROBE_CHUNK - 1) / PROBE_CHUNK;
  for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const uint64_t lo = e0 + c * PROBE_CHUNK;
    const uint64_t hi = lo + PROBE_CHUNK < e0 + n ? lo + PROBE_CHUNK : e0 + n;
    if (mode == 0) {
      deliver_span<WT, DEL_BLOCK>(a, w, nb, lo, hi, threadIdx.x, DEL_BLOCK, 0u, 0.0f, pol_stream, pol_ring);
      continue;
    }
    for (uint64_t b = lo + threadIdx.x; b < hi; b += 4ull * DEL_BLOCK) {
      const uint4 h = philox_stream(b, 0u, kPurposeProbe, 0ull);
      const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t e = b + (uint64_t)k * DEL_BLOCK;
        if (e < hi) {
          uint32_t slot = nb + __ldg(a.d + (e & ~255ull));
          if (slot >= a.ring_slots) slot -= a.ring_slots;
          red_add_keep(a.ring + (uint64_t)slot * a.n_rec * a.ring_stride + uniform_index(hw[k], a.N), 0.0f, pol_ring);
        }
      }
    }
  }
}

__global__ void advance_step_kernel(uint32_t* step, uint32_t by) { *step += by; }

__global__ void init_state_kernel(SimArgs a, const float* v0) {
  const uint64_t total = (uint64_t)a.N;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    a.V[i] = v0[i];
    a.Iex[i] = 0.f;
    a.Iin[i] = 0.f;
    a.refr[i] = 0;
  }
}

cudaError_t launch_update(const SimArgs& a, uint32_t k_step, cudaStream_t st, bool pdl) {
  const uint64_t need = ((uint64_t)a.N + UPD_BLOCK * UPD_Q - 1) / (UPD_BLOCK * UPD_Q);
  const unsigned grid = (unsigned)(need < a.update_grid ? need : a.update_grid);
  return launch_pdl(update_kernel, dim3(grid), dim3(UPD_BLOCK), st, pdl, a, k_step);
}

template <typename WT>
static cudaError_t launch_deliver_t(const SimArgs& a, const WT* w, uint32_t k_step, cudaStream_t st, bool pdl) {
  const dim3 grid((unsigned)a.deliver_grid);
  if (a.item_lanes) return launch_pdl(deliver_rows_kernel<WT>, grid, dim3(DEL_BLOCK), st, pdl, a, w, k_step);
  if (a.staged) return launch_pdl(deliver_staged_kernel<WT>, dim3((unsigned)a.staged_grid), dim3(TD_BLOCK), st, pdl,
                                  a, w, k_step);
  return launch_pdl(deliver_kernel<WT>, grid, dim3(DEL_BLOCK), st, pdl, a, w, k_step);
}

cudaError_t launch_deliver(const SimArgs& a, uint32_t k_step, cudaStream_t st, bool pdl) {
  if (a.w_format == 0) return launch_deliver_t(a, (const float*)a.w, k_step, st, pdl);
  if (a.w_format == 1) return launch_deliver_t(a, (const __nv_bfloat16*)a.w, k_step, st, pdl);
  return launch_deliver_t(a, (const __half*)a.w, k_step, st, pdl);
}

cudaError_t launch_ring_probe(const SimArgs& a, uint64_t e0, uint64_t n, uint32_t nb, uint32_t mode, unsigned grid,
                              cudaStream_t st) {
  if (a.w_format == 0) ring_probe_kernel<<<grid, DEL_BLOCK, 0, st>>>(a, (const float*)a.w, e0, n, nb, mode);
  else if (a.w_format == 1)
    ring_probe_kernel<<<grid, DEL_BLOCK, 0, st>>>(a, (const __nv_bfloat16*)a.w, e0, n, nb, mode);
  else ring_probe_kernel<<<grid, DEL_BLOCK, 0, st>>>(a, (const __half*)a.w, e0, n, nb, mode);
  return cudaGetLastError();
}

cudaError_t launch_step_update(const SimArgs& a, uint32_t k_step, uint32_t mode, cudaStream_t st) {
  const uint64_t need = ((uint64_t)a.N + UPD_BLOCK * UPD_Q - 1) / (UPD_BLOCK * UPD_Q);
  const unsigned grid = (unsigned)(need < a.update_grid ? need : a.update_grid);
  step_update_kernel<<<grid, UPD_BLOCK, 0, st>>>(a, k_step, mode);
  return cudaGetLastError();
}

cudaError_t launch_advance(const SimArgs& a, uint32_t by, cudaStream_t st) {
  advance_step_kernel<<<1, 1, 0, st>>>(a.step, by);
  return cudaGetLastError();
}

// Resident CTAs per SM of the staged delivery (its shared memory bounds them).
int staged_deliver_ctas_per_sm(uint32_t w_format) {
  int n = 0;
  cudaError_t e;
  if (w_format == 0) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, deliver_staged_kernel<float>, TD_BLOCK, 0);
  else if (w_format == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, deliver_staged_kernel<__nv_bfloat16>, TD_BLOCK, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, deliver_staged_kernel<__half>, TD_BLOCK, 0);
  return e == cudaSuccess ? n : 0;
}

cudaError_t launch_init_state(const SimArgs& a, const float* v0, cudaStream_t st) {
  init_state_kernel<<<256, 256, 0, st>>>(a, v0);
  return cudaGetLastError();
}

}  // namespace snn
