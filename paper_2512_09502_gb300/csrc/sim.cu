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
// One step = update_kernel (reads and clears ring slot n, integrates, appends spikes
// to the per-step delivery list) then deliver_kernel (walks the rows of every listed
// spike and red.add's the weights into slots n + d); the last deliver CTA to finish
// advances the device-side step counter, so the step needs no host involvement and
// is captured as a CUDA graph.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "sim_internal.cuh"

namespace snn {

constexpr int UPD_BLOCK = 256;
constexpr int DEL_BLOCK = 256;

__global__ void __launch_bounds__(UPD_BLOCK) update_kernel(SimArgs a) {
  __shared__ uint32_t s_tbl[256];
  __shared__ DevPop s_pop[64];
  const int tid = threadIdx.x;
  const uint32_t n = *a.step;
  for (uint32_t i = tid; i < a.poisson_tbl_len && i < 256; i += UPD_BLOCK) s_tbl[i] = a.poisson_tbl[i];
  for (uint32_t i = tid; i < a.npops && i < 64; i += UPD_BLOCK) s_pop[i] = a.pops[i];
  if (blockIdx.x == 0 && tid == 0) a.n_items[(n + 1) & 1] = 0;   // next step's list
  __syncthreads();
  const uint32_t i = blockIdx.x * UPD_BLOCK + tid;
  bool spike = false;
  uint32_t gid = 0;
  if (i < a.N) {
    const uint32_t pi = a.pop_of[i];
    const DevPop P = pi < 64 ? s_pop[pi] : a.pops[pi];
    gid = a.R == 1 ? i : a.gid_of[i];
    float V = a.V[i], Iex = a.Iex[i], Iin = a.Iin[i];
    uint32_t refr = a.refr[i];
    if (refr == 0) {
      V = P.P22 * V + P.P21ex * Iex + P.P21in * Iin + P.P20 * P.Ie;
    } else {
      --refr;
    }
    const uint32_t slot = n & a.ring_mask;
    float* rex = a.ring + ((uint64_t)slot * 2) * a.N;
    float* rin = rex + a.N;
    Iex = P.P11ex * Iex + rex[i];
    Iin = P.P11in * Iin + rin[i];
    rex[i] = 0.f;
    rin[i] = 0.f;
    for (uint32_t k = 0; k < a.ndrives; ++k) {
      const DevDrive dr = a.drives[k];
      if (gid - dr.first < dr.n) {
        const uint4 b = philox_stream((uint64_t)gid | ((uint64_t)n << 32), dr.idx, kPurposePoisson,
                                      dr.seed);
        const uint32_t cnt = upper_bound_u32(s_tbl + dr.tbl_off, dr.tbl_len, b.x);
        if (dr.weight >= 0.f) Iex += (float)cnt * dr.weight; else Iin += (float)cnt * dr.weight;
      }
    }
    if (V >= P.Vth) {
      V = P.Vreset;
      refr = P.ref_steps;
      spike = true;
    }
    a.V[i] = V;
    a.Iex[i] = Iex;
    a.Iin[i] = Iin;
    a.refr[i] = (uint16_t)refr;
  }
  // warp-aggregated append of the step's spikes (delivery items = rows of rank 0 for
  // one rank, neuron positions for the router otherwise)
  const uint32_t mask = __ballot_sync(0xffffffffu, spike);
  if (mask) {
    const int lane = tid & 31;
    const int leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&a.n_items[n & 1], __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    const uint32_t off = __popc(mask & ((1u << lane) - 1));
    if (spike) {
      a.items[(uint64_t)(n & 1) * a.N + base + off] = i;
      unsigned long long lb = 0;
      if (lane == leader) lb = atomicAdd(a.n_logged, (unsigned long long)__popc(mask));
      lb = __shfl_sync(mask, lb, leader);
      const unsigned long long slot = lb + off;
      if (slot < a.log_cap) a.log[slot] = make_uint2(n, gid);
    }
  }
}

template <typename WT>
__device__ __forceinline__ float load_w(const WT* w, uint64_t e);
template <>
__device__ __forceinline__ float load_w<float>(const float* w, uint64_t e) { return __ldg(w + e); }
template <>
__device__ __forceinline__ float load_w<__nv_bfloat16>(const __nv_bfloat16* w, uint64_t e) {
  return __bfloat162float(w[e]);
}
template <>
__device__ __forceinline__ float load_w<__half>(const __half* w, uint64_t e) {
  return __half2float(w[e]);
}

template <typename WT>
__global__ void __launch_bounds__(DEL_BLOCK) deliver_kernel(SimArgs a, const WT* __restrict__ w) {
  const uint32_t n = *a.step;
  const uint32_t nitems = a.n_items[n & 1];
  const uint32_t* items = a.items + (uint64_t)(n & 1) * a.N;
  const uint32_t slices = a.slices;
  const uint64_t total = (uint64_t)nitems * slices;
  for (uint64_t it = blockIdx.x; it < total; it += gridDim.x) {
    const uint32_t si = (uint32_t)(it / slices), sl = (uint32_t)(it - (uint64_t)si * slices);
    const uint32_t row = items[si];
    const uint64_t ra = a.row_ptr[row], rb = a.row_ptr[row + 1];
    const uint64_t len = rb - ra;
    const uint64_t lo = ra + len * sl / slices, hi = ra + len * (sl + 1) / slices;
    const float sc = a.row_scale ? a.row_scale[row] : 1.0f;
    for (uint64_t e = lo + threadIdx.x; e < hi; e += DEL_BLOCK) {
      const float ww = load_w<WT>(w, e) * sc;
      const uint32_t t = __ldg(a.tgt + e);
      const uint32_t slot = (n + __ldg(a.d + e)) & a.ring_mask;
      if (t < a.N) atomicAdd(a.ring + ((uint64_t)slot * 2 + (ww < 0.f ? 1 : 0)) * a.N + t, ww);
    }
    if (sl == 0 && threadIdx.x == 0) atomicAdd(a.n_events, (unsigned long long)len);
  }
  // the last CTA to finish advances the step counter
  __shared__ bool s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const uint32_t ticket = atomicAdd(a.done, 1u);
    s_last = ticket == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    *a.n_spikes_total += nitems;
    *a.done = 0;
    __threadfence();
    *a.step = n + 1;
  }
}

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

cudaError_t launch_update(const SimArgs& a, cudaStream_t st) {
  update_kernel<<<(a.N + UPD_BLOCK - 1) / UPD_BLOCK, UPD_BLOCK, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_deliver(const SimArgs& a, cudaStream_t st) {
  const unsigned grid = (unsigned)a.deliver_grid;
  if (a.w_format == 0)
    deliver_kernel<float><<<grid, DEL_BLOCK, 0, st>>>(a, (const float*)a.w);
  else if (a.w_format == 1)
    deliver_kernel<__nv_bfloat16><<<grid, DEL_BLOCK, 0, st>>>(a, (const __nv_bfloat16*)a.w);
  else
    deliver_kernel<__half><<<grid, DEL_BLOCK, 0, st>>>(a, (const __half*)a.w);
  return cudaGetLastError();
}

cudaError_t launch_init_state(const SimArgs& a, const float* v0, cudaStream_t st) {
  init_state_kernel<<<256, 256, 0, st>>>(a, v0);
  return cudaGetLastError();
}

}  // namespace snn
