// sim_internal.cuh -- device state of the simulation phase and its launchers.
#pragma once
#include "snn_internal.cuh"

namespace snn {

struct SimArgs {
  uint32_t N, R;
  float* V; float* Iex; float* Iin; uint16_t* refr;
  const uint16_t* pop_of;      // population of each neuron position
  const uint32_t* gid_of;      // gid of each neuron position (R > 1)
  const DevPop* pops; uint32_t npops;
  const DevDrive* drives; uint32_t ndrives;
  const uint32_t* poisson_tbl; uint32_t poisson_tbl_len;
  float* ring; uint32_t ring_slots;           // [D][n_rec][ring_stride], D = largest delay + 1
  uint32_t ring_stride;                       // N rounded up to a multiple of 4
  uint32_t n_rec;                             // 2 receptors, or 1 when tau_ex == tau_in
  uint32_t* step;                             // device step counter (first step of a batch)
  uint32_t* n_spk; uint32_t* spk;             // [2] counts, [2][N] spiking positions
  uint32_t* n_work; uint32_t* work;           // [2] counts, [2][stride] rows to deliver
  const uint32_t* work_rank;                  // [2][stride] rank of each row (R > 1) or null
  uint64_t work_stride;
  uint32_t item_lanes;                        // lanes per row for short rows; 0 = CTA per row slice
  unsigned long long* n_logged; uint2* log; unsigned long long log_cap;
  unsigned long long* n_events; unsigned long long* n_spikes_total;
  const uint64_t* rows;                       // row starts (absolute); one rank: gid rows
  const uint64_t* rows_off;                   // [R+1] first row of each rank (R > 1)
  const uint32_t* rank_off;                   // [R+1] first neuron position of each rank
  const uint32_t* tgt; const void* w; const uint8_t* d; uint32_t w_format;
  const float* row_scale;                     // per row (fp16 format) or null
  uint32_t slices;                            // slices of one row (several CTAs per row)
  uint32_t deliver_grid, update_grid;
  uint32_t lists;                             // spike / work lists cycled: 2, or 3 (overlapped steps)
  uint32_t* err;                              // device error word (kErrBounds: an event's target out of range)
  uint32_t staged;                            // long rows: chunks staged in shared memory by bulk copies
  uint32_t staged_grid;                       // CTAs of the staged delivery (all resident at once)
};

// Overlapped steps (one rank): the neuron work of step k and the delivery of step k run
// as two concurrent kernels.  step_update(k) takes the synaptic input of step k (POST)
// and decides the spikes of step k + 1 (PRE); a batch starts with PRE alone for its first
// step and ends with POST alone.  Lists cycle modulo 3.
constexpr uint32_t kStepPost = 1, kStepPre = 2;
cudaError_t launch_step_update(const SimArgs& a, uint32_t k_step, uint32_t mode, cudaStream_t st);

// Programmatic dependent launch (sm_90 and later).  A kernel launched with the
// programmatic stream serialization attribute may start while the previous kernel of the
// stream still runs.  pdl_wait blocks until that kernel has completed and its writes are
// visible; under a normal launch it returns at once.  pdl_trigger lets the next kernel's
// CTAs be scheduled before this one ends.  Only work that touches nothing the previous
// kernel writes may precede pdl_wait.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches kern<<<grid, block, 0, st>>>(args...), with programmatic serialization when pdl.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// pdl: start while the previous kernel of the stream runs (every kernel of a step
// but the first update of a batch)
cudaError_t launch_update(const SimArgs& a, uint32_t k_step, cudaStream_t st, bool pdl);
cudaError_t launch_deliver(const SimArgs& a, uint32_t k_step, cudaStream_t st, bool pdl);
cudaError_t launch_advance(const SimArgs& a, uint32_t by, cudaStream_t st);
cudaError_t launch_init_state(const SimArgs& a, const float* v0, cudaStream_t st);
int staged_deliver_ctas_per_sm(uint32_t w_format);
// Ceiling probe of the ring reductions (adds zeros; mode 0 streamed layout, mode 1 hashed targets)
cudaError_t launch_ring_probe(const SimArgs& a, uint64_t e0, uint64_t n, uint32_t nb, uint32_t mode, unsigned grid,
                              cudaStream_t st);

}  // namespace snn
