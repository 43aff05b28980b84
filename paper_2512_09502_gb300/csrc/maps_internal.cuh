// maps_internal.cuh -- image neurons, communication maps and spike routing of the
// logical ranks (maps.cu), plus row accessors used by the inspection calls.
#pragma once
#include <vector>

#include "../../include/snn.h"
#include "sim_internal.cuh"
#include "snn_internal.cuh"

namespace snn {

struct RouteArgs {
  uint32_t R, N, exchange;
  const uint32_t* rank_off; const uint32_t* M; const uint64_t* rows_off;
  const uint64_t* tp_ptr; const uint32_t* T; const uint32_t* P; const uint64_t* img_off;
  const uint64_t* h_pos; const int32_t* I;
  const uint32_t* step; uint32_t* err;
  const uint32_t* spk; const uint32_t* n_spk;
  uint32_t* work; uint32_t* work_tau; uint32_t* n_work; uint64_t work_cap;
};

struct MapsState {
  uint32_t R = 0, N = 0, Mmax = 0;
  std::vector<uint32_t> M, rank_off;
  uint32_t* d_M = nullptr; uint32_t* d_rank_off = nullptr;
  // target side
  uint64_t n_images_total = 0;
  std::vector<uint64_t> n_img, img_first, rows_off, img_off;   // img_off: [R][R+1] by slot
  uint64_t* d_rows_off = nullptr; uint64_t* d_img_first = nullptr; uint64_t* d_img_off = nullptr;
  uint64_t* rows = nullptr;             // concatenated per-rank row starts (absolute)
  uint32_t* img_gid = nullptr;          // gid of every image, rank-major
  uint32_t* img_s = nullptr;            // its local index on the source rank (R maps)
  // source side
  uint64_t* spos = nullptr;             // [R][R][Mmax] prefix positions of S entries
  std::vector<uint64_t> S_off;          // [R*R+1] start of S_{tau,sigma} at sigma*R+tau
  uint64_t* d_S_off = nullptr; uint32_t* S_vals = nullptr;
  uint64_t* tp_ptr = nullptr; uint32_t* T = nullptr; uint32_t* P = nullptr; uint64_t n_tp = 0;
  uint64_t* h_pos = nullptr; std::vector<uint64_t> h_off; uint64_t* d_h_off = nullptr;
  uint32_t* H = nullptr; int32_t* I = nullptr; uint64_t n_h = 0;
  RouteArgs route{};
  uint32_t t0 = 0, nt = 0;              // ranks the target-side arrays cover: t0 .. t0 + nt - 1
  bool dry = false;                     // one rank's share only: no source-side maps
};

// accessors of the context (api.cu)
void* ctx_alloc(snn_ctx* c, size_t bytes);
void ctx_free(snn_ctx* c, void* p);
int ctx_fail(snn_ctx* c, int code, const char* msg);
cudaStream_t ctx_stream(snn_ctx* c);
MapsState& ctx_maps(snn_ctx* c);
SimArgs& ctx_sim(snn_ctx* c);
const Geom& ctx_geom(snn_ctx* c);
uint64_t ctx_geom_synapses(snn_ctx* c);   // synapses over all ranks
const std::vector<uint64_t>& ctx_seg_start(snn_ctx* c);
const std::vector<uint32_t>& ctx_rank_sizes(snn_ctx* c);
const std::vector<uint32_t>& ctx_rank_off(snn_ctx* c);
uint64_t* ctx_dense(snn_ctx* c);
const uint32_t* ctx_dense_off(snn_ctx* c);
const uint64_t* ctx_dseg_start(snn_ctx* c);
const float* ctx_scale_src(snn_ctx* c);
int ctx_num_sms(snn_ctx* c);
uint32_t* ctx_err(snn_ctx* c);
int ctx_exchange(snn_ctx* c);
uint32_t ctx_N(snn_ctx* c);

// all_src[p * R + tau] != 0: projection p gives all its sources images on rank tau
// (threshold xi); set only where p has targets on tau
int build_maps_dry(snn_ctx* c, uint32_t rank, const std::vector<DevProj>& projs,
                   const std::vector<uint8_t>& all_src);   // target side of one rank (dry run)
int build_maps(snn_ctx* c, const std::vector<DevProj>& projs, const DevProj* d_projs,
               const uint64_t* d_cbase, const uint32_t* d_tables, const std::vector<uint8_t>& all_src);
int setup_routing(snn_ctx* c);
cudaError_t launch_route(snn_ctx* c, uint32_t k_step, bool pdl);
uint32_t route_kernels_per_step(snn_ctx* c);
int rank_row_ptr(snn_ctx* c, uint32_t rank, std::vector<uint64_t>* rp);
int rank_row_scales(snn_ctx* c, uint32_t rank, std::vector<float>* scales);
int rank_row_bounds(snn_ctx* c, uint32_t rank, uint64_t row, uint64_t ab[2], float* scale);

}  // namespace snn
