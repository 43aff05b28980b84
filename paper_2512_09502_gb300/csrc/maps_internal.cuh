// maps_internal.cuh -- image neurons, communication maps and spike routing of the
// logical ranks (maps.cu), plus row accessors used by the inspection calls.
#pragma once
#include <vector>

#include "../../include/snn.h"
#include "sim_internal.cuh"
#include "snn_internal.cuh"

namespace snn {

struct MapsState {
  uint64_t n_images_total = 0;
  std::vector<uint64_t> n_img;          // images per rank
  std::vector<uint64_t> rp_off;         // first entry of each rank's row_ptr in rows
  uint64_t* rows = nullptr;             // concatenated per-rank row_ptr (absolute)
  uint32_t* img_gid = nullptr;          // gid of every image row, per rank concatenated
  std::vector<uint64_t> img_off;        // first image of each rank in img_gid
};

// accessors of the context (api.cu)
void* ctx_alloc(snn_ctx* c, size_t bytes);
void ctx_free(snn_ctx* c, void* p);
int ctx_fail(snn_ctx* c, int code, const char* msg);
cudaStream_t ctx_stream(snn_ctx* c);
MapsState& ctx_maps(snn_ctx* c);
SimArgs& ctx_sim(snn_ctx* c);
const Geom& ctx_geom(snn_ctx* c);
const std::vector<uint64_t>& ctx_seg_start(snn_ctx* c);
const std::vector<uint32_t>& ctx_rank_sizes(snn_ctx* c);
const std::vector<uint32_t>& ctx_rank_off(snn_ctx* c);
uint64_t* ctx_dense(snn_ctx* c);
const uint64_t* ctx_dseg_start(snn_ctx* c);
const float* ctx_scale_src(snn_ctx* c);
int ctx_num_sms(snn_ctx* c);
uint32_t* ctx_err(snn_ctx* c);
int ctx_exchange(snn_ctx* c);
uint32_t ctx_N(snn_ctx* c);

int build_maps(snn_ctx* c, const std::vector<DevProj>& projs, const DevProj* d_projs,
               const uint64_t* d_cbase);
int setup_routing(snn_ctx* c);
cudaError_t launch_route(snn_ctx* c);
uint32_t route_kernels_per_step(snn_ctx* c);
int rank_row_ptr(snn_ctx* c, uint32_t rank, std::vector<uint64_t>* rp);
int rank_row_scales(snn_ctx* c, uint32_t rank, std::vector<float>* scales);
int rank_row_bounds(snn_ctx* c, uint32_t rank, uint64_t row, uint64_t ab[2], float* scale);

}  // namespace snn
