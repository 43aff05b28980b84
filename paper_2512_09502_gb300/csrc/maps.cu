// maps.cu -- image neurons and the point-to-point / collective communication maps
// of the logical ranks (paper, Methods, "Remote connections"), and the row accessors
// of the inspection calls.
#include <cstring>
#include <vector>

#include "maps_internal.cuh"

namespace snn {

int build_maps(snn_ctx* c, const std::vector<DevProj>&, const DevProj*, const uint64_t*) {
  return ctx_fail(c, SNN_EINVAL, "logical ranks > 1 are not built yet");
}

int setup_routing(snn_ctx* c) { return ctx_fail(c, SNN_EINVAL, "logical ranks > 1 are not built yet"); }

cudaError_t launch_route(snn_ctx*) { return cudaErrorNotSupported; }

uint32_t route_kernels_per_step(snn_ctx*) { return 0; }

int rank_row_ptr(snn_ctx* c, uint32_t rank, std::vector<uint64_t>* rp) {
  const Geom& g = ctx_geom(c);
  if (g.R != 1) return ctx_fail(c, SNN_EINVAL, "logical ranks > 1 are not built yet");
  rp->resize((size_t)g.N + 1);
  if (cudaMemcpy(rp->data(), ctx_dense(c), ((size_t)g.N + 1) * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ctx_fail(c, SNN_ECUDA, "row_ptr copy failed");
  (void)rank;
  return SNN_OK;
}

int rank_row_scales(snn_ctx* c, uint32_t rank, std::vector<float>* scales) {
  const Geom& g = ctx_geom(c);
  if (g.R != 1) return ctx_fail(c, SNN_EINVAL, "logical ranks > 1 are not built yet");
  scales->assign(g.N, 1.0f);
  if (ctx_scale_src(c) &&
      cudaMemcpy(scales->data(), ctx_scale_src(c), (size_t)g.N * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ctx_fail(c, SNN_ECUDA, "scale copy failed");
  (void)rank;
  return SNN_OK;
}

int rank_row_bounds(snn_ctx* c, uint32_t rank, uint64_t row, uint64_t ab[2], float* scale) {
  const Geom& g = ctx_geom(c);
  if (g.R != 1) return ctx_fail(c, SNN_EINVAL, "logical ranks > 1 are not built yet");
  if (row >= g.N) return ctx_fail(c, SNN_EINVAL, "row out of range");
  if (cudaMemcpy(ab, ctx_dense(c) + row, 16, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ctx_fail(c, SNN_ECUDA, "row bounds copy failed");
  *scale = 1.0f;
  if (ctx_scale_src(c) &&
      cudaMemcpy(scale, ctx_scale_src(c) + row, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return ctx_fail(c, SNN_ECUDA, "scale copy failed");
  (void)rank;
  return SNN_OK;
}

}  // namespace snn

extern "C" int snn_get_maps(snn_ctx* c, uint32_t tau, uint32_t sigma, int32_t which, int64_t* host_buf,
                            uint64_t cap, uint64_t* n_out) {
  if (!c) return SNN_EINVAL;
  (void)tau; (void)sigma; (void)which; (void)host_buf; (void)cap;
  if (n_out) *n_out = 0;
  return snn::ctx_fail(c, SNN_EINVAL, "maps exist only with more than one logical rank");
}
