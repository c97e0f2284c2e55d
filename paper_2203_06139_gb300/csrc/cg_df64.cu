// cg_df64.cu -- double-float (FP32-pipe) variants of the fused kernels.
#include "cg_internal.cuh"
#include "cg_models.cuh"

namespace cg {

bool df64_supported(const cg_problem*) { return false; }

cg_status launch_df64(const cg_problem*, const double*, int64_t, double*, WsHeader*, TileGrid*, cudaStream_t) {
    return CG_ERR_UNSUPPORTED;
}

}  // namespace cg
