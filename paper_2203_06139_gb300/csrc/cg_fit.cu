// cg_fit.cu -- histogram batches and the BFGS fitters of libcg.
#include "cg_internal.cuh"
#include "cg_models.cuh"

namespace cg {
size_t grad_workspace_bytes(const cg_problem* pb, int64_t n_theta);
cg_status grad_points(const cg_problem* pb, const double* theta, int64_t n_theta, double* value, double* grad,
                      void* ws, size_t ws_bytes, cudaStream_t st);
}  // namespace cg

using namespace cg;

extern "C" {

size_t cg_batch_workspace_size(const cg_batch* b) {
    if (!b || b->n_hist < 1) return 0;
    if (!b->offsets) return grad_workspace_bytes(&b->tmpl, b->n_hist);
    return 0;
}

cg_status cg_batch_gradient(const cg_batch* b, const double* theta, double* value, double* grad, void* ws,
                            size_t ws_bytes, void* stream) {
    if (!b || b->n_hist < 1) return CG_ERR_INVALID_ARG;
    if (!b->offsets) return grad_points(&b->tmpl, theta, b->n_hist, value, grad, ws, ws_bytes, (cudaStream_t)stream);
    return CG_ERR_UNSUPPORTED;
}

size_t cg_fit_workspace_size(const cg_batch*) { return 0; }
cg_status cg_fit_plan(const cg_batch*, const int64_t*, const cg_tile_map*, void*, size_t, void*) { return CG_ERR_UNSUPPORTED; }
cg_status cg_fit_init(const cg_batch*, const double*, cg_fit_state*, void*, size_t, void*) { return CG_ERR_UNSUPPORTED; }
cg_status cg_fit_step(const cg_batch*, cg_fit_state*, int, double, void*, size_t, void*) { return CG_ERR_UNSUPPORTED; }
size_t cg_fit_single_workspace_size(const cg_problem*) { return 0; }
cg_status cg_fit_single_init(const cg_problem*, const double*, cg_fit_state*, void*, size_t, void*) { return CG_ERR_UNSUPPORTED; }
cg_status cg_fit_single_step(const cg_problem*, cg_fit_state*, int, double, void*, size_t, void*) { return CG_ERR_UNSUPPORTED; }

}  // extern "C"
