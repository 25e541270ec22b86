// gf_fmm.cu -- placeholder until the FMM path lands.
#include "gf_internal.cuh"

namespace gf {
gf_status fmm_create(gf_plan_s *, const double *, cudaStream_t) {
    set_error("FMM mode is not built yet");
    return GF_ERR_UNSUPPORTED;
}
gf_status fmm_forward(gf_plan_s *, const void *, int, int, double *, double *, cudaStream_t) {
    set_error("FMM mode is not built yet");
    return GF_ERR_UNSUPPORTED;
}
gf_status fmm_adjoint(gf_plan_s *, const double *, int, int, double *, cudaStream_t) {
    set_error("FMM mode is not built yet");
    return GF_ERR_UNSUPPORTED;
}
void fmm_destroy(gf_plan_s *) {}
gf_status fmm_info(const gf_plan_s *, gf_plan_info *) { return GF_OK; }
gf_status fmm_export_tree(gf_plan_s *, int, int32_t *, uint64_t *, uint64_t *, int64_t *, int64_t *) {
    set_error("FMM mode is not built yet");
    return GF_ERR_UNSUPPORTED;
}
size_t fmm_bytes_estimate(const gf_grid *, int, int64_t, const gf_options *) { return 0; }
}  // namespace gf
