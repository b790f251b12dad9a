// Stage instantiations for the PhysKPP physics policy: the FP32-mixed form
// (all degrees).
#include "stage.cuh"

namespace cgl {
StageFn stage_fn_kpp32(int p) { return select_stage_r<PhysKPP, float>(p); }

cudaError_t upload_kpp32(const Tab<double>* td, const Tab<float>* tf, const double* a2d, const float* a2f) {
    return upload_tables_here(td, tf, a2d, a2f);
}
}  // namespace cgl
