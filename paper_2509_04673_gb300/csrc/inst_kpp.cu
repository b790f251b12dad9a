// Stage instantiations for the PhysKPP physics policy: the FP64 form (all
// degrees); the FP32-mixed form is compiled in inst_kpp_f32.cu.
#include "stage.cuh"

namespace cgl {
StageFn stage_fn_kpp(int prec, int p) {
    return prec == 0 ? select_stage_r<PhysKPP, double>(p) : stage_fn_kpp32(p);
}

cudaError_t upload_kpp(const Tab<double>* td, const Tab<float>* tf, const double* a2d, const float* a2f) {
    return upload_tables_here(td, tf, a2d, a2f);
}
}  // namespace cgl
