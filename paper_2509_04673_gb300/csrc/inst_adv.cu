// Stage instantiations for the PhysAdv physics policy: the FP64 form (all
// degrees); the FP32-mixed form is compiled in inst_adv_f32.cu.
#include "stage.cuh"

namespace cgl {
StageFn stage_fn_adv(int prec, int p) {
    return prec == 0 ? select_stage_r<PhysAdv, double>(p) : stage_fn_adv32(p);
}

cudaError_t upload_adv(const Tab<double>* td, const Tab<float>* tf, const double* a2d, const float* a2f) {
    return upload_tables_here(td, tf, a2d, a2f);
}
}  // namespace cgl
