// Stage instantiations for the PhysKPP physics policy (all degrees, both precisions).
#include "stage.cuh"

namespace cgl {
StageFn stage_fn_kpp(int prec, int p) { return select_stage<PhysKPP>(prec, p); }
}  // namespace cgl

namespace cgl {
cudaError_t upload_kpp(const Tab<double>* td, const Tab<float>* tf, const double* a2d,
                        const float* a2f) {
    return upload_tables_here(td, tf, a2d, a2f);
}
}  // namespace cgl
