// noalloc.cu — the lumped gradient projection g = M_L^-1 sum_e int phi_i grad u_h
// as an entry point that allocates no memory.
//
// Some callers cannot allocate device memory while they run: code inside a
// host callback or a custom allocator hook, real-time loops that must not
// hit the driver's allocator, or embedders that hand over fixed buffers only.
// For them this entry point keeps the element-vector scratch that the pass
// needs between its element loop and its node gather in a file-scope device
// array instead of a cudaMalloc'd buffer. The array lives as long as the
// library is loaded, on every GPU that loads it.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "state.h"

namespace cgl {

cudaError_t upload_host_tables(UploadFn f);  // api.cu

// scratch capacity in doubles: 2 values per (element, local node) are needed,
// so the limit is nx * ny * (p + 1)^2 <= 2^20 (16 MiB of scratch)
constexpr long long NOALLOC_SCRATCH = 1LL << 21;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH];

template <int P>
__global__ void k_noalloc_grad(MeshDev m, const double* __restrict__ u, double* __restrict__ EV) {
    int ex, ey, e;
    if (!elem_of_thread(m, ex, ey, e)) return;
    double U[1][Dim<P>::N2];
    load_block<double, P, 1>(u, m, ex, ey, U);
    grad_vectors<double, P, 1>(m, U, m.h, m.E, e, EV);
}

template <int P>
__global__ void k_noalloc_gather(MeshDev m, const double* __restrict__ EV, double* __restrict__ g) {
    int gx, gy;
    long long node;
    if (!node_of_thread(m, gx, gy, node)) return;
    gather_init_at<double, P, 2>(m, EV, nullptr, g, gx, gy, node);
}

static cudaError_t upload_noalloc(const Tab<double>* td, const Tab<float>* tf, const double* a2d,
                                  const float* a2f) {
    return upload_tables_here(td, tf, a2d, a2f);
}

struct NoallocSetup {
    int device;
    double* scratch;
};

static std::mutex g_noalloc_mu;
static std::vector<NoallocSetup> g_noalloc_setups;

// once per device, with that device current: tables into this unit's
// constant memory and the device address of the scratch array
static cgl_status noalloc_setup(int dev, double** scratch) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    for (const NoallocSetup& s : g_noalloc_setups)
        if (s.device == dev) {
            *scratch = s.scratch;
            return CGL_OK;
        }
    cudaError_t e = upload_host_tables(upload_noalloc);
    if (e != cudaSuccess) return set_error(CGL_ECUDA, "table upload: %s", cudaGetErrorString(e));
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
        return set_error(CGL_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_setups.push_back(NoallocSetup{dev, (double*)ptr});
    *scratch = (double*)ptr;
    return CGL_OK;
}

}  // namespace cgl

using namespace cgl;

extern "C" cgl_status cgl_gradient_noalloc(const cgl_mesh* mesh, const double* u, double* g, void* stream) {
    if (!mesh || !u || !g) return set_error(CGL_EINVAL, "null argument");
    const MeshDev& m = mesh->m;
    const long long need = (long long)m.E * (m.p + 1) * (m.p + 1) * 2;
    if (need > NOALLOC_SCRATCH)
        return set_error(CGL_EINVAL,
                         "mesh too large for the no-allocation scratch: nx*ny*(p+1)^2 = %lld > %lld",
                         need / 2, NOALLOC_SCRATCH / 2);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(CGL_ECUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    double* scratch = nullptr;
    cgl_status rc = noalloc_setup(dev, &scratch);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 be(64, 2), bn(128, 1);
    const dim3 ge((m.nx + 63) / 64, (m.ny + 1) / 2), gn((m.nnx + 127) / 128, m.nny);
    switch (m.p) {
        case 1:
            k_noalloc_grad<1><<<ge, be, 0, st>>>(m, u, scratch);
            k_noalloc_gather<1><<<gn, bn, 0, st>>>(m, scratch, g);
            break;
        case 2:
            k_noalloc_grad<2><<<ge, be, 0, st>>>(m, u, scratch);
            k_noalloc_gather<2><<<gn, bn, 0, st>>>(m, scratch, g);
            break;
        case 3:
            k_noalloc_grad<3><<<ge, be, 0, st>>>(m, u, scratch);
            k_noalloc_gather<3><<<gn, bn, 0, st>>>(m, scratch, g);
            break;
        default:
            k_noalloc_grad<4><<<ge, be, 0, st>>>(m, u, scratch);
            k_noalloc_gather<4><<<gn, bn, 0, st>>>(m, scratch, g);
            break;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(CGL_ECUDA, "launch: %s", cudaGetErrorString(e));
    return CGL_OK;
}
