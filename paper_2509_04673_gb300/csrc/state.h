// state.h — internal layout of the library's mesh and state objects
// (shared by the C-ABI implementation and the batched launcher).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/cgl.h"
#include "stage.cuh"

struct cgl_mesh {
    cgl_mesh_desc d;
    cgl::MeshDev m;
};

struct cgl_state {
    const cgl_mesh* mesh;
    int nc, prec, device;
    cudaStream_t st;
    bool own_stream;
    bool has_problem;
    cgl_problem prob;
    bool has_bnd;          // a cgl_set_boundary table is in force
    cgl_boundary bnd;
    cgl::ProbDev pd;
    cgl::StageFn stage;
    cgl::Bufs B;
    size_t rsz;  // bytes per bulk value
    cudaGraphExec_t step_graph;
    double* diag;       // device partials for diagnostics
    double* host_stage; // float64 staging of host copies (nc*NN values), allocated at first use
    // pipelined host copies (cgl_set_state_async / cgl_get_state_async), set
    // up at first use: two float64 staging buffers per direction, one copy
    // stream per direction, events that order the buffers' reuse
    double* stage_in[2];
    double* stage_out[2];
    int in_k, out_k;
    cudaStream_t cst_in, cst_out;
    cudaEvent_t ev_in_ready[2], ev_in_free[2], ev_out_ready[2], ev_out_free[2];
    std::vector<void*> allocs;
};

namespace cgl {
// shared helpers of the C-ABI units
cgl_status set_error(cgl_status st, const char* fmt, ...);
}  // namespace cgl
