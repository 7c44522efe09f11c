// Interface between the context (lskum_host.cpp) and the warm-start network
// (lskum_mlp.cu): the device view of a context that the network reads and
// writes, and the kernel launchers both files use.
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lskum.h"

namespace lskum {

// Device arrays of a context, internal point order (k < n), for the network.
struct MlpView {
    int32_t n, ld, n_cases;
    const float *x, *y, *dwall;    // [ld] coordinates and distance to the case's wall polygon
    const uint8_t *flag;           // [ld]
    const int32_t *case_of;        // [ld]
    const float *case_mach, *case_aoa;  // [n_cases] (AoA in degrees), network inputs
    const double *case_Uinf;       // [n_cases][4] conserved free stream, bitwise the context's own
    const double *case_uv;         // [n_cases][2] free-stream velocity (u_inf, v_inf)
    double *U;                     // [4][ld] conserved state of the current state set
    cudaStream_t stream;
};

// Host copies of a context (caller order unless stated).
struct CtxHost {
    int32_t n, n_cases;
    const int32_t *perm;            // internal position -> caller index
    const int32_t *inv;             // caller index -> internal position
    const uint8_t *flag;            // [n]
    const int32_t *case_of_caller;  // [n]
};

// Context side (lskum_host.cpp).
CtxHost ctx_host(lskum_ctx *c);
lskum_status ctx_case_status(lskum_ctx *c, std::vector<int32_t> &status);  // LSKUM_OK or the failure
lskum_status ctx_mlp_view(lskum_ctx *c, MlpView *v);        // builds the geometry on first use
lskum_status ctx_state_written(lskum_ctx *c);                // after U was written on the device
lskum_status ctx_case_norms(lskum_ctx *c, std::vector<double> &norms);  // first residual norm per case
lskum_status ctx_fail(lskum_ctx *c, lskum_status s, const char *msg);

// Network side (lskum_mlp.cu): the wall distance of every point of a view,
// from the per-case wall segments seg[s] = (ax, ay, bx, by), seg_off[n_cases + 1].
cudaError_t launch_wall_distance(const float *x, const float *y, const int32_t *case_of, int32_t n,
                                 const float4 *seg, const int32_t *seg_off, float *dwall, cudaStream_t s);

}  // namespace lskum
