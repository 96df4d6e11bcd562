// FP64 diagnostics of the particle state (energy and momentum), shared by the
// kernels (sph_integrate.cu) and the C ABI (sph_api.cu).
#pragma once

#include "sph_internal.cuh"

namespace sph {

// FP64 energy and momentum of the state at tick ti (partials: DIAG_BLOCKS x
// DIAG_FIELDS doubles of scratch; out: DIAG_FIELDS doubles, device)
constexpr int DIAG_FIELDS = 8, DIAG_BLOCKS = 304, DIAG_THREADS = 256;
cudaError_t launch_diagnostics(const sph_particles &p, long long ti, double dt_min, double gamma,
                               double *partials, double *out, cudaStream_t st);

}  // namespace sph
