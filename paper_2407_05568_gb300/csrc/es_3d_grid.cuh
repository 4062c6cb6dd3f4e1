// es_3d_grid.cuh -- index and ghost helpers of the 3D meshes, shared by the FP64 (es_3d.cu) and the
// mixed (es_3d_mixed.cu) kernels.
#pragma once
#include <cuda_runtime.h>

#include "es_3d.h"
#include "es_device.cuh"

namespace es {

__device__ __forceinline__ size_t idx3(const Grid3& g, int i1, int i2, int i3) {
    return (size_t(i3) * g.n[1] + i2) * g.n[0] + i1;
}

// extended grid (3 ghosts in every direction)
__device__ __forceinline__ size_t eidx(const Grid3& g, int e1, int e2, int e3) {
    return (size_t(e3) * (g.n[1] + 6) + e2) * (g.n[0] + 6) + e1;
}

// value of a mesh field at a possibly-ghost node: tensor product of the per-direction ghost
// terms (odd reflection / wrap) of f + c2 f2, plus the period shift for coordinate component
// `comp` (-1: none)
__device__ __forceinline__ double ghost_value3(const Grid3& g, const double* f, const double* f2, double c2,
                                               int i1, int i2, int i3, int comp) {
    // a coordinate / velocity component other than direction d lies along that direction's planes
    const GhostTerms t1 = ghost_terms(i1, g.n[0], g.bc[0], comp != 0);
    const GhostTerms t2 = ghost_terms(i2, g.n[1], g.bc[1], comp != 1);
    const GhostTerms t3 = ghost_terms(i3, g.n[2], g.bc[2], comp != 2);
    double acc = 0.0;
    for (int c = 0; c < t3.nterm; ++c)
        for (int b = 0; b < t2.nterm; ++b)
            for (int a = 0; a < t1.nterm; ++a) {
                const size_t id = (size_t(t3.idx[c]) * g.n[1] + t2.idx[b]) * g.n[0] + t1.idx[a];
                const double v = f2 ? f[id] + c2 * f2[id] : f[id];
                acc += t1.w[a] * t2.w[b] * t3.w[c] * v;
            }
    if (comp == 0) acc += t1.q * g.period[0];
    if (comp == 1) acc += t2.q * g.period[1];
    if (comp == 2) acc += t3.q * g.period[2];
    return acc;
}

// node at least `m` nodes inside the mesh in every direction (its stencil needs no ghost rule)
__device__ __forceinline__ bool inside3(const Grid3& g, int i1, int i2, int i3, int m) {
    return i1 >= m && i1 < g.n[0] - m && i2 >= m && i2 < g.n[1] - m && i3 >= m && i3 < g.n[2] - m;
}

}  // namespace es
