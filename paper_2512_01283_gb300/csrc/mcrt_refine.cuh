// mcrt_refine.cuh -- the composite grid of static mesh refinement (Kratos-polrad,
// arXiv:2512.01283, Sec. 2: a composite mesh, optionally with static mesh refinement).
// One level of disjoint patches over the root grid; a root cell covered by patch p
// carries p + 1 in the last word of its record.  Shared by the transport and the
// imaging kernels.
#pragma once

#include "mcrt_device.cuh"
#include "mcrt_internal.h"
#include "mcrt_packet.cuh"

namespace mcrt {

// Patch covering a root cell, from its record; -1 when none.
__device__ __forceinline__ int covering_patch(const float4& r) { return (int)__float_as_uint(r.w) - 1; }

template <typename T> __device__ __forceinline__ T patch_lo(const PatchDev& q, int a) { return pick<T>(q.lo_f[a], q.lo[a]); }
template <typename T> __device__ __forceinline__ T patch_d(const PatchDev& q, int a) { return pick<T>(q.d_f[a], q.d[a]); }

// Cell of patch q holding p for travel along n (a point on a face belongs to the cell n
// points into), clamped to the patch: the entry cell when p lies on the patch's box.
template <typename T>
__device__ __forceinline__ void patch_locate(const PatchDev& q, T px, T py, T pz, T nx, T ny, T nz, int idx[3]) {
    const T p[3] = {px, py, pz}, n[3] = {nx, ny, nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T x = (p[a] - patch_lo<T>(q, a)) / patch_d<T>(q, a);
        int i = (int)floor(x);
        if (T(i) == x && n[a] < T(0)) i -= 1;
        i = i < 0 ? 0 : (i >= q.n[a] ? q.n[a] - 1 : i);
        idx[a] = i;
    }
}

__device__ __forceinline__ long long patch_cell(const PatchDev& q, int ix, int iy, int iz) {
    return q.offset + ((long long)iz * q.n[1] + iy) * q.n[0] + ix;
}

}  // namespace mcrt
