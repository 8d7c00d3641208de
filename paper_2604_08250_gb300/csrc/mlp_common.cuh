// mlp_common.cuh -- device pieces of the MLP site energy (MLPNet, Sec. IV-B)
// shared by the sweep, energy and gradient kernels: species lookups, packed
// neighbour histograms and BF16 packing.
#pragma once

#include <cuda_bf16.h>

#include "smc_common.cuh"

namespace smc {

extern __shared__ __align__(16) unsigned char g_smem[];

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}


// Species at cell (xx, yy, zz) of sublattice sb (coordinates within one box
// length of the box).
__device__ __forceinline__ int occ_at(const int8_t *occ, int nx, int ny, int nz, int sb, int xx, int yy, int zz)
{
    return occ[((size_t)((sb * nz + wrapc(zz, nz)) * ny + wrapc(yy, ny))) * nx + wrapc(xx, nx)] & 7;
}

// Packed neighbour histograms of the site at cell (x, y, z) of sublattice
// sub, read through `spec(sublattice, x, y, z)`.
template <class Spec>
__device__ __forceinline__ void site_hist(const Spec &spec, int sub, int x, int y, int z, uint32_t &h1,
                                          uint32_t &h2, uint32_t &h3)
{
    const int o = sub == 0 ? -1 : 0;
    h1 = h2 = h3 = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
        h1 += 1u << (4 * spec(1 - sub, x + o + ((u >> 2) & 1), y + o + ((u >> 1) & 1), z + o + (u & 1)));
    h2 = (1u << (4 * spec(sub, x - 1, y, z))) + (1u << (4 * spec(sub, x + 1, y, z))) +
         (1u << (4 * spec(sub, x, y - 1, z))) + (1u << (4 * spec(sub, x, y + 1, z))) +
         (1u << (4 * spec(sub, x, y, z - 1))) + (1u << (4 * spec(sub, x, y, z + 1)));
#pragma unroll
    for (int p = -1; p <= 1; p += 2)
#pragma unroll
        for (int r = -1; r <= 1; r += 2)
            h3 += (1u << (4 * spec(sub, x + p, y + r, z))) + (1u << (4 * spec(sub, x + p, y, z + r))) +
                  (1u << (4 * spec(sub, x, y + p, z + r)));
}

}  // namespace smc
