// mlp_common.cuh -- device pieces of the MLP site energy (MLPNet, Sec. IV-B)
// shared by the sweep, energy and gradient kernels: feature rows, the
// m16n8k16 BF16 tensor-core instruction and the SiLU.
#pragma once

#include <cuda_bf16.h>

#include "smc_common.cuh"

namespace smc {

constexpr int kARowB = 80;    // feature row stride (bytes): 32 BF16 used, padded against bank conflicts
constexpr int kW1RowB = 80;   // W1 row stride in shared memory (32 BF16 + pad)
constexpr int kW2RowB = 144;  // W2 row stride (64 BF16 + pad)

extern __shared__ __align__(16) unsigned char g_smem[];

__device__ __forceinline__ uint32_t lds32(uint32_t off) { return *(const uint32_t *)(g_smem + off); }

__device__ __forceinline__ void mma_bf16(float *d, uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// SiLU through the identity z sigmoid(z) = h (1 + tanh(h)), h = z/2, with the
// hardware tanh approximation (relative error about 2^-11).
__device__ __forceinline__ float silu(float z)
{
    const float h = 0.5f * z;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Feature row of a site from its species q0 and packed 4-bit neighbour counts
// per shell: 32 BF16 values [onehot(5) | h1(5) | h2(5) | h3(5) | 0 ...].
__device__ __forceinline__ void write_feature_row(uint32_t row, int q0, uint32_t h1, uint32_t h2, uint32_t h3)
{
    uint32_t w[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int col = 2 * c + u;
            float x = 0.f;
            if (col < 5)
                x = (col == q0) ? 1.f : 0.f;
            else if (col < 10)
                x = (float)((h1 >> (4 * (col - 5))) & 15u);
            else if (col < 15)
                x = (float)((h2 >> (4 * (col - 10))) & 15u);
            else if (col < 20)
                x = (float)((h3 >> (4 * (col - 15))) & 15u);
            v[u] = x;
        }
        w[c] = pack_bf16(v[0], v[1]);  // small integers: exact in BF16
    }
#pragma unroll
    for (int c = 0; c < 16; c += 4)
        *(uint4 *)(g_smem + row + 4 * c) = make_uint4(w[c], w[c + 1], w[c + 2], w[c + 3]);
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
