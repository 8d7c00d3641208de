// observables.cu -- pair counts, energy, Warren-Cowley SRO, pair-parameter
// gradient, and the device Philox used by tests.
//
// The ordered pair counts n_m^{pq} = #{(i, v in shell m): s_i = p, s_{i+v} = q}
// (the pair numbers behind pi_m^{pp'} of Eq. 2) are one streaming pass over
// the lattice.  Energy, SRO and the pair gradient are small finishing kernels
// on the counts:
//   E = 1/2 sum_{m,p,q} V_m(p,q) n_m^{pq},
//   alpha_m^{pq} = 1 - n_m^{pq} / (N c_p z_m c_q),
//   dE/dV_m^{pq} = n_m^{pq} (p < q),  n_m^{pp} / 2 (p = q).
#include <algorithm>
#include <cstdint>

#include "smc_common.cuh"

namespace smc {

// Ordered pair counts by bonds.  Every unordered bond is visited once: shell 1
// from its sublattice-0 end (all 8 vectors), shells 2 and 3 along half of
// their vectors (+x, +y, +z; the 6 shell-3 vectors whose first non-zero
// component is positive).  With c_m^{pq} the number of visited (site, vector)
// pairs with s_i = p, s_{i+v} = q, the ordered count is
// n_m^{pq} = c_m^{pq} + c_m^{qp} (the map (i, v) -> (i + v, -v) is a bijection
// of the torus, aliasing included).  A warp walks whole rows (sub, z, y), lane
// = x; each lane keeps 8-bit counters packed per (shell, own species) in
// 64-bit words and the warp folds them into shared memory every 16 sites.
template <int NSH>
__global__ void __launch_bounds__(256) k_pair_counts(const int8_t *__restrict__ occ, int nx, int ny, int nz, int S,
                                                     unsigned long long *counts)
{
    __shared__ unsigned long long bins[NSH * 64];
    for (int i = threadIdx.x; i < NSH * 64; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long nrows = 2LL * nz * ny;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned char *o = (const unsigned char *)occ;
    for (long long row = w0; row < nrows; row += nw) {
        const int sub = (int)(row / ((long long)nz * ny));
        const int rem = (int)(row - (long long)sub * nz * ny);
        const int z = rem / ny, y = rem - (rem / ny) * ny;
        auto R = [&](int sb, int zz, int yy) {
            return o + ((size_t)((sb * nz + wrapc(zz, nz)) * ny + wrapc(yy, ny))) * nx;
        };
        const unsigned char *self = R(sub, z, y);
        const unsigned char *ry1 = R(sub, z, y + 1), *rym = R(sub, z, y - 1);
        const unsigned char *rz1 = R(sub, z + 1, y), *rzm = R(sub, z - 1, y);
        const unsigned char *rz1y1 = R(sub, z + 1, y + 1), *rzmy1 = R(sub, z - 1, y + 1);
        // shell 1 from sublattice 0: the other sublattice's cells (x-1..x, y-1..y, z-1..z)
        const unsigned char *p00 = R(1, z - 1, y - 1), *p01 = R(1, z - 1, y), *p10 = R(1, z, y - 1), *p11 = R(1, z, y);
        for (int x0 = 0; x0 < nx; x0 += 32 * 16) {
            unsigned long long acc[NSH][8];
#pragma unroll
            for (int m = 0; m < NSH; ++m)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[m][q] = 0;
            const int x1 = min(nx, x0 + 32 * 16);
            for (int x = x0 + lane; x < x1; x += 32) {
                const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
                const int p = self[x] & 7;
                unsigned long long h[3];
                h[0] = 0;
                if (sub == 0)
                    h[0] = (1ull << (8 * (p00[xm] & 7))) + (1ull << (8 * (p00[x] & 7))) +
                           (1ull << (8 * (p01[xm] & 7))) + (1ull << (8 * (p01[x] & 7))) +
                           (1ull << (8 * (p10[xm] & 7))) + (1ull << (8 * (p10[x] & 7))) +
                           (1ull << (8 * (p11[xm] & 7))) + (1ull << (8 * (p11[x] & 7)));
                if (NSH >= 2)
                    h[1] = (1ull << (8 * (self[xp] & 7))) + (1ull << (8 * (ry1[x] & 7))) + (1ull << (8 * (rz1[x] & 7)));
                if (NSH >= 3)
                    h[2] = (1ull << (8 * (ry1[xp] & 7))) + (1ull << (8 * (rym[xp] & 7))) +
                           (1ull << (8 * (rz1[xp] & 7))) + (1ull << (8 * (rzm[xp] & 7))) +
                           (1ull << (8 * (rz1y1[x] & 7))) + (1ull << (8 * (rzmy1[x] & 7)));
#pragma unroll
                for (int m = 0; m < NSH; ++m)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[m][q] += (p == q) ? h[m] : 0ull;
            }
            // at most 16 sites per lane x 8 per bin: no 8-bit field has overflowed
#pragma unroll
            for (int m = 0; m < NSH; ++m)
#pragma unroll
                for (int pp = 0; pp < 8; ++pp)
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (pp < S && q < S) {
                            const unsigned v =
                                __reduce_add_sync(0xffffffffu, (unsigned)((acc[m][pp] >> (8 * q)) & 0xFFu));
                            if (lane == 0 && v) atomicAdd(&bins[m * 64 + pp * 8 + q], (unsigned long long)v);
                        }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NSH * 64; i += blockDim.x) {
        const int m = i / 64, pp = (i / 8) % 8, q = i % 8;
        if (pp < S && q < S) {
            const unsigned long long c = bins[i] + bins[m * 64 + q * 8 + pp];
            if (c) atomicAdd(counts + (m * S + pp) * S + q, c);
        }
    }
}

// The same counts for rows of nx % 16 == 0 bytes (and a 16-byte aligned
// occupancy array), with 16-byte loads: lane l of a warp takes sites
// x = 16 l .. 16 l + 15 of a 512-site chunk of the row and reads each
// neighbour row once as a uint4 (plus one 4-byte word for the byte before or
// after the 16).  A site's neighbour histogram per shell is 8 4-bit fields in
// one word (at most 8 neighbours per shell); its even and odd fields are
// added, as 8-bit fields, to the lane's counters of its own species, kept in
// shared memory [shell][species][lane] (at most 16 x 8 per field per chunk).
constexpr int kCountWarps = 4;

__device__ __forceinline__ unsigned fcount_byte(const uint4 &w, int k)
{
    const unsigned v = k < 4 ? w.x : (k < 8 ? w.y : (k < 12 ? w.z : w.w));
    return (v >> (8 * (k & 3))) & 7u;
}

__device__ __forceinline__ unsigned fcount_nib(unsigned species) { return 1u << (4 * species); }

template <int NSH, int S>
__global__ void __launch_bounds__(32 * kCountWarps) k_pair_counts16(const int8_t *__restrict__ occ, int nx, int ny,
                                                                    int nz, unsigned long long *counts)
{
    __shared__ unsigned long long bins[NSH * 64];
    __shared__ uint2 acc_all[kCountWarps][NSH][S][32];
    for (int i = threadIdx.x; i < NSH * 64; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint2(*acc)[S][32] = acc_all[warp];
    const long long nrows = 2LL * nz * ny;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned char *o = (const unsigned char *)occ;
    const int nw4 = nx >> 2;
    for (long long row = w0; row < nrows; row += nw) {
        const int sub = (int)(row / ((long long)nz * ny));
        const int rem = (int)(row - (long long)sub * nz * ny);
        const int z = rem / ny, y = rem - (rem / ny) * ny;
        auto R = [&](int sb, int zz, int yy) {
            return o + ((size_t)((sb * nz + wrapc(zz, nz)) * ny + wrapc(yy, ny))) * nx;
        };
        for (int x0 = 0; x0 < nx; x0 += 32 * 16) {
#pragma unroll
            for (int m = 0; m < NSH; ++m)
#pragma unroll
                for (int p = 0; p < S; ++p) acc[m][p][lane] = make_uint2(0u, 0u);
            const int xb = x0 + 16 * lane;
            if (xb < nx) {
                const int wprev = (xb >> 2) == 0 ? nw4 - 1 : (xb >> 2) - 1, wnext = ((xb + 16) >> 2) % nw4;
                auto V = [&](const unsigned char *r) { return __ldg(reinterpret_cast<const uint4 *>(r + xb)); };
                auto PREV = [&](const unsigned char *r) { return (__ldg(reinterpret_cast<const unsigned *>(r) + wprev) >> 24) & 7u; };
                auto NEXT = [&](const unsigned char *r) { return __ldg(reinterpret_cast<const unsigned *>(r) + wnext) & 7u; };
                const unsigned char *self = R(sub, z, y);
                const uint4 vs = V(self);
                unsigned ns = 0;
                uint4 v00, v01, v10, v11, vy1, vz1, vym, vzm, vz1y1, vzmy1;
                unsigned p00 = 0, p01 = 0, p10 = 0, p11 = 0, ny1 = 0, nym = 0, nz1 = 0, nzm = 0;
                if (sub == 0) {
                    const unsigned char *r00 = R(1, z - 1, y - 1), *r01 = R(1, z - 1, y), *r10 = R(1, z, y - 1),
                                        *r11 = R(1, z, y);
                    v00 = V(r00);
                    v01 = V(r01);
                    v10 = V(r10);
                    v11 = V(r11);
                    p00 = PREV(r00);
                    p01 = PREV(r01);
                    p10 = PREV(r10);
                    p11 = PREV(r11);
                }
                if (NSH >= 2) {
                    const unsigned char *ry1 = R(sub, z, y + 1), *rz1 = R(sub, z + 1, y);
                    ns = NEXT(self);
                    vy1 = V(ry1);
                    vz1 = V(rz1);
                    if (NSH >= 3) {
                        const unsigned char *rym = R(sub, z, y - 1), *rzm = R(sub, z - 1, y);
                        ny1 = NEXT(ry1);
                        nz1 = NEXT(rz1);
                        vym = V(rym);
                        vzm = V(rzm);
                        nym = NEXT(rym);
                        nzm = NEXT(rzm);
                        vz1y1 = V(R(sub, z + 1, y + 1));
                        vzmy1 = V(R(sub, z - 1, y + 1));
                    }
                }
                // byte k of a row window, k = -1 and 16 from the neighbouring words
                auto B = [&](const uint4 &w, unsigned prev, unsigned next, int k) -> unsigned {
                    return k < 0 ? prev : (k > 15 ? next : fcount_byte(w, k));
                };
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const unsigned p = fcount_byte(vs, k);
                    unsigned h[3] = {0u, 0u, 0u};
                    if (sub == 0)
                        h[0] = fcount_nib(B(v00, p00, 0, k - 1)) + fcount_nib(fcount_byte(v00, k)) +
                               fcount_nib(B(v01, p01, 0, k - 1)) + fcount_nib(fcount_byte(v01, k)) +
                               fcount_nib(B(v10, p10, 0, k - 1)) + fcount_nib(fcount_byte(v10, k)) +
                               fcount_nib(B(v11, p11, 0, k - 1)) + fcount_nib(fcount_byte(v11, k));
                    if (NSH >= 2)
                        h[1] = fcount_nib(B(vs, 0, ns, k + 1)) + fcount_nib(fcount_byte(vy1, k)) +
                               fcount_nib(fcount_byte(vz1, k));
                    if (NSH >= 3)
                        h[2] = fcount_nib(B(vy1, 0, ny1, k + 1)) + fcount_nib(B(vym, 0, nym, k + 1)) +
                               fcount_nib(B(vz1, 0, nz1, k + 1)) + fcount_nib(B(vzm, 0, nzm, k + 1)) +
                               fcount_nib(fcount_byte(vz1y1, k)) + fcount_nib(fcount_byte(vzmy1, k));
                    if (p < (unsigned)S) {
#pragma unroll
                        for (int m = 0; m < NSH; ++m) {
                            if (m == 0 && sub != 0) continue;  // shell 1 is counted from sublattice 0
                            uint2 a = acc[m][p][lane];
                            a.x += h[m] & 0x0F0F0F0Fu;         // q = 0, 2, 4, 6
                            a.y += (h[m] >> 4) & 0x0F0F0F0Fu;  // q = 1, 3, 5, 7
                            acc[m][p][lane] = a;
                        }
                    }
                }
            }
            __syncwarp();
            // 16 sites per lane x at most 8 per field: no 8-bit field has overflowed
#pragma unroll
            for (int m = 0; m < NSH; ++m)
#pragma unroll
                for (int pp = 0; pp < S; ++pp) {
                    const uint2 a = acc[m][pp][lane];
#pragma unroll
                    for (int q = 0; q < S; ++q) {
                        const unsigned f = ((q & 1) ? a.y : a.x) >> (8 * (q >> 1));
                        const unsigned v = __reduce_add_sync(0xffffffffu, f & 0xFFu);
                        if (lane == 0 && v) atomicAdd(&bins[m * 64 + pp * 8 + q], (unsigned long long)v);
                    }
                }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NSH * 64; i += blockDim.x) {
        const int m = i / 64, pp = (i / 8) % 8, q = i % 8;
        if (pp < S && q < S) {
            const unsigned long long c = bins[i] + bins[m * 64 + q * 8 + pp];
            if (c) atomicAdd(counts + (m * S + pp) * S + q, c);
        }
    }
}

// The same counts from bit planes, for rows of nx % 32 == 0 sites.  A word
// of a row holds 32 consecutive sites; plane k bit i is bit k of the species
// of site i, so the sites of species p in a word are one three-input logic
// function of the planes, M_p.  For a vector v (one of the visited half of a
// shell, as above) and the word's sites i with neighbours i + v,
//   c_m^{pq} = popc(M_p(i) & M_q(i + v)),
// where M_q(i + v) comes from the neighbour row's word, funnel-shifted by one
// site (with the wrap of the row) when v has an x component.  Only the sums
// n_m^{pq} = c_m^{pq} + c_m^{qp} are needed, and for p != q the two bit sets
// are disjoint (a site has one species), so each unordered pair costs one
// popcount: popc((M_p(i) & M_q(i + v)) | (M_q(i) & M_p(i + v))).
__global__ void k_planes(const int8_t *__restrict__ occ, long long nwords, uint4 *__restrict__ planes)
{
    const uint4 *o = reinterpret_cast<const uint4 *>(occ);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nwords;
         t += (long long)gridDim.x * blockDim.x) {
        const uint4 a = __ldg(o + 2 * t), b = __ldg(o + 2 * t + 1);
        const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t P[3] = {0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // bit k of the four bytes at bits 0, 8, 16, 24; the product
                // gathers them at bits 24..27 (no two partial products meet)
                const uint32_t x = (w[j] >> k) & 0x01010101u;
                P[k] |= ((x * 0x01020408u) >> 24) << (4 * j);
            }
        planes[t] = make_uint4(P[0], P[1], P[2], 0u);
    }
}

template <int S>
__device__ __forceinline__ void species_masks(const uint4 &w, uint32_t (&M)[S])
{
#pragma unroll
    for (int p = 0; p < S; ++p)
        M[p] = ((p & 1) ? w.x : ~w.x) & ((p & 2) ? w.y : ~w.y) & ((p & 4) ? w.z : ~w.z);
}
// the word of sites x - 1 (from the previous word's last site) and x + 1
__device__ __forceinline__ uint4 site_minus1(const uint4 &prev, const uint4 &cur)
{
    return make_uint4(__funnelshift_l(prev.x, cur.x, 1), __funnelshift_l(prev.y, cur.y, 1),
                      __funnelshift_l(prev.z, cur.z, 1), 0u);
}
__device__ __forceinline__ uint4 site_plus1(const uint4 &cur, const uint4 &next)
{
    return make_uint4(__funnelshift_r(cur.x, next.x, 1), __funnelshift_r(cur.y, next.y, 1),
                      __funnelshift_r(cur.z, next.z, 1), 0u);
}

template <int NSH, int S>
__global__ void __launch_bounds__(256) k_pair_counts_planes(const uint4 *__restrict__ planes, int nw, int ny, int nz,
                                                            unsigned long long *counts)
{
    constexpr int NP = S * (S + 1) / 2;  // pairs p <= q
    __shared__ unsigned long long bins[NSH * NP];
    for (int i = threadIdx.x; i < NSH * NP; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    uint32_t acc[NSH][NP];  // p < q: n^{pq}; p = q: c^{pp} = n^{pp} / 2
#pragma unroll
    for (int m = 0; m < NSH; ++m)
#pragma unroll
        for (int k = 0; k < NP; ++k) acc[m][k] = 0u;
    const long long total = 2LL * ny * nz * nw;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long row = t / nw;
        const int w = (int)(t - row * nw);
        const int sub = (int)(row / ((long long)ny * nz));
        const int rem = (int)(row - (long long)sub * ny * nz);
        const int z = rem / ny, y = rem - z * ny;
        auto PL = [&](int sb, int zz, int yy, int ww) {
            ww = ww < 0 ? ww + nw : (ww >= nw ? ww - nw : ww);
            return __ldg(planes + ((size_t)((sb * nz + wrapc(zz, nz)) * ny + wrapc(yy, ny))) * nw + ww);
        };
        uint32_t A[S];
        const uint4 c = PL(sub, z, y, w);
        species_masks<S>(c, A);
        auto count = [&](int m, const uint4 &nb) {
            uint32_t B[S];
            species_masks<S>(nb, B);
            int k = 0;
#pragma unroll
            for (int p = 0; p < S; ++p) {
                acc[m][k++] += __popc(A[p] & B[p]);
#pragma unroll
                for (int q = p + 1; q < S; ++q) acc[m][k++] += __popc((A[p] & B[q]) | (A[q] & B[p]));
            }
        };
        if (sub == 0) {
            // shell 1: partners (1, y + dy, z + dz), dy, dz in {-1, 0}, at x - 1 and x
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int dy = (k & 1) - 1, dz = (k >> 1) - 1;
                const uint4 r = PL(1, z + dz, y + dy, w), rp = PL(1, z + dz, y + dy, w - 1);
                count(0, r);
                count(0, site_minus1(rp, r));
            }
        }
        if constexpr (NSH >= 2) {
            // shell 2: +x, +y, +z
            const uint4 ry = PL(sub, z, y + 1, w), rz = PL(sub, z + 1, y, w);
            count(1, site_plus1(c, PL(sub, z, y, w + 1)));
            count(1, ry);
            count(1, rz);
            if constexpr (NSH >= 3) {
                // shell 3: (+x, +-y), (+x, +-z), (+y, +-z)
                count(2, site_plus1(ry, PL(sub, z, y + 1, w + 1)));
                count(2, site_plus1(PL(sub, z, y - 1, w), PL(sub, z, y - 1, w + 1)));
                count(2, site_plus1(rz, PL(sub, z + 1, y, w + 1)));
                count(2, site_plus1(PL(sub, z - 1, y, w), PL(sub, z - 1, y, w + 1)));
                count(2, PL(sub, z + 1, y + 1, w));
                count(2, PL(sub, z - 1, y + 1, w));
            }
        }
    }
    // at most 8 visited vectors per shell x 32 sites per word: the 32-bit
    // counters hold 2^32 / 256 words per thread
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < NSH; ++m)
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const unsigned v = __reduce_add_sync(0xffffffffu, acc[m][k]);
            if (lane == 0 && v) atomicAdd(&bins[m * NP + k], (unsigned long long)v);
        }
    __syncthreads();
    for (int i = threadIdx.x; i < NSH * S * S; i += blockDim.x) {
        const int m = i / (S * S), p = (i / S) % S, q = i % S;
        const int a = p < q ? p : q, b = p < q ? q : p;
        const int k = a * S - a * (a - 1) / 2 + (b - a);  // index of (a, b) among the pairs a <= b
        const unsigned long long v = bins[m * NP + k];
        const unsigned long long cnt = p == q ? 2 * v : v;
        if (cnt) atomicAdd(counts + i, cnt);
    }
}

// A grow-only device buffer for the planes (kept apart from the workspace,
// whose scratch the callers already use for the counts).
void *planes_buffer(size_t bytes, smc_status *st)
{
    static void *buf = nullptr;
    static size_t cap = 0;
    static int dev = -1;
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    if (buf && (bytes <= cap) && d == dev) return buf;
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess && buf) e = cudaFree(buf);
    buf = nullptr;
    cap = 0;
    if (e == cudaSuccess) e = cudaMalloc(&buf, bytes);
    if (e != cudaSuccess) {
        buf = nullptr;
        *st = cuda_fail(e, "cudaMalloc(planes)");
        return nullptr;
    }
    cap = bytes;
    dev = d;
    return buf;
}

template <int NSH, int S>
void launch_planes_counts(int blocks, const uint4 *planes, int nw, int ny, int nz, unsigned long long *counts,
                          cudaStream_t stream)
{
    k_pair_counts_planes<NSH, S><<<blocks, 256, 0, stream>>>(planes, nw, ny, nz, counts);
}

// Dispatch on (shells, species) with at most 84 counters per thread; false
// when the pair is not covered.
bool planes_counts(int NSH, int S, int blocks, const uint4 *planes, int nw, int ny, int nz,
                   unsigned long long *counts, cudaStream_t stream)
{
#define SMC_PC(n, s)                                                              \
    if (NSH == n && S == s) {                                                    \
        launch_planes_counts<n, s>(blocks, planes, nw, ny, nz, counts, stream); \
        return true;                                                             \
    }
    SMC_PC(1, 2) SMC_PC(1, 3) SMC_PC(1, 4) SMC_PC(1, 5) SMC_PC(1, 6) SMC_PC(1, 7) SMC_PC(1, 8)
    SMC_PC(2, 2) SMC_PC(2, 3) SMC_PC(2, 4) SMC_PC(2, 5) SMC_PC(2, 6) SMC_PC(2, 7) SMC_PC(2, 8)
    SMC_PC(3, 2) SMC_PC(3, 3) SMC_PC(3, 4) SMC_PC(3, 5) SMC_PC(3, 6) SMC_PC(3, 7)
#undef SMC_PC
    return false;
}

template <int NSH>
void launch_counts16(int S, int blocks, int threads, const int8_t *occ, int nx, int ny, int nz,
                     unsigned long long *counts, cudaStream_t stream)
{
    switch (S) {
    case 1: k_pair_counts16<NSH, 1><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    case 2: k_pair_counts16<NSH, 2><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    case 3: k_pair_counts16<NSH, 3><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    case 4: k_pair_counts16<NSH, 4><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    case 5: k_pair_counts16<NSH, 5><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    case 6: k_pair_counts16<NSH, 6><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    case 7: k_pair_counts16<NSH, 7><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    default: k_pair_counts16<NSH, 8><<<blocks, threads, 0, stream>>>(occ, nx, ny, nz, counts); break;
    }
}

smc_status launch_pair_counts(const smc_lattice *lat, int nshells, const int8_t *occ, unsigned long long *counts,
                              cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const int S = lat->nspecies;
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * nshells * S * S, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counts)");
    const long long rows = 2LL * lat->ny * lat->nz;
    if (lat->nx % 32 == 0 && reinterpret_cast<uintptr_t>(occ) % 16 == 0 && S >= 2 &&
        S * (S + 1) / 2 * nshells <= 84) {
        const int nw = lat->nx / 32;
        const long long nwords = rows * nw;
        uint4 *planes = (uint4 *)planes_buffer((size_t)nwords * sizeof(uint4), &st);
        if (!planes) return st;
        const int grid = (int)std::max(1LL, std::min<long long>((nwords + 255) / 256, (long long)ws->num_sms * 8));
        k_planes<<<grid, 256, 0, stream>>>(occ, nwords, planes);
        if (planes_counts(nshells, S, ws->num_sms * 4, planes, nw, lat->ny, lat->nz, counts, stream)) {
            e = cudaGetLastError();
            return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_pair_counts_planes");
        }
    }
    const int threads = 256;
    const long long want = (rows + 7) / 8;
    const int blocks = (int)std::max(1LL, std::min<long long>(want, (long long)ws->num_sms * 8));
    if (lat->nx % 16 == 0 && reinterpret_cast<uintptr_t>(occ) % 16 == 0) {
        const int t16 = 32 * kCountWarps;
        const int b16 = (int)std::max(1LL, std::min<long long>((rows + kCountWarps - 1) / kCountWarps,
                                                               (long long)ws->num_sms * 16));
        if (nshells == 1)
            launch_counts16<1>(S, b16, t16, occ, lat->nx, lat->ny, lat->nz, counts, stream);
        else if (nshells == 2)
            launch_counts16<2>(S, b16, t16, occ, lat->nx, lat->ny, lat->nz, counts, stream);
        else
            launch_counts16<3>(S, b16, t16, occ, lat->nx, lat->ny, lat->nz, counts, stream);
    } else if (nshells == 1)
        k_pair_counts<1><<<blocks, threads, 0, stream>>>(occ, lat->nx, lat->ny, lat->nz, S, counts);
    else if (nshells == 2)
        k_pair_counts<2><<<blocks, threads, 0, stream>>>(occ, lat->nx, lat->ny, lat->nz, S, counts);
    else
        k_pair_counts<3><<<blocks, threads, 0, stream>>>(occ, lat->nx, lat->ny, lat->nz, S, counts);
    e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_pair_counts");
}

__constant__ int c_shell_z[3] = {8, 6, 12};

__global__ void k_sro_finish(int nshells, int S, long long N, const unsigned long long *counts, double *alpha)
{
    const int i = threadIdx.x;
    if (i >= nshells * S * S) return;
    const int m = i / (S * S), p = (i / S) % S, q = i % S;
    // N_p from the first-shell row sums: sum_q n_1^{pq} = 8 N_p
    long long Np = 0, Nq = 0;
    for (int t = 0; t < S; ++t) {
        Np += (long long)counts[p * S + t];
        Nq += (long long)counts[q * S + t];
    }
    Np /= 8;
    Nq /= 8;
    if (Np == 0 || Nq == 0) {
        alpha[i] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    const double cp = __ddiv_rn((double)Np, (double)N), cq = __ddiv_rn((double)Nq, (double)N);
    const double den = __dmul_rn(__dmul_rn(__dmul_rn((double)N, cp), (double)c_shell_z[m]), cq);
    alpha[i] = __dsub_rn(1.0, __ddiv_rn((double)counts[i], den));
}

smc_status launch_sro_finish(const smc_lattice *lat, int nshells, const unsigned long long *counts, double *alpha,
                             cudaStream_t stream)
{
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    k_sro_finish<<<1, 256, 0, stream>>>(nshells, lat->nspecies, N, counts, alpha);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_sro_finish");
}

struct VBlock {
    int vi[kMaxShells * kMaxSpecies * kMaxSpecies];
    float vf[kMaxShells * kMaxSpecies * kMaxSpecies];
};

__global__ void k_energy_finish(VBlock V, int is_int, int nshells, int S, const unsigned long long *counts,
                                double *e, long long *e_int, double *e_add)
{
    if (threadIdx.x != 0) return;
    if (is_int) {
        long long tot = 0;
        for (int i = 0; i < nshells * S * S; ++i) tot += (long long)V.vi[i] * (long long)counts[i];
        tot /= 2;  // every bond is counted from both ends
        if (e_int) *e_int = tot;
        if (e) *e = (double)tot;
    } else {
        double tot = 0.0;
        for (int i = 0; i < nshells * S * S; ++i) tot = __dadd_rn(tot, __dmul_rn((double)V.vf[i], (double)counts[i]));
        tot = __dmul_rn(0.5, tot);
        if (e_add) tot = __dadd_rn(tot, *e_add);
        if (e) *e = tot;
    }
}

smc_status launch_energy_finish(const smc_lattice *lat, const smc_model *m, const unsigned long long *counts,
                                double *e, int64_t *e_int, cudaStream_t stream)
{
    VBlock V;
    const int S = lat->nspecies, n = m->nshells * S * S;
    for (int i = 0; i < n; ++i) {
        if (m->kind == SMC_PAIR_I32)
            V.vi[i] = m->v_i32[i];
        else
            V.vf[i] = m->v_f32[i];
    }
    k_energy_finish<<<1, 32, 0, stream>>>(V, m->kind == SMC_PAIR_I32, m->nshells, S, counts, e,
                                          (long long *)e_int, nullptr);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? SMC_OK : cuda_fail(err, "k_energy_finish");
}

__global__ void k_pair_grad_finish(int nshells, int S, const unsigned long long *counts, float *grad)
{
    const int i = threadIdx.x;
    const int per = S * (S + 1) / 2;
    if (i >= nshells * per) return;
    const int m = i / per;
    int r = i % per, p = 0;
    while (r >= S - p) {
        r -= S - p;
        ++p;
    }
    const int q = p + r;
    const unsigned long long c = counts[(m * S + p) * S + q];
    grad[i] = p == q ? (float)((double)c * 0.5) : (float)c;
}

smc_status launch_pair_grad_finish(const smc_lattice *lat, const smc_model *m, const unsigned long long *counts,
                                   float *grad, cudaStream_t stream)
{
    k_pair_grad_finish<<<1, 256, 0, stream>>>(m->nshells, lat->nspecies, counts, grad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_pair_grad_finish");
}

__global__ void k_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    U4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
    U4 w = philox10(c, key[2 * i], key[2 * i + 1]);
    out[4 * i] = w.x;
    out[4 * i + 1] = w.y;
    out[4 * i + 2] = w.z;
    out[4 * i + 3] = w.w;
}

smc_status launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n, cudaStream_t stream)
{
    if (n <= 0) return SMC_OK;
    const int threads = 256;
    k_philox<<<(unsigned)((n + threads - 1) / threads), threads, 0, stream>>>(ctr, key, out, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_philox");
}

}  // namespace smc
