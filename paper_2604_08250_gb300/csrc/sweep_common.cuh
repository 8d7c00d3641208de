// sweep_common.cuh -- parameter block and warp-level helpers shared by the
// pair and MLP sweep kernels.
#pragma once

#include "smc_common.cuh"

namespace smc {

constexpr int kMaxBeta = 1024;
constexpr int kMaxGroups = 64;
// Fixed-point pair tables (pair_fixed.cuh): 64 rows (A * 8 + B) of at most
// 28 words.
constexpr int kPairQWords = 64 * 28;

// MLP weights as the kernels read them (device memory, one copy per call):
// W1 padded from 20 to 32 inputs, BF16 bit patterns, row = output unit; W2
// BF16; W3, biases FP32 (W3 widened exactly from BF16).
struct MlpBlock {
    uint16_t w1[64 * 32];
    uint16_t w2[64 * 64];
    float b1[64], b2[64], w3[64];
    float b3;
    float pad[3];
};

// Fills the kernels' weight block from a model's MLP weights (host).
void make_mlp_block(const smc_model *m, MlpBlock &W);

struct RepDesc {
    int8_t *occ;
    double *e_acc;
    long long *n_acc;
    int nx, ny, nz;
    int NLx, NLy, NLz;
    int NTy, NTz;  // tiles along y, z
    int tile0;     // first global tile of this replica
    uint32_t rep;  // RNG replica index
    int vec;       // rows are 16-byte aligned: copy with 16-byte transactions
};

struct SweepParams {
    int R, ntiles, G;
    int Lx, Ly, Lz;
    int TY, TZ, CB;
    int nshells, S;
    int nsweeps;
    int beta_stride;  // 0: one value per replica; else values per (replica, sweep)
    int tpc;          // accumulator slots per CTA (>= tiles owned by any CTA)
    int skip_tile;
    int maxNLx;           // fast kernel: most link cells along x of any replica
    int team;             // fast kernel: warps sharing one column (1, 2 or 4)
    int team_bytes;       // fast kernel: shared-memory bytes per team
    int nbuf;             // fast kernel: row buffers per team (1 or 2)
    int stage;            // fast kernel: row staging by bulk copies (0) or 16-byte cp.async (1)
    uint64_t seed, sweep0;
    long long timeout_ns;
    uint32_t *flags;
    double *part_e;
    long long *part_n;
    unsigned *ticket;
    int *abort_flag;
    int *status;
    const uint32_t *tab;  // integer acceptance tables
    int lag[kMaxGroups];  // group g may start once neighbours completed g+1-lag[g] groups
    int warp_bytes;       // fast kernel: shared-memory bytes per warp
    int nap_cap;          // fast kernel: longest sleep between progress polls (ns)
    int kind;             // model kind (SMC_PAIR_I32 .. SMC_PAIR_F32_MLP_BF16)
    const void *mlpw;     // network weights (device MlpBlock or NetBlock), MLP kinds only
    float *ecache;        // per-site MLP energy f(x_i) (device, N floats), MLP kinds only
    uint4 *fcache;        // per-site MLP features {species, shell-1, -2, -3 packed counts} (device, N)
    int rowB;             // fast kernel: row stride in shared memory
    int mlp_chunk;        // MLP sweep: trials of a mini-step evaluated together
    int qrow;             // pair kernels: words per fixed-point table row
    int pad1;
    double escale;        // pair kernels: eV (integer models: units) per dE_fix unit, 2^-sigma
    union {
        float beta[kMaxBeta];        // MLP and qSRO kernels: 1 / kT; pair kernels: cx = -log2(e) 2^-sigma / kT
        int2 tabinfo[kMaxBeta / 2];  // (offset, length) into tab
    } temp;
    // resident kernel: block descriptors, exchange lists, the lattice at the
    // start of the launch (species x 8), the published row versions (words of
    // 4 species bytes | 32-bit tag, two copies by sweep parity), window of
    // rows per sublattice, block grid
    const int *rdesc;
    const uint32_t *rlists;
    int8_t *exch;
    unsigned long long *xver;
    int nver, rxw;  // version slots; exchange warps of the resident kernel
    int Wy, Wz, NBy, NBz, rcols, rblob;
    uint32_t qtab[kPairQWords];  // pair kernels: fixed-point table rows (pair_fixed.cuh)
    union {
        int di[kMaxShells * kMaxSpecies * kMaxSpecies * kMaxSpecies];
        float df[kMaxShells * kMaxSpecies * kMaxSpecies * kMaxSpecies];
    } D;  // D[m][A][B][q] = V_m(B, q) - V_m(A, q)
    RepDesc rep[kMaxReplicas];
};
static_assert(sizeof(SweepParams) < 32000, "kernel parameter block too large");

constexpr int kDEntries = kMaxShells * kMaxSpecies * kMaxSpecies * kMaxSpecies;


template <bool IS_INT>
struct Acc;
template <>
struct Acc<true> {
    using T = int;
};
template <>
struct Acc<false> {
    using T = float;
};

template <bool IS_INT>
__device__ __forceinline__ bool metropolis(typename Acc<IS_INT>::T dE, uint32_t r, float beta, const uint32_t *tab,
                                           int2 ti)
{
    if constexpr (IS_INT) {
        if (dE <= 0) return true;
        return (int)dE < ti.y && r < __ldg(tab + ti.x + (int)dE);
    } else {
        const float u = ((float)r + 0.5f) * 1.862645149230957e-09f;  // 2^-29
        return (dE <= 0.f) | (u < expf(-beta * (float)dE));
    }
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

extern __shared__ __align__(16) unsigned char g_smem[];

#define SM8(off) ((uint32_t)g_smem[(off)])
// Bounded wait of one warp for the 8 neighbouring tiles of (ty, tz).
static __device__ bool wait_tile_warp(const SweepParams &P, const RepDesc &D, int ty, int tz, uint32_t need, int lane)
{
    const uint32_t *fp = nullptr;
    if (lane < 9 && lane != 4) {
        int nty = ty + (lane % 3) - 1, ntz = tz + (lane / 3) - 1;
        nty = nty < 0 ? nty + D.NTy : (nty >= D.NTy ? nty - D.NTy : nty);
        ntz = ntz < 0 ? ntz + D.NTz : (ntz >= D.NTz ? ntz - D.NTz : ntz);
        fp = P.flags + D.tile0 + ntz * D.NTy + nty;
    }
    uint64_t t0 = 0;  // read at the first miss: most waits end at the first look
    unsigned nap = 32;
    for (;;) {
        const bool ok = (fp == nullptr) || ld_acquire_u32(fp) >= need;
        if (__all_sync(0xffffffffu, ok)) return true;
        if (t0 == 0) t0 = global_ns();
        int stop = 0;
        if (lane == 0) {
            if (ld_volatile_i32(P.abort_flag)) {
                stop = 1;
            } else if ((long long)(global_ns() - t0) > P.timeout_ns) {
                atomicCAS(P.status, 0, (int)SMC_ERR_TIMEOUT);
                atomicExch(P.abort_flag, 1);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        __nanosleep(nap);
        nap = nap < (unsigned)P.nap_cap ? nap * 2 : (unsigned)P.nap_cap;
    }
}

// Stores v at x (in [-1, nx]) of the halo-framed row whose body starts at
// byte offset `row`, and at the cell's halo copy when it is one of the first
// or last four cells (elsewhere the second store repeats the first).
__device__ __forceinline__ void halo_store(uint32_t row, int x, int nx, unsigned char v)
{
    const int xr = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    const int xm = xr < 4 ? xr + nx : (xr >= nx - 4 ? xr - nx : xr);
    g_smem[row + xr] = v;
    g_smem[row + xm] = v;
}

}  // namespace smc
