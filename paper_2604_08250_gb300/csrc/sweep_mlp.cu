// sweep_mlp.cu -- swap-MC sweep, lock-step trace and energies with the MLP
// site energy (MLPNet, Sec. IV-B; BF16 weights and activations on the tensor
// cores, FP32 accumulation and SiLU).
//
// Site energy e_i = f(x_i), x_i = [onehot(s_i) | counts of each species among
// the shell-1, shell-2 and shell-3 neighbours] (20 inputs), f = W3 silu(W2
// silu(W1 x + b1) + b2) + b3.  A trial (a <-> b) changes x_j exactly for the
// sites j of its local interaction zone Omega = {a, b} and their neighbours
// within three shells (40 sites on BCC), so (Algorithm 1, the reduction of the
// local energies over Omega before and after the swap)
//   dE = sum_{j in Omega} f(x'_j) - f(x_j).
// The post-swap energies f(x'_j) are evaluated on the tensor cores; the
// pre-swap energies come from a per-site cache E[i] = f(x_i) that the same
// tile routine fills (so both sides are bit-identical) and that accepted
// trials update over their whole Omega.
//
// Sweep organisation follows the pair kernel: link-cell columns staged in
// shared memory, 4 mini-steps per group, one warp per tile, neighbour progress
// flags with bounded waits.  A column here stages 61 rows (the 5x5
// trial-sublattice and 6x6 partner-sublattice rows of its 3-shell reach).
// Within a mini-step the warp handles its trials in batches of 4: swap in
// shared memory, build the 160 post-swap feature rows, run the MLP on them,
// compare with the cached energies, keep or undo each swap.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "mlp_common.cuh"
#include "sweep_common.cuh"

namespace smc {

constexpr int kOmega = 40;    // sites of a trial's interaction zone
constexpr int kMlpTB = 4;     // trials per batch
constexpr int kMlpRows = kMlpTB * kOmega;
constexpr int kMlpWinRows = 61;  // 25 trial-sublattice + 36 partner-sublattice rows
constexpr int kMlpMaxWarps = 8;

// Omega of a trial for each (trial sublattice, partner direction), relative
// to the trial site's byte in row (0, 0) of its column window: `same` is the
// site's own offset, `other` the offset of the same cell in the other
// sublattice's window (the anchor of its shell-1 neighbours); rel = 0 for the
// trial sublattice, 1 for the partner's; (dxo, dy, dz) its cell offset.
// Entry 0 is a, entry 1 is b.
struct OmegaEntry {
    int same, other;
    signed char rel, dy, dz, dxo;
};
struct MlpGeo {
    OmegaEntry om[2][8][kOmega];
    int pat1[2][2][8];    // shell-1 neighbour offsets from `other`, per (trial sublattice, rel)
    int pat23[2][2][18];  // shell-2 then shell-3 neighbour offsets from `same`
};

// Layout of the CTA-wide part of the MLP kernels' shared memory.
struct MlpSmem {
    static constexpr uint32_t D = 0;                    // pair table (kDEntries floats)
    static constexpr uint32_t W1 = D + kDEntries * 4;   // 64 rows x 80 B
    static constexpr uint32_t W2 = W1 + 64 * kW1RowB;   // 64 rows x 144 B
    static constexpr uint32_t B1 = W2 + 64 * kW2RowB;   // 64 floats each
    static constexpr uint32_t B2 = B1 + 256;
    static constexpr uint32_t W3 = B2 + 256;
    static constexpr uint32_t B3 = W3 + 256;
    static constexpr uint32_t GEO = B3 + 16;
    static constexpr uint32_t END = (uint32_t)((GEO + sizeof(MlpGeo) + 15) / 16 * 16);
};

// f for the 16 feature rows at shared offset `rows` (stride kARowB).  Lane
// (g = lane/4, t = lane%4) returns f of rows g and g+8 (the four lanes of a
// quad agree).  A row's arithmetic does not depend on the other rows of the
// tile or on its position in it, so a site's f is the same wherever it is
// evaluated.
__device__ __forceinline__ void mlp_tile16(uint32_t rows, int lane, float &f_lo, float &f_hi)
{
    const int g = lane >> 2, t = lane & 3;
    const float *b1 = (const float *)(g_smem + MlpSmem::B1);
    const float *b2 = (const float *)(g_smem + MlpSmem::B2);
    const float *w3 = (const float *)(g_smem + MlpSmem::W3);
    const float b3 = *(const float *)(g_smem + MlpSmem::B3);
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
        const uint32_t ar = rows + kc * 32 + 4 * t;
        const uint32_t a0 = lds32(ar + g * kARowB), a1 = lds32(ar + (g + 8) * kARowB);
        const uint32_t a2 = lds32(ar + g * kARowB + 16), a3 = lds32(ar + (g + 8) * kARowB + 16);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t br = MlpSmem::W1 + (8 * j + g) * kW1RowB + kc * 32 + 4 * t;
            mma_bf16(acc[j], a0, a1, a2, a3, lds32(br), lds32(br + 16));
        }
    }
    // hidden layer 1: bias, SiLU, BF16 -> the A fragments of layer 2 (the
    // m16n8k16 accumulator of n-block j holds columns 8j + 2t, 8j + 2t + 1
    // of rows g, g+8, which is the A-fragment layout of k-chunk j/2)
    uint32_t ha[4][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        const float h0 = silu(acc[j][0] + b1[c]), h1 = silu(acc[j][1] + b1[c + 1]);
        const float h2 = silu(acc[j][2] + b1[c]), h3 = silu(acc[j][3] + b1[c + 1]);
        ha[j >> 1][(j & 1) * 2 + 0] = pack_bf16(h0, h1);
        ha[j >> 1][(j & 1) * 2 + 1] = pack_bf16(h2, h3);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t br = MlpSmem::W2 + (8 * j + g) * kW2RowB + kc * 32 + 4 * t;
            mma_bf16(acc[j], ha[kc][0], ha[kc][1], ha[kc][2], ha[kc][3], lds32(br), lds32(br + 16));
        }
    }
    // hidden layer 2 and the output layer (FP32)
    float s_lo = 0.f, s_hi = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = 8 * j + 2 * t;
        s_lo = fmaf(w3[c], silu(acc[j][0] + b2[c]), s_lo);
        s_lo = fmaf(w3[c + 1], silu(acc[j][1] + b2[c + 1]), s_lo);
        s_hi = fmaf(w3[c], silu(acc[j][2] + b2[c]), s_hi);
        s_hi = fmaf(w3[c + 1], silu(acc[j][3] + b2[c + 1]), s_hi);
    }
    s_lo += __shfl_xor_sync(0xffffffffu, s_lo, 1);
    s_lo += __shfl_xor_sync(0xffffffffu, s_lo, 2);
    s_hi += __shfl_xor_sync(0xffffffffu, s_hi, 1);
    s_hi += __shfl_xor_sync(0xffffffffu, s_hi, 2);
    f_lo = s_lo + b3;
    f_hi = s_hi + b3;
}

// Copies the MLP weights (and the pair table and Omega geometry when given)
// into the CTA's shared memory in the layout mlp_tile16 reads.
__device__ void load_mlp_smem(const MlpBlock *W, const float *Dsrc, const MlpGeo *geo)
{
    const int tid = threadIdx.x, n = blockDim.x;
    for (int i = tid; i < 64 * 16; i += n) {
        const int r = i >> 4, c = i & 15;
        *(uint32_t *)(g_smem + MlpSmem::W1 + r * kW1RowB + 4 * c) = ((const uint32_t *)W->w1)[r * 16 + c];
    }
    for (int i = tid; i < 64 * 32; i += n) {
        const int r = i >> 5, c = i & 31;
        *(uint32_t *)(g_smem + MlpSmem::W2 + r * kW2RowB + 4 * c) = ((const uint32_t *)W->w2)[r * 32 + c];
    }
    for (int i = tid; i < 64; i += n) {
        ((float *)(g_smem + MlpSmem::B1))[i] = W->b1[i];
        ((float *)(g_smem + MlpSmem::B2))[i] = W->b2[i];
        ((float *)(g_smem + MlpSmem::W3))[i] = W->w3[i];
    }
    if (tid == 0) *(float *)(g_smem + MlpSmem::B3) = W->b3;
    if (Dsrc)
        for (int i = tid; i < kDEntries; i += n) ((float *)(g_smem + MlpSmem::D))[i] = Dsrc[i];
    if (geo)
        for (int i = tid; i < (int)(sizeof(MlpGeo) / 4); i += n)
            ((int *)(g_smem + MlpSmem::GEO))[i] = ((const int *)geo)[i];
}

// ---------------------------------------------------------------------------
// Per-site energies of the whole lattice: e[i] = f(x_i), optionally stored
// (the sweep's cache), and their sum per CTA in a fixed order.  One warp per
// 16 consecutive sites.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_mlp_site_energy(const MlpBlock *W, const int8_t *__restrict__ occ, int nx,
                                                         int ny, int nz, float *ecache, double *part)
{
    load_mlp_smem(W, nullptr, nullptr);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const uint32_t tile = MlpSmem::END + warp * 16 * kARowB;
    const long long N = 2LL * nx * ny * nz;
    const long long ntile = (N + 15) / 16;
    auto spec = [&](int sb, int xx, int yy, int zz) { return occ_at(occ, nx, ny, nz, sb, xx, yy, zz); };
    double wsum = 0.0;
    for (long long tl = (long long)blockIdx.x * nwarp + warp; tl < ntile; tl += (long long)gridDim.x * nwarp) {
        if (lane < 16) {
            const long long s = tl * 16 + lane;
            int q0 = 0;
            uint32_t h1 = 0, h2 = 0, h3 = 0;
            if (s < N) {
                long long r = s;
                const int x = (int)(r % nx);
                r /= nx;
                const int y = (int)(r % ny);
                r /= ny;
                const int z = (int)(r % nz);
                const int sub = (int)(r / nz);
                q0 = occ[s] & 7;
                site_hist(spec, sub, x, y, z, h1, h2, h3);
            }
            write_feature_row(tile + lane * kARowB, q0, h1, h2, h3);
        }
        __syncwarp();
        float f_lo, f_hi;
        mlp_tile16(tile, lane, f_lo, f_hi);
        const int g = lane >> 2;
        const long long s_lo = tl * 16 + g, s_hi = tl * 16 + g + 8;
        if ((lane & 3) == 0 && ecache) {
            if (s_lo < N) ecache[s_lo] = f_lo;
            if (s_hi < N) ecache[s_hi] = f_hi;
        }
        // the 16 values in site order, summed by every lane alike
        const float v_lo = (s_lo < N) ? f_lo : 0.f, v_hi = (s_hi < N) ? f_hi : 0.f;
        double tsum = 0.0;
        for (int gg = 0; gg < 8; ++gg) tsum += (double)__shfl_sync(0xffffffffu, v_lo, 4 * gg);
        for (int gg = 0; gg < 8; ++gg) tsum += (double)__shfl_sync(0xffffffffu, v_hi, 4 * gg);
        wsum += tsum;
        __syncwarp();
    }
    __shared__ double wpart[32];
    if (lane == 0) wpart[warp] = wsum;
    __syncthreads();
    if (threadIdx.x == 0 && part) {
        double s = 0.0;
        for (int w = 0; w < nwarp; ++w) s += wpart[w];
        part[blockIdx.x] = s;
    }
}

// out (+)= sum of part[0 .. n-1], in index order.
__global__ void k_sum_parts(const double *part, int n, double *out, int accumulate)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    if (accumulate)
        *out += s;
    else
        *out = s;
}

// Pair part of dE (pair + MLP models) from the post-swap feature rows of a
// (row ra: species B now) and b (row rb: species A now).  Their shell counts
// include the swapped partner, which is subtracted from shell 1.
__device__ __forceinline__ float pair_part(const SweepParams &P, const float *Dt, uint32_t ra, uint32_t rbv, int A,
                                           int B)
{
    const __nv_bfloat16 *xa = (const __nv_bfloat16 *)(g_smem + ra);
    const __nv_bfloat16 *xb = (const __nv_bfloat16 *)(g_smem + rbv);
    float dp = 0.f;
    for (int m = 0; m < P.nshells; ++m) {
        const float *D = Dt + ((m * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
        for (int q = 0; q < P.S; ++q) {
            float ca = __bfloat162float(xa[5 + 5 * m + q]);
            float cb = __bfloat162float(xb[5 + 5 * m + q]);
            if (m == 0) {
                ca -= (q == A) ? 1.f : 0.f;
                cb -= (q == B) ? 1.f : 0.f;
            }
            dp = fmaf(ca - cb, D[q], dp);
        }
    }
    return dp;
}

// ---------------------------------------------------------------------------
// The sweep.
// ---------------------------------------------------------------------------
struct MlpWarp {  // per-warp shared memory (offsets from the warp's base)
    uint32_t win, A, fnew, eold, site, words, tinfo, end;
};

__host__ __device__ __forceinline__ MlpWarp mlp_warp_layout(int rb, int nk, int tpc)
{
    MlpWarp L;
    L.win = (uint32_t)(16 * tpc + 15) / 16 * 16;  // accumulator slots first
    L.A = L.win + (uint32_t)((kMlpWinRows * rb + 16 + 15) / 16 * 16);
    L.fnew = L.A + kMlpRows * kARowB;
    L.eold = L.fnew + kMlpRows * 4;
    L.site = L.eold + kMlpRows * 4;
    L.words = L.site + kMlpRows * 4;
    L.tinfo = L.words + (uint32_t)nk * 512;
    L.end = L.tinfo + kMlpTB * 32;
    return L;
}

template <bool HAS_PAIR, int SOFF>
__device__ __forceinline__ void mlp_column(const SweepParams &P, const RepDesc &RD, uint32_t wb, const MlpWarp &L,
                                           int y0, int z0, uint64_t sweep, float beta, int lane, double &accEd,
                                           long long &accN)
{
    constexpr int sub = SOFF == -1 ? 0 : 1;
    constexpr int lo = SOFF - 2;  // first partner-sublattice row (dy, dz) of the window
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NLx = RD.NLx;
    const uint32_t rb = (uint32_t)P.rowB;
    const uint32_t col0 = wb + L.win + 16;  // row 0's body (4-byte halos on both sides)
    const MlpGeo &geo = *(const MlpGeo *)(g_smem + MlpSmem::GEO);
    // ---- stage the 61 rows ----
    {
        const bool vec = RD.vec != 0;
        const int cpr = vec ? (nx >> 4) : (nx >> 2);
        const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(g_smem);
        for (int rr = 0; rr < kMlpWinRows; ++rr) {
            int gsub, dy, dz;
            if (rr < 25) {
                dy = rr % 5 - 2;
                dz = rr / 5 - 2;
                gsub = sub;
            } else {
                dy = (rr - 25) % 6 + lo;
                dz = (rr - 25) / 6 + lo;
                gsub = 1 - sub;
            }
            const int gy = wrapc(y0 + dy, ny), gz = wrapc(z0 + dz, nz);
            const int8_t *src = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx;
            const uint32_t dst = col0 + (uint32_t)rr * rb;
            if (vec) {
                for (int c = lane; c < cpr; c += 32)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem0 + dst + 16 * c),
                                 "l"(src + 16 * c)
                                 : "memory");
            } else {
                for (int c = lane; c < cpr; c += 32)
                    *(unsigned *)(g_smem + dst + 4 * c) = __ldcg((const unsigned *)src + c);
            }
        }
        if (vec) asm volatile("cp.async.wait_all;" ::: "memory");
        __syncwarp();
        for (int rr = lane; rr < kMlpWinRows; rr += 32) {
            unsigned char *row = g_smem + col0 + rr * rb;
            for (int c = 0; c < nx; c += 4) *(unsigned *)(row + c) &= 0x07070707u;
            *(unsigned *)(row - 4) = *(const unsigned *)(row + nx - 4);
            *(unsigned *)(row + nx) = *(const unsigned *)row;
        }
        __syncwarp();
    }
    // ---- Philox words of the column's trial sites: [k][word][lane] ----
    uint32_t *wsm = (uint32_t *)(g_smem + wb + L.words);
    const int nk = (NLx + 31) >> 5;
    const uint32_t rowsite = (uint32_t)(((sub * nz + z0) * ny + y0) * nx);
    for (int k = 0; k < nk; ++k) {
        const int i = lane + 32 * k;
        if (i < NLx) {
            const U4 w = philox10(U4{(rowsite >> 2) + (uint32_t)i, RD.rep, (uint32_t)sweep, (uint32_t)(sweep >> 32)},
                                  (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
            wsm[(k * 4 + 0) * 32 + lane] = w.x;
            wsm[(k * 4 + 1) * 32 + lane] = w.y;
            wsm[(k * 4 + 2) * 32 + lane] = w.z;
            wsm[(k * 4 + 3) * 32 + lane] = w.w;
        }
    }
    __syncwarp();
    int *tinfo = (int *)(g_smem + wb + L.tinfo);  // per trial: dir, r, A, B, b row, b x, x, accepted
    float *fnew = (float *)(g_smem + wb + L.fnew);
    float *eold = (float *)(g_smem + wb + L.eold);
    int *sites = (int *)(g_smem + wb + L.site);
    const uint32_t A_tile = wb + L.A;
    const float *Dt = (const float *)(g_smem + MlpSmem::D);
    const uint32_t arow = col0 + 12 * rb;
    for (int dx = 0; dx < 4; ++dx) {
        for (int i0 = 0; i0 < NLx; i0 += kMlpTB) {
            const int nb = min(kMlpTB, NLx - i0);
            // -- decode the trials and swap in shared memory --
            if (lane < nb) {
                const int i = i0 + lane, x = 4 * i + dx;
                const uint32_t w = wsm[((i >> 5) * 4 + dx) * 32 + (i & 31)];
                const int dir = (int)(w >> kRBits);
                const int kx = (dir >> 2) & 1, ky = (dir >> 1) & 1, kz = dir & 1;
                const uint32_t brow = col0 + (uint32_t)(25 + (kz + 2) * 6 + (ky + 2)) * rb;
                const int xb = x + SOFF + kx;
                const int A = g_smem[arow + x], B = g_smem[brow + xb];
                halo_store(arow, x, nx, (unsigned char)B);
                halo_store(brow, xb, nx, (unsigned char)A);
                int *ti = tinfo + lane * 8;
                ti[0] = dir;
                ti[1] = (int)(w & kRMask);
                ti[2] = A;
                ti[3] = B;
                ti[4] = (int)brow;
                ti[5] = xb;
                ti[6] = x;
            }
            __syncwarp();
            // -- post-swap feature rows; cached pre-swap energies --
            const int nrow = nb * kOmega;
            float eo[5];
#pragma unroll
            for (int it = 0; it < 5; ++it) {
                const int q = lane + 32 * it;
                eo[it] = 0.f;
                if (q < nrow) {
                    const int t = q / kOmega, e = q - t * kOmega;
                    const OmegaEntry oe = geo.om[sub][tinfo[t * 8]][e];
                    const int ssub = oe.rel ? 1 - sub : sub;
                    const int x = tinfo[t * 8 + 6];
                    const int gx = wrapc(x + oe.dxo, nx), gy = wrapc(y0 + oe.dy, ny), gz = wrapc(z0 + oe.dz, nz);
                    const int site = ((ssub * nz + gz) * ny + gy) * nx + gx;
                    sites[q] = site;
                    eo[it] = __ldcg(P.ecache + site);
                }
            }
#pragma unroll
            for (int it = 0; it < 5; ++it) {
                const int q = lane + 32 * it;
                if (q < nrow) {
                    const int t = q / kOmega, e = q - t * kOmega;
                    const OmegaEntry oe = geo.om[sub][tinfo[t * 8]][e];
                    const int x = tinfo[t * 8 + 6];
                    const uint32_t bs = col0 + (uint32_t)(oe.same + x), bo = col0 + (uint32_t)(oe.other + x);
                    const int *p1 = geo.pat1[sub][oe.rel];
                    const int *p23 = geo.pat23[sub][oe.rel];
                    uint32_t h1 = 0, h2 = 0, h3 = 0;
#pragma unroll
                    for (int k = 0; k < 8; ++k) h1 += 1u << (4 * g_smem[bo + p1[k]]);
#pragma unroll
                    for (int k = 0; k < 6; ++k) h2 += 1u << (4 * g_smem[bs + p23[k]]);
#pragma unroll
                    for (int k = 6; k < 18; ++k) h3 += 1u << (4 * g_smem[bs + p23[k]]);
                    write_feature_row(A_tile + q * kARowB, g_smem[bs], h1, h2, h3);
                    eold[q] = eo[it];
                }
            }
            __syncwarp();
            // -- the MLP on the rows, 16 at a time --
            const int ntl = (nrow + 15) / 16;
            for (int m = 0; m < ntl; ++m) {
                float f_lo, f_hi;
                mlp_tile16(A_tile + m * 16 * kARowB, lane, f_lo, f_hi);
                if ((lane & 3) == 0) {
                    fnew[m * 16 + (lane >> 2)] = f_lo;
                    fnew[m * 16 + (lane >> 2) + 8] = f_hi;
                }
            }
            __syncwarp();
            // -- decisions; rejected swaps are undone --
            if (lane < nb) {
                int *ti = tinfo + lane * 8;
                float dE = 0.f;
                for (int e = 0; e < kOmega; ++e) dE += fnew[lane * kOmega + e] - eold[lane * kOmega + e];
                const int A = ti[2], B = ti[3];
                if (HAS_PAIR && A != B)
                    dE += pair_part(P, Dt, A_tile + (lane * kOmega) * kARowB, A_tile + (lane * kOmega + 1) * kARowB,
                                    A, B);
                const bool acc = metropolis<false>(dE, (uint32_t)ti[1], beta, nullptr, make_int2(0, 0));
                ti[7] = acc ? 1 : 0;
                if (!acc) {
                    halo_store(arow, ti[6], nx, (unsigned char)A);
                    halo_store((uint32_t)ti[4], ti[5], nx, (unsigned char)B);
                } else {
                    accEd += (double)dE;
                    accN += 1;
                }
            }
            __syncwarp();
            // -- cached energies over the accepted trials' Omega --
            for (int q = lane; q < nrow; q += 32)
                if (tinfo[(q / kOmega) * 8 + 7]) P.ecache[sites[q]] = fnew[q];
            __syncwarp();
        }
    }
    // ---- write back the trial row (0, 0) and the partner rows (SOFF..SOFF+1)^2 ----
    {
        const bool vec = RD.vec != 0;
        const int cpr = vec ? (nx >> 4) : (nx >> 2);
        for (int wr = 0; wr < 5; ++wr) {
            int rr, gsub, gy, gz;
            if (wr == 0) {
                rr = 12;
                gsub = sub;
                gy = y0;
                gz = z0;
            } else {
                const int ddy = SOFF + ((wr - 1) & 1), ddz = SOFF + ((wr - 1) >> 1);
                rr = 25 + (ddz - lo) * 6 + (ddy - lo);
                gsub = 1 - sub;
                gy = wrapc(y0 + ddy, ny);
                gz = wrapc(z0 + ddz, nz);
            }
            int8_t *dstg = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx;
            const unsigned char *srcs = g_smem + col0 + (uint32_t)rr * rb;
            if (vec) {
                for (int c = lane; c < cpr; c += 32) *((int4 *)dstg + c) = *((const int4 *)srcs + c);
            } else {
                for (int c = lane; c < cpr; c += 32) *((unsigned *)dstg + c) = *((const unsigned *)srcs + c);
            }
        }
    }
    __syncwarp();
}

template <bool HAS_PAIR>
__global__ void __launch_bounds__(32 * kMlpMaxWarps, 1) k_sweep_mlp(const __grid_constant__ SweepParams P,
                                                                    const __grid_constant__ MlpGeo G)
{
    load_mlp_smem(P.mlpw, HAS_PAIR ? P.D.df : nullptr, &G);
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int gw = blockIdx.x * nwarp + warp, NW = gridDim.x * nwarp;
    const RepDesc &RD = P.rep[0];
    const int nk = (RD.NLx + 31) >> 5;
    const MlpWarp L = mlp_warp_layout(P.rowB, nk, P.tpc);
    const uint32_t wb = MlpSmem::END + (uint32_t)warp * P.warp_bytes;
    double *slot_e = (double *)(g_smem + wb);
    long long *slot_n = (long long *)(g_smem + wb + 8 * P.tpc);
    for (int i = lane; i < P.tpc; i += 32) {
        slot_e[i] = 0.0;
        slot_n[i] = 0;
    }
    __syncwarp();
    bool aborted = false;
    for (int t = 0; t < P.nsweeps && !aborted; ++t) {
        const uint64_t sweep = P.sweep0 + (uint64_t)t;
        const float beta = P.temp.beta[P.beta_stride ? t : 0];
        for (int g = 0; g < P.G && !aborted; ++g) {
            const uint32_t gstep = (uint32_t)(t * P.G + g);
            const int dy = g & 3, dz = (g >> 2) & 3, sub = g >> 4;
            int slotk = 0;
            for (int tile = gw; tile < P.ntiles; tile += NW, ++slotk) {
                const int ty = tile % RD.NTy, tz = tile / RD.NTy;
                // every earlier group of the 8 neighbouring tiles must be done
                if (!wait_tile_warp(P, RD, ty, tz, gstep, lane)) {
                    aborted = true;
                    break;
                }
                double accEd = 0.0;
                long long accN = 0;
                const int j0 = ty * P.TY, j1 = min(j0 + P.TY, RD.NLy);
                const int l0 = tz * P.TZ, l1 = min(l0 + P.TZ, RD.NLz);
                for (int l = l0; l < l1; ++l)
                    for (int j = j0; j < j1; ++j) {
                        if (sub == 0)
                            mlp_column<HAS_PAIR, -1>(P, RD, wb, L, 4 * j + dy, 4 * l + dz, sweep, beta, lane, accEd,
                                                     accN);
                        else
                            mlp_column<HAS_PAIR, 0>(P, RD, wb, L, 4 * j + dy, 4 * l + dz, sweep, beta, lane, accEd,
                                                    accN);
                    }
                const double e_w = warp_sum<double>(accEd);
                const long long n_w = warp_sum<long long>(accN);
                if (lane == 0) {
                    slot_e[slotk] += e_w;
                    slot_n[slotk] += n_w;
                }
                __syncwarp();
                if (lane == 0 && tile != P.skip_tile) st_release_u32(P.flags + tile, gstep + 1);
            }
        }
    }
    if (aborted) return;
    // per-tile partial sums, then the last warp to finish adds them in tile order
    if (lane == 0) {
        int k = 0;
        for (int tile = gw; tile < P.ntiles; tile += NW, ++k) {
            P.part_e[tile] = slot_e[k];
            P.part_n[tile] = slot_n[k];
        }
    }
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicAdd(P.ticket, 1u) == (unsigned)NW - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last || lane != 0) return;
    __threadfence();
    double se = 0.0;
    long long sn = 0;
    for (int k = 0; k < P.ntiles; ++k) {
        se += __ldcg(P.part_e + k);
        sn += __ldcg(P.part_n + k);
    }
    if (RD.e_acc) *RD.e_acc += se;
    if (RD.n_acc) *RD.n_acc += sn;
}

// ---------------------------------------------------------------------------
// Lock-step trace of one mini-step: one warp per batch of 4 trials, features
// read from global memory, pre-swap energies recomputed rather than cached;
// same tile routine and summation order as the sweep.  Phase 2 (the pair
// kernel's k_ministep_apply) applies the accepted swaps.
// ---------------------------------------------------------------------------
constexpr uint32_t kTraceWarpBytes = 2 * kMlpRows * kARowB + 2 * kMlpRows * 4 + kMlpTB * 32;

template <bool HAS_PAIR>
__global__ void __launch_bounds__(128) k_mlp_trace_eval(const __grid_constant__ SweepParams P,
                                                        const __grid_constant__ MlpGeo G, int k, float *dE_out,
                                                        uint8_t *acc_out, int *swap_a, int *swap_b)
{
    load_mlp_smem(P.mlpw, HAS_PAIR ? P.D.df : nullptr, &G);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const RepDesc &RD = P.rep[0];
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz;
    const int ntr = RD.NLx * RD.NLy * RD.NLz;
    const int dx = k % 4, dy = (k / 4) % 4, dz = (k / 16) % 4, sub = k / 64;
    const int soff = sub == 0 ? -1 : 0;
    const uint32_t wb = MlpSmem::END + warp * kTraceWarpBytes;
    const uint32_t Apost = wb, Apre = wb + kMlpRows * kARowB;
    float *fpost = (float *)(g_smem + wb + 2 * kMlpRows * kARowB);
    float *fpre = fpost + kMlpRows;
    int *tinfo = (int *)(fpre + kMlpRows);  // per trial: a, b, r, A, B, x, y, z
    const float *Dt = (const float *)(g_smem + MlpSmem::D);
    const MlpGeo &geo = *(const MlpGeo *)(g_smem + MlpSmem::GEO);
    const int8_t *occ = RD.occ;
    for (int c0 = (blockIdx.x * nwarp + warp) * kMlpTB; c0 < ntr; c0 += gridDim.x * nwarp * kMlpTB) {
        const int nb = min(kMlpTB, ntr - c0);
        int mydir = 0;
        if (lane < nb) {
            const int c = c0 + lane;
            const int cx = c % RD.NLx, cy = (c / RD.NLx) % RD.NLy, cz = c / (RD.NLx * RD.NLy);
            const int x = 4 * cx + dx, y = 4 * cy + dy, z = 4 * cz + dz;
            const uint32_t s = (uint32_t)(((sub * nz + z) * ny + y) * nx + x);
            const uint32_t w = site_word(P.seed, RD.rep, P.sweep0, s);
            mydir = (int)(w >> kRBits);
            const int kx = (mydir >> 2) & 1, ky = (mydir >> 1) & 1, kz = mydir & 1;
            const int bx = wrapc(x + soff + kx, nx), by = wrapc(y + soff + ky, ny), bz = wrapc(z + soff + kz, nz);
            int *ti = tinfo + lane * 8;
            ti[0] = (int)s;
            ti[1] = (((1 - sub) * nz + bz) * ny + by) * nx + bx;
            ti[2] = (int)(w & kRMask);
            ti[3] = occ[s] & 7;
            ti[4] = occ[ti[1]] & 7;
            ti[5] = x;
            ti[6] = y;
            ti[7] = z;
        }
        int dirs[kMlpTB];
#pragma unroll
        for (int t = 0; t < kMlpTB; ++t) dirs[t] = __shfl_sync(0xffffffffu, mydir, t);
        __syncwarp();
        for (int q = lane; q < 2 * nb * kOmega; q += 32) {
            const bool post = q < nb * kOmega;
            const int qq = post ? q : q - nb * kOmega;
            const int t = qq / kOmega, e = qq - t * kOmega;
            const int *ti = tinfo + t * 8;
            const int a = ti[0], b = ti[1], A = ti[3], B = ti[4];
            int dir = dirs[0];
#pragma unroll
            for (int u = 1; u < kMlpTB; ++u)
                if (t == u) dir = dirs[u];
            const OmegaEntry oe = geo.om[sub][dir][e];
            const int ssub = oe.rel ? 1 - sub : sub;
            const int gx = wrapc(ti[5] + oe.dxo, nx), gy = wrapc(ti[6] + oe.dy, ny), gz = wrapc(ti[7] + oe.dz, nz);
            auto spec = [&](int sb, int xx, int yy, int zz) -> int {
                const int id = ((sb * nz + wrapc(zz, nz)) * ny + wrapc(yy, ny)) * nx + wrapc(xx, nx);
                const int v = occ[id] & 7;
                return post ? (id == a ? B : (id == b ? A : v)) : v;
            };
            uint32_t h1, h2, h3;
            site_hist(spec, ssub, gx, gy, gz, h1, h2, h3);
            write_feature_row((post ? Apost : Apre) + qq * kARowB, spec(ssub, gx, gy, gz), h1, h2, h3);
        }
        __syncwarp();
        const int ntl = (nb * kOmega + 15) / 16;
        for (int m = 0; m < 2 * ntl; ++m) {
            const bool post = m < ntl;
            const int mm = post ? m : m - ntl;
            float f_lo, f_hi;
            mlp_tile16((post ? Apost : Apre) + mm * 16 * kARowB, lane, f_lo, f_hi);
            if ((lane & 3) == 0) {
                float *dst = post ? fpost : fpre;
                dst[mm * 16 + (lane >> 2)] = f_lo;
                dst[mm * 16 + (lane >> 2) + 8] = f_hi;
            }
        }
        __syncwarp();
        if (lane < nb) {
            const int c = c0 + lane;
            const int *ti = tinfo + lane * 8;
            float dE = 0.f;
            for (int e = 0; e < kOmega; ++e) dE += fpost[lane * kOmega + e] - fpre[lane * kOmega + e];
            const int A = ti[3], B = ti[4];
            if (HAS_PAIR && A != B)
                dE += pair_part(P, Dt, Apost + (lane * kOmega) * kARowB, Apost + (lane * kOmega + 1) * kARowB, A, B);
            const bool acc = metropolis<false>(dE, (uint32_t)ti[2], P.temp.beta[0], nullptr, make_int2(0, 0));
            if (dE_out) dE_out[c] = dE;
            if (acc_out) acc_out[c] = acc ? 1 : 0;
            swap_a[c] = (acc && A != B) ? ti[0] : -1;
            swap_b[c] = ti[1];
        }
        __syncwarp();
    }
}

__global__ void k_mlp_trace_apply(int8_t *occ, int ntr, const int *swap_a, const int *swap_b)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ntr) return;
    const int a = swap_a[c];
    if (a < 0) return;
    const int b = swap_b[c];
    const int8_t t = occ[a];
    occ[a] = occ[b];
    occ[b] = t;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
static float bf16_bits_to_float(uint16_t b)
{
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// The kernels' weight block: W1 padded to 32 inputs, W3 widened to FP32.
void make_mlp_block(const smc_model *m, MlpBlock &W)
{
    memset(&W, 0, sizeof W);
    for (int j = 0; j < 64; ++j)
        for (int i = 0; i < 20; ++i) W.w1[j * 32 + i] = m->mlp_w1[j * 20 + i];
    for (int i = 0; i < 64 * 64; ++i) W.w2[i] = m->mlp_w2[i];
    for (int i = 0; i < 64; ++i) {
        W.b1[i] = m->mlp_b1[i];
        W.b2[i] = m->mlp_b2[i];
        W.w3[i] = bf16_bits_to_float(m->mlp_w3[i]);
    }
    W.b3 = m->mlp_b3;
}

namespace {

// Window row (0 .. 60) of cell offset (dy, dz) in window w (0: trial
// sublattice, rows -2..2; 1: partner sublattice, rows lo..lo+5), or -1.
int win_row(int w, int lo, int dy, int dz)
{
    if (w == 0) return (dy < -2 || dy > 2 || dz < -2 || dz > 2) ? -1 : (dz + 2) * 5 + (dy + 2);
    return (dy < lo || dy > lo + 5 || dz < lo || dz > lo + 5) ? -1 : 25 + (dz - lo) * 6 + (dy - lo);
}

struct Cell {
    int w, x, y, z;  // window (sublattice relative to the trial's) and cell offset
};

// The 26 neighbours (8 shell-1, 6 shell-2, 12 shell-3) of a site of
// sublattice s at window w, cell c, in that order.
void neighbours(int s, const Cell &c, Cell out[26])
{
    int n = 0;
    const int o = s == 0 ? -1 : 0;
    for (int u = 0; u < 8; ++u)
        out[n++] = Cell{1 - c.w, c.x + o + ((u >> 2) & 1), c.y + o + ((u >> 1) & 1), c.z + o + (u & 1)};
    const int s2[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (auto &v : s2) out[n++] = Cell{c.w, c.x + v[0], c.y + v[1], c.z + v[2]};
    for (int p = -1; p <= 1; p += 2)
        for (int r = -1; r <= 1; r += 2) {
            out[n++] = Cell{c.w, c.x + p, c.y + r, c.z};
            out[n++] = Cell{c.w, c.x + p, c.y, c.z + r};
            out[n++] = Cell{c.w, c.x, c.y + p, c.z + r};
        }
}

// Builds Omega and the neighbour patterns for row stride rb; fails if a site
// or a neighbour falls outside the staged window (a geometry error).
bool build_mlp_geo(int rb, MlpGeo &G)
{
    memset(&G, 0, sizeof G);
    for (int ts = 0; ts < 2; ++ts) {
        const int soff = ts == 0 ? -1 : 0, lo = soff - 2;
        const int width[2] = {5, 6};
        for (int w = 0; w < 2; ++w) {
            const int s = w == 0 ? ts : 1 - ts;
            const int o = s == 0 ? -1 : 0;
            for (int u = 0; u < 8; ++u) {
                const int ex = o + ((u >> 2) & 1), ey = o + ((u >> 1) & 1), ez = o + (u & 1);
                G.pat1[ts][w][u] = (ez * width[1 - w] + ey) * rb + ex;
            }
            Cell nb[26];
            neighbours(s, Cell{w, 0, 0, 0}, nb);
            for (int k = 0; k < 18; ++k) {
                const Cell &c = nb[8 + k];
                G.pat23[ts][w][k] = (c.z * width[w] + c.y) * rb + c.x;
            }
        }
        for (int dir = 0; dir < 8; ++dir) {
            std::vector<Cell> om;
            auto add = [&](const Cell &c) {
                for (auto &e : om)
                    if (e.w == c.w && e.x == c.x && e.y == c.y && e.z == c.z) return;
                om.push_back(c);
            };
            const Cell a{0, 0, 0, 0};
            const Cell b{1, soff + ((dir >> 2) & 1), soff + ((dir >> 1) & 1), soff + (dir & 1)};
            add(a);
            add(b);
            for (const Cell &c : {a, b}) {
                Cell nb[26];
                neighbours(c.w == 0 ? ts : 1 - ts, c, nb);
                for (auto &n : nb) add(n);
            }
            if ((int)om.size() != kOmega) return false;
            for (int e = 0; e < kOmega; ++e) {
                const Cell &c = om[e];
                const int r_same = win_row(c.w, lo, c.y, c.z), r_other = (1 - c.w) == 0
                                                                          ? (c.z + 2) * 5 + (c.y + 2)
                                                                          : 25 + (c.z - lo) * 6 + (c.y - lo);
                if (r_same < 0 || c.x < -3 || c.x > 3) return false;
                OmegaEntry &oe = G.om[ts][dir][e];
                oe.same = r_same * rb + c.x;
                oe.other = r_other * rb + c.x;
                oe.rel = (signed char)c.w;
                oe.dxo = (signed char)c.x;
                oe.dy = (signed char)c.y;
                oe.dz = (signed char)c.z;
                // every neighbour read must land on its own row of the window
                Cell nb[26];
                neighbours(c.w == 0 ? ts : 1 - ts, c, nb);
                for (int k = 0; k < 26; ++k) {
                    const int r = win_row(nb[k].w, lo, nb[k].y, nb[k].z);
                    if (r < 0 || nb[k].x < -4 || nb[k].x > 4) return false;
                    const int off = k < 8 ? oe.other + G.pat1[ts][c.w][k] : oe.same + G.pat23[ts][c.w][k - 8];
                    if (off != r * rb + nb[k].x) return false;
                }
            }
        }
    }
    return true;
}

bool mlp_shape_ok(const smc_lattice *lat, const int8_t *occ)
{
    return lc_edge(lat->nx) == 4 && lc_edge(lat->ny) == 4 && lc_edge(lat->nz) == 4 && lat->nx <= 1024 &&
           ((uintptr_t)occ % 4 == 0);
}

int mlp_rowB(int nx) { return ((nx + 15) & ~15) + 16; }

void fill_pair_D(const smc_model *m, int S, SweepParams &P)
{
    for (int mm = 0; mm < m->nshells; ++mm)
        for (int A = 0; A < S; ++A)
            for (int B = 0; B < S; ++B)
                for (int q = 0; q < S; ++q)
                    P.D.df[((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies + q] =
                        (float)((double)m->v_f32[(mm * S + B) * S + q] - (double)m->v_f32[(mm * S + A) * S + q]);
}

size_t round16(size_t v) { return (v + 15) / 16 * 16; }

}  // namespace

// E (+)= sum_i f(x_i); writes the per-site energies to ecache when non-NULL.
// W is a device MlpBlock; part needs room for the grid's CTA count (<= 8 per SM).
static smc_status mlp_energy_launch(Workspace *ws, const smc_lattice *lat, const MlpBlock *W, const int8_t *occ,
                                    float *ecache, double *part, double *e, int accumulate, cudaStream_t stream)
{
    const int threads = 128;
    const size_t smem = MlpSmem::END + (size_t)(threads / 32) * 16 * kARowB;
    cudaError_t err = cudaFuncSetAttribute(k_mlp_site_energy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(k_mlp_site_energy)");
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_site_energy, threads, smem);
    if (err != cudaSuccess) return cuda_fail(err, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    per_sm = std::max(1, std::min(per_sm, 8));
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const long long tiles = (N + 15) / 16;
    const int grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * ws->num_sms, (tiles + 3) / 4));
    k_mlp_site_energy<<<grid, threads, smem, stream>>>(W, occ, lat->nx, lat->ny, lat->nz, ecache, part);
    err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "k_mlp_site_energy");
    if (e) {
        k_sum_parts<<<1, 32, 0, stream>>>(part, grid, e, accumulate);
        err = cudaGetLastError();
        if (err != cudaSuccess) return cuda_fail(err, "k_sum_parts");
    }
    return SMC_OK;
}

smc_status launch_mlp_energy(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e,
                             cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    // scratch: [pair counts | MlpBlock | CTA partial sums]
    const size_t off_w = round16(sizeof(unsigned long long) * kMaxShells * 64);
    const size_t off_part = round16(off_w + sizeof(MlpBlock));
    const size_t need = off_part + sizeof(double) * 8 * (size_t)std::max(ws->num_sms, 1);
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, need, &st);
    if (!scr) return st;
    static MlpBlock W;
    make_mlp_block(m, W);
    cudaError_t err = cudaMemcpyAsync(scr + off_w, &W, sizeof W, cudaMemcpyHostToDevice, stream);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemcpyAsync(MLP weights)");
    int accumulate = 0;
    if (m->kind == SMC_PAIR_F32_MLP_BF16) {
        unsigned long long *cnt = (unsigned long long *)scr;
        st = launch_pair_counts(lat, m->nshells, occ, cnt, stream);
        if (st != SMC_OK) return st;
        st = launch_energy_finish(lat, m, cnt, e, nullptr, stream);
        if (st != SMC_OK) return st;
        accumulate = 1;
    }
    return mlp_energy_launch(ws, lat, (const MlpBlock *)(scr + off_w), occ, nullptr, (double *)(scr + off_part), e,
                             accumulate, stream);
}

namespace {
struct MlpPlan {
    int threads = 0, grid = 0, tpc = 0, ntiles = 0, warp_bytes = 0;
    size_t smem = 0;
};

smc_status make_mlp_plan(Workspace *ws, const smc_lattice *lat, const void *kernel, MlpPlan &pl)
{
    const Tuning tu = current_tuning();
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    const int rb = mlp_rowB(lat->nx), nk = (lat->nx / 4 + 31) / 32;
    pl.ntiles = (lat->ny / 4) * (lat->nz / 4);
    int best = 0;
    for (int nw_cta = kMlpMaxWarps; nw_cta >= 1; --nw_cta) {
        if (tu.threads && tu.threads != 32 * nw_cta) continue;
        for (int tpc_guess = 1; tpc_guess <= 4096; tpc_guess *= 2) {
            const size_t wbytes = round16(mlp_warp_layout(rb, nk, tpc_guess).end);
            const size_t smem = MlpSmem::END + (size_t)nw_cta * wbytes;
            if (smem > dyn_max) break;
            int per_sm = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * nw_cta, smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            if (tu.ctas_per_sm > 0) per_sm = std::min(per_sm, tu.ctas_per_sm);
            if (per_sm < 1) break;
            const long long res = (long long)per_sm * ws->num_sms * nw_cta;
            long long nw = 0;
            for (long long c = std::min<long long>(res, pl.ntiles) / nw_cta * nw_cta; c >= nw_cta; c -= nw_cta)
                if (pl.ntiles % c == 0) {
                    nw = c;
                    break;
                }
            const long long fill = std::min<long long>(res, pl.ntiles) / nw_cta * nw_cta;
            if (nw * 2 < fill) nw = fill;
            if (nw < nw_cta) nw = nw_cta;
            const int tpc = (int)((pl.ntiles + nw - 1) / nw);
            if (tpc <= tpc_guess) {
                if (nw > best) {
                    best = (int)nw;
                    pl.threads = 32 * nw_cta;
                    pl.grid = (int)(nw / nw_cta);
                    pl.tpc = tpc_guess;
                    pl.smem = smem;
                    pl.warp_bytes = (int)wbytes;
                }
                break;
            }
        }
    }
    if (!best) {
        set_error("MLP sweep kernel does not fit on an SM (rows of %d bytes)", rb);
        return SMC_ERR_UNSUPPORTED;
    }
    return SMC_OK;
}
}  // namespace

smc_status launch_mlp_sweep(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                            int64_t *n_acc, cudaStream_t stream)
{
    if (!mlp_shape_ok(lat, occ)) {
        set_error("MLP sweeps need every axis a multiple of 4 cells and >= 8, nx <= 1024 and 4-byte aligned occ");
        return SMC_ERR_UNSUPPORTED;
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const bool has_pair = m->kind == SMC_PAIR_F32_MLP_BF16;
    const void *kernel = has_pair ? (const void *)k_sweep_mlp<true> : (const void *)k_sweep_mlp<false>;
    MlpPlan pl;
    st = make_mlp_plan(ws, lat, kernel, pl);
    if (st != SMC_OK) return st;
    const int rb = mlp_rowB(lat->nx);
    static MlpGeo G;
    if (!build_mlp_geo(rb, G)) {
        set_error("internal error: MLP interaction-zone geometry");
        return SMC_ERR_STATE;
    }
    static SweepParams P;
    memset(&P, 0, sizeof P);
    P.R = 1;
    P.G = 32;
    P.Lx = P.Ly = P.Lz = 4;
    P.TY = P.TZ = P.CB = 1;
    P.nshells = has_pair ? m->nshells : 0;
    P.S = lat->nspecies;
    P.tpc = pl.tpc;
    P.warp_bytes = pl.warp_bytes;
    P.nap_cap = 1024;
    P.rowB = rb;
    P.kind = m->kind;
    for (int g = 0; g < kMaxGroups; ++g) P.lag[g] = 1;
    P.skip_tile = (int)debug_skip_tile();
    P.seed = seed;
    P.timeout_ns = debug_timeout_ns();
    P.ntiles = pl.ntiles;
    RepDesc &d = P.rep[0];
    d.occ = occ;
    d.e_acc = e_acc;
    d.n_acc = (long long *)n_acc;
    d.nx = lat->nx;
    d.ny = lat->ny;
    d.nz = lat->nz;
    d.NLx = d.nx / 4;
    d.NLy = d.ny / 4;
    d.NLz = d.nz / 4;
    d.NTy = d.NLy;
    d.NTz = d.NLz;
    d.tile0 = 0;
    d.rep = replica;
    d.vec = (d.nx % 16 == 0) && ((uintptr_t)occ % 16 == 0);
    if (has_pair) fill_pair_D(m, P.S, P);

    // workspace: [flags | part_e | part_n | ticket, abort | MlpBlock | energy parts | E cache]
    const size_t nt = (size_t)P.ntiles;
    const size_t N = 2ull * lat->nx * lat->ny * lat->nz;
    const size_t off_pe = round16(nt * 4), off_pn = off_pe + nt * 8, off_misc = off_pn + nt * 8;
    const size_t off_w = round16(off_misc + 16);
    const size_t off_parts = round16(off_w + sizeof(MlpBlock));
    const size_t off_cache = round16(off_parts + sizeof(double) * 8 * (size_t)std::max(ws->num_sms, 1));
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_cache + N * 4, &st);
    if (!scr) return st;
    P.flags = (uint32_t *)scr;
    P.part_e = (double *)(scr + off_pe);
    P.part_n = (long long *)(scr + off_pn);
    P.ticket = (unsigned *)(scr + off_misc);
    P.abort_flag = (int *)(scr + off_misc + 4);
    P.status = ws->status;
    P.mlpw = (const MlpBlock *)(scr + off_w);
    P.ecache = (float *)(scr + off_cache);
    static MlpBlock W;
    make_mlp_block(m, W);
    cudaError_t e = cudaMemcpyAsync(scr + off_w, &W, sizeof W, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(MLP weights)");
    st = mlp_energy_launch(ws, lat, P.mlpw, occ, P.ecache, (double *)(scr + off_parts), nullptr, 0, stream);
    if (st != SMC_OK) return st;

    bool constant = true;
    for (int t = 1; t < nsweeps; ++t)
        if (kT[t] != kT[0]) constant = false;
    const int chunk = constant ? nsweeps : kMaxBeta;
    for (int t0 = 0; t0 < nsweeps; t0 += chunk) {
        const int nc = std::min(chunk, nsweeps - t0);
        P.sweep0 = sweep0 + (uint64_t)t0;
        P.nsweeps = nc;
        P.beta_stride = constant ? 0 : 1;
        for (int t = 0; t < (constant ? 1 : nc); ++t) P.temp.beta[t] = (float)(1.0 / kT[t0 + t]);
        e = cudaMemsetAsync(scr, 0, off_misc + 16, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sweep scratch)");
        void *args[] = {(void *)&P, (void *)&G};
        e = cudaLaunchCooperativeKernel(kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(MLP sweep)");
    }
    return SMC_OK;
}

smc_status launch_mlp_trace(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep, int k, double kT, float *dE, uint8_t *acc,
                            cudaStream_t stream)
{
    if (lc_edge(lat->nx) != 4 || lc_edge(lat->ny) != 4 || lc_edge(lat->nz) != 4) {
        set_error("MLP traces need every axis a multiple of 4 cells and >= 8");
        return SMC_ERR_UNSUPPORTED;
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const bool has_pair = m->kind == SMC_PAIR_F32_MLP_BF16;
    static MlpGeo G;
    if (!build_mlp_geo(mlp_rowB(lat->nx), G)) {
        set_error("internal error: MLP interaction-zone geometry");
        return SMC_ERR_STATE;
    }
    static SweepParams P;
    memset(&P, 0, sizeof P);
    P.R = 1;
    P.Lx = P.Ly = P.Lz = 4;
    P.nshells = has_pair ? m->nshells : 0;
    P.S = lat->nspecies;
    P.seed = seed;
    P.sweep0 = sweep;
    P.kind = m->kind;
    P.temp.beta[0] = (float)(1.0 / kT);
    RepDesc &d = P.rep[0];
    d.occ = occ;
    d.nx = lat->nx;
    d.ny = lat->ny;
    d.nz = lat->nz;
    d.NLx = d.nx / 4;
    d.NLy = d.ny / 4;
    d.NLz = d.nz / 4;
    d.rep = replica;
    if (has_pair) fill_pair_D(m, P.S, P);
    const int ntr = d.NLx * d.NLy * d.NLz;
    const size_t off_w = round16((size_t)ntr * 8);
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_w + sizeof(MlpBlock), &st);
    if (!scr) return st;
    int *swap_a = (int *)scr, *swap_b = swap_a + ntr;
    P.mlpw = (const MlpBlock *)(scr + off_w);
    static MlpBlock W;
    make_mlp_block(m, W);
    cudaError_t e = cudaMemcpyAsync(scr + off_w, &W, sizeof W, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(MLP weights)");
    const int threads = 128;
    const size_t smem = MlpSmem::END + (size_t)(threads / 32) * kTraceWarpBytes;
    auto kern = has_pair ? k_mlp_trace_eval<true> : k_mlp_trace_eval<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_trace_eval)");
    const int per_block = (threads / 32) * kMlpTB;
    const int blocks = (ntr + per_block - 1) / per_block;
    kern<<<blocks, threads, smem, stream>>>(P, G, k, dE, acc, swap_a, swap_b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_trace_eval");
    k_mlp_trace_apply<<<(ntr + 127) / 128, 128, 0, stream>>>(occ, ntr, swap_a, swap_b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_trace_apply");
    return SMC_OK;
}

}  // namespace smc
