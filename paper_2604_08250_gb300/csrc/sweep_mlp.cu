// sweep_mlp.cu -- swap-MC sweep, lock-step trace and energies with the MLP
// site energy (MLPNet, Sec. IV-B), evaluated on the tcgen05 tensor cores.
//
// Site energy e_i = f(x_i), x_i = [onehot(s_i) | counts of each species among
// the shell-1, shell-2 and shell-3 neighbours] (20 inputs), f = W3 silu(W2
// silu(W1 x + b1) + b2) + b3.  A trial (a <-> b) changes x_j exactly for the
// sites j of its local interaction zone Omega = {a, b} and their neighbours
// within three shells (40 sites on BCC), so (Algorithm 1, the reduction of the
// local energies over Omega before and after the swap)
//   dE = sum_{j in Omega} f(x'_j) - f(x_j).
// The sweep keeps two per-site caches, filled at the start of a call by the
// energy kernel: the energies E[i] = f(x_i) and the features F[i] = {s_i,
// packed shell counts}.  A trial reads F[j] and E[j] of its 40 zone sites;
// x'_j = x_j with species A of a moved to B and B of b moved to A in the
// shells where j sees them (a table from the geometry), so the post-swap rows
// need no neighbour gathers.  The rows are evaluated on the tensor cores
// (mlp_tc.cuh) and compared with E[j]; an accepted trial stores x'_j, f(x'_j)
// and the two swapped species.  Energies of rows come from one evaluator
// everywhere, so cached and fresh values are bit-identical.
//
// Scheduling as in the pair kernel: link-cell columns, 4 mini-steps per
// group, neighbour progress flags with bounded waits; one CTA of 4
// warpgroups per tile evaluates up to 64 trials of a mini-step at a time in
// 128-row tiles alternating between warpgroups.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "mlp_common.cuh"
#include "mlp_tc.cuh"
#include "mlpnet_tc.cuh"
#include "sweep_common.cuh"

namespace smc {

constexpr int kOmega = 40;       // sites of a trial's interaction zone
constexpr int kMlpChunk = 64;    // most trials of a mini-step evaluated together (40 rows each)
constexpr int kTraceTB = 3;      // trials per trace step (120 rows: one tile)
constexpr int kTcMaxCtasPerSm = 512 / (2 * kTcCols);  // for the 2-warpgroup kernels
constexpr int kTinfo = 16;       // ints of per-trial information

// Omega of a trial for each (trial sublattice, partner direction): rel = 0
// for a site of the trial sublattice, 1 for the partner's; (dxo, dy, dz) its
// cell offset from the trial site's cell.  Entry 0 is a, entry 1 is b.
struct OmegaEntry {
    signed char rel, dy, dz, dxo;
    signed char ma, mb;  // shell (1-3) in which the site sees a / b, 0 if none
    signed char pad[2];
};
struct MlpGeo {
    OmegaEntry om[2][8][kOmega];
};

// Shared memory of the MLP kernels: weights, the warpgroups' tiles, then
// kernel-specific parts from END on.
template <int NWG>
struct MlpSmem {
    static constexpr uint32_t W1 = 0;
    static constexpr uint32_t W2 = W1 + kTcW1;
    static constexpr uint32_t X = W2 + kTcW2;        // [NWG] tiles
    static constexpr uint32_t H = X + NWG * kTcX;    // [NWG] tiles
    static constexpr uint32_t B1 = H + NWG * kTcH;
    static constexpr uint32_t B2 = B1 + 256;
    static constexpr uint32_t W3 = B2 + 256;
    static constexpr uint32_t B3 = W3 + 256;
    static constexpr uint32_t MBAR = B3 + 16;        // [NWG][2]
    static constexpr uint32_t TSLOT = MBAR + 16 * NWG;
    static constexpr uint32_t CTL = TSLOT + 4;       // CTA-wide flag
    static constexpr uint32_t RED = (CTL + 4 + 15) / 16 * 16;  // 4 doubles / long longs for reductions
    static constexpr uint32_t TINFO = RED + 64;      // int [kMlpChunk][kTinfo]
    static constexpr uint32_t ACT = TINFO + kMlpChunk * kTinfo * 4;  // int [kMlpChunk]: trials with A != B
    static constexpr uint32_t D = ACT + kMlpChunk * 4;  // pair table (kDEntries floats)
    static constexpr uint32_t GEO = D + kDEntries * 4;
    static constexpr uint32_t END = (uint32_t)((GEO + sizeof(MlpGeo) + 127) / 128 * 128);
    static_assert(X % 128 == 0 && H % 128 == 0 && W2 % 128 == 0, "tile alignment");
    static_assert(MBAR % 8 == 0 && RED % 8 == 0, "alignment");
};
constexpr int kSweepWG = 4;  // warpgroups of the sweep kernel (64-wide network)
constexpr int kEvalWG = 2;   // warpgroups of the energy and trace kernels

// Shared memory of the MLPNet kernels (96-wide, three ReLU layers): the same
// kernel-specific parts as MlpSmem from CTL on, without the pair table.
template <int NWG>
struct NetSmem {
    static constexpr uint32_t W0 = 0;
    static constexpr uint32_t W1 = W0 + kNetW0;
    static constexpr uint32_t W2 = W1 + kNetW12;
    static constexpr uint32_t X = W2 + kNetW12;      // [NWG] tiles
    static constexpr uint32_t H = X + NWG * kNetX;   // [NWG] tiles
    static constexpr uint32_t W3 = H + NWG * kNetHt;
    static constexpr uint32_t B3 = W3 + kNetHid * 4;
    static constexpr uint32_t MBAR = B3 + 16;        // [NWG][2]
    static constexpr uint32_t TSLOT = MBAR + 16 * NWG;
    static constexpr uint32_t CTL = TSLOT + 4;
    static constexpr uint32_t RED = (CTL + 4 + 15) / 16 * 16;
    static constexpr uint32_t TINFO = RED + 64;
    static constexpr uint32_t ACT = TINFO + kMlpChunk * kTinfo * 4;
    static constexpr uint32_t GEO = ACT + kMlpChunk * 4;
    static constexpr uint32_t END = (uint32_t)((GEO + sizeof(MlpGeo) + 127) / 128 * 128);
    static_assert(X % 128 == 0 && H % 128 == 0 && W1 % 128 == 0 && W2 % 128 == 0, "tile alignment");
    static_assert(MBAR % 8 == 0 && RED % 8 == 0, "alignment");
};

// The two site-energy networks the MLP kernels run: evaluator, layouts and
// warpgroups of the sweep.
struct NetSilu64 {  // MLP of mlp_tc.cuh: 20 -> 64 -> 64 -> 1, SiLU
    using Eval = TcEval;
    using Block = MlpBlock;
    template <int NWG>
    using Smem = MlpSmem<NWG>;
    static constexpr int kSweepNWG = kSweepWG;
    template <int NWG>
    static __device__ TcLayout layout(uint32_t wg)
    {
        using M = MlpSmem<NWG>;
        return TcLayout{M::X + wg * kTcX, M::H + wg * kTcH, M::W1, M::W2, M::B1, M::B2, M::W3, M::B3,
                        M::MBAR + 16 * wg, M::TSLOT};
    }
};
struct NetRelu96 {  // MLPNet of mlpnet_tc.cuh: 20 -> 96 -> 96 -> 96 -> 1, ReLU
    using Eval = NetEval;
    using Block = NetBlock;
    template <int NWG>
    using Smem = NetSmem<NWG>;
    static constexpr int kSweepNWG = 2;  // the 28 KB hidden tiles of four would not fit
    template <int NWG>
    static __device__ NetLayout layout(uint32_t wg)
    {
        using M = NetSmem<NWG>;
        return NetLayout{M::X + wg * kNetX, M::H + wg * kNetHt, M::W0, M::W1, M::W2, M::W3, M::B3, M::MBAR + 16 * wg,
                         M::TSLOT};
    }
};

// Site-energy models of the tensor-core sweep.
constexpr int kModeMlp = 0, kModeMlpPair = 1;

// The evaluator of this thread's warpgroup.
template <class Net, int NWG>
__device__ __forceinline__ typename Net::Eval mlp_evaluator(long long timeout_ns, int *status, int *abort_flag)
{
    const uint32_t wg = threadIdx.x >> 7;
    typename Net::Eval E;
    E.L = Net::template layout<NWG>(wg);
    E.timeout_ns = timeout_ns;
    E.status = status;
    E.abort_flag = abort_flag;
    E.tmem = 0;
    E.phase1 = E.phase2 = 0;
    E.bar = 1 + wg;
    return E;
}

// Pair part of dE (pair + MLP models) from the packed post-swap neighbour
// histograms of a (species B now) and b (species A now), 3 shells each; the
// swapped partner is removed from shell 1.
template <int NWG>
__device__ __forceinline__ float pair_part(const SweepParams &P, const int *ha, const int *hb, int A, int B)
{
    const float *Dt = (const float *)(g_smem + MlpSmem<NWG>::D);
    float dp = 0.f;
    for (int m = 0; m < P.nshells; ++m) {
        const float *D = Dt + ((m * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
        for (int q = 0; q < P.S; ++q) {
            float ca = (float)(((uint32_t)ha[m] >> (4 * q)) & 15u);
            float cb = (float)(((uint32_t)hb[m] >> (4 * q)) & 15u);
            if (m == 0) {
                ca -= (q == A) ? 1.f : 0.f;
                cb -= (q == B) ? 1.f : 0.f;
            }
            dp = fmaf(ca - cb, D[q], dp);
        }
    }
    return dp;
}

// Copies the model (weights, pair table, geometry) and sets up the evaluators.
template <class Net, int NWG>
__device__ void mlp_cta_setup(typename Net::Eval &E, const void *W, const float *Dsrc, const MlpGeo *geo)
{
    using M = typename Net::template Smem<NWG>;
    tc_load_weights((const typename Net::Block *)W, E.L);
    const int tid = threadIdx.x, n = blockDim.x;
    if constexpr (std::is_same<Net, NetSilu64>::value) {
        if (Dsrc)
            for (int i = tid; i < kDEntries; i += n) ((float *)(g_smem + M::D))[i] = Dsrc[i];
    }
    if (geo)
        for (int i = tid; i < (int)(sizeof(MlpGeo) / 4); i += n) ((int *)(g_smem + M::GEO))[i] = ((const int *)geo)[i];
    tc_setup(E, NWG);
}

// ---------------------------------------------------------------------------
// Per-site energies of the whole lattice: e[i] = f(x_i), optionally stored
// (the sweep's cache), and their sum per CTA in a fixed order.  Each
// warpgroup takes 128 consecutive sites per tile.
// ---------------------------------------------------------------------------
template <class Net>
__global__ void __launch_bounds__(128 * kEvalWG) k_mlp_site_energy(const void *W, const int8_t *__restrict__ occ,
                                                                   int nx, int ny, int nz, float *ecache,
                                                                   uint4 *fcache, double *part, long long timeout_ns,
                                                                   int *status, int *abort_flag)
{
    constexpr int NWG = kEvalWG;
    using M = typename Net::template Smem<NWG>;
    typename Net::Eval E = mlp_evaluator<Net, NWG>(timeout_ns, status, abort_flag);
    mlp_cta_setup<Net, NWG>(E, W, nullptr, nullptr);
    const int tid = threadIdx.x, r = tid & 127, wg = tid >> 7;
    const long long N = 2LL * nx * ny * nz;
    const long long ntile = (N + kTcRows - 1) / kTcRows;
    auto spec = [&](int sb, int xx, int yy, int zz) { return occ_at(occ, nx, ny, nz, sb, xx, yy, zz); };
    double sum = 0.0;
    // one tile's features into the X tile (zeros past the end)
    auto build = [&](long long tl) {
        const long long s = tl * kTcRows + r;
        int q0 = -1;
        uint32_t h1 = 0, h2 = 0, h3 = 0;
        if (s < N) {
            long long t = s;
            const int x = (int)(t % nx);
            t /= nx;
            const int y = (int)(t % ny);
            t /= ny;
            const int z = (int)(t % nz);
            const int sub = (int)(t / nz);
            q0 = occ[s] & 7;
            site_hist(spec, sub, x, y, z, h1, h2, h3);
            if (fcache) fcache[s] = make_uint4((uint32_t)q0, h1, h2, h3);
        }
        tc_write_features(E.L, r, q0, h1, h2, h3);
        fence_async_smem();
    };
    const long long step = (long long)NWG * gridDim.x;
    long long tl = (long long)NWG * blockIdx.x + wg;
    if (tl < ntile) {
        build(tl);
        tc_issue1(E);
    }
    while (tl < ntile) {
        tc_stage2(E);
        const long long nx_tl = tl + step;
        if (nx_tl < ntile) {  // the next tile's gathers and layer-1 products overlap this tile's layer 2
            build(nx_tl);
            tc_issue1(E);
        }
        const float f = tc_finish(E);
        const long long s = tl * kTcRows + r;
        if (s < N) {
            if (ecache) ecache[s] = f;
            sum += (double)f;
        }
        tl = nx_tl;
    }
    // CTA sum in thread order (the X tiles are free once both warpgroups are done)
    double *red = (double *)(g_smem + M::X);
    tc_fence_before();
    __syncthreads();
    red[tid] = sum;
    __syncthreads();
    if (tid == 0 && part) {
        double t = 0.0;
        for (int i = 0; i < 128 * NWG; ++i) t += red[i];
        part[blockIdx.x] = t;
    }
    tc_teardown(E, NWG);
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

// ---------------------------------------------------------------------------
// The sweep.
// ---------------------------------------------------------------------------
struct SweepLayout {  // offsets after MlpSmem<kSweepWG>::END
    uint32_t words, fval, diff, site, feat, slots, end;
};

__host__ __device__ __forceinline__ SweepLayout mlp_sweep_layout(int NLx, int tpc, int chunk,
                                                                 uint32_t base = MlpSmem<kSweepWG>::END)
{
    SweepLayout L;
    const uint32_t rows = (uint32_t)kOmega * (uint32_t)(NLx < chunk ? NLx : chunk);
    L.words = base;
    L.fval = L.words + (uint32_t)((NLx * 16 + 15) / 16 * 16);
    L.diff = L.fval + rows * 4;
    L.site = L.diff + rows * 4;
    L.feat = (L.site + rows * 4 + 15) / 16 * 16;
    L.slots = L.feat + rows * 16;
    L.end = L.slots + (uint32_t)(16 * tpc);
    return L;
}

__device__ __forceinline__ int warp_of(int tid) { return tid >> 5; }

// Rank of an evaluated trial among the evaluated trials of its warp (or -1).
__device__ __forceinline__ void tinfo_rank_store(int *tinfo, int tid, bool active, unsigned mask)
{
    if (active) tinfo[tid * kTinfo + 15] = __popc(mask & ((1u << (tid & 31)) - 1u));
    else if (tid < kMlpChunk) tinfo[tid * kTinfo + 15] = -1;
}

// The 4 mini-steps of one link-cell column (cells y0, z0 of the trial
// sublattice; trials at x = 4 i + dx).
template <class Net, int MODE, int SOFF>
__device__ __forceinline__ void mlp_column(const SweepParams &P, const RepDesc &RD, const SweepLayout &SL,
                                           typename Net::Eval &E, int y0, int z0, uint64_t sweep, float beta,
                                           double &accEd, long long &accN)
{
    constexpr bool HAS_PAIR = MODE == kModeMlpPair;
    constexpr int sub = SOFF == -1 ? 0 : 1;
    constexpr int NWG = Net::kSweepNWG, kThreads = 128 * NWG;
    const int tid = threadIdx.x, r = tid & 127, wg = tid >> 7;
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NLx = RD.NLx;
    using M = typename Net::template Smem<NWG>;
    const MlpGeo &geo = *(const MlpGeo *)(g_smem + M::GEO);
    int8_t *occ = RD.occ;
    // ---- Philox words of the column's trial sites: [link cell][word] ----
    uint32_t *wsm = (uint32_t *)(g_smem + SL.words);
    const int rowsite = ((sub * nz + z0) * ny + y0) * nx;
    for (int i = tid; i < NLx; i += kThreads) {
        const U4 w = philox10(U4{((uint32_t)rowsite >> 2) + (uint32_t)i, RD.rep, (uint32_t)sweep,
                                 (uint32_t)(sweep >> 32)},
                              (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
        *(uint4 *)(wsm + 4 * i) = make_uint4(w.x, w.y, w.z, w.w);
    }
    __syncthreads();
    // per trial: dir, r, A, B, a, b, x, accepted, post-swap histograms of a (8-10) and b (11-13), rank (15)
    int *tinfo = (int *)(g_smem + M::TINFO);
    int *act = (int *)(g_smem + M::ACT);
    const int *red_i = (const int *)(g_smem + M::RED);
    float *fval = (float *)(g_smem + SL.fval);
    float *diff = (float *)(g_smem + SL.diff);
    int *sites = (int *)(g_smem + SL.site);
    uint4 *feat = (uint4 *)(g_smem + SL.feat);
    for (int dx = 0; dx < 4; ++dx) {
        for (int i0 = 0; i0 < NLx; i0 += P.mlp_chunk) {
            const int T = min(P.mlp_chunk, NLx - i0);
            // -- decode the trials; a swap of two equal species changes nothing
            //    (dE = 0, accepted): it is counted but not evaluated --
            if (tid < T) {
                const int i = i0 + tid, x = 4 * i + dx;
                const uint32_t w = wsm[4 * i + dx];
                const int dir = (int)(w >> kRBits);
                const int kx = (dir >> 2) & 1, ky = (dir >> 1) & 1, kz = dir & 1;
                const int a = rowsite + x;
                const int b = (((1 - sub) * nz + wrapc(z0 + SOFF + kz, nz)) * ny + wrapc(y0 + SOFF + ky, ny)) * nx +
                              wrapc(x + SOFF + kx, nx);
                int *ti = tinfo + tid * kTinfo;
                ti[0] = dir;
                ti[1] = (int)(w & kRMask);
                ti[2] = __ldcg(occ + a) & 7;
                ti[3] = __ldcg(occ + b) & 7;
                ti[4] = a;
                ti[5] = b;
                ti[6] = x;
                ti[7] = 0;
            }
            if (warp_of(tid) < 2) {  // rank of each evaluated trial (warps 0 and 1 hold the T <= 64 trials)
                const bool active = tid < T && tinfo[tid * kTinfo + 2] != tinfo[tid * kTinfo + 3];
                const unsigned m = __ballot_sync(0xffffffffu, active);
                if ((tid & 31) == 0) ((int *)(g_smem + M::RED))[tid >> 5] = __popc(m);
                __syncwarp();
                tinfo_rank_store(tinfo, tid, active, m);
            }
            __syncthreads();
            const int nact = red_i[0] + (T > 32 ? red_i[1] : 0);
            if (tid < T && tinfo[tid * kTinfo + 15] >= 0)
                act[tinfo[tid * kTinfo + 15] + (tid >= 32 ? red_i[0] : 0)] = tid;
            __syncthreads();
            const int nrow_act = nact * kOmega;
            // -- post-swap rows from the cached features: 128 per tile, tiles
            //    alternating between the warpgroups; each warpgroup builds
            //    tile n+1 and runs its layer-1 products while tile n's layer 2
            //    is in flight --
            const int ntile = (nrow_act + kTcRows - 1) / kTcRows;
            auto build = [&](int n, float &eo, int &site) {
                const int row = n * kTcRows + r;
                eo = 0.f;
                site = 0;
                if (row < nrow_act) {
                    const int t = act[row / kOmega], e = row - (row / kOmega) * kOmega;
                    int *ti = tinfo + t * kTinfo;
                    const OmegaEntry oe = geo.om[sub][ti[0]][e];
                    const int ssub = oe.rel ? 1 - sub : sub;
                    const int gx = wrapc(ti[6] + oe.dxo, nx), gy = wrapc(y0 + oe.dy, ny), gz = wrapc(z0 + oe.dz, nz);
                    site = ((ssub * nz + gz) * ny + gy) * nx + gx;
                    const uint4 f = __ldcg(P.fcache + site);
                    eo = __ldcg(P.ecache + site);
                    const int A = ti[2], B = ti[3];
                    uint32_t q0 = f.x, h[3] = {f.y, f.z, f.w};
                    if (e == 0) q0 = (uint32_t)B;
                    if (e == 1) q0 = (uint32_t)A;
                    const uint32_t dAB = (1u << (4 * B)) - (1u << (4 * A));  // a: A -> B (mod 2^32)
#pragma unroll
                    for (int m = 0; m < 3; ++m) {
                        if (oe.ma == m + 1) h[m] += dAB;
                        if (oe.mb == m + 1) h[m] -= dAB;
                    }
                    tc_write_features(E.L, r, (int)q0, h[0], h[1], h[2]);
                    feat[row] = make_uint4(q0, h[0], h[1], h[2]);
                    if (e < 2) {
                        ti[8 + 3 * e] = (int)h[0];
                        ti[9 + 3 * e] = (int)h[1];
                        ti[10 + 3 * e] = (int)h[2];
                    }
                } else {
                    tc_write_features(E.L, r, -1, 0, 0, 0);
                }
                fence_async_smem();
            };
            int n = wg;
            float eo = 0.f;
            int site = 0;
            if (n < ntile) {
                build(n, eo, site);
                tc_issue1(E);
            }
            while (n < ntile) {
                tc_stage2(E);
                const int nn = n + NWG;
                float eo_n = 0.f;
                int site_n = 0;
                if (nn < ntile) {
                    build(nn, eo_n, site_n);
                    tc_issue1(E);
                }
                const float f = tc_finish(E);
                const int row = n * kTcRows + r;
                if (row < nrow_act) {
                    fval[row] = f;
                    diff[row] = f - eo;
                    sites[row] = site;
                }
                n = nn;
                eo = eo_n;
                site = site_n;
            }
            __syncthreads();
            // -- decisions; an accepted swap is written to the occupancy --
            if (tid < T) {
                int *ti = tinfo + tid * kTinfo;
                const int A = ti[2], B = ti[3];
                if (A == B) {
                    ti[7] = 1;  // dE = 0: accepted, nothing changes
                    accN += 1;
                } else {
                    const int base = (ti[15] + (tid >= 32 ? red_i[0] : 0)) * kOmega;
                    float dE = 0.f;
                    for (int e = 0; e < kOmega; ++e) dE += diff[base + e];
                    if (HAS_PAIR) dE += pair_part<NWG>(P, ti + 8, ti + 11, A, B);
                    const bool acc = metropolis<false>(dE, (uint32_t)ti[1], beta, nullptr, make_int2(0, 0));
                    ti[7] = acc ? 1 : 0;
                    if (acc) {
                        occ[ti[4]] = (int8_t)B;
                        occ[ti[5]] = (int8_t)A;
                        accEd += (double)dE;
                        accN += 1;
                    }
                }
            }
            __syncthreads();
            // -- caches over the accepted trials' Omega --
            for (int row = tid; row < nrow_act; row += kThreads)
                if (tinfo[act[row / kOmega] * kTinfo + 7]) {
                    P.fcache[sites[row]] = feat[row];
                    P.ecache[sites[row]] = fval[row];
                }
            __syncthreads();
        }
    }
}

template <class Net, int MODE>
__global__ void __launch_bounds__(128 * Net::kSweepNWG, 1) k_sweep_mlp(const __grid_constant__ SweepParams P,
                                                                       const __grid_constant__ MlpGeo G)
{
    constexpr int NWG = Net::kSweepNWG, kThreads = 128 * NWG;
    using M = typename Net::template Smem<NWG>;
    typename Net::Eval E = mlp_evaluator<Net, NWG>(P.timeout_ns, P.status, P.abort_flag);
    mlp_cta_setup<Net, NWG>(E, P.mlpw, MODE == kModeMlpPair ? P.D.df : nullptr, &G);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const RepDesc &RD = P.rep[0];
    const SweepLayout SL = mlp_sweep_layout(RD.NLx, P.tpc, P.mlp_chunk, M::END);
    double *slot_e = (double *)(g_smem + SL.slots);
    long long *slot_n = (long long *)(g_smem + SL.slots + 8 * P.tpc);
    double *red_e = (double *)(g_smem + M::RED);
    long long *red_n = (long long *)(g_smem + M::RED + 16);
    for (int i = tid; i < P.tpc; i += kThreads) {
        slot_e[i] = 0.0;
        slot_n[i] = 0;
    }
    volatile int *ctl = (volatile int *)(g_smem + M::CTL);
    __syncthreads();
    bool aborted = false;
    for (int t = 0; t < P.nsweeps && !aborted; ++t) {
        const uint64_t sweep = P.sweep0 + (uint64_t)t;
        const float beta = P.temp.beta[P.beta_stride ? t : 0];
        for (int g = 0; g < P.G && !aborted; ++g) {
            const uint32_t gstep = (uint32_t)(t * P.G + g);
            const int dy = g & 3, dz = (g >> 2) & 3, sub = g >> 4;
            int slotk = 0;
            for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++slotk) {
                const int ty = tile % RD.NTy, tz = tile / RD.NTy;
                // every earlier group of the 8 neighbouring tiles must be done
                if (warp == 0) {
                    const bool ok = wait_tile_warp(P, RD, ty, tz, gstep, lane);
                    if (lane == 0) *ctl = ok ? 0 : 1;
                }
                __syncthreads();
                if (*ctl) {
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
                            mlp_column<Net, MODE, -1>(P, RD, SL, E, 4 * j + dy, 4 * l + dz, sweep, beta, accEd, accN);
                        else
                            mlp_column<Net, MODE, 0>(P, RD, SL, E, 4 * j + dy, 4 * l + dz, sweep, beta, accEd, accN);
                    }
                // the deciding threads are 0 .. kMlpChunk-1 (warps 0 and 1)
                if (warp < 2) {
                    const double e_w = warp_sum<double>(accEd);
                    const long long n_w = warp_sum<long long>(accN);
                    if (lane == 0) {
                        red_e[warp] = e_w;
                        red_n[warp] = n_w;
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    slot_e[slotk] += red_e[0] + red_e[1];
                    slot_n[slotk] += red_n[0] + red_n[1];
                    if (tile != P.skip_tile) st_release_u32(P.flags + tile, gstep + 1);
                }
            }
        }
    }
    if (!aborted && tid == 0) {
        // per-tile partial sums; the last CTA to finish adds them in tile order
        int k = 0;
        for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++k) {
            P.part_e[tile] = slot_e[k];
            P.part_n[tile] = slot_n[k];
        }
        __threadfence();
        const bool last = atomicAdd(P.ticket, 1u) == gridDim.x - 1;
        if (last) {
            __threadfence();
            double se = 0.0;
            long long sn = 0;
            for (int k2 = 0; k2 < P.ntiles; ++k2) {
                se += __ldcg(P.part_e + k2);
                sn += __ldcg(P.part_n + k2);
            }
            if (RD.e_acc) *RD.e_acc += se;
            if (RD.n_acc) *RD.n_acc += sn;
        }
    }
    tc_teardown(E, NWG);
}

// ---------------------------------------------------------------------------
// Lock-step trace of one mini-step: a CTA per batch of 3 trials, features
// read from global memory, pre-swap energies recomputed rather than cached
// (warpgroup 0 evaluates the pre-swap rows, warpgroup 1 the post-swap rows);
// same evaluator and summation order as the sweep.  k_mlp_trace_apply
// applies the accepted swaps.
// ---------------------------------------------------------------------------
template <class Net, bool HAS_PAIR>
__global__ void __launch_bounds__(128 * kEvalWG) k_mlp_trace_eval(const __grid_constant__ SweepParams P,
                                                                const __grid_constant__ MlpGeo G, int k,
                                                                float *dE_out, uint8_t *acc_out, int *swap_a,
                                                                int *swap_b)
{
    using M = typename Net::template Smem<kEvalWG>;
    typename Net::Eval E = mlp_evaluator<Net, kEvalWG>(P.timeout_ns, P.status, P.abort_flag);
    mlp_cta_setup<Net, kEvalWG>(E, P.mlpw, HAS_PAIR ? P.D.df : nullptr, &G);
    const int tid = threadIdx.x, r = tid & 127, wg = tid >> 7;
    const bool post = wg == 1;
    const RepDesc &RD = P.rep[0];
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz;
    const int ntr = RD.NLx * RD.NLy * RD.NLz;
    const int dx = k % 4, dy = (k / 4) % 4, dz = (k / 16) % 4, sub = k / 64;
    const int soff = sub == 0 ? -1 : 0;
    // per trial: a, b, r, A, B, x, y, z, dir, post-swap histograms of a (9-11) and b (12-14)
    int *tinfo = (int *)(g_smem + M::TINFO);
    float *fpre = (float *)(g_smem + M::END);
    float *fpost = fpre + kTcRows;
    const MlpGeo &geo = *(const MlpGeo *)(g_smem + M::GEO);
    const int8_t *occ = RD.occ;
    for (int c0 = blockIdx.x * kTraceTB; c0 < ntr; c0 += gridDim.x * kTraceTB) {
        const int nb = min(kTraceTB, ntr - c0);
        if (tid < nb) {
            const int c = c0 + tid;
            const int cx = c % RD.NLx, cy = (c / RD.NLx) % RD.NLy, cz = c / (RD.NLx * RD.NLy);
            const int x = 4 * cx + dx, y = 4 * cy + dy, z = 4 * cz + dz;
            const uint32_t s = (uint32_t)(((sub * nz + z) * ny + y) * nx + x);
            const uint32_t w = site_word(P.seed, RD.rep, P.sweep0, s);
            const int dir = (int)(w >> kRBits);
            const int kx = (dir >> 2) & 1, ky = (dir >> 1) & 1, kz = dir & 1;
            const int bx = wrapc(x + soff + kx, nx), by = wrapc(y + soff + ky, ny), bz = wrapc(z + soff + kz, nz);
            int *ti = tinfo + tid * kTinfo;
            ti[0] = (int)s;
            ti[1] = (((1 - sub) * nz + bz) * ny + by) * nx + bx;
            ti[2] = (int)(w & kRMask);
            ti[3] = occ[s] & 7;
            ti[4] = occ[ti[1]] & 7;
            ti[5] = x;
            ti[6] = y;
            ti[7] = z;
            ti[8] = dir;
        }
        __syncthreads();
        if (r < nb * kOmega) {
            const int t = r / kOmega, e = r - t * kOmega;
            int *ti = tinfo + t * kTinfo;
            const int a = ti[0], b = ti[1], A = ti[3], B = ti[4];
            const OmegaEntry oe = geo.om[sub][ti[8]][e];
            const int ssub = oe.rel ? 1 - sub : sub;
            const int gx = wrapc(ti[5] + oe.dxo, nx), gy = wrapc(ti[6] + oe.dy, ny), gz = wrapc(ti[7] + oe.dz, nz);
            auto spec = [&](int sb, int xx, int yy, int zz) -> int {
                const int id = ((sb * nz + wrapc(zz, nz)) * ny + wrapc(yy, ny)) * nx + wrapc(xx, nx);
                const int v = occ[id] & 7;
                return post ? (id == a ? B : (id == b ? A : v)) : v;
            };
            uint32_t h1, h2, h3;
            site_hist(spec, ssub, gx, gy, gz, h1, h2, h3);
            tc_write_features(E.L, r, spec(ssub, gx, gy, gz), h1, h2, h3);
            if (post && e < 2) {
                ti[9 + 3 * e] = (int)h1;
                ti[10 + 3 * e] = (int)h2;
                ti[11 + 3 * e] = (int)h3;
            }
        } else {
            tc_write_features(E.L, r, -1, 0, 0, 0);
        }
        fence_async_smem();
        const float f = tc_eval(E);
        (post ? fpost : fpre)[r] = f;
        __syncthreads();
        if (tid < nb) {
            const int c = c0 + tid;
            const int *ti = tinfo + tid * kTinfo;
            float dE = 0.f;
            for (int e = 0; e < kOmega; ++e) dE += fpost[tid * kOmega + e] - fpre[tid * kOmega + e];
            const int A = ti[3], B = ti[4];
            if (HAS_PAIR && A != B) dE += pair_part<kEvalWG>(P, ti + 9, ti + 12, A, B);
            const bool acc = metropolis<false>(dE, (uint32_t)ti[2], P.temp.beta[0], nullptr, make_int2(0, 0));
            if (dE_out) dE_out[c] = dE;
            if (acc_out) acc_out[c] = acc ? 1 : 0;
            swap_a[c] = (acc && A != B) ? ti[0] : -1;
            swap_b[c] = ti[1];
        }
        __syncthreads();
    }
    tc_teardown(E, kEvalWG);
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
// qSRO per-site pass: per shell m and species p, Q_m^p = sum over sites of
// species p of c_m[p]^2 (the same-element counts squared), reduced across
// each warp and added with 64-bit atomics: exact integers whatever the launch
// shape.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_qsro_sites(const int8_t *__restrict__ occ, int nx, int ny, int nz, int nsh,
                                                    unsigned long long *quad)
{
    const long long N = 2LL * nx * ny * nz;
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w0 = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    auto spec = [&](int sb, int xx, int yy, int zz) { return occ_at(occ, nx, ny, nz, sb, xx, yy, zz); };
    unsigned long long acc[kMaxShells][kMaxSpecies];
#pragma unroll
    for (int m = 0; m < kMaxShells; ++m)
#pragma unroll
        for (int p = 0; p < kMaxSpecies; ++p) acc[m][p] = 0;
    for (long long base = w0 * 32; base < N; base += nwarps * 32) {
        const long long s = base + lane;
        int q0 = -1;
        uint32_t h[3] = {0, 0, 0};
        if (s < N) {
            long long t = s;
            const int x = (int)(t % nx);
            t /= nx;
            const int y = (int)(t % ny);
            t /= ny;
            const int z = (int)(t % nz);
            const int sub = (int)(t / nz);
            q0 = occ[s] & 7;
            site_hist(spec, sub, x, y, z, h[0], h[1], h[2]);
        }
        {
#pragma unroll
            for (int m = 0; m < kMaxShells; ++m) {
                const uint32_t c = q0 >= 0 ? (h[m] >> (4 * q0)) & 15u : 0u;
#pragma unroll
                for (int p = 0; p < kMaxSpecies; ++p) {
                    const uint32_t v = (m < nsh && q0 == p) ? c * c : 0u;
                    const uint32_t w = __reduce_add_sync(0xffffffffu, v);
                    if (lane == 0) acc[m][p] += w;
                }
            }
        }
    }
    if (lane == 0)
#pragma unroll
        for (int m = 0; m < kMaxShells; ++m)
#pragma unroll
            for (int p = 0; p < kMaxSpecies; ++p)
                if (acc[m][p]) atomicAdd(quad + m * kMaxSpecies + p, acc[m][p]);
}

// qSRO parameters in FP64 (exact widenings of the FP32 inputs).
struct QsroRaw {
    double v[kMaxShells][kMaxSpecies][kMaxSpecies];
    double w[kMaxShells][kMaxSpecies];
    double c;
    int nsh, S;
};

// E = sum_m sum_{p,q} V_m^{pq} n_m^{pq} / z_m + sum_{m,p} W_m^p Q_m^p / z_m^2 + N C
// from the ordered pair counts n_m^{pq} (sum over sites of species p of their
// shell-m species-q counts) and the Q_m^p; dE/dtheta in the layout
// [V_m^{pq}, p <= q][W_m^p][C] (one parameter per unordered pair).
__global__ void k_qsro_finish(QsroRaw Q, const unsigned long long *cnt, const unsigned long long *quad, long long N,
                              double *e, float *grad)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double z[3] = {8.0, 6.0, 12.0};
    const int S = Q.S;
    if (e) {
        double E = 0.0;
        for (int m = 0; m < Q.nsh; ++m)
            for (int p = 0; p < S; ++p)
                for (int q = 0; q < S; ++q) E += Q.v[m][p][q] * (double)cnt[(m * S + p) * S + q] / z[m];
        for (int m = 0; m < Q.nsh; ++m)
            for (int p = 0; p < S; ++p) E += Q.w[m][p] * (double)quad[m * kMaxSpecies + p] / (z[m] * z[m]);
        *e = E + (double)N * Q.c;
    }
    if (grad) {
        int i = 0;
        for (int m = 0; m < Q.nsh; ++m)
            for (int p = 0; p < S; ++p)
                for (int q = p; q < S; ++q) {
                    const double n = p == q ? (double)cnt[(m * S + p) * S + p]
                                            : (double)cnt[(m * S + p) * S + q] + (double)cnt[(m * S + q) * S + p];
                    grad[i++] = (float)(n / z[m]);
                }
        for (int m = 0; m < Q.nsh; ++m)
            for (int p = 0; p < S; ++p) grad[i++] = (float)((double)quad[m * kMaxSpecies + p] / (z[m] * z[m]));
        grad[i] = (float)N;
    }
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

struct Cell {
    int w, x, y, z;  // sublattice relative to the trial's (0 same, 1 other) and cell offset
};

// The 26 neighbours (8 shell-1, 6 shell-2, 12 shell-3) of a site of
// sublattice s at relative sublattice w, cell c.
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

// Shell (1-3) of the vector between two sites given by their sublattice and
// cell, from its squared length in half-cell units (3, 4, 8), else 0.
int shell_between(int sa, const Cell &a, int sb, const Cell &b)
{
    const int dx = 2 * (a.x - b.x) + (sa - sb), dy = 2 * (a.y - b.y) + (sa - sb), dz = 2 * (a.z - b.z) + (sa - sb);
    const int d2 = dx * dx + dy * dy + dz * dz;
    return d2 == 3 ? 1 : (d2 == 4 ? 2 : (d2 == 8 ? 3 : 0));
}

// Omega of every (trial sublattice, partner direction) with the shells in
// which each zone site sees a and b; fails on a geometry inconsistency.
bool build_mlp_geo(MlpGeo &G)
{
    memset(&G, 0, sizeof G);
    for (int ts = 0; ts < 2; ++ts) {
        const int soff = ts == 0 ? -1 : 0;
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
            if ((int)om.size() != kOmega || shell_between(ts, a, 1 - ts, b) != 1) return false;
            for (int e = 0; e < kOmega; ++e) {
                const Cell &c = om[e];
                const int sc = c.w == 0 ? ts : 1 - ts;
                OmegaEntry &oe = G.om[ts][dir][e];
                oe.rel = (signed char)c.w;
                oe.dxo = (signed char)c.x;
                oe.dy = (signed char)c.y;
                oe.dz = (signed char)c.z;
                oe.ma = (signed char)shell_between(sc, c, ts, a);
                oe.mb = (signed char)shell_between(sc, c, 1 - ts, b);
                if (c.x < -3 || c.x > 3 || c.y < -3 || c.y > 3 || c.z < -3 || c.z > 3) return false;
                if (e >= 2 && oe.ma == 0 && oe.mb == 0) return false;  // every zone site sees a or b
            }
        }
    }
    return true;
}

bool mlp_shape_ok(const smc_lattice *lat)
{
    return lc_edge(lat->nx) == 4 && lc_edge(lat->ny) == 4 && lc_edge(lat->nz) == 4;
}

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

bool is_mlpnet(const smc_model *m) { return m->kind == SMC_MLPNET_BF16; }

// The MLPNet kernels' weight block: W0 padded to 32 inputs, W3 widened to FP32.
void make_net_block(const smc_model *m, NetBlock &W)
{
    memset(&W, 0, sizeof W);
    for (int j = 0; j < kNetHid; ++j)
        for (int i = 0; i < 20; ++i) W.w0[j * 32 + i] = m->net_w0[j * 20 + i];
    for (int i = 0; i < kNetHid * kNetHid; ++i) {
        W.w1[i] = m->net_w1[i];
        W.w2[i] = m->net_w2[i];
    }
    for (int j = 0; j < kNetHid; ++j) {
        W.b0[j] = m->net_b0[j];
        W.b1[j] = m->net_b1[j];
        W.b2[j] = m->net_b2[j];
        W.w3[j] = bf16_bits_to_float(m->net_w3[j]);
    }
    W.b3 = m->net_b3;
}

// Copies the model's weight block (MlpBlock or NetBlock) to dst (device).
smc_status copy_weights(const smc_model *m, void *dst, cudaStream_t stream)
{
    static MlpBlock Wm;
    static NetBlock Wn;
    const void *src;
    size_t n;
    if (is_mlpnet(m)) {
        make_net_block(m, Wn);
        src = &Wn;
        n = sizeof Wn;
    } else {
        make_mlp_block(m, Wm);
        src = &Wm;
        n = sizeof Wm;
    }
    const cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, stream);
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "cudaMemcpyAsync(network weights)");
}

constexpr size_t kWeightBytes = sizeof(MlpBlock) > sizeof(NetBlock) ? sizeof(MlpBlock) : sizeof(NetBlock);

}  // namespace

// E (+)= sum_i f(x_i); writes the per-site energies to ecache and the
// features to fcache when non-NULL.
// W is the device weight block of Net; part needs room for kTcMaxCtasPerSm CTAs per SM;
// abort_flag is a device word that starts at zero.
template <class Net>
static smc_status mlp_energy_launch(Workspace *ws, const smc_lattice *lat, const void *W, const int8_t *occ,
                                    float *ecache, uint4 *fcache, double *part, int *abort_flag, double *e,
                                    int accumulate, cudaStream_t stream)
{
    const size_t smem = Net::template Smem<kEvalWG>::END;
    auto kern = k_mlp_site_energy<Net>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return cuda_fail(err, "cudaFuncSetAttribute(k_mlp_site_energy)");
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128 * kEvalWG, smem);
    if (err != cudaSuccess) return cuda_fail(err, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm > kTcMaxCtasPerSm) {
        // more resident CTAs than tensor-memory allocations: a CTA would wait in tcgen05.alloc
        set_error("internal error: MLP energy kernel occupancy exceeds tensor memory");
        return SMC_ERR_STATE;
    }
    per_sm = std::max(1, per_sm);
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const long long tiles = (N + kTcRows - 1) / kTcRows;
    const int grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * ws->num_sms, tiles));
    kern<<<grid, 128 * kEvalWG, smem, stream>>>(W, occ, lat->nx, lat->ny, lat->nz, ecache, fcache, part,
                                                           debug_timeout_ns(), ws->status, abort_flag);
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
    // scratch: [pair counts | abort word | weight block | CTA partial sums]
    const size_t off_abort = round16(sizeof(unsigned long long) * kMaxShells * 64);
    const size_t off_w = off_abort + 16;
    const size_t off_part = round16(off_w + kWeightBytes);
    const size_t need = off_part + sizeof(double) * kTcMaxCtasPerSm * (size_t)std::max(ws->num_sms, 1);
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, need, &st);
    if (!scr) return st;
    st = copy_weights(m, scr + off_w, stream);
    if (st != SMC_OK) return st;
    cudaError_t err = cudaMemsetAsync(scr + off_abort, 0, 16, stream);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync(abort word)");
    int accumulate = 0;
    if (m->kind == SMC_PAIR_F32_MLP_BF16) {
        unsigned long long *cnt = (unsigned long long *)scr;
        st = launch_pair_counts(lat, m->nshells, occ, cnt, stream);
        if (st != SMC_OK) return st;
        st = launch_energy_finish(lat, m, cnt, e, nullptr, stream);
        if (st != SMC_OK) return st;
        accumulate = 1;
    }
    if (is_mlpnet(m))
        return mlp_energy_launch<NetRelu96>(ws, lat, scr + off_w, occ, nullptr, nullptr, (double *)(scr + off_part),
                                            (int *)(scr + off_abort), e, accumulate, stream);
    return mlp_energy_launch<NetSilu64>(ws, lat, scr + off_w, occ, nullptr, nullptr, (double *)(scr + off_part),
                                        (int *)(scr + off_abort), e, accumulate, stream);
}

namespace {
struct MlpPlan {
    int grid = 0, tpc = 0, ntiles = 0, chunk = kMlpChunk;
    size_t smem = 0;
};

// One CTA per tile at a time; all CTAs resident (cooperative launch), at most
// as many per SM as tensor memory holds (kSweepWG x kTcCols columns each)
// when the kernel uses it.  `base`: end of the kernel's fixed shared memory.
smc_status make_mlp_plan(Workspace *ws, const smc_lattice *lat, const void *kernel, uint32_t base, int threads,
                         int tmem_cols, MlpPlan &pl)
{
    const Tuning tu = current_tuning();
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    const int NLx = lat->nx / 4;
    pl.ntiles = (lat->ny / 4) * (lat->nz / 4);
    // the largest trial chunk (a multiple of 16, up to kMlpChunk) that fits
    while (pl.chunk > 16 && mlp_sweep_layout(NLx, 1, pl.chunk, base).end > dyn_max) pl.chunk -= 16;
    for (int tpc_guess = 1; tpc_guess <= 4096; tpc_guess *= 2) {
        const size_t smem = mlp_sweep_layout(NLx, tpc_guess, pl.chunk, base).end;
        if (smem > dyn_max) break;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (tmem_cols > 0) per_sm = std::min(per_sm, 512 / tmem_cols);  // tensor-memory columns
        if (tu.ctas_per_sm > 0) per_sm = std::min(per_sm, tu.ctas_per_sm);
        if (per_sm < 1) break;
        // the CTA with the most tiles sets the pace: fill the GPU, then use as
        // few CTAs as give that same maximum
        const long long res = std::min<long long>((long long)per_sm * ws->num_sms, pl.ntiles);
        const long long most = (pl.ntiles + res - 1) / res;
        const long long nc = (pl.ntiles + most - 1) / most;
        const int tpc = (int)most;
        if (tpc <= tpc_guess) {
            pl.grid = (int)nc;
            pl.tpc = tpc_guess;
            pl.smem = smem;
            return SMC_OK;
        }
    }
    set_error("MLP sweep kernel does not fit on an SM (nx = %d)", lat->nx);
    return SMC_ERR_UNSUPPORTED;
}
}  // namespace

smc_status launch_mlp_sweep(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                            int64_t *n_acc, cudaStream_t stream)
{
    if (!mlp_shape_ok(lat)) {
        set_error("MLP sweeps need every axis a multiple of 4 cells and >= 8");
        return SMC_ERR_UNSUPPORTED;
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const bool has_pair = m->kind == SMC_PAIR_F32_MLP_BF16, net = is_mlpnet(m);
    const void *kernel = net ? (const void *)k_sweep_mlp<NetRelu96, kModeMlp>
                             : (has_pair ? (const void *)k_sweep_mlp<NetSilu64, kModeMlpPair>
                                         : (const void *)k_sweep_mlp<NetSilu64, kModeMlp>);
    const int threads = 128 * (net ? NetRelu96::kSweepNWG : NetSilu64::kSweepNWG);
    MlpPlan pl;
    st = net ? make_mlp_plan(ws, lat, kernel, NetSmem<NetRelu96::kSweepNWG>::END, threads,
                             NetRelu96::kSweepNWG * (int)kNetCols, pl)
             : make_mlp_plan(ws, lat, kernel, MlpSmem<kSweepWG>::END, threads, kSweepWG * (int)kTcCols, pl);
    if (st != SMC_OK) return st;
    static MlpGeo G;
    if (!build_mlp_geo(G)) {
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
    P.nap_cap = 1024;
    P.mlp_chunk = pl.chunk;
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

    // workspace: [flags | part_e | part_n | ticket, abort | weights | energy parts | E cache | F cache]
    const size_t nt = (size_t)P.ntiles;
    const size_t N = 2ull * lat->nx * lat->ny * lat->nz;
    const size_t off_pe = round16(nt * 4), off_pn = off_pe + nt * 8, off_misc = off_pn + nt * 8;
    const size_t off_w = round16(off_misc + 16);
    const size_t off_parts = round16(off_w + kWeightBytes);
    const size_t off_cache =
        round16(off_parts + sizeof(double) * kTcMaxCtasPerSm * (size_t)std::max(ws->num_sms, 1));
    const size_t off_fcache = round16(off_cache + N * 4);
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_fcache + N * 16, &st);
    if (!scr) return st;
    P.flags = (uint32_t *)scr;
    P.part_e = (double *)(scr + off_pe);
    P.part_n = (long long *)(scr + off_pn);
    P.ticket = (unsigned *)(scr + off_misc);
    P.abort_flag = (int *)(scr + off_misc + 4);
    P.status = ws->status;
    P.mlpw = scr + off_w;
    P.ecache = (float *)(scr + off_cache);
    P.fcache = (uint4 *)(scr + off_fcache);
    st = copy_weights(m, scr + off_w, stream);
    if (st != SMC_OK) return st;
    cudaError_t e = cudaMemsetAsync(scr, 0, off_misc + 16, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sweep scratch)");
    st = net ? mlp_energy_launch<NetRelu96>(ws, lat, P.mlpw, occ, P.ecache, P.fcache, (double *)(scr + off_parts),
                                            P.abort_flag, nullptr, 0, stream)
             : mlp_energy_launch<NetSilu64>(ws, lat, P.mlpw, occ, P.ecache, P.fcache, (double *)(scr + off_parts),
                                            P.abort_flag, nullptr, 0, stream);
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
        e = cudaLaunchCooperativeKernel(kernel, dim3(pl.grid), dim3(threads), args, pl.smem, stream);
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
    if (!build_mlp_geo(G)) {
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
    P.timeout_ns = debug_timeout_ns();
    P.status = ws->status;
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
    const size_t off_abort = round16((size_t)ntr * 8);
    const size_t off_w = off_abort + 16;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_w + kWeightBytes, &st);
    if (!scr) return st;
    int *swap_a = (int *)scr, *swap_b = swap_a + ntr;
    P.abort_flag = (int *)(scr + off_abort);
    P.mlpw = scr + off_w;
    st = copy_weights(m, scr + off_w, stream);
    if (st != SMC_OK) return st;
    cudaError_t e = cudaMemsetAsync(scr + off_abort, 0, 16, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(abort word)");
    const bool net = is_mlpnet(m);
    const size_t smem = (net ? NetSmem<kEvalWG>::END : MlpSmem<kEvalWG>::END) + 2 * kTcRows * sizeof(float);
    auto kern = net ? k_mlp_trace_eval<NetRelu96, false>
                    : (has_pair ? k_mlp_trace_eval<NetSilu64, true> : k_mlp_trace_eval<NetSilu64, false>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_trace_eval)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128 * kEvalWG, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm > kTcMaxCtasPerSm) {
        set_error("internal error: MLP trace kernel occupancy exceeds tensor memory");
        return SMC_ERR_STATE;
    }
    const int blocks = std::max(1, std::min((ntr + kTraceTB - 1) / kTraceTB, std::max(per_sm, 1) * ws->num_sms));
    kern<<<blocks, 128 * kEvalWG, smem, stream>>>(P, G, k, dE, acc, swap_a, swap_b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_trace_eval");
    k_mlp_trace_apply<<<(ntr + 127) / 128, 128, 0, stream>>>(occ, ntr, swap_a, swap_b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_trace_apply");
    return SMC_OK;
}

// ---------------------------------------------------------------------------
// qSRO host side.
// ---------------------------------------------------------------------------
namespace {
constexpr double kShellZ[3] = {8.0, 6.0, 12.0};

QsroRaw make_qsro_raw(const smc_model *m, int S)
{
    QsroRaw Q;
    memset(&Q, 0, sizeof Q);
    for (int mm = 0; mm < m->nshells; ++mm) {
        for (int p = 0; p < S; ++p)
            for (int q = 0; q < S; ++q) Q.v[mm][p][q] = (double)m->v_f32[(mm * S + p) * S + q];
        for (int p = 0; p < S; ++p) Q.w[mm][p] = (double)m->qsro_w[mm * S + p];
    }
    Q.c = (double)m->qsro_c;
    Q.nsh = m->nshells;
    Q.S = S;
    return Q;
}

smc_status qsro_sites_launch(Workspace *ws, const smc_lattice *lat, int nsh, const int8_t *occ,
                             unsigned long long *quad, cudaStream_t stream)
{
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const int blocks = (int)std::max(1LL, std::min<long long>((N + 255) / 256, (long long)ws->num_sms * 8));
    k_qsro_sites<<<blocks, 256, 0, stream>>>(occ, lat->nx, lat->ny, lat->nz, nsh, quad);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_qsro_sites");
}

// Pair counts and Q_m^p into scratch, then the FP64 energy and/or gradient.
smc_status qsro_counts_finish(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e, float *grad,
                              cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const size_t off_quad = sizeof(unsigned long long) * kMaxShells * 64;
    unsigned char *scr =
        (unsigned char *)workspace_scratch(ws, off_quad + sizeof(unsigned long long) * kMaxShells * kMaxSpecies, &st);
    if (!scr) return st;
    unsigned long long *cnt = (unsigned long long *)scr, *quad = (unsigned long long *)(scr + off_quad);
    st = launch_pair_counts(lat, m->nshells, occ, cnt, stream);
    if (st != SMC_OK) return st;
    cudaError_t err = cudaMemsetAsync(quad, 0, sizeof(unsigned long long) * kMaxShells * kMaxSpecies, stream);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync(qSRO sums)");
    st = qsro_sites_launch(ws, lat, m->nshells, occ, quad, stream);
    if (st != SMC_OK) return st;
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    k_qsro_finish<<<1, 32, 0, stream>>>(make_qsro_raw(m, lat->nspecies), cnt, quad, N, e, grad);
    err = cudaGetLastError();
    return err == cudaSuccess ? SMC_OK : cuda_fail(err, "k_qsro_finish");
}
}  // namespace

smc_status launch_qsro_energy(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e,
                              cudaStream_t stream)
{
    return qsro_counts_finish(lat, m, occ, e, nullptr, stream);
}

smc_status launch_qsro_grad(const smc_lattice *lat, const smc_model *m, const int8_t *occ, float *grad,
                            cudaStream_t stream)
{
    return qsro_counts_finish(lat, m, occ, nullptr, grad, stream);
}

}  // namespace smc
