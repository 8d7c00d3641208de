// fcc.cu -- swap Monte Carlo on the FCC lattice (the paper's lattice, Sec.
// IV-C; 4x4x4 link cells and 256 mini-steps as in Sec. V-C) with pair models
// and the qSRO model (Sec. IV-B, Eq. quadratic_local_SRO).
//
// Geometry: nx x ny x nz cubic cells of 4 sites at half-unit offsets
// (0,0,0), (1,1,0), (1,0,1), (0,1,1) (sublattices 0-3), site id
// s = ((sub*nz + z)*ny + y)*nx + x.  Shell m holds the half-unit vectors of
// squared length 2m with an even component sum (12, 6, 24 of them), in
// lexicographic order of (vx, vy, vz).  A sweep is n_A = 4 * 64 mini-steps,
// k = ((sub*4 + dz)*4 + dy)*4 + dx, each trying the site at that offset of
// every 4x4x4 link cell against the partner floor(12 w1 / 2^32) of its first
// shell, w = Philox4x32-10(key seed, counter (s, replica, sweep lo, hi)),
// Metropolis on r = w0 & (2^29 - 1) as for the BCC lattice.
//
// One thread per trial and one launch per mini-step: the trials of a
// mini-step touch disjoint read and write sets (pinned exhaustively on the
// CPU for 1-3 shells), and consecutive launches are ordered by the stream.
// dE sums the changed bonds: with every axis at least 8 cells no shell
// aliases, so a's neighbours other than b and b's other than a each flip
// one bond, dE = sum_j D_m(q_j) over a's zone - sum_j D_m(q_j) over b's,
// D_m(q) = V_m(B, q) - V_m(A, q).  The same kernel records the trace (dE,
// decision) of a mini-step, so a sweep equals its traced mini-steps bit for
// bit.
//
// Link cells away from the box faces (1 <= c < NL-1 on every axis) reach
// every neighbour of a and b without a periodic wrap: a neighbour is the
// site id plus a delta that depends only on the sublattice and the vector.
// Those trials run in the last blocks with the deltas, the D rows and the
// first-shell sublattice map in shared memory; the link cells on the faces
// run in the first blocks (their longer path starts early) with wrapped
// coordinates.  Both sum in the same order, so the split changes no result.
// No site read in a launch is written by another trial of it (the
// read/write-set pin), so the interior path reads species through the
// read-only data path.  (Staging the 4 x 5 x 5 rows around each row of
// link cells in shared memory instead was measured slower at 256^3: 400
// staged bytes per trial against 84 cached byte loads.)
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <vector>

#include "sweep_common.cuh"

namespace smc {

namespace {

// Per-call tables (32-bit words): D rows T[m][A][B][q] = V_m(B,q) - V_m(A,q)
// (stride 8), index deltas D[sub][t] of the 42 shell vectors without wrap,
// first-shell sublattice map N1[sub][dir], packed vectors (v + 2, 4 bits each).
constexpr int kFccT = kMaxShells * 8 * 8 * 8, kFccD = kFccT, kFccN1 = kFccD + 4 * 42, kFccVec = kFccN1 + 4 * 12,
              kFccWords = kFccVec + 42;

// What the mini-step and cache kernels read (a small launch parameter block:
// 256 launches per sweep).
struct FccStep {
    int nx, ny, nz, S, nshells, nA_cells;  // nA_cells: link cells (trials per mini-step)
    int NLx, NLy, NLz;
    int n_int, n_bnd, bnd_blocks;          // interior / face link cells, blocks of the face part (run first)
    const uint32_t *tables;
    uint64_t seed;
    uint32_t replica;
    uint64_t sweep;
    float beta;
    int2 tinfo;
    const uint32_t *tab;
    int8_t *occ;
    double *part_e;       // per link cell, accumulated over a call
    long long *part_n;
    float *dE_out;        // trace (nullable)
    uint8_t *acc_out;
    void *qcache;  // qSRO: own-species counts per shell of every site (1 byte for 1-2 shells, 2 for 3)
};

// The model as the energy kernels read it.
struct FccParams : FccStep {
    int vi[kMaxShells * kMaxSpecies * kMaxSpecies];
    float vf[kMaxShells * kMaxSpecies * kMaxSpecies];
    float wq[kMaxShells * kMaxSpecies];  // qSRO W_m^p
    double qc;                           // qSRO C
};

// Own-species count fields of the qSRO cache: shell 1 in bits 0-3 (<= 12),
// shell 2 in bits 4-6 (<= 6), shell 3 in bits 7-11 (<= 24).
__host__ __device__ constexpr int fcc_qoff(int m) { return m == 0 ? 0 : (m == 1 ? 4 : 7); }
__host__ __device__ constexpr int fcc_qmask(int m) { return m == 0 ? 15 : (m == 1 ? 7 : 31); }

// Zone categories of a qSRO trial, (shell to a) * 4 + (shell to b), with their
// sizes: the same for every partner direction (the 12 are equivalent under
// the cubic point group, which keeps shells).  The zone table of each
// direction lists its sites in this category order.
__host__ __device__ constexpr int fcc_zone_ncat(int nsh) { return nsh == 1 ? 3 : (nsh == 2 ? 7 : 14); }
__host__ __device__ constexpr int fcc_zone_cat(int nsh, int i, int *count)
{
    constexpr int c1[3][2] = {{4, 7}, {1, 7}, {5, 4}};
    constexpr int c2[7][2] = {{4, 5}, {8, 4}, {1, 5}, {2, 4}, {5, 4}, {6, 2}, {9, 2}};
    constexpr int c3[14][2] = {{4, 1},  {8, 2},  {12, 14}, {1, 1}, {2, 2},  {3, 14}, {5, 4},
                               {6, 2},  {7, 4},  {9, 2},   {11, 2}, {13, 4}, {14, 2}, {15, 4}};
    const int *e = nsh == 1 ? c1[i] : (nsh == 2 ? c2[i] : c3[i]);
    *count = e[1];
    return e[0];
}
// category code of the e-th zone site
__host__ __device__ constexpr int fcc_zone_code(int nsh, int e)
{
    int n = 0, code = 0;
    for (int i = 0; i < fcc_zone_ncat(nsh); ++i) {
        code = fcc_zone_cat(nsh, i, &n);
        if (e < n) return code;
        e -= n;
    }
    return 0;
}

// qSRO per-call tables (32-bit words): Dz[m][A][B][q] = (V_m(B,q) - V_m(A,q)) / z_m,
// Wz[m][p] = W_m^p / z_m^2, per partner direction the zone entries (half-unit
// offset index w = (x+3) + 7 (y+3) + 49 (z+3), shell to a at bit 9, shell to
// b at bit 11), the offset index of each first-shell vector, and the index
// deltas of every offset per sublattice.
constexpr int kQZmax = 58, kQT = kMaxShells * 512, kQW = kQT, kQZ = kQW + kMaxShells * 8, kQV1 = kQZ + 12 * kQZmax,
              kQDel = kQV1 + 12, kQWords = kQDel + 4 * 343;

__constant__ signed char c_fcc_vec[4][24][3];  // shells 1-3 at [1..3]
__constant__ int c_fcc_n[4];

// Half-unit position of a site and its wrapped neighbour along v.
struct FccPos {
    int x, y, z;  // 2 * cell + basis
};

__device__ __forceinline__ FccPos fcc_pos(int sub, int x, int y, int z)
{
    return FccPos{2 * x + ((sub == 1 || sub == 2) ? 1 : 0), 2 * y + ((sub == 1 || sub == 3) ? 1 : 0),
                  2 * z + ((sub == 2 || sub == 3) ? 1 : 0)};
}

__device__ __forceinline__ int fcc_site_at(const FccStep &P, int px, int py, int pz)
{
    const int ox = px & 1, oy = py & 1;
    const int nsub = (0x6C >> ((ox << 2) | (oy << 1))) & 3;  // parities (1,1) -> 1, (1,0) -> 2, (0,1) -> 3
    const int cx = wrapc(px >> 1, P.nx), cy = wrapc(py >> 1, P.ny), cz = wrapc(pz >> 1, P.nz);
    return ((nsub * P.nz + cz) * P.ny + cy) * P.nx + cx;
}

__device__ __forceinline__ int3 fcc_unpack(int w) { return make_int3((w & 15) - 2, ((w >> 4) & 15) - 2, ((w >> 8) & 15) - 2); }

// Shell-vector index t (shell 1: 0-11, shell 2: 12-17, shell 3: 18-41) -> D-row offset.
__host__ __device__ constexpr int fcc_shell_off(int t) { return t < 12 ? 0 : (t < 18 ? 512 : 1024); }

// The t-th link cell on the box faces: z faces, then y faces, then x faces.
__device__ __forceinline__ int3 fcc_face_cell(int j, int NLx, int NLy, int NLz)
{
    const int fz = NLx * NLy;
    if (j < 2 * fz) {
        const int r = j % fz;
        return make_int3(r % NLx, r / NLx, j < fz ? 0 : NLz - 1);
    }
    j -= 2 * fz;
    const int fy = NLx * (NLz - 2);
    if (j < 2 * fy) {
        const int r = j % fy;
        return make_int3(r % NLx, j < fy ? 0 : NLy - 1, 1 + r / NLx);
    }
    j -= 2 * fy;
    const int fx = (NLy - 2) * (NLz - 2);
    const int r = j % fx;
    return make_int3(j < fx ? 0 : NLx - 1, 1 + r % (NLy - 2), 1 + r / (NLy - 2));
}

template <bool IS_INT, int NSH>
__global__ void __launch_bounds__(256) k_fcc_ministep(const __grid_constant__ FccStep P, int k)
{
    using T = typename Acc<IS_INT>::T;
    using Word = typename std::conditional<IS_INT, int, float>::type;
    // integer models sum in 64 bits (84 terms of |V| <= 2^24 can pass 2^31)
    using Wide = typename std::conditional<IS_INT, long long, float>::type;
    constexpr int NV = NSH == 1 ? 12 : (NSH == 2 ? 18 : 42);
    __shared__ uint32_t sm[kFccWords];
    for (int i = threadIdx.x; i < kFccWords; i += blockDim.x) sm[i] = __ldg(P.tables + i);
    __syncthreads();
    const Word *sT = reinterpret_cast<const Word *>(sm);
    const int *sD = reinterpret_cast<const int *>(sm + kFccD);
    const int *sN1 = reinterpret_cast<const int *>(sm + kFccN1);
    const int *sV = reinterpret_cast<const int *>(sm + kFccVec);

    const int dx = k & 3, dy = (k >> 2) & 3, dz = (k >> 4) & 3, sub = k >> 6;
    const bool interior = (int)blockIdx.x >= P.bnd_blocks;
    int3 cc;
    if (interior) {
        const int i = (blockIdx.x - P.bnd_blocks) * blockDim.x + threadIdx.x;
        if (i >= P.n_int) return;
        const int wx = P.NLx - 2, wy = P.NLy - 2;
        cc = make_int3(1 + i % wx, 1 + (i / wx) % wy, 1 + i / (wx * wy));
    } else {
        const int j = blockIdx.x * blockDim.x + threadIdx.x;
        if (j >= P.n_bnd) return;
        cc = fcc_face_cell(j, P.NLx, P.NLy, P.NLz);
    }
    const int c = (cc.z * P.NLy + cc.y) * P.NLx + cc.x;
    const int x = 4 * cc.x + dx, y = 4 * cc.y + dy, z = 4 * cc.z + dz;
    const int a = ((sub * P.nz + z) * P.ny + y) * P.nx + x;
    const U4 w = philox10(U4{(uint32_t)a, P.replica, (uint32_t)P.sweep, (uint32_t)(P.sweep >> 32)}, (uint32_t)P.seed,
                          (uint32_t)(P.seed >> 32));
    const uint32_t r = w.x & kRMask;
    const int dir = (int)(((uint64_t)w.y * 12u) >> 32), opp = 11 - dir;  // shell 1 is centrally symmetric
    const FccPos pa = fcc_pos(sub, x, y, z);
    const int3 v1 = fcc_unpack(sV[dir]);
    const FccPos pb{pa.x + v1.x, pa.y + v1.y, pa.z + v1.z};
    int8_t *occ = P.occ;
    const int b = interior ? a + sD[sub * 42 + dir] : fcc_site_at(P, pb.x, pb.y, pb.z);
    const int A = occ[a] & 7, B = occ[b] & 7;
    const Word *row = sT + (A * 8 + B) * 8;
    Wide dw = Wide(0);
    if (interior) {
        // all 2 NV species loads first (independent, in flight together), then the sums
        const int *da = sD + sub * 42, *db = sD + sN1[sub * 12 + dir] * 42;
        int qa[NV], qb[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) qa[t] = __ldg(occ + a + da[t]);
#pragma unroll
        for (int t = 0; t < NV; ++t) qb[t] = __ldg(occ + b + db[t]);
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const Word v = row[fcc_shell_off(t) + (qa[t] & 7)];
            if (t >= 12 || t != dir) dw += (Wide)v;
        }
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            const Word v = row[fcc_shell_off(t) + (qb[t] & 7)];
            if (t >= 12 || t != opp) dw -= (Wide)v;
        }
    } else {
#pragma unroll 6
        for (int t = 0; t < NV; ++t) {
            const int3 v = fcc_unpack(sV[t]);
            const Word e = row[fcc_shell_off(t) + (occ[fcc_site_at(P, pa.x + v.x, pa.y + v.y, pa.z + v.z)] & 7)];
            if (t >= 12 || t != dir) dw += (Wide)e;
        }
#pragma unroll 6
        for (int t = 0; t < NV; ++t) {
            const int3 v = fcc_unpack(sV[t]);
            const Word e = row[fcc_shell_off(t) + (occ[fcc_site_at(P, pb.x + v.x, pb.y + v.y, pb.z + v.z)] & 7)];
            if (t >= 12 || t != opp) dw -= (Wide)e;
        }
    }
    // a dE beyond the int range is rejected anyway (the acceptance table is shorter)
    T dE;
    if constexpr (IS_INT)
        dE = (T)(dw > 0x7FFFFFFFLL ? 0x7FFFFFFFLL : (dw < -0x7FFFFFFFLL ? -0x7FFFFFFFLL : dw));
    else
        dE = dw;
    const bool acc = metropolis<IS_INT>(dE, r, P.beta, P.tab, P.tinfo);
    if (acc) {
        occ[a] = (int8_t)B;
        occ[b] = (int8_t)A;
        if (P.part_e) {
            P.part_e[c] += (double)dw;
            P.part_n[c] += 1;
        }
    }
    if (P.dE_out) P.dE_out[c] = (float)dw;
    if (P.acc_out) P.acc_out[c] = acc ? 1 : 0;
}

__device__ __forceinline__ int3 fcc_woff(int w) { return make_int3(w % 7 - 3, (w / 7) % 7 - 3, w / 49 - 3); }

// qSRO cache: for every site, the number of its shell-m neighbours of its own
// species, in field m (fcc_qoff).
__global__ void __launch_bounds__(256) k_fcc_qsro_cache(const __grid_constant__ FccStep P)
{
    const int N = 4 * P.nx * P.ny * P.nz;
    // 64-bit loop index: N may be within one stride of 2^31
    for (long long si = blockIdx.x * (long long)blockDim.x + threadIdx.x; si < N;
         si += (long long)gridDim.x * blockDim.x) {
        const int s = (int)si;
        const int p = P.occ[s] & 7;
        const int x = s % P.nx, y = (s / P.nx) % P.ny, z = (s / (P.nx * P.ny)) % P.nz, sub = s / (P.nx * P.ny * P.nz);
        const FccPos ps = fcc_pos(sub, x, y, z);
        uint32_t q = 0;
        for (int m = 1; m <= P.nshells; ++m)
            for (int t = 0; t < c_fcc_n[m]; ++t) {
                const signed char *v = c_fcc_vec[m][t];
                if ((P.occ[fcc_site_at(P, ps.x + v[0], ps.y + v[1], ps.z + v[2])] & 7) == p) q += 1u << fcc_qoff(m - 1);
            }
        if (P.nshells == 3)
            static_cast<uint16_t *>(P.qcache)[s] = (uint16_t)q;
        else
            static_cast<uint8_t *>(P.qcache)[s] = (uint8_t)q;
    }
}

// One qSRO trial per thread (Eq. quadratic_local_SRO with the FCC shells).
// Site j's energy changes only through the species of its neighbours a and
// b: with a in shell ma of j and b in shell mb (0 = neither),
//   linear part  D_ma(s_j)/z_ma - D_mb(s_j)/z_mb,  D_m(q) = V_m(B,q) - V_m(A,q),
//   W part       (s_j = A or B, ma != mb) from j's cached own-species counts.
// a and b change their own species: their linear parts sum to the same
// D terms again (V symmetric), and their W parts use the counts of A and B
// around each (b counted in a's shell 1 and a in b's).  C cancels.  The zone
// is walked in category order, so ma and mb are compile-time constants.
template <int NSH>
__global__ void __launch_bounds__(256) k_fcc_qsro_ministep(const __grid_constant__ FccStep P, int k)
{
    using QT = typename std::conditional<NSH == 3, uint16_t, uint8_t>::type;
    constexpr int NZ = NSH == 1 ? 18 : (NSH == 2 ? 26 : 58);
    __shared__ uint32_t sm[kQWords];
    for (int i = threadIdx.x; i < kQWords; i += blockDim.x) sm[i] = __ldg(P.tables + i);
    __syncthreads();
    const float *sT = reinterpret_cast<const float *>(sm);
    const float *sW = reinterpret_cast<const float *>(sm + kQW);
    const int *sZ = reinterpret_cast<const int *>(sm + kQZ);
    const int *sV1 = reinterpret_cast<const int *>(sm + kQV1);

    const int dx = k & 3, dy = (k >> 2) & 3, dz = (k >> 4) & 3, sub = k >> 6;
    const bool interior = (int)blockIdx.x >= P.bnd_blocks;
    int3 cc;
    if (interior) {
        const int i = (blockIdx.x - P.bnd_blocks) * blockDim.x + threadIdx.x;
        if (i >= P.n_int) return;
        const int wx = P.NLx - 2, wy = P.NLy - 2;
        cc = make_int3(1 + i % wx, 1 + (i / wx) % wy, 1 + i / (wx * wy));
    } else {
        const int j = blockIdx.x * blockDim.x + threadIdx.x;
        if (j >= P.n_bnd) return;
        cc = fcc_face_cell(j, P.NLx, P.NLy, P.NLz);
    }
    const int c = (cc.z * P.NLy + cc.y) * P.NLx + cc.x;
    const int x = 4 * cc.x + dx, y = 4 * cc.y + dy, z = 4 * cc.z + dz;
    const int a = ((sub * P.nz + z) * P.ny + y) * P.nx + x;
    const U4 w4 = philox10(U4{(uint32_t)a, P.replica, (uint32_t)P.sweep, (uint32_t)(P.sweep >> 32)}, (uint32_t)P.seed,
                           (uint32_t)(P.seed >> 32));
    const uint32_t r = w4.x & kRMask;
    const int dir = (int)(((uint64_t)w4.y * 12u) >> 32);
    const FccPos pa = fcc_pos(sub, x, y, z);
    const int *del = reinterpret_cast<const int *>(sm + kQDel) + sub * 343;
    const int wb = sV1[dir];
    const int3 v1 = fcc_woff(wb);
    const int b = interior ? a + del[wb] : fcc_site_at(P, pa.x + v1.x, pa.y + v1.y, pa.z + v1.z);
    int8_t *occ = P.occ;
    QT *Qc = static_cast<QT *>(P.qcache);
    const int A = occ[a] & 7, B = occ[b] & 7;
    const int *zone = sZ + dir * kQZmax;
    auto site = [&](int e) {
        const int w = zone[e];
        if (interior) return a + del[w];
        const int3 d = fcc_woff(w);
        return fcc_site_at(P, pa.x + d.x, pa.y + d.y, pa.z + d.z);
    };
    // packed per-shell counts (byte m-1): species A / B around a and around b
    uint32_t cAa = 0, cBa = 1u, cAb = 1u, cBb = 0;  // b (species B) is in a's shell 1, a (A) in b's
    // species | count cache << 4 of every zone site, kept for the update of
    // an accepted swap: reloading them there would put a global round trip
    // behind every cache store of the walk (the compiler cannot prove occ
    // and the cache apart)
    uint32_t zq[NZ];
    float dE = 0.f;
    if (A != B) {
        const float *row = sT + (A * 8 + B) * 8;
        float wA[NSH], wB[NSH];  // W_m^A / z_m^2, W_m^B / z_m^2
#pragma unroll
        for (int m = 0; m < NSH; ++m) {
            wA[m] = sW[m * 8 + A];
            wB[m] = sW[m * 8 + B];
        }
        float lin = 0.f, wz = 0.f;
#pragma unroll
        for (int e = 0; e < NZ; ++e) {
            const int code = fcc_zone_code(NSH, e), ma = code >> 2, mb = code & 3;
            const int j = site(e);
            const int sj = occ[j] & 7;
            const uint32_t isA = sj == A, isB = sj == B;
            if (ma) {
                lin += row[(ma - 1) * 512 + sj];
                cAa += isA << (8 * (ma - 1));
                cBa += isB << (8 * (ma - 1));
            }
            if (mb) {
                lin -= row[(mb - 1) * 512 + sj];
                cAb += isA << (8 * (mb - 1));
                cBb += isB << (8 * (mb - 1));
            }
            zq[e] = (uint32_t)sj;
            if (ma != mb) {
                const int q = Qc[j];
                zq[e] |= (uint32_t)q << 4;
                float t = 0.f;  // a leaves j's shell ma as A and arrives as B; b the reverse in shell mb
                if (ma) {
                    const int n = (q >> fcc_qoff(ma - 1)) & fcc_qmask(ma - 1);
                    t += isA ? wA[ma - 1] * (float)(1 - 2 * n) : (isB ? wB[ma - 1] * (float)(2 * n + 1) : 0.f);
                }
                if (mb) {
                    const int n = (q >> fcc_qoff(mb - 1)) & fcc_qmask(mb - 1);
                    t += isA ? wA[mb - 1] * (float)(2 * n + 1) : (isB ? wB[mb - 1] * (float)(1 - 2 * n) : 0.f);
                }
                wz += t;
            }
        }
        float wa = 0.f, wbb = 0.f;
#pragma unroll
        for (int m = 0; m < NSH; ++m) {
            const int nAa = (cAa >> (8 * m)) & 255, nBa = ((cBa >> (8 * m)) & 255) - (m == 0 ? 1 : 0);
            const int nAb = ((cAb >> (8 * m)) & 255) - (m == 0 ? 1 : 0), nBb = (cBb >> (8 * m)) & 255;
            wa += wB[m] * (float)(nBa * nBa) - wA[m] * (float)(nAa * nAa);
            wbb += wA[m] * (float)(nAb * nAb) - wB[m] * (float)(nBb * nBb);
        }
        dE = 2.f * lin + wa + wbb + wz;
    }
    const bool acc = metropolis<false>(dE, r, P.beta, P.tab, P.tinfo);
    if (acc) {
        if (A != B) {
            occ[a] = (int8_t)B;
            occ[b] = (int8_t)A;
            int qa = 0, qb = 0;  // a now B: its B neighbours other than b; b now A likewise
#pragma unroll
            for (int m = 0; m < NSH; ++m) {
                qa += (int)(((cBa >> (8 * m)) & 255u) - (m == 0 ? 1u : 0u)) << fcc_qoff(m);
                qb += (int)(((cAb >> (8 * m)) & 255u) - (m == 0 ? 1u : 0u)) << fcc_qoff(m);
            }
            Qc[a] = (QT)qa;
            Qc[b] = (QT)qb;
#pragma unroll
            for (int e = 0; e < NZ; ++e) {
                const int code = fcc_zone_code(NSH, e), ma = code >> 2, mb = code & 3;
                if (ma == mb) continue;
                const int sj = (int)(zq[e] & 15u), q = (int)(zq[e] >> 4);
                // A sites lose a (shell ma) and gain b (shell mb); B sites the reverse
                const int d = (ma ? 1 << fcc_qoff(ma - 1) : 0) - (mb ? 1 << fcc_qoff(mb - 1) : 0);
                if (sj == A) Qc[site(e)] = (QT)(q - d);
                if (sj == B) Qc[site(e)] = (QT)(q + d);
            }
        }
        if (P.part_e) {
            P.part_e[c] += (double)dE;
            P.part_n[c] += 1;
        }
    }
    if (P.dE_out) P.dE_out[c] = dE;
    if (P.acc_out) P.acc_out[c] = acc ? 1 : 0;
}

// e_acc += sum of part_e, n_acc += sum of part_n, in a fixed order: thread t
// sums link cells t, t + 1024, ... in turn, then a fixed pairwise tree over
// the 1024 partial sums (one block of kFccReduceThreads).
constexpr int kFccReduceThreads = 1024;
__global__ void __launch_bounds__(kFccReduceThreads) k_fcc_reduce(const double *part_e, const long long *part_n, int n,
                                                                  double *e_acc, long long *n_acc)
{
    __shared__ double se[kFccReduceThreads];
    __shared__ long long sn[kFccReduceThreads];
    const int t = threadIdx.x;
    double e = 0.0;
    long long c = 0;
    for (int i = t; i < n; i += kFccReduceThreads) {
        e += part_e[i];
        c += part_n[i];
    }
    se[t] = e;
    sn[t] = c;
    __syncthreads();
    for (int h = kFccReduceThreads / 2; h > 0; h >>= 1) {
        if (t < h) {
            se[t] += se[t + h];
            sn[t] += sn[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        if (e_acc) *e_acc += se[0];
        if (n_acc) *n_acc += sn[0];
    }
}

// Ordered pair counts n_m^{pq} (each site's shell-m neighbours), per-block
// shared counters flushed with 64-bit atomics.
// With sq non-null also Q_m^p = sum over sites of species p of the squared
// number of their shell-m neighbours of species p (the qSRO W term).
__global__ void __launch_bounds__(256) k_fcc_pair_counts(const __grid_constant__ FccParams P,
                                                         unsigned long long *counts, unsigned long long *sq)
{
    __shared__ unsigned int cnt[kMaxShells * kMaxSpecies * kMaxSpecies];
    __shared__ unsigned int csq[kMaxShells * kMaxSpecies];
    for (int i = threadIdx.x; i < kMaxShells * kMaxSpecies * kMaxSpecies; i += blockDim.x) cnt[i] = 0;
    for (int i = threadIdx.x; i < kMaxShells * kMaxSpecies; i += blockDim.x) csq[i] = 0;
    __syncthreads();
    const int N = 4 * P.nx * P.ny * P.nz, S = P.S;
    // 64-bit loop index: N may be within one stride of 2^31
    for (long long si = blockIdx.x * (long long)blockDim.x + threadIdx.x; si < N;
         si += (long long)gridDim.x * blockDim.x) {
        const int s = (int)si;
        const int p = P.occ[s] & 7;
        const int x = s % P.nx, y = (s / P.nx) % P.ny, z = (s / (P.nx * P.ny)) % P.nz, sub = s / (P.nx * P.ny * P.nz);
        const FccPos ps = fcc_pos(sub, x, y, z);
        for (int m = 1; m <= P.nshells; ++m) {
            unsigned int own = 0;
            for (int t = 0; t < c_fcc_n[m]; ++t) {
                const signed char *v = c_fcc_vec[m][t];
                const int q = P.occ[fcc_site_at(P, ps.x + v[0], ps.y + v[1], ps.z + v[2])] & 7;
                atomicAdd(&cnt[((m - 1) * S + p) * S + q], 1u);
                own += q == p;
            }
            if (sq && own) atomicAdd(&csq[(m - 1) * kMaxSpecies + p], own * own);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P.nshells * S * S; i += blockDim.x)
        if (cnt[i]) atomicAdd(counts + i, (unsigned long long)cnt[i]);
    if (sq)
        for (int i = threadIdx.x; i < kMaxShells * kMaxSpecies; i += blockDim.x)
            if (csq[i]) atomicAdd(sq + i, (unsigned long long)csq[i]);
}

// E = 1/2 sum_m sum_{p,q} V_m(p, q) n_m^{pq}, exactly in int64 (integer
// models, also returned in units) or FP64.
__global__ void k_fcc_energy_finish(const __grid_constant__ FccParams P, const unsigned long long *counts, int is_int,
                                    double unit, double *e, long long *e_int)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = P.nshells * P.S * P.S;
    if (is_int) {
        long long tot = 0;
        for (int i = 0; i < n; ++i) tot += (long long)P.vi[i] * (long long)counts[i];
        tot /= 2;  // every bond counted from both ends
        if (e_int) *e_int = tot;
        if (e) *e = (double)tot * unit;
    } else if (e && P.qcache) {  // qSRO: E = N C + sum V n / z_m + sum W Q / z_m^2
        const double z[3] = {12.0, 6.0, 24.0};
        const unsigned long long *sq = counts + kMaxShells * 64;
        double tot = 4.0 * P.nx * P.ny * P.nz * P.qc;
        for (int i = 0; i < n; ++i) tot += (double)P.vf[i] * (double)counts[i] / z[i / (P.S * P.S)];
        for (int m = 0; m < P.nshells; ++m)
            for (int p = 0; p < P.S; ++p)
                tot += (double)P.wq[m * P.S + p] * (double)sq[m * kMaxSpecies + p] / (z[m] * z[m]);
        *e = tot;
    } else if (e) {
        double tot = 0.0;
        for (int i = 0; i < n; ++i) tot += (double)P.vf[i] * (double)counts[i];
        *e = 0.5 * tot;
    }
}

uint64_t g_fcc_tables = 0;  // bit d: the constant tables are on device d (each device has its own copy)

smc_status fcc_tables()
{
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
    if (dev < 64 && (g_fcc_tables >> dev & 1u)) return SMC_OK;
    signed char v[4][24][3] = {};
    int n[4] = {0, 0, 0, 0};
    for (int m = 1; m <= 3; ++m)
        for (int x = -2; x <= 2; ++x)
            for (int y = -2; y <= 2; ++y)
                for (int z = -2; z <= 2; ++z)
                    if (x * x + y * y + z * z == 2 * m && ((x + y + z) & 1) == 0) {
                        v[m][n[m]][0] = (signed char)x;
                        v[m][n[m]][1] = (signed char)y;
                        v[m][n[m]][2] = (signed char)z;
                        ++n[m];
                    }
    if (n[1] != 12 || n[2] != 6 || n[3] != 24) {
        set_error("internal error: FCC shell vectors");
        return SMC_ERR_STATE;
    }
    cudaError_t e = cudaMemcpyToSymbol(c_fcc_vec, v, sizeof v);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_fcc_n, n, sizeof n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(FCC shells)");
    if (dev < 64) g_fcc_tables |= 1ull << dev;
    return SMC_OK;
}

smc_status fcc_params(const smc_lattice *lat, const smc_model *m, int8_t *occ, FccParams &P)
{
    memset(&P, 0, sizeof P);
    P.nx = lat->nx;
    P.ny = lat->ny;
    P.nz = lat->nz;
    P.S = lat->nspecies;
    P.nshells = m->nshells;
    P.NLx = lat->nx / 4;
    P.NLy = lat->ny / 4;
    P.NLz = lat->nz / 4;
    P.nA_cells = P.NLx * P.NLy * P.NLz;
    P.occ = occ;
    const int n = m->nshells * P.S * P.S;
    for (int i = 0; i < n; ++i) {
        if (m->kind == SMC_PAIR_I32)
            P.vi[i] = m->v_i32[i];
        else
            P.vf[i] = m->v_f32[i];
    }
    if (m->kind == SMC_QSRO_F32) {
        for (int i = 0; i < m->nshells * P.S; ++i) P.wq[i] = m->qsro_w[i];
        P.qc = m->qsro_c;
    }
    return fcc_tables();
}

// Shell of a half-unit offset (1-3 within nshells, else 0).
int fcc_shell_of(int x, int y, int z, int nshells)
{
    const int d = x * x + y * y + z * z;
    if (d == 0 || (d & 1) || ((x + y + z) & 1)) return 0;
    return d / 2 <= nshells ? d / 2 : 0;
}

// The per-call table block of k_fcc_qsro_ministep (layout at kQT .. kQWords).
smc_status fcc_qsro_tables(const smc_lattice *lat, const smc_model *m, std::vector<uint32_t> &w)
{
    const int S = lat->nspecies, nsh = m->nshells;
    const double z[3] = {12.0, 6.0, 24.0};
    w.assign(kQWords, 0u);
    for (int sh = 0; sh < nsh; ++sh) {
        for (int A = 0; A < S; ++A)
            for (int B = 0; B < S; ++B)
                for (int q = 0; q < S; ++q) {
                    const float d = (float)(((double)m->v_f32[(sh * S + B) * S + q] - m->v_f32[(sh * S + A) * S + q]) / z[sh]);
                    memcpy(&w[sh * 512 + (A * 8 + B) * 8 + q], &d, 4);
                }
        for (int p = 0; p < S; ++p) {
            const float v = (float)((double)m->qsro_w[sh * S + p] / (z[sh] * z[sh]));
            memcpy(&w[kQW + sh * 8 + p], &v, 4);
        }
    }
    auto widx = [](int x, int y, int z) { return (x + 3) + 7 * (y + 3) + 49 * (z + 3); };
    std::vector<std::array<int, 3>> v1;
    for (int x = -2; x <= 2; ++x)
        for (int y = -2; y <= 2; ++y)
            for (int zz = -2; zz <= 2; ++zz)
                if (x * x + y * y + zz * zz == 2 && ((x + y + zz) & 1) == 0) v1.push_back({x, y, zz});
    const int want = nsh == 1 ? 18 : (nsh == 2 ? 26 : 58);
    for (int d = 0; d < 12; ++d) {
        w[kQV1 + d] = (uint32_t)widx(v1[d][0], v1[d][1], v1[d][2]);
        int n = 0;
        for (int ci = 0; ci < fcc_zone_ncat(nsh); ++ci) {
            int cnt = 0;
            const int code = fcc_zone_cat(nsh, ci, &cnt);
            int got = 0;
            for (int x = -3; x <= 3; ++x)
                for (int y = -3; y <= 3; ++y)
                    for (int zz = -3; zz <= 3; ++zz) {
                        if ((x == 0 && y == 0 && zz == 0) || (x == v1[d][0] && y == v1[d][1] && zz == v1[d][2]))
                            continue;
                        const int ma = fcc_shell_of(x, y, zz, nsh);
                        const int mb = fcc_shell_of(x - v1[d][0], y - v1[d][1], zz - v1[d][2], nsh);
                        if (ma * 4 + mb != code) continue;
                        if (n < kQZmax) w[kQZ + d * kQZmax + n] = (uint32_t)widx(x, y, zz);
                        ++n;
                        ++got;
                    }
            if (got != cnt) {
                set_error("internal error: FCC qSRO zone category %d has %d sites (want %d)", code, got, cnt);
                return SMC_ERR_STATE;
            }
        }
        if (n != want) {
            set_error("internal error: FCC qSRO zone has %d sites (want %d)", n, want);
            return SMC_ERR_STATE;
        }
    }
    const long long NC = (long long)lat->nx * lat->ny * lat->nz;
    for (int sub = 0; sub < 4; ++sub) {
        const int b[3] = {(sub == 1 || sub == 2) ? 1 : 0, (sub == 1 || sub == 3) ? 1 : 0, (sub == 2 || sub == 3) ? 1 : 0};
        for (int x = -3; x <= 3; ++x)
            for (int y = -3; y <= 3; ++y)
                for (int zz = -3; zz <= 3; ++zz) {
                    if ((x + y + zz) & 1) continue;
                    const int q[3] = {b[0] + x, b[1] + y, b[2] + zz};
                    int dc[3];
                    for (int k = 0; k < 3; ++k) dc[k] = q[k] >= 0 ? q[k] / 2 : -((1 - q[k]) / 2);  // floor(q / 2)
                    const int par = ((q[0] & 1) << 2) | ((q[1] & 1) << 1) | (q[2] & 1);
                    const int nsub = par == 0 ? 0 : (par == 6 ? 1 : (par == 5 ? 2 : 3));
                    const long long delta = (nsub - sub) * NC + ((long long)dc[2] * lat->ny + dc[1]) * lat->nx + dc[0];
                    w[kQDel + sub * 343 + widx(x, y, zz)] = (uint32_t)(int32_t)delta;
                }
    }
    return SMC_OK;
}

// The per-call table block of k_fcc_ministep (layout at kFccT .. kFccWords).
smc_status fcc_sweep_tables(const smc_lattice *lat, const smc_model *m, std::vector<uint32_t> &w)
{
    std::vector<std::array<int, 3>> vec;
    for (int sh = 1; sh <= 3; ++sh)
        for (int x = -2; x <= 2; ++x)
            for (int y = -2; y <= 2; ++y)
                for (int z = -2; z <= 2; ++z)
                    if (x * x + y * y + z * z == 2 * sh && ((x + y + z) & 1) == 0) vec.push_back({x, y, z});
    bool ok = vec.size() == 42;
    for (int i = 0; ok && i < 12; ++i)
        for (int d = 0; d < 3; ++d) ok = ok && vec[11 - i][d] == -vec[i][d];
    for (int t = 0; ok && t < 42; ++t) ok = fcc_shell_off(t) == 512 * ((t >= 12) + (t >= 18));
    if (!ok) {
        set_error("internal error: FCC shell table");
        return SMC_ERR_STATE;
    }
    w.assign(kFccWords, 0u);
    const int S = lat->nspecies;
    for (int sh = 0; sh < m->nshells; ++sh)
        for (int A = 0; A < S; ++A)
            for (int B = 0; B < S; ++B)
                for (int q = 0; q < S; ++q) {
                    const int o = sh * 512 + (A * 8 + B) * 8 + q;
                    const int ib = (sh * S + B) * S + q, ia = (sh * S + A) * S + q;
                    if (m->kind == SMC_PAIR_I32) {
                        w[o] = (uint32_t)(m->v_i32[ib] - m->v_i32[ia]);
                    } else {
                        const float d = m->v_f32[ib] - m->v_f32[ia];
                        memcpy(&w[o], &d, 4);
                    }
                }
    const long long NC = (long long)lat->nx * lat->ny * lat->nz;
    for (int sub = 0; sub < 4; ++sub) {
        const int b[3] = {(sub == 1 || sub == 2) ? 1 : 0, (sub == 1 || sub == 3) ? 1 : 0, (sub == 2 || sub == 3) ? 1 : 0};
        for (int t = 0; t < 42; ++t) {
            int q[3], dc[3];
            for (int d = 0; d < 3; ++d) {
                q[d] = b[d] + vec[t][d];
                dc[d] = q[d] >= 0 ? q[d] / 2 : -((1 - q[d]) / 2);  // floor(q / 2)
            }
            const int par = ((q[0] & 1) << 2) | ((q[1] & 1) << 1) | (q[2] & 1);
            const int nsub = par == 0 ? 0 : (par == 6 ? 1 : (par == 5 ? 2 : 3));
            const long long delta = (nsub - sub) * NC + ((long long)dc[2] * lat->ny + dc[1]) * lat->nx + dc[0];
            w[kFccD + sub * 42 + t] = (uint32_t)(int32_t)delta;
            if (t < 12) w[kFccN1 + sub * 12 + t] = (uint32_t)nsub;
        }
    }
    for (int t = 0; t < 42; ++t)
        w[kFccVec + t] = (uint32_t)((vec[t][0] + 2) | ((vec[t][1] + 2) << 4) | ((vec[t][2] + 2) << 8));
    return SMC_OK;
}

using FccKernel = void (*)(FccStep, int);

template <bool IS_INT>
FccKernel pick_fcc(int nshells)
{
    return nshells == 1 ? k_fcc_ministep<IS_INT, 1> : (nshells == 2 ? k_fcc_ministep<IS_INT, 2> : k_fcc_ministep<IS_INT, 3>);
}

}  // namespace

bool fcc_shape_ok(const smc_lattice *lat)
{
    return lat->nx >= 8 && lat->ny >= 8 && lat->nz >= 8 && lat->nx % 4 == 0 && lat->ny % 4 == 0 && lat->nz % 4 == 0 &&
           4LL * lat->nx * lat->ny * lat->nz < (1LL << 31);
}

smc_status launch_fcc_sweep(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                            int64_t *n_acc, float *trace_dE, uint8_t *trace_acc, int trace_k, cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    static FccParams P;
    st = fcc_params(lat, m, occ, P);
    if (st != SMC_OK) return st;
    const bool is_int = m->kind == SMC_PAIR_I32;
    P.seed = seed;
    P.replica = replica;
    const int nc = P.nA_cells;
    // integer acceptance tables, one per distinct kT of the call, back to back
    std::vector<uint32_t> tabs;
    std::vector<int2> tinfo((size_t)std::max(nsweeps, 1));
    std::map<double, int2> tindex;
    if (is_int)
        for (int t = 0; t < nsweeps; ++t) {
            auto it = tindex.find(kT[t]);
            if (it == tindex.end()) {
                const std::vector<uint32_t> tb = int_table(m->unit_ev, kT[t]);
                it = tindex.emplace(kT[t], make_int2((int)tabs.size(), (int)tb.size())).first;
                tabs.insert(tabs.end(), tb.begin(), tb.end());
            }
            tinfo[t] = it->second;
        }
    const bool is_qsro = m->kind == SMC_QSRO_F32;
    std::vector<uint32_t> words;
    st = is_qsro ? fcc_qsro_tables(lat, m, words) : fcc_sweep_tables(lat, m, words);
    if (st != SMC_OK) return st;
    // workspace: [part_e | part_n | ministep tables | acceptance tables | qSRO count cache]
    const size_t off_pn = (size_t)nc * 8, off_w = off_pn + (size_t)nc * 8, off_tab = off_w + words.size() * 4;
    const size_t off_q = (off_tab + tabs.size() * 4 + 255) / 256 * 256;
    const size_t N = 4ull * lat->nx * lat->ny * lat->nz;
    const size_t qbytes = m->nshells == 3 ? 2 : 1;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_q + (is_qsro ? N * qbytes : 16), &st);
    if (!scr) return st;
    cudaError_t e = cudaMemsetAsync(scr, 0, off_w, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(FCC partial sums)");
    e = cudaMemcpyAsync(scr + off_w, words.data(), words.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(FCC tables)");
    if (!tabs.empty()) {
        e = cudaMemcpyAsync(scr + off_tab, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(acceptance tables)");
    }
    P.tables = (const uint32_t *)(scr + off_w);
    P.tab = (const uint32_t *)(scr + off_tab);
    P.part_e = (double *)scr;
    P.part_n = (long long *)(scr + off_pn);
    const int threads = 256;
    P.n_int = (P.NLx > 2 && P.NLy > 2 && P.NLz > 2) ? (P.NLx - 2) * (P.NLy - 2) * (P.NLz - 2) : 0;
    P.n_bnd = nc - P.n_int;
    P.bnd_blocks = (P.n_bnd + threads - 1) / threads;
    const int blocks = P.bnd_blocks + (P.n_int + threads - 1) / threads;
    const FccKernel kern = is_qsro ? (m->nshells == 1 ? k_fcc_qsro_ministep<1>
                                                       : (m->nshells == 2 ? k_fcc_qsro_ministep<2> : k_fcc_qsro_ministep<3>))
                                   : (is_int ? pick_fcc<true>(m->nshells) : pick_fcc<false>(m->nshells));
    if (is_qsro) {  // the count cache, from the occupancy at the start of every call
        P.qcache = scr + off_q;
        const int cb = (int)std::max<size_t>(1, std::min<size_t>((N + 255) / 256, (size_t)ws->num_sms * 16));
        k_fcc_qsro_cache<<<cb, 256, 0, stream>>>(static_cast<const FccStep &>(P));
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_fcc_qsro_cache");
    }
    for (int t = 0; t < nsweeps; ++t) {
        P.sweep = sweep0 + (uint64_t)t;
        P.beta = (float)(1.0 / kT[t]);
        P.tinfo = tinfo[t];
        const int k0 = trace_k >= 0 ? trace_k : 0, k1 = trace_k >= 0 ? trace_k + 1 : 256;
        P.dE_out = trace_dE;
        P.acc_out = trace_acc;
        const FccStep step = P;
        for (int k = k0; k < k1; ++k) kern<<<blocks, threads, 0, stream>>>(step, k);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_fcc_ministep");
    }
    if (e_acc || n_acc) {
        k_fcc_reduce<<<1, kFccReduceThreads, 0, stream>>>(P.part_e, P.part_n, nc, e_acc, (long long *)n_acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_fcc_reduce");
    }
    return SMC_OK;
}

smc_status launch_fcc_energy(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e,
                             int64_t *e_int, cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    static FccParams P;
    st = fcc_params(lat, m, const_cast<int8_t *>(occ), P);
    if (st != SMC_OK) return st;
    // [ordered pair counts n_m^{pq} | qSRO squared own-species counts Q_m^p]
    const size_t cbytes = sizeof(unsigned long long) * kMaxShells * (64 + kMaxSpecies);
    unsigned long long *cnt = (unsigned long long *)workspace_scratch(ws, cbytes, &st);
    if (!cnt) return st;
    cudaError_t err = cudaMemsetAsync(cnt, 0, cbytes, stream);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync(FCC counts)");
    const bool is_qsro = m->kind == SMC_QSRO_F32;
    if (is_qsro) P.qcache = cnt;  // marks the qSRO energy (not dereferenced)
    const long long N = 4LL * lat->nx * lat->ny * lat->nz;
    const int blocks = (int)std::max(1LL, std::min<long long>((N + 255) / 256, (long long)ws->num_sms * 8));
    k_fcc_pair_counts<<<blocks, 256, 0, stream>>>(P, cnt, is_qsro ? cnt + kMaxShells * 64 : nullptr);
    err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "k_fcc_pair_counts");
    k_fcc_energy_finish<<<1, 32, 0, stream>>>(P, cnt, m->kind == SMC_PAIR_I32 ? 1 : 0, m->unit_ev, e,
                                              (long long *)e_int);
    err = cudaGetLastError();
    return err == cudaSuccess ? SMC_OK : cuda_fail(err, "k_fcc_energy_finish");
}

}  // namespace smc
