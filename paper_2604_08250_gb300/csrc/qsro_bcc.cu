// qsro_bcc.cu -- qSRO sweeps on the BCC lattice (Sec. IV-B, Eq.
// quadratic_local_SRO; Algorithm 1 with 4x4x4 link cells, 128 mini-steps):
// one thread per trial and one launch per mini-step, the trials of a
// mini-step being independent (read/write sets pinned on the CPU).
//
// Site j's energy changes only through the species of its neighbours a and
// b: with a in shell ma of j and b in shell mb (0 = neither),
//   linear part  D_ma(s_j) - D_mb(s_j),  D_m(q) = (V_m(B,q) - V_m(A,q)) / z_m,
//   W part       (s_j = A or B) from j's cached own-species counts,
// and a and b, changing their own species, add the same linear terms again
// (V symmetric) and W parts from the A / B counts around each (b in a's
// shell 1, a in b's).  C cancels.  On the BCC lattice no site has a and b in
// one shell (they sit on different sublattices), so every zone site of
// species A or B changes its W term.  The zone (14 / 20 / 38 sites besides a
// and b for 1 / 2 / 3 shells) is walked from a per-direction table of
// half-unit offsets sorted by (shell to a, shell to b), so both shells are
// compile-time constants in the unrolled walk.  Link cells off every box
// face reach the zone as id + delta(sublattice, offset); those on the faces
// run in the first blocks with wrapped coordinates.  The own-species count
// cache (bit fields of 4, 3, 4 bits for shells 1-3) is built from the
// occupancy at the start of every call and updated by accepting trials; the
// traced mini-step rebuilds it, so a sweep equals its traced mini-steps bit
// for bit.  Random numbers as for the pair sweep: word s & 3 of
// Philox4x32-10(key seed, counter (s >> 2, replica, sweep lo, sweep hi)),
// partner direction word >> 29, r = word & (2^29 - 1).
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "sweep_common.cuh"

namespace smc {

namespace {

// Per-call tables (32-bit words, staged into shared memory by every block):
// Dz[m][A][B][q] = (V_m(B,q) - V_m(A,q)) / z_m at m * 512 + (A * 8 + B) * 8 + q,
// Wz[m][p] = W_m^p / z_m^2 at kBqW + m * 8 + p, per partner direction the
// zone's offset indices w = (x+3) + 7 (y+3) + 49 (z+3) (half units) in
// category order at kBqZ, the partner's offset index at kBqV1 + dir, and the
// site-index delta of every offset per sublattice at kBqDel + sub * 343.
constexpr int kBqZmax = 38, kBqT = kMaxShells * 512, kBqW = kBqT, kBqZ = kBqW + kMaxShells * 8,
              kBqV1 = kBqZ + 8 * kBqZmax, kBqDel = kBqV1 + 8, kBqWords = kBqDel + 2 * 343;

struct BqStep {
    int nx, ny, nz, nshells, nA_cells;
    int NLx, NLy, NLz;
    int n_int, n_bnd, bnd_blocks;  // interior / face link cells, blocks of the face part (run first)
    const uint32_t *tables;
    uint64_t seed;
    uint32_t replica;
    uint64_t sweep;
    float beta;
    int8_t *occ;
    double *part_e;  // per link cell, accumulated over a call
    long long *part_n;
    float *dE_out;  // trace (nullable)
    uint8_t *acc_out;
    void *qcache;  // own-species counts per shell of every site (1 byte for 1-2 shells, 2 for 3)
};

__host__ __device__ constexpr int bq_qoff(int m) { return m == 0 ? 0 : (m == 1 ? 4 : 7); }
__host__ __device__ constexpr int bq_qmask(int m) { return m == 1 ? 7 : 15; }

// Zone categories, (shell to a) * 4 + (shell to b), and their sizes (the same
// for all 8 partner directions, equivalent under the cubic point group).
__host__ __device__ constexpr int bq_ncat(int nsh) { return nsh == 1 ? 2 : (nsh == 2 ? 6 : 10); }
__host__ __device__ constexpr int bq_cat(int nsh, int i, int *count)
{
    constexpr int c1[2][2] = {{4, 7}, {1, 7}};
    constexpr int c2[6][2] = {{4, 4}, {8, 3}, {1, 4}, {2, 3}, {6, 3}, {9, 3}};
    constexpr int c3[10][2] = {{4, 1}, {8, 3}, {12, 9}, {1, 1}, {2, 3}, {3, 9}, {6, 3}, {7, 3}, {9, 3}, {13, 3}};
    const int *e = nsh == 1 ? c1[i] : (nsh == 2 ? c2[i] : c3[i]);
    *count = e[1];
    return e[0];
}
__host__ __device__ constexpr int bq_code(int nsh, int e)
{
    int n = 0, code = 0;
    for (int i = 0; i < bq_ncat(nsh); ++i) {
        code = bq_cat(nsh, i, &n);
        if (e < n) return code;
        e -= n;
    }
    return 0;
}

__device__ __forceinline__ int3 bq_woff(int w) { return make_int3(w % 7 - 3, (w / 7) % 7 - 3, w / 49 - 3); }

// Site at half-unit position (px, py, pz) (equal parities), wrapped.
__device__ __forceinline__ int bq_site_at(const BqStep &P, int px, int py, int pz)
{
    const int sub = px & 1;
    const int cx = wrapc((px - sub) >> 1, P.nx), cy = wrapc((py - sub) >> 1, P.ny), cz = wrapc((pz - sub) >> 1, P.nz);
    return ((sub * P.nz + cz) * P.ny + cy) * P.nx + cx;
}

// The t-th link cell on the box faces: z faces, then y faces, then x faces.
__device__ __forceinline__ int3 bq_face_cell(int j, int NLx, int NLy, int NLz)
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

__constant__ signed char c_bq_vec[4][12][3];  // shells 1-3 at [1..3]
__constant__ int c_bq_n[4];

__global__ void __launch_bounds__(256) k_bq_cache(const __grid_constant__ BqStep P)
{
    const long long N = 2LL * P.nx * P.ny * P.nz;
    for (long long si = blockIdx.x * (long long)blockDim.x + threadIdx.x; si < N;
         si += (long long)gridDim.x * blockDim.x) {
        const int s = (int)si;
        const int p = P.occ[s] & 7;
        const int x = s % P.nx, y = (s / P.nx) % P.ny, z = (s / (P.nx * P.ny)) % P.nz, sub = s / (P.nx * P.ny * P.nz);
        const int px = 2 * x + sub, py = 2 * y + sub, pz = 2 * z + sub;
        uint32_t q = 0;
        for (int m = 1; m <= P.nshells; ++m)
            for (int t = 0; t < c_bq_n[m]; ++t) {
                const signed char *v = c_bq_vec[m][t];
                if ((P.occ[bq_site_at(P, px + v[0], py + v[1], pz + v[2])] & 7) == p) q += 1u << bq_qoff(m - 1);
            }
        if (P.nshells == 3)
            static_cast<uint16_t *>(P.qcache)[s] = (uint16_t)q;
        else
            static_cast<uint8_t *>(P.qcache)[s] = (uint8_t)q;
    }
}

template <int NSH>
__global__ void __launch_bounds__(256) k_bq_ministep(const __grid_constant__ BqStep P, int k)
{
    using QT = typename std::conditional<NSH == 3, uint16_t, uint8_t>::type;
    constexpr int NZ = NSH == 1 ? 14 : (NSH == 2 ? 20 : 38);
    __shared__ uint32_t sm[kBqWords];
    for (int i = threadIdx.x; i < kBqWords; i += blockDim.x) sm[i] = __ldg(P.tables + i);
    __syncthreads();
    const float *sT = reinterpret_cast<const float *>(sm);
    const float *sW = reinterpret_cast<const float *>(sm + kBqW);
    const int *sZ = reinterpret_cast<const int *>(sm + kBqZ);
    const int *sV1 = reinterpret_cast<const int *>(sm + kBqV1);

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
        cc = bq_face_cell(j, P.NLx, P.NLy, P.NLz);
    }
    const int c = (cc.z * P.NLy + cc.y) * P.NLx + cc.x;
    const int x = 4 * cc.x + dx, y = 4 * cc.y + dy, z = 4 * cc.z + dz;
    const int a = ((sub * P.nz + z) * P.ny + y) * P.nx + x;
    const uint32_t word = site_word(P.seed, P.replica, P.sweep, (uint32_t)a);
    const uint32_t r = word & kRMask;
    const int dir = (int)(word >> kRBits);
    const int pax = 2 * x + sub, pay = 2 * y + sub, paz = 2 * z + sub;
    const int *del = reinterpret_cast<const int *>(sm + kBqDel) + sub * 343;
    const int wb = sV1[dir];
    const int3 v1 = bq_woff(wb);
    const int b = interior ? a + del[wb] : bq_site_at(P, pax + v1.x, pay + v1.y, paz + v1.z);
    int8_t *occ = P.occ;
    QT *Qc = static_cast<QT *>(P.qcache);
    const int A = occ[a] & 7, B = occ[b] & 7;
    const int *zone = sZ + dir * kBqZmax;
    auto site = [&](int e) {
        const int w = zone[e];
        if (interior) return a + del[w];
        const int3 d = bq_woff(w);
        return bq_site_at(P, pax + d.x, pay + d.y, paz + d.z);
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
            const int code = bq_code(NSH, e), ma = code >> 2, mb = code & 3;
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
            const int q = Qc[j];
            zq[e] = (uint32_t)sj | (uint32_t)q << 4;
            float t = 0.f;  // a leaves j's shell ma as A and arrives as B; b the reverse in shell mb
            if (ma) {
                const int n = (q >> bq_qoff(ma - 1)) & bq_qmask(ma - 1);
                t += isA ? wA[ma - 1] * (float)(1 - 2 * n) : (isB ? wB[ma - 1] * (float)(2 * n + 1) : 0.f);
            }
            if (mb) {
                const int n = (q >> bq_qoff(mb - 1)) & bq_qmask(mb - 1);
                t += isA ? wA[mb - 1] * (float)(2 * n + 1) : (isB ? wB[mb - 1] * (float)(1 - 2 * n) : 0.f);
            }
            wz += t;
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
    const bool acc = metropolis<false>(dE, r, P.beta, nullptr, make_int2(0, 0));
    if (acc) {
        if (A != B) {
            occ[a] = (int8_t)B;
            occ[b] = (int8_t)A;
            int qa = 0, qb = 0;  // a now B: its B neighbours other than b; b now A likewise
#pragma unroll
            for (int m = 0; m < NSH; ++m) {
                qa += (int)(((cBa >> (8 * m)) & 255u) - (m == 0 ? 1u : 0u)) << bq_qoff(m);
                qb += (int)(((cAb >> (8 * m)) & 255u) - (m == 0 ? 1u : 0u)) << bq_qoff(m);
            }
            Qc[a] = (QT)qa;
            Qc[b] = (QT)qb;
#pragma unroll
            for (int e = 0; e < NZ; ++e) {
                const int code = bq_code(NSH, e), ma = code >> 2, mb = code & 3;
                const int sj = (int)(zq[e] & 15u), q = (int)(zq[e] >> 4);
                // A sites lose a (shell ma) and gain b (shell mb); B sites the reverse
                const int d = (ma ? 1 << bq_qoff(ma - 1) : 0) - (mb ? 1 << bq_qoff(mb - 1) : 0);
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

// e_acc += sum of part_e, n_acc += sum of part_n, in a fixed order.
constexpr int kBqReduceThreads = 1024;
__global__ void __launch_bounds__(kBqReduceThreads) k_bq_reduce(const double *part_e, const long long *part_n, int n,
                                                                double *e_acc, long long *n_acc)
{
    __shared__ double se[kBqReduceThreads];
    __shared__ long long sn[kBqReduceThreads];
    const int t = threadIdx.x;
    double e = 0.0;
    long long cnt = 0;
    for (int i = t; i < n; i += kBqReduceThreads) {
        e += part_e[i];
        cnt += part_n[i];
    }
    se[t] = e;
    sn[t] = cnt;
    __syncthreads();
    for (int h = kBqReduceThreads / 2; h > 0; h >>= 1) {
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

// BCC shells in half units: (+-1,+-1,+-1), (+-2,0,0) and permutations,
// (+-2,+-2,0) and permutations.
int bq_shell(int x, int y, int z, int nsh)
{
    const bool same = ((x & 1) == (y & 1)) && ((y & 1) == (z & 1));
    if (!same) return 0;
    int ax[3] = {std::abs(x), std::abs(y), std::abs(z)};
    std::sort(ax, ax + 3);
    const int m = (ax[0] == 1 && ax[1] == 1 && ax[2] == 1) ? 1
                  : (ax[0] == 0 && ax[1] == 0 && ax[2] == 2) ? 2
                  : (ax[0] == 0 && ax[1] == 2 && ax[2] == 2) ? 3
                                                              : 0;
    return m <= nsh ? m : 0;
}

uint64_t g_bq_shells = 0;  // bit d: the shell vectors are on device d (each device has its own copy)

smc_status bq_shell_tables()
{
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return cuda_fail(de, "cudaGetDevice");
    if (dev < 64 && (g_bq_shells >> dev & 1u)) return SMC_OK;
    signed char v[4][12][3] = {};
    int n[4] = {0, 0, 0, 0};
    for (int x = -2; x <= 2; ++x)
        for (int y = -2; y <= 2; ++y)
            for (int z = -2; z <= 2; ++z) {
                const int m = bq_shell(x, y, z, 3);
                if (!m) continue;
                v[m][n[m]][0] = (signed char)x;
                v[m][n[m]][1] = (signed char)y;
                v[m][n[m]][2] = (signed char)z;
                ++n[m];
            }
    if (n[1] != 8 || n[2] != 6 || n[3] != 12) {
        set_error("internal error: BCC shell vectors");
        return SMC_ERR_STATE;
    }
    cudaError_t e = cudaMemcpyToSymbol(c_bq_vec, v, sizeof v);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_bq_n, n, sizeof n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(BCC shells)");
    if (dev < 64) g_bq_shells |= 1ull << dev;
    return SMC_OK;
}

smc_status bq_tables(const smc_lattice *lat, const smc_model *m, std::vector<uint32_t> &w)
{
    const int S = lat->nspecies, nsh = m->nshells;
    const double z[3] = {8.0, 6.0, 12.0};
    w.assign(kBqWords, 0u);
    for (int sh = 0; sh < nsh; ++sh) {
        for (int A = 0; A < S; ++A)
            for (int B = 0; B < S; ++B)
                for (int q = 0; q < S; ++q) {
                    const float d =
                        (float)(((double)m->v_f32[(sh * S + B) * S + q] - m->v_f32[(sh * S + A) * S + q]) / z[sh]);
                    memcpy(&w[sh * 512 + (A * 8 + B) * 8 + q], &d, 4);
                }
        for (int p = 0; p < S; ++p) {
            const float v = (float)((double)m->qsro_w[sh * S + p] / (z[sh] * z[sh]));
            memcpy(&w[kBqW + sh * 8 + p], &v, 4);
        }
    }
    auto widx = [](int x, int y, int zz) { return (x + 3) + 7 * (y + 3) + 49 * (zz + 3); };
    const int want = nsh == 1 ? 14 : (nsh == 2 ? 20 : 38);
    for (int d = 0; d < 8; ++d) {  // direction bits (kx, ky, kz) -> (2kx-1, 2ky-1, 2kz-1)
        const int v1[3] = {2 * ((d >> 2) & 1) - 1, 2 * ((d >> 1) & 1) - 1, 2 * (d & 1) - 1};
        w[kBqV1 + d] = (uint32_t)widx(v1[0], v1[1], v1[2]);
        std::vector<int> by_code[16];  // offsets by category code, each in lexicographic order
        for (int x = -3; x <= 3; ++x)
            for (int y = -3; y <= 3; ++y)
                for (int zz = -3; zz <= 3; ++zz) {
                    if ((x == 0 && y == 0 && zz == 0) || (x == v1[0] && y == v1[1] && zz == v1[2])) continue;
                    const int ma = bq_shell(x, y, zz, nsh), mb = bq_shell(x - v1[0], y - v1[1], zz - v1[2], nsh);
                    if (ma * 4 + mb) by_code[ma * 4 + mb].push_back(widx(x, y, zz));
                }
        int n = 0;
        for (int ci = 0; ci < bq_ncat(nsh); ++ci) {
            int cnt = 0;
            const int code = bq_cat(nsh, ci, &cnt);
            const int got = (int)by_code[code].size();
            if (got != cnt) {
                set_error("internal error: BCC qSRO zone category %d has %d sites (want %d)", code, got, cnt);
                return SMC_ERR_STATE;
            }
            for (int o : by_code[code])
                if (n < kBqZmax) w[kBqZ + d * kBqZmax + n++] = (uint32_t)o;
        }
        size_t total = 0;  // every zone site in a listed category
        for (int code = 0; code < 16; ++code) total += by_code[code].size();
        if (n != want || (int)total != want) {
            set_error("internal error: BCC qSRO zone has %d sites (want %d)", (int)total, want);
            return SMC_ERR_STATE;
        }
    }
    const long long NC = (long long)lat->nx * lat->ny * lat->nz;
    for (int sub = 0; sub < 2; ++sub)
        for (int x = -3; x <= 3; ++x)
            for (int y = -3; y <= 3; ++y)
                for (int zz = -3; zz <= 3; ++zz) {
                    const int qx = sub + x, qy = sub + y, qz = sub + zz;
                    const int ns = qx & 1;
                    if ((qy & 1) != ns || (qz & 1) != ns) continue;  // not a lattice site
                    const int dcx = (qx - ns) / 2, dcy = (qy - ns) / 2, dcz = (qz - ns) / 2;
                    const long long delta = (ns - sub) * NC + ((long long)dcz * lat->ny + dcy) * lat->nx + dcx;
                    w[kBqDel + sub * 343 + widx(x, y, zz)] = (uint32_t)(int32_t)delta;
                }
    return SMC_OK;
}

using BqKernel = void (*)(BqStep, int);

}  // namespace

smc_status launch_qsro_ministeps(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                                 uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                                 int64_t *n_acc, float *trace_dE, uint8_t *trace_acc, int trace_k,
                                 cudaStream_t stream)
{
    if (lc_edge(lat->nx) != 4 || lc_edge(lat->ny) != 4 || lc_edge(lat->nz) != 4) {
        set_error("qSRO sweeps need every axis a multiple of 4 cells and >= 8");
        return SMC_ERR_UNSUPPORTED;
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    st = bq_shell_tables();
    if (st != SMC_OK) return st;
    BqStep P;
    memset(&P, 0, sizeof P);
    P.nx = lat->nx;
    P.ny = lat->ny;
    P.nz = lat->nz;
    P.nshells = m->nshells;
    P.NLx = lat->nx / 4;
    P.NLy = lat->ny / 4;
    P.NLz = lat->nz / 4;
    P.nA_cells = P.NLx * P.NLy * P.NLz;
    P.occ = occ;
    P.seed = seed;
    P.replica = replica;
    const int nc = P.nA_cells;
    std::vector<uint32_t> words;
    st = bq_tables(lat, m, words);
    if (st != SMC_OK) return st;
    // workspace: [part_e | part_n | tables | count cache]
    const size_t off_pn = (size_t)nc * 8, off_w = off_pn + (size_t)nc * 8, off_q = (off_w + words.size() * 4 + 255) / 256 * 256;
    const size_t N = 2ull * lat->nx * lat->ny * lat->nz;
    const size_t qbytes = m->nshells == 3 ? 2 : 1;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_q + N * qbytes, &st);
    if (!scr) return st;
    cudaError_t e = cudaMemsetAsync(scr, 0, off_w, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(qSRO partial sums)");
    e = cudaMemcpyAsync(scr + off_w, words.data(), words.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(qSRO tables)");
    P.tables = (const uint32_t *)(scr + off_w);
    P.part_e = (double *)scr;
    P.part_n = (long long *)(scr + off_pn);
    P.qcache = scr + off_q;
    const int threads = 256;
    P.n_int = (P.NLx > 2 && P.NLy > 2 && P.NLz > 2) ? (P.NLx - 2) * (P.NLy - 2) * (P.NLz - 2) : 0;
    P.n_bnd = nc - P.n_int;
    P.bnd_blocks = (P.n_bnd + threads - 1) / threads;
    const int blocks = P.bnd_blocks + (P.n_int + threads - 1) / threads;
    const BqKernel kern = m->nshells == 1 ? k_bq_ministep<1> : (m->nshells == 2 ? k_bq_ministep<2> : k_bq_ministep<3>);
    const int cb = (int)std::max<size_t>(1, std::min<size_t>((N + 255) / 256, (size_t)ws->num_sms * 16));
    k_bq_cache<<<cb, 256, 0, stream>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_bq_cache");
    P.dE_out = trace_dE;
    P.acc_out = trace_acc;
    for (int t = 0; t < nsweeps; ++t) {
        P.sweep = sweep0 + (uint64_t)t;
        P.beta = (float)(1.0 / kT[t]);
        const int k0 = trace_k >= 0 ? trace_k : 0, k1 = trace_k >= 0 ? trace_k + 1 : 128;
        for (int k = k0; k < k1; ++k) kern<<<blocks, threads, 0, stream>>>(P, k);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_bq_ministep");
    }
    if (e_acc || n_acc) {
        k_bq_reduce<<<1, kBqReduceThreads, 0, stream>>>(P.part_e, P.part_n, nc, e_acc, (long long *)n_acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_bq_reduce");
    }
    return SMC_OK;
}

}  // namespace smc
