// fcc.cu -- swap Monte Carlo on the FCC lattice (the paper's lattice, Sec.
// IV-C; 4x4x4 link cells and 256 mini-steps as in Sec. V-C) with pair models.
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
// one bond.  The same kernel records the trace (dE, decision) of a
// mini-step, so a sweep equals its traced mini-steps bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "sweep_common.cuh"

namespace smc {

namespace {

struct FccParams {
    int nx, ny, nz, S, nshells, nA_cells;  // nA_cells: link cells (trials per mini-step)
    int NLx, NLy;
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
    int vi[kMaxShells * kMaxSpecies * kMaxSpecies];
    float vf[kMaxShells * kMaxSpecies * kMaxSpecies];
};

__constant__ signed char c_fcc_vec[4][24][3];  // shells 1-3 at [1..3]
__constant__ int c_fcc_n[4];

__device__ __forceinline__ int fcc_neighbor(const FccParams &P, int s, const signed char *v)
{
    int t = s;
    const int x = t % P.nx;
    t /= P.nx;
    const int y = t % P.ny;
    t /= P.ny;
    const int z = t % P.nz;
    const int sub = t / P.nz;
    const int bx = (sub == 1 || sub == 2) ? 1 : 0, by = (sub == 1 || sub == 3) ? 1 : 0,
              bz = (sub == 2 || sub == 3) ? 1 : 0;
    const int px = 2 * x + bx + v[0], py = 2 * y + by + v[1], pz = 2 * z + bz + v[2];
    const int ox = px & 1, oy = py & 1, oz = pz & 1;
    const int nsub = ox ? (oy ? 1 : 2) : (oy ? 3 : 0);
    const int cx = wrapc((px - ox) >> 1, P.nx), cy = wrapc((py - oy) >> 1, P.ny), cz = wrapc((pz - oz) >> 1, P.nz);
    return ((nsub * P.nz + cz) * P.ny + cy) * P.nx + cx;
}

template <bool IS_INT>
__global__ void __launch_bounds__(256) k_fcc_ministep(const __grid_constant__ FccParams P, int k)
{
    using T = typename Acc<IS_INT>::T;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= P.nA_cells) return;
    const int dx = k & 3, dy = (k >> 2) & 3, dz = (k >> 4) & 3, sub = k >> 6;
    const int cx = c % P.NLx, cy = (c / P.NLx) % P.NLy, cz = c / (P.NLx * P.NLy);
    const int a = ((sub * P.nz + 4 * cz + dz) * P.ny + 4 * cy + dy) * P.nx + 4 * cx + dx;
    const U4 w = philox10(U4{(uint32_t)a, P.replica, (uint32_t)P.sweep, (uint32_t)(P.sweep >> 32)}, (uint32_t)P.seed,
                          (uint32_t)(P.seed >> 32));
    const uint32_t r = w.x & kRMask;
    const int dir = (int)(((uint64_t)w.y * 12u) >> 32);
    const int b = fcc_neighbor(P, a, c_fcc_vec[1][dir]);
    int8_t *occ = P.occ;
    const int A = occ[a] & 7, B = occ[b] & 7, S = P.S;
    // integer models sum in 64 bits (84 terms of |V| <= 2^24 can pass 2^31)
    using Wide = typename std::conditional<IS_INT, long long, float>::type;
    Wide dw = Wide(0);
    for (int m = 1; m <= P.nshells; ++m) {
        const int base = (m - 1) * S * S;
        for (int t = 0; t < c_fcc_n[m]; ++t) {
            const int ja = fcc_neighbor(P, a, c_fcc_vec[m][t]);
            if (ja != b) {
                const int q = occ[ja] & 7;
                if constexpr (IS_INT)
                    dw += (long long)P.vi[base + B * S + q] - P.vi[base + A * S + q];
                else
                    dw += P.vf[base + B * S + q] - P.vf[base + A * S + q];
            }
            const int jb = fcc_neighbor(P, b, c_fcc_vec[m][t]);
            if (jb != a) {
                const int q = occ[jb] & 7;
                if constexpr (IS_INT)
                    dw += (long long)P.vi[base + A * S + q] - P.vi[base + B * S + q];
                else
                    dw += P.vf[base + A * S + q] - P.vf[base + B * S + q];
            }
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

// e_acc += sum of part_e, n_acc += sum of part_n, in link-cell order.
__global__ void k_fcc_reduce(const double *part_e, const long long *part_n, int n, double *e_acc, long long *n_acc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double e = 0.0;
    long long c = 0;
    for (int i = 0; i < n; ++i) {
        e += part_e[i];
        c += part_n[i];
    }
    if (e_acc) *e_acc += e;
    if (n_acc) *n_acc += c;
}

// Ordered pair counts n_m^{pq} (each site's shell-m neighbours), per-block
// shared counters flushed with 64-bit atomics.
__global__ void __launch_bounds__(256) k_fcc_pair_counts(const __grid_constant__ FccParams P,
                                                         unsigned long long *counts)
{
    __shared__ unsigned int cnt[kMaxShells * kMaxSpecies * kMaxSpecies];
    for (int i = threadIdx.x; i < kMaxShells * kMaxSpecies * kMaxSpecies; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    const int N = 4 * P.nx * P.ny * P.nz, S = P.S;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int p = P.occ[s] & 7;
        for (int m = 1; m <= P.nshells; ++m)
            for (int t = 0; t < c_fcc_n[m]; ++t) {
                const int q = P.occ[fcc_neighbor(P, s, c_fcc_vec[m][t])] & 7;
                atomicAdd(&cnt[((m - 1) * S + p) * S + q], 1u);
            }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P.nshells * S * S; i += blockDim.x)
        if (cnt[i]) atomicAdd(counts + i, (unsigned long long)cnt[i]);
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
    } else if (e) {
        double tot = 0.0;
        for (int i = 0; i < n; ++i) tot += (double)P.vf[i] * (double)counts[i];
        *e = 0.5 * tot;
    }
}

bool g_fcc_tables = false;

smc_status fcc_tables()
{
    if (g_fcc_tables) return SMC_OK;
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
    g_fcc_tables = true;
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
    P.nA_cells = (lat->nx / 4) * (lat->ny / 4) * (lat->nz / 4);
    P.occ = occ;
    const int n = m->nshells * P.S * P.S;
    for (int i = 0; i < n; ++i) {
        if (m->kind == SMC_PAIR_I32)
            P.vi[i] = m->v_i32[i];
        else
            P.vf[i] = m->v_f32[i];
    }
    return fcc_tables();
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
    // workspace: [part_e | part_n | acceptance tables]
    std::vector<uint32_t> tabs;
    std::vector<int2> tinfo((size_t)std::max(nsweeps, 1));
    if (is_int)
        for (int t = 0; t < nsweeps; ++t) {
            const std::vector<uint32_t> tb = int_table(m->unit_ev, kT[t]);
            tinfo[t] = make_int2((int)tabs.size(), (int)tb.size());
            tabs.insert(tabs.end(), tb.begin(), tb.end());
        }
    const size_t off_pn = (size_t)nc * 8, off_tab = off_pn + (size_t)nc * 8;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_tab + tabs.size() * 4 + 16, &st);
    if (!scr) return st;
    cudaError_t e = cudaMemsetAsync(scr, 0, off_tab, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(FCC partial sums)");
    if (!tabs.empty()) {
        e = cudaMemcpyAsync(scr + off_tab, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(acceptance tables)");
    }
    P.tab = (const uint32_t *)(scr + off_tab);
    P.part_e = (double *)scr;
    P.part_n = (long long *)(scr + off_pn);
    const int threads = 256, blocks = (nc + threads - 1) / threads;
    auto kern = is_int ? k_fcc_ministep<true> : k_fcc_ministep<false>;
    for (int t = 0; t < nsweeps; ++t) {
        P.sweep = sweep0 + (uint64_t)t;
        P.beta = (float)(1.0 / kT[t]);
        P.tinfo = tinfo[t];
        const int k0 = trace_k >= 0 ? trace_k : 0, k1 = trace_k >= 0 ? trace_k + 1 : 256;
        P.dE_out = trace_dE;
        P.acc_out = trace_acc;
        for (int k = k0; k < k1; ++k) kern<<<blocks, threads, 0, stream>>>(P, k);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_fcc_ministep");
    }
    if (e_acc || n_acc) {
        k_fcc_reduce<<<1, 32, 0, stream>>>(P.part_e, P.part_n, nc, e_acc, (long long *)n_acc);
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
    unsigned long long *cnt =
        (unsigned long long *)workspace_scratch(ws, sizeof(unsigned long long) * kMaxShells * 64, &st);
    if (!cnt) return st;
    cudaError_t err = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * kMaxShells * 64, stream);
    if (err != cudaSuccess) return cuda_fail(err, "cudaMemsetAsync(FCC counts)");
    const long long N = 4LL * lat->nx * lat->ny * lat->nz;
    const int blocks = (int)std::max(1LL, std::min<long long>((N + 255) / 256, (long long)ws->num_sms * 8));
    k_fcc_pair_counts<<<blocks, 256, 0, stream>>>(P, cnt);
    err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "k_fcc_pair_counts");
    k_fcc_energy_finish<<<1, 32, 0, stream>>>(P, cnt, m->kind == SMC_PAIR_I32 ? 1 : 0, m->unit_ev, e,
                                              (long long *)e_int);
    err = cudaGetLastError();
    return err == cudaSuccess ? SMC_OK : cuda_fail(err, "k_fcc_energy_finish");
}

}  // namespace smc
