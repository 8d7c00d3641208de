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

#include "smc_common.cuh"

namespace smc {

// Per-site neighbour histograms, packed 8 bits per species, reduced across
// the warp with redux.sync per (p, q) and accumulated in shared memory.
__global__ void __launch_bounds__(256) k_pair_counts(const int8_t *__restrict__ occ, int nx, int ny, int nz,
                                                     int nshells, int S, unsigned long long *counts)
{
    __shared__ unsigned int bins[kMaxShells * kMaxSpecies * kMaxSpecies];
    for (int i = threadIdx.x; i < kMaxShells * kMaxSpecies * kMaxSpecies; i += blockDim.x) bins[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const long long N = 2LL * nx * ny * nz;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwt = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long s0 = wid * 32; s0 < N; s0 += nwt * 32) {
        const long long s = s0 + lane;
        const bool valid = s < N;
        int p = -1, x = 0, y = 0, z = 0, sub = 0;
        if (valid) {
            long long t = s;
            x = (int)(t % nx);
            t /= nx;
            y = (int)(t % ny);
            t /= ny;
            z = (int)(t % nz);
            sub = (int)(t / nz);
            p = occ[s] & 7;
        }
        auto at = [&](int sb, int xx, int yy, int zz) -> int {
            xx = wrapc(xx, nx);
            yy = wrapc(yy, ny);
            zz = wrapc(zz, nz);
            return occ[((size_t)((sb * nz + zz) * ny + yy)) * nx + xx] & 7;
        };
        for (int m = 0; m < nshells; ++m) {
            unsigned long long h = 0;
            if (valid) {
                if (m == 0) {
                    const int o = sub == 0 ? -1 : 0;  // other-sublattice cells x+o .. x+o+1
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        h += 1ull << (8 * at(1 - sub, x + o + ((u >> 2) & 1), y + o + ((u >> 1) & 1), z + o + (u & 1)));
                } else if (m == 1) {
                    h += 1ull << (8 * at(sub, x - 1, y, z));
                    h += 1ull << (8 * at(sub, x + 1, y, z));
                    h += 1ull << (8 * at(sub, x, y - 1, z));
                    h += 1ull << (8 * at(sub, x, y + 1, z));
                    h += 1ull << (8 * at(sub, x, y, z - 1));
                    h += 1ull << (8 * at(sub, x, y, z + 1));
                } else {
#pragma unroll
                    for (int a = -1; a <= 1; a += 2)
#pragma unroll
                        for (int b = -1; b <= 1; b += 2) {
                            h += 1ull << (8 * at(sub, x + a, y + b, z));
                            h += 1ull << (8 * at(sub, x + a, y, z + b));
                            h += 1ull << (8 * at(sub, x, y + a, z + b));
                        }
                }
            }
            for (int q = 0; q < S; ++q) {
                const unsigned cnt = (unsigned)((h >> (8 * q)) & 0xFFu);
                for (int pp = 0; pp < S; ++pp) {
                    const unsigned tot = __reduce_add_sync(0xffffffffu, p == pp ? cnt : 0u);
                    if (lane == 0 && tot) atomicAdd(&bins[(m * kMaxSpecies + pp) * kMaxSpecies + q], tot);
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nshells * kMaxSpecies * kMaxSpecies; i += blockDim.x) {
        const int m = i / (kMaxSpecies * kMaxSpecies), p = (i / kMaxSpecies) % kMaxSpecies, q = i % kMaxSpecies;
        if (p < S && q < S && bins[i]) atomicAdd(counts + (m * S + p) * S + q, (unsigned long long)bins[i]);
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
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const int threads = 256;
    const long long want = (N + threads - 1) / threads;
    const int blocks = (int)std::min<long long>(want, (long long)ws->num_sms * 8);
    k_pair_counts<<<blocks, threads, 0, stream>>>(occ, lat->nx, lat->ny, lat->nz, nshells, S, counts);
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
