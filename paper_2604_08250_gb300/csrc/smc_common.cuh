// smc_common.cuh -- device helpers and internal interfaces of libsmc.so.
//
// Independent of the oracle: Philox, the BCC geometry and the link-cell
// schedule are written here from their definitions (Salmon et al., SC'11 for
// Philox4x32-10; Sec. II-A and Algorithm 1 of the paper for the schedule).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/smc.h"

namespace smc {

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds; each round multiplies words 0 and 2 by the two
// Philox constants, swaps the halves with a key-dependent xor, and the key
// advances by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ void mul_hilo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo)
{
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umulhi(a, b);
#else
    uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        uint32_t h0, l0, h1, l1;
        mul_hilo(0xD2511F53u, c.x, h0, l0);
        mul_hilo(0xCD9E8D57u, c.z, h1, l1);
        U4 n;
        n.x = h1 ^ c.y ^ k0;
        n.y = l1;
        n.z = h0 ^ c.w ^ k1;
        n.w = l0;
        c = n;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__host__ __device__ __forceinline__ uint32_t pick_word(const U4 &w, uint32_t idx)
{
    return idx == 0 ? w.x : (idx == 1 ? w.y : (idx == 2 ? w.z : w.w));
}

// Random word of canonical site s in sweep `sweep` of replica `rep`.
__device__ __forceinline__ uint32_t site_word(uint64_t seed, uint32_t rep, uint64_t sweep, uint32_t s)
{
    U4 c{s >> 2, rep, (uint32_t)sweep, (uint32_t)(sweep >> 32)};
    U4 w = philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    return pick_word(w, s & 3u);
}

constexpr int kRBits = 29;
constexpr uint32_t kRMask = (1u << kRBits) - 1u;
constexpr int kMaxSpecies = 8;
constexpr int kMaxShells = 3;
constexpr int kMaxReplicas = 64;

// Link-cell edge along an axis of n cells (Sec. II-A): 4 when the axis holds
// at least two 4-cell link cells, otherwise the whole axis.
__host__ __device__ __forceinline__ int lc_edge(int n)
{
    return (n >= 8 && (n % 4) == 0) ? 4 : n;
}

__device__ __forceinline__ int wrapc(int v, int n)
{
    // v in [-n, 2n)
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

// ---------------------------------------------------------------------------
// Device status word and bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Two 64-bit words with relaxed (single-copy atomic per word) semantics at
// GPU scope: the tagged exchange of the resident sweep.
__device__ __forceinline__ ulonglong2 ld_relaxed_v2u64(const unsigned long long *p)
{
    ulonglong2 v;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_v2u64(unsigned long long *p, unsigned long long a, unsigned long long b)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int *p)
{
    return *(volatile const int *)p;
}

// ---------------------------------------------------------------------------
// Host-side internals shared by the translation units.
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
smc_status cuda_fail(cudaError_t e, const char *what);

// Per-device workspace (grown with cudaMalloc, never shrunk).
struct Workspace {
    int device = -1;
    void *buf = nullptr;
    size_t cap = 0;
    int *status = nullptr;  // latched device status (first 16 bytes of buf)
    int num_sms = 0;
    size_t smem_optin = 0;
};
Workspace *workspace(smc_status *st);
// Ensures at least `bytes` of scratch after the status header; returns it.
void *workspace_scratch(Workspace *ws, size_t bytes, smc_status *st);

struct Tuning {
    int tile_y = 0, tile_z = 0, threads = 0, ctas_per_sm = 0;
};
Tuning current_tuning();
int64_t debug_timeout_ns();
int64_t debug_skip_tile();
int debug_fast_team();
int debug_fast_nbuf();
int debug_fast_stage();

bool lattice_valid(const smc_lattice *lat, bool mlp);
bool model_valid(const smc_lattice *lat, const smc_model *m);

// Launchers implemented in the .cu files.
smc_status launch_pair_sweep(int R, const smc_lattice *lats, const smc_model *m, int8_t *const *occ,
                             uint64_t seed, uint32_t replica0, uint64_t sweep0, int nsweeps,
                             const double *kT, double *e_acc, int64_t *n_acc, cudaStream_t stream);
smc_status launch_pair_sweep_noalloc(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                                     uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT,
                                     double *e_acc, int64_t *n_acc, int32_t *status, cudaStream_t stream);
smc_status launch_ministep_trace(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                                 uint32_t replica, uint64_t sweep, int k, double kT, float *dE,
                                 uint8_t *acc, cudaStream_t stream);
smc_status launch_slab_ministep(const smc_lattice *lat, const smc_model *m, int8_t *win, int x0, int w, int g,
                                uint64_t seed, uint32_t replica, uint64_t sweep, int k, double kT, double *e_acc,
                                int64_t *n_acc, int part, cudaStream_t stream);
// Warp count of a warp-per-tile kernel (warp w owns tiles w, w + NW, ...)
// that gives the busiest SM the fewest tiles (defined in sweep_pair.cu).
long long balanced_warps(long long ntiles, int nwarps, int per_sm, int num_sms);
std::vector<uint32_t> int_table(double unit_ev, double kT);
bool fcc_shape_ok(const smc_lattice *lat);
smc_status launch_fcc_sweep(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                            int64_t *n_acc, float *trace_dE, uint8_t *trace_acc, int trace_k, cudaStream_t stream);
smc_status launch_fcc_energy(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e,
                             int64_t *e_int, cudaStream_t stream);
smc_status launch_qsro_ministeps(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                                 uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                                 int64_t *n_acc, float *trace_dE, uint8_t *trace_acc, int trace_k,
                                 cudaStream_t stream);
smc_status launch_qsro_energy(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e,
                              cudaStream_t stream);
smc_status launch_qsro_grad(const smc_lattice *lat, const smc_model *m, const int8_t *occ, float *grad,
                            cudaStream_t stream);
smc_status launch_mlp_sweep(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                            int64_t *n_acc, cudaStream_t stream);
smc_status launch_mlp_trace(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep, int k, double kT, float *dE, uint8_t *acc,
                            cudaStream_t stream);
smc_status launch_mlp_energy(const smc_lattice *lat, const smc_model *m, const int8_t *occ, double *e,
                             cudaStream_t stream);
smc_status launch_mlp_grad(const smc_lattice *lat, const smc_model *m, const int8_t *occ, float *grad,
                           cudaStream_t stream);
smc_status launch_pair_counts(const smc_lattice *lat, int nshells, const int8_t *occ, unsigned long long *counts,
                              cudaStream_t stream);
smc_status launch_init(const smc_lattice *lat, const int64_t *counts, uint64_t seed, uint32_t replica,
                       int8_t *occ, cudaStream_t stream);
smc_status launch_philox(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                         cudaStream_t stream);
smc_status launch_sro_finish(const smc_lattice *lat, int nshells, const unsigned long long *counts,
                             double *alpha, cudaStream_t stream);
smc_status launch_energy_finish(const smc_lattice *lat, const smc_model *m,
                                const unsigned long long *counts, double *e, int64_t *e_int,
                                cudaStream_t stream);
smc_status launch_pair_grad_finish(const smc_lattice *lat, const smc_model *m,
                                   const unsigned long long *counts, float *grad, cudaStream_t stream);

}  // namespace smc
