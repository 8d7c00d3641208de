// init.cu -- composition-conserving random initial configuration.
//
// Definition: sites ordered by the compound key K(s) = (k64(s), s), with
// k64(s) = (hi(s) << 32) | lo(s), hi/lo the Philox words of site s at the two
// reserved sweep indices; the sites at sorted positions [C_{p}, C_{p+1}) get
// species p (C = cumulative counts).
//
// No sort is needed: species(s) = #{t : K(s) >= T_t}, where T_t is the
// element of rank C_t.  Each T_t is found by a most-significant-digit radix
// select over the 12 bytes of K (one histogram pass per byte, all thresholds
// at once), recomputing the keys from Philox on every pass.
#include <algorithm>
#include <vector>

#include "smc_common.cuh"

namespace smc {

constexpr int kMaxTargets = kMaxSpecies - 1;

struct SelState {
    unsigned long long p64[kMaxTargets];  // known leading bytes of the key
    unsigned int p32[kMaxTargets];        // known leading bytes of the site id
    unsigned int rank[kMaxTargets];       // rank still to skip inside the prefix
    int active[kMaxTargets];              // 0: target beyond the last site
};

__device__ __forceinline__ void site_keys(uint64_t seed, uint32_t rep, uint32_t q, U4 &hi, U4 &lo)
{
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    hi = philox10(U4{q, rep, 0xFFFFFFFEu, 0xFFFFFFFFu}, k0, k1);
    lo = philox10(U4{q, rep, 0xFFFFFFFFu, 0xFFFFFFFFu}, k0, k1);
}

__device__ __forceinline__ bool prefix_match(unsigned long long k64, unsigned s, unsigned long long p64, unsigned p32,
                                             int d)
{
    if (d == 0) return true;
    if (d <= 8) {
        const int sh = 64 - 8 * d;
        return (k64 >> sh) == (p64 >> sh);
    }
    if (k64 != p64) return false;
    const int sh = 32 - 8 * (d - 8);
    return sh >= 32 ? true : (s >> sh) == (p32 >> sh);
}

__device__ __forceinline__ unsigned key_byte(unsigned long long k64, unsigned s, int d)
{
    return d < 8 ? (unsigned)((k64 >> (56 - 8 * d)) & 0xFF) : (s >> (24 - 8 * (d - 8))) & 0xFF;
}

__global__ void __launch_bounds__(256) k_init_hist(uint64_t seed, uint32_t rep, long long N, int ntarget, int d,
                                                   const SelState *st, unsigned *hist)
{
    __shared__ unsigned h[kMaxTargets * 256];
    __shared__ SelState ss;
    for (int i = threadIdx.x; i < ntarget * 256; i += blockDim.x) h[i] = 0;
    if (threadIdx.x == 0) ss = *st;
    __syncthreads();
    const long long nq = (N + 3) / 4;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        U4 hi, lo;
        site_keys(seed, rep, (uint32_t)q, hi, lo);
        for (int i = 0; i < 4; ++i) {
            const long long s = 4 * q + i;
            if (s >= N) break;
            const unsigned long long k64 = ((unsigned long long)pick_word(hi, i) << 32) | pick_word(lo, i);
            for (int t = 0; t < ntarget; ++t) {
                if (!ss.active[t]) continue;
                if (prefix_match(k64, (unsigned)s, ss.p64[t], ss.p32[t], d))
                    atomicAdd(&h[t * 256 + key_byte(k64, (unsigned)s, d)], 1u);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ntarget * 256; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, h[i]);
}

__global__ void k_init_select(int ntarget, int d, SelState *st, unsigned *hist)
{
    const int t = threadIdx.x;
    if (t < ntarget && st->active[t]) {
        unsigned r = st->rank[t], acc = 0;
        int b = 0;
        for (; b < 256; ++b) {
            const unsigned c = hist[t * 256 + b];
            if (acc + c > r) break;
            acc += c;
        }
        if (b == 256) b = 255;  // unreachable when the rank lies inside the prefix
        st->rank[t] = r - acc;
        if (d < 8)
            st->p64[t] |= (unsigned long long)b << (56 - 8 * d);
        else
            st->p32[t] |= (unsigned)b << (24 - 8 * (d - 8));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ntarget * 256; i += blockDim.x) hist[i] = 0;
}

__global__ void __launch_bounds__(256) k_init_assign(uint64_t seed, uint32_t rep, long long N, int ntarget,
                                                     const SelState *st, int8_t *occ)
{
    __shared__ SelState ss;
    if (threadIdx.x == 0) ss = *st;
    __syncthreads();
    const long long nq = (N + 3) / 4;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nq; q += (long long)gridDim.x * blockDim.x) {
        U4 hi, lo;
        site_keys(seed, rep, (uint32_t)q, hi, lo);
        for (int i = 0; i < 4; ++i) {
            const long long s = 4 * q + i;
            if (s >= N) break;
            const unsigned long long k64 = ((unsigned long long)pick_word(hi, i) << 32) | pick_word(lo, i);
            int sp = 0;
            for (int t = 0; t < ntarget; ++t)
                if (ss.active[t] && (k64 > ss.p64[t] || (k64 == ss.p64[t] && (unsigned)s >= ss.p32[t]))) ++sp;
            occ[s] = (int8_t)sp;
        }
    }
}

smc_status launch_init(const smc_lattice *lat, const int64_t *counts, uint64_t seed, uint32_t replica, int8_t *occ,
                       cudaStream_t stream)
{
    smc_status stt;
    Workspace *ws = workspace(&stt);
    if (!ws) return stt;
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const int ntarget = lat->nspecies - 1;
    SelState h0{};
    long long cum = 0;
    for (int t = 0; t < ntarget; ++t) {
        cum += counts[t];
        h0.rank[t] = (unsigned)cum;
        h0.active[t] = cum < N ? 1 : 0;
    }
    const size_t need = sizeof(SelState) + 16 + (size_t)kMaxTargets * 256 * 4;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, need, &stt);
    if (!scr) return stt;
    SelState *st = (SelState *)scr;
    unsigned *hist = (unsigned *)(scr + ((sizeof(SelState) + 15) / 16) * 16);
    cudaError_t e = cudaMemcpyAsync(st, &h0, sizeof h0, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(init state)");
    e = cudaMemsetAsync(hist, 0, (size_t)kMaxTargets * 256 * 4, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(init hist)");
    const int threads = 256;
    const long long nq = (N + 3) / 4;
    const int blocks = (int)std::max<long long>(1, std::min<long long>((nq + threads - 1) / threads, ws->num_sms * 8LL));
    if (ntarget > 0) {
        for (int d = 0; d < 12; ++d) {
            k_init_hist<<<blocks, threads, 0, stream>>>(seed, replica, N, ntarget, d, st, hist);
            k_init_select<<<1, 256, 0, stream>>>(ntarget, d, st, hist);
        }
    }
    k_init_assign<<<blocks, threads, 0, stream>>>(seed, replica, N, ntarget, st, occ);
    e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "init kernels");
}

}  // namespace smc
