// mlp_grad.cu -- dE/dtheta of the MLP energy E = sum_i f(x_i) with respect to
// every MLP parameter (W1, b1, W2, b2, W3, b3), by back-propagation at every
// site, on the tcgen05 tensor cores.
//
// For one site, with z1 = W1 x + b1, h1 = silu(z1), z2 = W2 h1 + b2,
// h2 = silu(z2), f = W3 h2 + b3:
//   d2 = W3 .* silu'(z2),  d1 = (W2^T d2) .* silu'(z1),
//   dE/dW3 = sum_i h2,  dE/db3 = N,  dE/dW2 = sum_i d2 h1^T,  dE/db2 = sum_i d2,
//   dE/dW1 = sum_i d1 x^T,  dE/db1 = sum_i d1.
// A warpgroup takes 128 sites per tile, thread t owning site t (TMEM lane t):
//   layer 1   D1 = [X | 1] [W1 | b1]^T / 2 = z1/2                (2 MMAs)
//   epilogue  h1 = silu(z1) -> H tile (BF16), silu'(z1) kept in registers
//   layer 2   D2 = [H | 1] [W2 | b2]^T / 2 = z2/2                (5 MMAs)
//   epilogue  h2, d2 -> columns 0-63, 64-127 of the Z tile (BF16)
//   back      D3 = D2tile W2 (d2 rows, W2 unscaled)             (4 MMAs)
//   epilogue  d1 = D3 .* silu'(z1) -> columns 128-191 of Z
// The tiles are site-major (each site's values contiguous), which makes them,
// read with MN-major descriptors (leading byte offset = stride between 8-site
// groups, stride byte offset = 128 B between 8-value groups), the operands of
// the contractions over sites, accumulated in TMEM across tiles:
//   G1[128 x 80] += [h2 | d2]^T [h1 | 1]  ->  rows 64-127: dW2, db2 (col 64);
//                                           rows 0-63, col 64: dW3
//   G2[128 x 32] += [d2 | d1]^T [x | 1]   ->  rows 64-127: dW1 (cols 0-19),
//                                           db1 (col 20)
// (8 MMAs each, K = 16 sites).  Every kFlushEvery tile rounds the
// accumulators are added into an FP64 copy per CTA; a second kernel adds the
// CTA copies in CTA order, so the result is bit-reproducible for a device.
#include <algorithm>
#include <cstring>

#include "mlp_common.cuh"
#include "mlp_tc.cuh"
#include "sweep_common.cuh"

namespace smc {

constexpr int kGradWG = 2;
constexpr int kGradThreads = 128 * kGradWG;
constexpr int kMlpParams = 64 * 20 + 64 + 64 * 64 + 64 + 64 + 1;
constexpr int kFlushEvery = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 64 * 20, kOffW2 = kOffB1 + 64, kOffB2 = kOffW2 + 64 * 64,
              kOffW3 = kOffB2 + 64, kOffB3 = kOffW3 + 64;
constexpr uint32_t kZRow = 3 * 64 * 2;     // Z tile: h2 | d2 | d1, 192 BF16 per site
constexpr uint32_t kZ = 128 * kZRow;       // 48 KB
constexpr uint32_t kW2T = 64 * 64 * 2;     // W2 transposed, K-major [j][k], K = 64
// TMEM columns of a warpgroup (256 allocated per warpgroup)
constexpr uint32_t kColD1 = 0, kColD2 = 64, kColG1 = 128, kColG2 = 208;

struct GradSmem {
    static constexpr uint32_t W1 = 0;
    static constexpr uint32_t W2 = W1 + kTcW1;
    static constexpr uint32_t W2T = W2 + kTcW2;
    static constexpr uint32_t W3 = W2T + kW2T;
    static constexpr uint32_t B3 = W3 + 256;
    static constexpr uint32_t WG = (B3 + 16 + 127) / 128 * 128;  // per-warpgroup tiles from here
    static constexpr uint32_t X = 0, H = X + kTcX, Z = H + kTcH, WGSIZE = Z + kZ;  // offsets within a warpgroup
    static constexpr uint32_t MBAR = WG + kGradWG * WGSIZE;      // [kGradWG][4]
    static constexpr uint32_t TSLOT = MBAR + 32 * kGradWG;
    static constexpr uint32_t CNT = TSLOT + 8;                   // long long [kGradWG]
    static constexpr uint32_t ACC = (CNT + 8 * kGradWG + 15) / 16 * 16;  // FP64 [kMlpParams]
    static constexpr uint32_t END = ACC + kMlpParams * 8;
};
static_assert(GradSmem::WG % 128 == 0 && GradSmem::WGSIZE % 128 == 0, "tile alignment");

// Byte offset of chunk kc (8 BF16) of row r in the K = 64 transposed-W2 tile.
__host__ __device__ constexpr uint32_t w2t_off(uint32_t r, uint32_t kc) { return (r >> 3) * 1024 + kc * 128 + (r & 7) * 16; }
// Z-tile byte offset of BF16 chunk kc (8 values) of site row r.
__host__ __device__ constexpr uint32_t z_off(uint32_t r, uint32_t kc) { return (r >> 3) * (kZRow * 8) + kc * 128 + (r & 7) * 16; }

// silu(2h) and silu'(2h) from h with t = tanh(h): h + h t and (1+t)(1+h(1-t))/2.
__device__ __forceinline__ void silu_pair(float h, float &s, float &ds)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    s = fmaf(h, t, h);
    ds = 0.5f * (1.f + t) * fmaf(h, 1.f - t, 1.f);
}

__device__ __forceinline__ void grad_wait(uint32_t mbar, uint32_t &phase, long long timeout_ns, int *status,
                                          int *abort_flag)
{
    if (!mbar_wait(mbar, phase, timeout_ns)) {
        atomicCAS(status, 0, (int)SMC_ERR_TIMEOUT);
        atomicExch(abort_flag, 1);
    }
    phase ^= 1;
    tc_fence_after();
}

__global__ void __launch_bounds__(kGradThreads, 1) k_mlp_grad(const MlpBlock *W, const int8_t *__restrict__ occ,
                                                              int nx, int ny, int nz, double *part,
                                                              long long timeout_ns, int *status, int *abort_flag)
{
    const int tid = threadIdx.x, r = tid & 127, wg = tid >> 7, wq = r >> 5;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const uint32_t base = GradSmem::WG + wg * GradSmem::WGSIZE;
    TcLayout L{base + GradSmem::X, base + GradSmem::H, GradSmem::W1, GradSmem::W2, 0, 0, GradSmem::W3, GradSmem::B3,
               GradSmem::MBAR + 32 * wg, GradSmem::TSLOT};
    const uint32_t Zt = base + GradSmem::Z;
    // weights: W1, W2 halved with the biases folded in; W2 transposed, unscaled
    tc_load_weights(W, L);
    for (int i = tid; i < 64 * 64; i += kGradThreads) {
        const int k = i >> 6, j = i & 63;  // W2[k][j] -> W2T[j][k]
        *(uint16_t *)(g_smem + GradSmem::W2T + w2t_off(j, k >> 3) + 2 * (k & 7)) = W->w2[i];
    }
    double *acc64 = (double *)(g_smem + GradSmem::ACC);
    for (int i = tid; i < kMlpParams; i += kGradThreads) acc64[i] = 0.0;
    tc_init_h_row(L, r);
    if (r == 0)
        for (int b = 0; b < 4; ++b) mbar_init(s0 + L.mbar + 8 * b, 1);
    if (tid < 32) tc_alloc(s0 + GradSmem::TSLOT, 512);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *(const uint32_t *)(g_smem + GradSmem::TSLOT) + 256 * wg;
    const uint32_t bar = 1 + wg;
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    uint32_t ph[4] = {0, 0, 0, 0};
    const float4 *w3 = (const float4 *)(g_smem + GradSmem::W3);
    auto spec = [&](int sb, int xx, int yy, int zz) { return occ_at(occ, nx, ny, nz, sb, xx, yy, zz); };
    constexpr uint32_t kIdG1 = tc_idesc(128, 80, true, true), kIdG2 = tc_idesc(128, 32, true, true);
    const long long N = 2LL * nx * ny * nz;
    const long long ntile = (N + kTcRows - 1) / kTcRows;
    const long long rounds = (ntile + (long long)kGradWG * gridDim.x - 1) / ((long long)kGradWG * gridDim.x);
    long long nvalid = 0;
    uint32_t g_acc = 0;  // 0: the next weight-gradient products start the accumulators afresh

    // adds the TMEM accumulators of this warpgroup into the FP64 copy
    auto flush = [&]() {
        uint32_t v[32];
        if (r >= 64) {
            const int k = r - 64;
            for (int c = 0; c < 64; c += 32) {
                tc_ld32(tmem + lane_base + kColG1 + c, v);
                tc_wait_ld(v);
                for (int j = 0; j < 32; ++j) acc64[kOffW2 + k * 64 + c + j] += (double)__uint_as_float(v[j]);
            }
        }
        uint32_t u[16];
        tc_ld16(tmem + lane_base + kColG1 + 64, u);
        tc_wait_ld16(u);
        if (r < 64)
            acc64[kOffW3 + r] += (double)__uint_as_float(u[0]);
        else
            acc64[kOffB2 + r - 64] += (double)__uint_as_float(u[0]);
        tc_ld32(tmem + lane_base + kColG2, v);
        tc_wait_ld(v);
        if (r >= 64) {
            const int j = r - 64;
            for (int i = 0; i < 20; ++i) acc64[kOffW1 + j * 20 + i] += (double)__uint_as_float(v[i]);
            acc64[kOffB1 + j] += (double)__uint_as_float(v[20]);
        }
        tc_fence_before();
    };

    for (long long rd = 0; rd < rounds; ++rd) {
        const long long tl = (rd * gridDim.x + blockIdx.x) * kGradWG + wg;
        if (tl < ntile) {
            // ---- features of site s (row r) ----
            const long long s = tl * kTcRows + r;
            const bool valid = s < N;
            int q0 = -1;
            uint32_t h1 = 0, h2 = 0, h3 = 0;
            if (valid) {
                long long t = s;
                const int x = (int)(t % nx);
                t /= nx;
                const int y = (int)(t % ny);
                t /= ny;
                const int z = (int)(t % nz);
                const int sub = (int)(t / nz);
                q0 = occ[s] & 7;
                site_hist(spec, sub, x, y, z, h1, h2, h3);
                ++nvalid;
            }
            tc_write_features(L, r, q0, h1, h2, h3);
            fence_async_smem();
            tc_fence_before();
            wg_sync(bar);
            if (r == 0) {
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < 2; ++k)
                    tc_mma(tmem + kColD1, tc_desc(s0 + L.x + k * 256, 128, 512), tc_desc(s0 + L.w1 + k * 256, 128, 512),
                           k > 0);
                tc_commit(s0 + L.mbar);
            }
            grad_wait(s0 + L.mbar, ph[0], timeout_ns, status, abort_flag);
            // ---- layer-1 epilogue: h1 -> H, silu'(z1) kept ----
            float ds1[64];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc_ld32(tmem + lane_base + kColD1 + 32 * half, v);
                tc_wait_ld(v);
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    uint32_t w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 32 * half + 8 * kc + 2 * u;
                        float sa, sb;
                        silu_pair(__uint_as_float(v[8 * kc + 2 * u]), sa, ds1[c]);
                        silu_pair(__uint_as_float(v[8 * kc + 2 * u + 1]), sb, ds1[c + 1]);
                        w[u] = pack_bf16(sa, sb);
                    }
                    *(uint4 *)(g_smem + L.h + tc_off80(r, 4 * half + kc)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            wg_sync(bar);
            if (r == 0) {
                tc_fence_after();
#pragma unroll
                for (int k = 0; k < kTcK2 / 16; ++k)
                    tc_mma(tmem + kColD2, tc_desc(s0 + L.h + k * 256, 128, 1280),
                           tc_desc(s0 + L.w2 + k * 256, 128, 1280), k > 0);
                tc_commit(s0 + L.mbar + 8);
            }
            grad_wait(s0 + L.mbar + 8, ph[1], timeout_ns, status, abort_flag);
            // ---- layer-2 epilogue: h2 and d2 = W3 .* silu'(z2) -> Z ----
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc_ld32(tmem + lane_base + kColD2 + 32 * half, v);
                tc_wait_ld(v);
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    uint32_t wh[4], wd[4];
                    const float4 wa = w3[8 * half + 2 * kc], wb = w3[8 * half + 2 * kc + 1];
                    const float wv[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float sa, sb, da, db;
                        silu_pair(__uint_as_float(v[8 * kc + 2 * u]), sa, da);
                        silu_pair(__uint_as_float(v[8 * kc + 2 * u + 1]), sb, db);
                        const float m = valid ? 1.f : 0.f;
                        wh[u] = pack_bf16(m * sa, m * sb);
                        wd[u] = pack_bf16(m * wv[2 * u] * da, m * wv[2 * u + 1] * db);
                    }
                    *(uint4 *)(g_smem + Zt + z_off(r, 4 * half + kc)) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
                    *(uint4 *)(g_smem + Zt + z_off(r, 8 + 4 * half + kc)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            wg_sync(bar);
            if (r == 0) {
                tc_fence_after();
                // back-propagation through W2: D3 = d2 W2 (into the D1 columns)
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc_mma(tmem + kColD1, tc_desc(s0 + Zt + 1024 + k * 256, 128, kZRow * 8),
                           tc_desc(s0 + GradSmem::W2T + k * 256, 128, 1024), k > 0);
                // G1 += [h2 | d2]^T [h1 | 1], contraction over the 128 sites
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    tc_mma_i(tmem + kColG1, tc_desc(s0 + Zt + k * 2 * kZRow * 8, kZRow * 8, 128),
                             tc_desc(s0 + L.h + k * 2 * 1280, 1280, 128), kIdG1, (k > 0) | g_acc);
                tc_commit(s0 + L.mbar + 16);
            }
            grad_wait(s0 + L.mbar + 16, ph[2], timeout_ns, status, abort_flag);
            // ---- back epilogue: d1 = D3 .* silu'(z1) -> Z ----
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                uint32_t v[32];
                tc_ld32(tmem + lane_base + kColD1 + 32 * half, v);
                tc_wait_ld(v);
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {
                    uint32_t w[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int c = 32 * half + 8 * kc + 2 * u;
                        const float m = valid ? 1.f : 0.f;
                        w[u] = pack_bf16(m * __uint_as_float(v[8 * kc + 2 * u]) * ds1[c],
                                         m * __uint_as_float(v[8 * kc + 2 * u + 1]) * ds1[c + 1]);
                    }
                    *(uint4 *)(g_smem + Zt + z_off(r, 16 + 4 * half + kc)) = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            wg_sync(bar);
            if (r == 0) {
                tc_fence_after();
                // G2 += [d2 | d1]^T [x | 1]
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    tc_mma_i(tmem + kColG2, tc_desc(s0 + Zt + 1024 + k * 2 * kZRow * 8, kZRow * 8, 128),
                             tc_desc(s0 + L.x + k * 2 * 512, 512, 128), kIdG2, (k > 0) | g_acc);
                tc_commit(s0 + L.mbar + 24);
            }
            grad_wait(s0 + L.mbar + 24, ph[3], timeout_ns, status, abort_flag);  // X, H, Z free again
            g_acc = 1;
        }
        // ---- every kFlushEvery rounds (and after the last): FP64 accumulation ----
        if ((rd + 1) % kFlushEvery == 0 || rd + 1 == rounds) {
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            for (int w = 0; w < kGradWG; ++w) {
                if (wg == w && g_acc) flush();
                __syncthreads();
            }
            tc_fence_after();
            g_acc = 0;
        }
    }
    // site count, then the CTA's FP64 vector
    for (int o = 16; o > 0; o >>= 1) nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    long long *cnt = (long long *)(g_smem + GradSmem::CNT);
    __syncthreads();
    if (tid == 0)
        for (int w = 0; w < kGradWG; ++w) cnt[w] = 0;
    __syncthreads();
    if ((tid & 31) == 0) atomicAdd((unsigned long long *)&cnt[wg], (unsigned long long)nvalid);
    __syncthreads();
    if (tid == 0) {
        long long n = 0;
        for (int w = 0; w < kGradWG; ++w) n += cnt[w];
        acc64[kOffB3] = (double)n;
    }
    __syncthreads();
    double *dst = part + (size_t)blockIdx.x * kMlpParams;
    for (int i = tid; i < kMlpParams; i += kGradThreads) dst[i] = acc64[i];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) tc_dealloc(*(const uint32_t *)(g_smem + GradSmem::TSLOT), 512);
}

// grad[i] = sum over CTAs of part[cta][i], in CTA order.
__global__ void k_mlp_grad_finish(const double *part, int nparts, float *grad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(size_t)b * kMlpParams + i];
    grad[i] = (float)s;
}

smc_status launch_mlp_grad(const smc_lattice *lat, const smc_model *m, const int8_t *occ, float *grad,
                           cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const size_t smem = GradSmem::END;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_grad)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_grad, kGradThreads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm != 1) {  // each CTA holds all 512 tensor-memory columns of its SM
        set_error("MLP gradient kernel occupancy %d (expected 1 CTA per SM)", per_sm);
        return SMC_ERR_STATE;
    }
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const long long ntile = (N + kTcRows - 1) / kTcRows;
    const int grid = (int)std::max(1LL, std::min<long long>((long long)ws->num_sms, (ntile + kGradWG - 1) / kGradWG));
    // scratch: [pair counts | abort word | MlpBlock | CTA partials]
    const size_t off_abort = (sizeof(unsigned long long) * kMaxShells * 64 + 15) / 16 * 16;
    const size_t off_w = off_abort + 16;
    const size_t off_part = (off_w + sizeof(MlpBlock) + 15) / 16 * 16;
    unsigned char *scr =
        (unsigned char *)workspace_scratch(ws, off_part + sizeof(double) * kMlpParams * (size_t)grid, &st);
    if (!scr) return st;
    int npair = 0;
    if (m->kind == SMC_PAIR_F32_MLP_BF16) {
        npair = m->nshells * lat->nspecies * (lat->nspecies + 1) / 2;
        unsigned long long *cnt = (unsigned long long *)scr;
        st = launch_pair_counts(lat, m->nshells, occ, cnt, stream);
        if (st != SMC_OK) return st;
        st = launch_pair_grad_finish(lat, m, cnt, grad, stream);
        if (st != SMC_OK) return st;
    }
    static MlpBlock W;
    make_mlp_block(m, W);
    e = cudaMemcpyAsync(scr + off_w, &W, sizeof W, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(MLP weights)");
    e = cudaMemsetAsync(scr + off_abort, 0, 16, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(abort word)");
    double *part = (double *)(scr + off_part);
    k_mlp_grad<<<grid, kGradThreads, smem, stream>>>((const MlpBlock *)(scr + off_w), occ, lat->nx, lat->ny, lat->nz,
                                                     part, debug_timeout_ns(), ws->status, (int *)(scr + off_abort));
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_grad");
    k_mlp_grad_finish<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(part, grid, grad + npair);
    e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_mlp_grad_finish");
}

}  // namespace smc
