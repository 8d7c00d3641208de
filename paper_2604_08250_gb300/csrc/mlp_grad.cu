// mlp_grad.cu -- dE/dtheta of the MLP energy E = sum_i f(x_i) with respect to
// every MLP parameter (W1, b1, W2, b2, W3, b3), by back-propagation at every
// site, on the tensor cores.
//
// For one site, with z1 = W1 x + b1, h1 = silu(z1), z2 = W2 h1 + b2,
// h2 = silu(z2), f = W3 h2 + b3:
//   d2 = W3 .* silu'(z2),  d1 = (W2^T d2) .* silu'(z1),
//   dE/dW3 = sum_i h2,  dE/db3 = N,  dE/dW2 = sum_i d2 h1^T,  dE/db2 = sum_i d2,
//   dE/dW1 = sum_i d1 x^T,  dE/db1 = sum_i d1.
// A CTA of 4 warps takes 64 sites at a time: each warp runs the forward and
// backward passes of 16 sites (m16n8k16 BF16 products with the sites as rows)
// and leaves x, h1, d2 and d1 in shared memory as BF16; then the weight
// gradients, contractions over the 64 sites, are split across the warps by
// output rows (ldmatrix.trans turns the site-major tiles into operands).
// Register accumulators are flushed into an FP64 per-CTA copy every
// kFlushEvery blocks; the CTA copies are added in CTA order by a second
// kernel, so the result is bit-reproducible for a given device.
#include <algorithm>
#include <cstring>

#include "mlp_common.cuh"
#include "sweep_common.cuh"

namespace smc {

constexpr int kGradWarps = 4;
constexpr int kGradSites = 16 * kGradWarps;
constexpr int kMlpParams = 64 * 20 + 64 + 64 * 64 + 64 + 64 + 1;
constexpr int kFlushEvery = 32;
// offsets of the parameter groups in the gradient vector
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + 64 * 20, kOffW2 = kOffB1 + 64, kOffB2 = kOffW2 + 64 * 64,
              kOffW3 = kOffB2 + 64, kOffB3 = kOffW3 + 64;

struct GradSmem {
    static constexpr uint32_t W1 = 0;                          // [64 out][32 in] BF16, stride 80 B
    static constexpr uint32_t W2 = W1 + 64 * kW1RowB;          // [64 out][64 in], stride 144 B
    static constexpr uint32_t W2T = W2 + 64 * kW2RowB;         // transposed: [64 in][64 out]
    static constexpr uint32_t B1 = W2T + 64 * kW2RowB;         // FP32 [64]
    static constexpr uint32_t B2 = B1 + 256;
    static constexpr uint32_t W3 = B2 + 256;
    static constexpr uint32_t X = W3 + 256;                    // [64 sites][32] BF16, stride 80 B
    static constexpr uint32_t H1 = X + kGradSites * kARowB;    // [64 sites][64] BF16, stride 144 B
    static constexpr uint32_t D2 = H1 + kGradSites * kW2RowB;
    static constexpr uint32_t DL = D2 + kGradSites * kW2RowB;  // d1
    static constexpr uint32_t ACC = DL + kGradSites * kW2RowB;  // FP64 [kMlpParams]
    static constexpr uint32_t WACC = (ACC + kMlpParams * 8 + 15) / 16 * 16;  // FP64 [warps][3][64]
    static constexpr uint32_t END = WACC + kGradWarps * 3 * 64 * 8;
};

__device__ __forceinline__ float sigmoid_approx(float z)
{
    float t;
    const float h = 0.5f * z;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(0.5f, t, 0.5f);
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__global__ void __launch_bounds__(32 * kGradWarps) k_mlp_grad(const MlpBlock *W, const int8_t *__restrict__ occ,
                                                              int nx, int ny, int nz, double *part)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    for (int i = tid; i < 64 * 16; i += blockDim.x) {
        const int r = i >> 4, c = i & 15;
        *(uint32_t *)(g_smem + GradSmem::W1 + r * kW1RowB + 4 * c) = ((const uint32_t *)W->w1)[r * 16 + c];
    }
    for (int i = tid; i < 64 * 64; i += blockDim.x) {
        const int k = i >> 6, j = i & 63;  // W2[k][j]
        const uint16_t v = W->w2[i];
        *(uint16_t *)(g_smem + GradSmem::W2 + k * kW2RowB + 2 * j) = v;
        *(uint16_t *)(g_smem + GradSmem::W2T + j * kW2RowB + 2 * k) = v;
    }
    for (int i = tid; i < 64; i += blockDim.x) {
        ((float *)(g_smem + GradSmem::B1))[i] = W->b1[i];
        ((float *)(g_smem + GradSmem::B2))[i] = W->b2[i];
        ((float *)(g_smem + GradSmem::W3))[i] = W->w3[i];
    }
    double *acc64 = (double *)(g_smem + GradSmem::ACC);
    double *wacc = (double *)(g_smem + GradSmem::WACC);
    for (int i = tid; i < kMlpParams; i += blockDim.x) acc64[i] = 0.0;
    for (int i = tid; i < kGradWarps * 3 * 64; i += blockDim.x) wacc[i] = 0.0;
    __syncthreads();
    const float *b1 = (const float *)(g_smem + GradSmem::B1);
    const float *b2 = (const float *)(g_smem + GradSmem::B2);
    const float *w3 = (const float *)(g_smem + GradSmem::W3);
    const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    auto spec = [&](int sb, int xx, int yy, int zz) { return occ_at(occ, nx, ny, nz, sb, xx, yy, zz); };

    float gw2[8][4], gw1[4][4], aw3[16], ab2[16], ab1[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) gw2[j][0] = gw2[j][1] = gw2[j][2] = gw2[j][3] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) gw1[j][0] = gw1[j][1] = gw1[j][2] = gw1[j][3] = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) aw3[j] = ab2[j] = ab1[j] = 0.f;
    long long nvalid = 0;

    // adds the register accumulators into the CTA's FP64 copy and clears them
    auto flush = [&]() {
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = 16 * warp + g + 8 * (e >> 1), n = 8 * j + 2 * t + (e & 1);
                acc64[kOffW2 + m * 64 + n] += (double)gw2[j][e];
                gw2[j][e] = 0.f;
            }
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = 16 * warp + g + 8 * (e >> 1), n = 8 * j + 2 * t + (e & 1);
                if (n < 20) acc64[kOffW1 + m * 20 + n] += (double)gw1[j][e];
                gw1[j][e] = 0.f;
            }
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float a = aw3[q], b = ab2[q], c = ab1[q];
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
                c += __shfl_xor_sync(0xffffffffu, c, o);
            }
            if (g == 0) {
                const int col = 8 * (q >> 1) + 2 * t + (q & 1);
                wacc[(warp * 3 + 0) * 64 + col] += (double)a;
                wacc[(warp * 3 + 1) * 64 + col] += (double)b;
                wacc[(warp * 3 + 2) * 64 + col] += (double)c;
            }
            aw3[q] = ab2[q] = ab1[q] = 0.f;
        }
    };

    const long long N = 2LL * nx * ny * nz;
    const long long nblk = (N + kGradSites - 1) / kGradSites;
    const uint32_t xrow = GradSmem::X + (uint32_t)(warp * 16) * kARowB;
    int it = 0;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long sbase = blk * kGradSites + warp * 16;
        if (lane < 16) {
            const long long s = sbase + lane;
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
                ++nvalid;
            }
            write_feature_row(xrow + lane * kARowB, q0, h1, h2, h3);
        }
        __syncwarp();
        const float v_lo = (sbase + g < N) ? 1.f : 0.f, v_hi = (sbase + g + 8 < N) ? 1.f : 0.f;
        // ---- forward, layer 1 ----
        float acc[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            const uint32_t ar = xrow + kc * 32 + 4 * t;
            const uint32_t a0 = lds32(ar + g * kARowB), a1 = lds32(ar + (g + 8) * kARowB);
            const uint32_t a2 = lds32(ar + g * kARowB + 16), a3 = lds32(ar + (g + 8) * kARowB + 16);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t br = GradSmem::W1 + (8 * j + g) * kW1RowB + kc * 32 + 4 * t;
                mma_bf16(acc[j], a0, a1, a2, a3, lds32(br), lds32(br + 16));
            }
        }
        uint32_t ha[4][4];
        float sp1[8][4];
        const uint32_t h1row = GradSmem::H1 + (uint32_t)(warp * 16 + g) * kW2RowB;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * t;
            float h[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float z = acc[j][e] + b1[c + (e & 1)];
                const float sg = sigmoid_approx(z);
                h[e] = z * sg;
                sp1[j][e] = sg * fmaf(z, 1.f - sg, 1.f);
            }
            ha[j >> 1][(j & 1) * 2 + 0] = pack_bf16(h[0], h[1]);
            ha[j >> 1][(j & 1) * 2 + 1] = pack_bf16(h[2], h[3]);
            *(uint32_t *)(g_smem + h1row + 2 * c) = ha[j >> 1][(j & 1) * 2 + 0];
            *(uint32_t *)(g_smem + h1row + 8 * kW2RowB + 2 * c) = ha[j >> 1][(j & 1) * 2 + 1];
        }
        // ---- forward, layer 2; output-layer gradients ----
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t br = GradSmem::W2 + (8 * j + g) * kW2RowB + kc * 32 + 4 * t;
                mma_bf16(acc[j], ha[kc][0], ha[kc][1], ha[kc][2], ha[kc][3], lds32(br), lds32(br + 16));
            }
        uint32_t da[4][4];
        const uint32_t d2row = GradSmem::D2 + (uint32_t)(warp * 16 + g) * kW2RowB;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * t;
            float d[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float z = acc[j][e] + b2[c + (e & 1)];
                const float sg = sigmoid_approx(z);
                const float v = (e < 2) ? v_lo : v_hi;
                aw3[2 * j + (e & 1)] = fmaf(z * sg, v, aw3[2 * j + (e & 1)]);
                d[e] = w3[c + (e & 1)] * (sg * fmaf(z, 1.f - sg, 1.f)) * v;
                ab2[2 * j + (e & 1)] += d[e];
            }
            da[j >> 1][(j & 1) * 2 + 0] = pack_bf16(d[0], d[1]);
            da[j >> 1][(j & 1) * 2 + 1] = pack_bf16(d[2], d[3]);
            *(uint32_t *)(g_smem + d2row + 2 * c) = da[j >> 1][(j & 1) * 2 + 0];
            *(uint32_t *)(g_smem + d2row + 8 * kW2RowB + 2 * c) = da[j >> 1][(j & 1) * 2 + 1];
        }
        // ---- backward to layer 1: d1 = (d2 W2) .* silu'(z1) ----
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
        for (int kc = 0; kc < 4; ++kc)
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t br = GradSmem::W2T + (8 * j + g) * kW2RowB + kc * 32 + 4 * t;
                mma_bf16(acc[j], da[kc][0], da[kc][1], da[kc][2], da[kc][3], lds32(br), lds32(br + 16));
            }
        const uint32_t dlrow = GradSmem::DL + (uint32_t)(warp * 16 + g) * kW2RowB;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * j + 2 * t;
            float d[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                d[e] = acc[j][e] * sp1[j][e];
                ab1[2 * j + (e & 1)] += d[e];
            }
            *(uint32_t *)(g_smem + dlrow + 2 * c) = pack_bf16(d[0], d[1]);
            *(uint32_t *)(g_smem + dlrow + 8 * kW2RowB + 2 * c) = pack_bf16(d[2], d[3]);
        }
        __syncthreads();
        // ---- weight gradients over the 64 sites: warp w owns output rows 16w..16w+15 ----
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            const int sa = kc * 16 + (lane & 7) + ((lane >> 4) << 3);  // A: sites of matrix (lane >> 3)
            const int ca = 16 * warp + ((lane >> 3) & 1) * 8;
            const int sb = kc * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;  // B: sites of matrix (lane >> 3)
            uint32_t a0, a1, a2, a3;
            ldsm_x4_trans(smem0 + GradSmem::D2 + sa * kW2RowB + 2 * ca, a0, a1, a2, a3);
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t b0, b1v, b2v, b3;
                const int cb = 8 * (2 * np + (lane >> 4));
                ldsm_x4_trans(smem0 + GradSmem::H1 + sb * kW2RowB + 2 * cb, b0, b1v, b2v, b3);
                mma_bf16(gw2[2 * np], a0, a1, a2, a3, b0, b1v);
                mma_bf16(gw2[2 * np + 1], a0, a1, a2, a3, b2v, b3);
            }
            ldsm_x4_trans(smem0 + GradSmem::DL + sa * kW2RowB + 2 * ca, a0, a1, a2, a3);
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                uint32_t b0, b1v, b2v, b3;
                const int cb = 8 * (2 * np + (lane >> 4));
                ldsm_x4_trans(smem0 + GradSmem::X + sb * kARowB + 2 * cb, b0, b1v, b2v, b3);
                mma_bf16(gw1[2 * np], a0, a1, a2, a3, b0, b1v);
                mma_bf16(gw1[2 * np + 1], a0, a1, a2, a3, b2v, b3);
            }
        }
        __syncthreads();
        if (++it == kFlushEvery) {
            flush();
            it = 0;
        }
    }
    flush();
    // site count of the CTA (each valid site was counted by one lane)
    for (int o = 16; o > 0; o >>= 1) nvalid += __shfl_xor_sync(0xffffffffu, nvalid, o);
    __shared__ long long cnt[kGradWarps];
    if (lane == 0) cnt[warp] = nvalid;
    __syncthreads();
    for (int c = tid; c < 64; c += blockDim.x) {
        double sw3 = 0.0, sb2 = 0.0, sb1 = 0.0;
        for (int w = 0; w < kGradWarps; ++w) {
            sw3 += wacc[(w * 3 + 0) * 64 + c];
            sb2 += wacc[(w * 3 + 1) * 64 + c];
            sb1 += wacc[(w * 3 + 2) * 64 + c];
        }
        acc64[kOffW3 + c] = sw3;
        acc64[kOffB2 + c] = sb2;
        acc64[kOffB1 + c] = sb1;
    }
    if (tid == 0) {
        long long n = 0;
        for (int w = 0; w < kGradWarps; ++w) n += cnt[w];
        acc64[kOffB3] = (double)n;
    }
    __syncthreads();
    double *dst = part + (size_t)blockIdx.x * kMlpParams;
    for (int i = tid; i < kMlpParams; i += blockDim.x) dst[i] = acc64[i];
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
    const int threads = 32 * kGradWarps;
    const size_t smem = GradSmem::END;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_mlp_grad)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mlp_grad, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) {
        set_error("MLP gradient kernel does not fit on an SM");
        return SMC_ERR_UNSUPPORTED;
    }
    const Tuning tu = current_tuning();
    if (tu.ctas_per_sm > 0) per_sm = std::min(per_sm, tu.ctas_per_sm);
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    const long long nblk = (N + kGradSites - 1) / kGradSites;
    const int grid = (int)std::max(1LL, std::min<long long>((long long)per_sm * ws->num_sms, nblk));
    // scratch: [pair counts | MlpBlock | CTA partials]
    const size_t off_w = (sizeof(unsigned long long) * kMaxShells * 64 + 15) / 16 * 16;
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
    double *part = (double *)(scr + off_part);
    k_mlp_grad<<<grid, threads, smem, stream>>>((const MlpBlock *)(scr + off_w), occ, lat->nx, lat->ny, lat->nz,
                                                part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_mlp_grad");
    k_mlp_grad_finish<<<(kMlpParams + 255) / 256, 256, 0, stream>>>(part, grid, grad + npair);
    e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_mlp_grad_finish");
}

}  // namespace smc
