// mlpnet_tc.cuh -- MLPNet at the paper's shape (Sec. IV-B: an input layer and
// two hidden layers of 96 units, each followed by ReLU, then a linear
// regression layer) on the tcgen05 tensor cores.
//
// A warpgroup of 128 threads evaluates f for a tile of 128 feature rows,
// thread t owning row t, in one 96-column TMEM region:
//   L0  D = [X | 1] [W0 | b0]^T              (K = 32: 2 MMAs, N = 96)
//   epilogue relu(D) -> BF16 rows of the hidden-layer operand H (K = 112:
//        96 activations, 3 constant ones against the bias parts, zero pad)
//   L1  D = [H | 1] [W1 | b1]^T              (7 MMAs), epilogue into H again
//   L2  D = [H | 1] [W2 | b2]^T              (7 MMAs)
//   f = b3 + sum_k W3[k] relu(D)[k]          (FP32, k in order)
// BF16 weights and activations, FP32 accumulation; the FP32 biases enter as
// three exact BF16 parts.  The stages follow the interface of mlp_tc.cuh
// (tc_write_features, tc_issue1, tc_stage2, tc_finish) so that the sweep,
// energy and trace kernels run either network: here tc_issue1 does nothing
// and tc_stage2 runs L0, L1 and L2 (each waits for the one before), so
// between tc_stage2 of a tile and its tc_finish the X tile is already free
// for the next tile's rows.  A row's f does not depend on the other rows.
#pragma once

#include "mlp_tc.cuh"

namespace smc {

constexpr int kNetHid = 96;
constexpr int kNetK = 112;                     // hidden-layer K
constexpr uint32_t kNetX = 128 * 64;           // X tile: 128 rows x 32 BF16
constexpr uint32_t kNetHt = 128 * kNetK * 2;   // H tile: 128 rows x 112 BF16
constexpr uint32_t kNetW0 = kNetHid * 64;      // W0: 96 rows x 32 BF16
constexpr uint32_t kNetW12 = kNetHid * kNetK * 2;  // W1, W2: 96 rows x 112 BF16
constexpr uint32_t kNetCols = 128;             // TMEM columns per warpgroup (96 used)
constexpr uint32_t kNetIdesc = tc_idesc(128, kNetHid, false, false);

// Byte offset of element chunk kc (8 BF16) of row r in a K = 112 tile.
__host__ __device__ constexpr uint32_t tn_off112(uint32_t r, uint32_t kc) { return (r >> 3) * 1792 + kc * 128 + (r & 7) * 16; }

// The kernels' MLPNet weight block: W0 padded to 32 inputs.
struct NetBlock {
    uint16_t w0[kNetHid * 32];
    uint16_t w1[kNetHid * kNetHid];
    uint16_t w2[kNetHid * kNetHid];
    float b0[kNetHid], b1[kNetHid], b2[kNetHid], w3[kNetHid];
    float b3;
    float pad[3];
};

struct NetLayout {
    uint32_t x, h, w0, w1, w2, w3, b3, mbar, tmem_slot;
};

struct NetEval {
    NetLayout L;
    uint32_t tmem;
    uint32_t phase1, phase2;  // mbarrier 1 (L0, L1) and 2 (L2)
    uint32_t bar;
    long long timeout_ns;
    int *status, *abort_flag;
};

__device__ __forceinline__ uint4 bias_chunk(float b, bool front)
{
    __nv_bfloat16 hi, mid, lo;
    split3_bf16(b, hi, mid, lo);
    __nv_bfloat162 p0 = __halves2bfloat162(hi, mid), p1 = __halves2bfloat162(lo, __float2bfloat16_rn(0.f));
    const uint32_t a = *reinterpret_cast<uint32_t *>(&p0), c = *reinterpret_cast<uint32_t *>(&p1);
    return front ? make_uint4(a, c, 0u, 0u) : make_uint4(0u, 0u, a, c);
}

static __device__ void tc_load_weights(const NetBlock *W, const NetLayout &L)
{
    const int tid = threadIdx.x, n = blockDim.x;
    for (int i = tid; i < kNetHid * 4; i += n) {  // W0: 96 rows x 4 chunks; b0 in columns 20-22
        const int r = i >> 2, kc = i & 3;
        uint4 v = ((const uint4 *)W->w0)[r * 4 + kc];
        if (kc == 2) {  // columns 16-19 inputs, 20-22 bias parts
            const uint4 b = bias_chunk(W->b0[r], false);
            v.z = b.z;
            v.w = b.w;
        }
        *(uint4 *)(g_smem + L.w0 + tc_off32(r, kc)) = v;
    }
    for (int l = 0; l < 2; ++l) {
        const uint16_t *w = l == 0 ? W->w1 : W->w2;
        const float *b = l == 0 ? W->b1 : W->b2;
        const uint32_t dst = l == 0 ? L.w1 : L.w2;
        for (int i = tid; i < kNetHid * 14; i += n) {  // 96 rows x 14 chunks; bias parts in columns 96-98
            const int r = i / 14, kc = i - 14 * (i / 14);
            uint4 v = make_uint4(0, 0, 0, 0);
            if (kc < 12)
                v = ((const uint4 *)w)[r * 12 + kc];
            else if (kc == 12)
                v = bias_chunk(b[r], true);
            *(uint4 *)(g_smem + dst + tn_off112(r, kc)) = v;
        }
    }
    for (int i = tid; i < kNetHid; i += n) ((float *)(g_smem + L.w3))[i] = W->w3[i];
    if (tid == 0) *(float *)(g_smem + L.b3) = W->b3;
}

// Constant columns 96-111 of row r of the H tile: ones in 96-98, zeros after.
__device__ __forceinline__ void tc_init_h_row(const NetLayout &L, uint32_t r)
{
    *(uint4 *)(g_smem + L.h + tn_off112(r, 12)) = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
    *(uint4 *)(g_smem + L.h + tn_off112(r, 13)) = make_uint4(0u, 0u, 0u, 0u);
}

static __device__ void tc_setup(NetEval &E, int nwg)
{
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const int wg = threadIdx.x >> 7;
    tc_init_h_row(E.L, threadIdx.x & 127);
    if ((threadIdx.x & 127) == 0) {
        mbar_init(s0 + E.L.mbar, 1);
        mbar_init(s0 + E.L.mbar + 8, 1);
    }
    if (threadIdx.x < 32) tc_alloc(s0 + E.L.tmem_slot, kNetCols * nwg);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    E.tmem = *(const uint32_t *)(g_smem + E.L.tmem_slot) + kNetCols * wg;
    E.phase1 = E.phase2 = 0;
    E.bar = 1 + wg;
}

static __device__ void tc_teardown(NetEval &E, int nwg)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tc_dealloc(*(const uint32_t *)(g_smem + E.L.tmem_slot), kNetCols * nwg);
}

// The X tile has the layout of the 64-wide network's: same features.
__device__ __forceinline__ void tc_write_features(const NetLayout &L, uint32_t r, int q0, uint32_t h1, uint32_t h2,
                                                  uint32_t h3)
{
    TcLayout T{};
    T.x = L.x;
    tc_write_features(T, r, q0, h1, h2, h3);
}

__device__ __forceinline__ void tc_timeout(NetEval &E)
{
    atomicCAS(E.status, 0, (int)SMC_ERR_TIMEOUT);
    atomicExch(E.abort_flag, 1);
}

// relu of this warp's 32 rows x 96 columns of D, as BF16, into the H tile.
__device__ __forceinline__ void net_epilogue(NetEval &E, uint32_t r, uint32_t lane_base)
{
#pragma unroll
    for (int third = 0; third < 3; ++third) {
        uint32_t v[32];
        tc_ld32(E.tmem + lane_base + 32 * third, v);
        tc_wait_ld(v);
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                w[u] = pack_bf16(fmaxf(__uint_as_float(v[8 * kc + 2 * u]), 0.f),
                                 fmaxf(__uint_as_float(v[8 * kc + 2 * u + 1]), 0.f));
            *(uint4 *)(g_smem + E.L.h + tn_off112(r, 4 * third + kc)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Issues the products of a hidden layer (A = the H tile, B = w) after the
// warpgroup's H rows are written.
__device__ __forceinline__ void net_issue_hidden(NetEval &E, uint32_t r, uint32_t s0, uint32_t w, uint32_t mbar)
{
    fence_async_smem();
    tc_fence_before();
    wg_sync(E.bar);
    if (r == 0) {
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < kNetK / 16; ++k)
            tc_mma_i(E.tmem, tc_desc(s0 + E.L.h + k * 256, 128, 1792), tc_desc(s0 + w + k * 256, 128, 1792), kNetIdesc,
                     k > 0);
        tc_commit(mbar);
    }
}

static __device__ __forceinline__ void tc_issue1(NetEval &E) { (void)E; }

static __device__ __forceinline__ void tc_stage2(NetEval &E)
{
    const int r = threadIdx.x & 127, wq = r >> 5;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    // L0 (the X rows were written and fenced by their threads)
    tc_fence_before();
    wg_sync(E.bar);
    if (r == 0) {
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < 2; ++k)
            tc_mma_i(E.tmem, tc_desc(s0 + E.L.x + k * 256, 128, 512), tc_desc(s0 + E.L.w0 + k * 256, 128, 512),
                     kNetIdesc, k > 0);
        tc_commit(s0 + E.L.mbar);
    }
    if (!mbar_wait(s0 + E.L.mbar, E.phase1, E.timeout_ns)) tc_timeout(E);
    E.phase1 ^= 1;
    tc_fence_after();
    net_epilogue(E, r, lane_base);
    net_issue_hidden(E, r, s0, E.L.w1, s0 + E.L.mbar);
    if (!mbar_wait(s0 + E.L.mbar, E.phase1, E.timeout_ns)) tc_timeout(E);
    E.phase1 ^= 1;
    tc_fence_after();
    net_epilogue(E, r, lane_base);
    net_issue_hidden(E, r, s0, E.L.w2, s0 + E.L.mbar + 8);
}

static __device__ __forceinline__ float tc_finish(NetEval &E)
{
    const int r = threadIdx.x & 127, wq = r >> 5;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    if (!mbar_wait(s0 + E.L.mbar + 8, E.phase2, E.timeout_ns)) tc_timeout(E);
    E.phase2 ^= 1;
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    const float4 *w3 = (const float4 *)(g_smem + E.L.w3);
    float acc = 0.f;
#pragma unroll
    for (int third = 0; third < 3; ++third) {
        uint32_t v[32];
        tc_ld32(E.tmem + lane_base + 32 * third, v);
        tc_wait_ld(v);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
            const float4 w = w3[8 * third + j4];
            acc = fmaf(w.x, fmaxf(__uint_as_float(v[4 * j4]), 0.f), acc);
            acc = fmaf(w.y, fmaxf(__uint_as_float(v[4 * j4 + 1]), 0.f), acc);
            acc = fmaf(w.z, fmaxf(__uint_as_float(v[4 * j4 + 2]), 0.f), acc);
            acc = fmaf(w.w, fmaxf(__uint_as_float(v[4 * j4 + 3]), 0.f), acc);
        }
    }
    tc_fence_before();
    return *(const float *)(g_smem + E.L.b3) + acc;
}

static __device__ __forceinline__ float tc_eval(NetEval &E)
{
    tc_issue1(E);
    tc_stage2(E);
    return tc_finish(E);
}

}  // namespace smc
