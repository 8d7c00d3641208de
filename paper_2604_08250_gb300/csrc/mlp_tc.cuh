// mlp_tc.cuh -- the MLP site energy on the 5th-generation tensor cores
// (tcgen05): operands in shared memory, accumulators in tensor memory (TMEM).
//
// A warpgroup of 128 threads evaluates f for a tile of 128 feature rows,
// thread t owning row t:
//   layer 1  D1[128 x 64] = [X | 1] [W1 | b1]^T / 2 = z1/2   (2 MMAs, K = 16 each)
//   epilogue silu(z1) = h + h tanh(h), h = D1 -> BF16 rows of the layer-2 operand
//   layer 2  D2[128 x 64] = [H1 | 1] [W2 | b2]^T / 2 = z2/2  (5 MMAs)
//   epilogue f = b3 + sum_k W3[k] silu(z2)[k]   (FP32, k in order)
// One thread issues the MMAs (tcgen05.mma.cta_group::1.kind::f16, BF16
// inputs, FP32 accumulation) and commits them to an mbarrier; every warp then
// reads its 32 TMEM lanes (rows) with tcgen05.ld.  A row's result does not
// depend on the other rows of the tile or on its position in it.
//
// Operand layout: K-major without swizzling, i.e. "core matrices" of 8 rows x
// 16 bytes stored as 128 contiguous bytes; the core matrices of one 8-row
// group follow each other along K (leading byte offset 128 B), and the 8-row
// groups follow each other (stride byte offset 8 rows x 2K bytes = 16 K B).
#pragma once

#include "mlp_common.cuh"
#include "sweep_common.cuh"

namespace smc {

constexpr int kTcRows = 128;
constexpr int kTcK2 = 80;               // layer-2 K: 64 activations, 3 ones for the bias, zero pad
constexpr uint32_t kTcX = 128 * 64;     // X tile: 128 rows x 32 BF16
constexpr uint32_t kTcH = 128 * kTcK2 * 2;  // H1 tile: 128 rows x 80 BF16
constexpr uint32_t kTcW1 = 64 * 64;     // W1: 64 x 32 BF16
constexpr uint32_t kTcW2 = 64 * kTcK2 * 2;  // W2: 64 x 80 BF16
constexpr uint32_t kTcCols = 128;       // TMEM columns per warpgroup (D1: 0-63, D2: 64-127)

// Byte offset of element chunk kc (8 BF16) of row r in a K = 32 / K = 80 tile.
__host__ __device__ constexpr uint32_t tc_off32(uint32_t r, uint32_t kc) { return (r >> 3) * 512 + kc * 128 + (r & 7) * 16; }
__host__ __device__ constexpr uint32_t tc_off80(uint32_t r, uint32_t kc) { return (r >> 3) * 1280 + kc * 128 + (r & 7) * 16; }

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), descriptor version 1
// (bit 46), no swizzle (bits 61-63 = 0).  Without swizzling the leading byte
// offset is the distance between core matrices along K and the stride byte
// offset the distance between core matrices along M (or N), for K-major and
// MN-major operands alike.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

// Instruction descriptor for other shapes / operand majors (transpose bits:
// 15 for A, 16 for B set = MN-major operand).
__host__ __device__ constexpr uint32_t tc_idesc(uint32_t M, uint32_t N, bool a_mn_major, bool b_mn_major)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) | ((b_mn_major ? 1u : 0u) << 16) |
           ((N >> 3) << 17) | ((M >> 4) << 24);
}
static_assert(tc_idesc(128, 64, false, false) == kTcIdesc, "instruction descriptor");

__device__ __forceinline__ void tc_mma_i(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM allocation by one whole warp; the address is written to shared memory.
__device__ __forceinline__ void tc_alloc(uint32_t dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier; false after timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, long long timeout_ns)
{
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(a, parity))
        if ((long long)(global_ns() - t0) > timeout_ns) return false;
    return true;
}

// 32 consecutive TMEM columns of this warp's 32 lanes (lane i -> register row i).
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
// 16 consecutive TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tc_wait_ld16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// Waits for this thread's tcgen05.ld; the registers pass through so that no
// use of them can be scheduled before the wait.
__device__ __forceinline__ void tc_wait_ld(uint32_t (&r)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]),
                   "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]),
                   "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// Shared-memory offsets (from g_smem) of the pieces the evaluator uses
// (mbar: two mbarriers, one per layer).
struct TcLayout {
    uint32_t x, h, w1, w2, b1, b2, w3, b3, mbar, tmem_slot;
};

// Evaluator state of one warpgroup (128 threads): its X and H tiles,
// mbarrier and TMEM columns; the weights are shared by the CTA.
struct TcEval {
    TcLayout L;
    uint32_t tmem;    // TMEM address of this warpgroup's first column (lane 0)
    uint32_t phase1, phase2;  // parities of the two mbarriers' next phases
    uint32_t bar;     // named barrier of the warpgroup (1 + warpgroup index)
    long long timeout_ns;
    int *status, *abort_flag;
};

__device__ __forceinline__ void wg_sync(uint32_t bar) { asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory"); }

// Copies the weights into the evaluator's layout, all scaled by 1/2 (exact:
// a power of two): the products then give h = z/2 directly and
// silu(z) = h + h tanh(h), bit for bit the values of the unscaled arithmetic.
// The FP32 biases ride along as three BF16 parts (hi + mid + lo = b/2
// exactly) in columns 20-22 of W1 and 64-66 of W2, against constant-one
// columns of the X and H tiles, so the products already include them.
__device__ __forceinline__ uint4 half_bf16x8(uint4 v)
{
    uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162 *>(&w[i]);
        const float2 f = __bfloat1622float2(b);
        b = __floats2bfloat162_rn(0.5f * f.x, 0.5f * f.y);
        w[i] = *reinterpret_cast<uint32_t *>(&b);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void split3_bf16(float b, __nv_bfloat16 &hi, __nv_bfloat16 &mid, __nv_bfloat16 &lo)
{
    hi = __float2bfloat16_rn(b);
    const float r1 = b - __bfloat162float(hi);
    mid = __float2bfloat16_rn(r1);
    lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

static __device__ void tc_load_weights(const MlpBlock *W, const TcLayout &L)
{
    const int tid = threadIdx.x, n = blockDim.x;
    for (int i = tid; i < 64 * 4; i += n) {  // W1: 64 rows x 4 chunks of 16 B
        const int r = i >> 2, kc = i & 3;
        uint4 v = half_bf16x8(((const uint4 *)W->w1)[r * 4 + kc]);
        if (kc == 2) {  // columns 16-23: inputs 16-19, then b1/2 in columns 20-22
            __nv_bfloat16 hi, mid, lo;
            split3_bf16(0.5f * W->b1[r], hi, mid, lo);
            __nv_bfloat162 p2 = __halves2bfloat162(hi, mid), p3 = __halves2bfloat162(lo, __float2bfloat16_rn(0.f));
            v.z = *reinterpret_cast<uint32_t *>(&p2);
            v.w = *reinterpret_cast<uint32_t *>(&p3);
        }
        *(uint4 *)(g_smem + L.w1 + tc_off32(r, kc)) = v;
    }
    for (int i = tid; i < 64 * 10; i += n) {  // W2: 64 rows x 10 chunks
        const int r = i / 10, kc = i - 10 * (i / 10);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (kc < 8) {
            v = half_bf16x8(((const uint4 *)W->w2)[r * 8 + kc]);
        } else if (kc == 8) {  // columns 64-66: b2/2
            __nv_bfloat16 hi, mid, lo;
            split3_bf16(0.5f * W->b2[r], hi, mid, lo);
            __nv_bfloat162 p0 = __halves2bfloat162(hi, mid), p1 = __halves2bfloat162(lo, __float2bfloat16_rn(0.f));
            v.x = *reinterpret_cast<uint32_t *>(&p0);
            v.y = *reinterpret_cast<uint32_t *>(&p1);
        }
        *(uint4 *)(g_smem + L.w2 + tc_off80(r, kc)) = v;
    }
    for (int i = tid; i < 64; i += n) ((float *)(g_smem + L.w3))[i] = W->w3[i];
    if (tid == 0) *(float *)(g_smem + L.b3) = W->b3;
}

// Constant columns 64-79 of this thread's row of its warpgroup's H tile:
// ones in 64-66 (the bias parts of W2), zeros after.
__device__ __forceinline__ void tc_init_h_row(const TcLayout &L, uint32_t r)
{
    *(uint4 *)(g_smem + L.h + tc_off80(r, 8)) = make_uint4(0x3F803F80u, 0x00003F80u, 0u, 0u);
    *(uint4 *)(g_smem + L.h + tc_off80(r, 9)) = make_uint4(0u, 0u, 0u, 0u);
}

// silu(2h) = h + h tanh(h), with the hardware tanh approximation.
__device__ __forceinline__ float silu_of_half(float h)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(h));
    return fmaf(h, t, h);
}

// Start of the kernel: one mbarrier per warpgroup, TMEM allocation (warp 0,
// kTcCols columns per warpgroup).  Every thread of the CTA calls it after the
// weights are loaded; it ends with a CTA barrier.  nwg = warpgroups per CTA.
static __device__ void tc_setup(TcEval &E, int nwg)
{
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const int wg = threadIdx.x >> 7;
    tc_init_h_row(E.L, threadIdx.x & 127);
    if ((threadIdx.x & 127) == 0) {
        mbar_init(s0 + E.L.mbar, 1);
        mbar_init(s0 + E.L.mbar + 8, 1);
    }
    if (threadIdx.x < 32) tc_alloc(s0 + E.L.tmem_slot, kTcCols * nwg);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    E.tmem = *(const uint32_t *)(g_smem + E.L.tmem_slot) + kTcCols * wg;
    E.phase1 = E.phase2 = 0;
    E.bar = 1 + wg;
}

static __device__ void tc_teardown(TcEval &E, int nwg)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tc_dealloc(*(const uint32_t *)(g_smem + E.L.tmem_slot), kTcCols * nwg);
}

// Writes the features of row r into the X tile (q0 < 0 and zero histograms
// give a row of zeros).
__device__ __forceinline__ void tc_write_features(const TcLayout &L, uint32_t r, int q0, uint32_t h1, uint32_t h2,
                                                  uint32_t h3)
{
    uint32_t w[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        float v[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int col = 2 * c + u;
            float x = 0.f;
            if (col < 5)
                x = (col == q0) ? 1.f : 0.f;
            else if (col < 10)
                x = (float)((h1 >> (4 * (col - 5))) & 15u);
            else if (col < 15)
                x = (float)((h2 >> (4 * (col - 10))) & 15u);
            else if (col < 20)
                x = (float)((h3 >> (4 * (col - 15))) & 15u);
            else if (col < 23)
                x = 1.f;  // against the bias parts of W1
            v[u] = x;
        }
        w[c] = pack_bf16(v[0], v[1]);
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
        *(uint4 *)(g_smem + L.x + tc_off32(r, kc)) = make_uint4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
}

// Feature value (BF16 -> float) of column k of row r of the X tile.
__device__ __forceinline__ float tc_feature(const TcLayout &L, uint32_t r, int k)
{
    const __nv_bfloat16 *p = (const __nv_bfloat16 *)(g_smem + L.x + tc_off32(r, (uint32_t)(k >> 3)));
    return __bfloat162float(p[k & 7]);
}

__device__ __forceinline__ void tc_timeout(TcEval &E)
{
    atomicCAS(E.status, 0, (int)SMC_ERR_TIMEOUT);
    atomicExch(E.abort_flag, 1);
}

// The evaluation of a tile in three stages, so that a warpgroup can overlap
// the products of one tile with the gathers and epilogue of another:
//   tc_issue1   (after the rows of the X tile are written and fenced)
//               layer-1 products X -> D1, committed to mbarrier 1
//   tc_stage2   waits for them, layer-1 epilogue D1 -> H, layer-2 products
//               H -> D2 committed to mbarrier 2; the X tile is free again
//   tc_finish   waits for them, returns f of row (threadIdx.x mod 128)
// All 128 threads of the warpgroup call every stage.  Between tc_stage2 of
// a tile and its tc_finish the warpgroup may write the next tile's X rows and
// call tc_issue1 for it (D1 and D2 are distinct TMEM columns).
static __device__ __forceinline__ void tc_issue1(TcEval &E)
{
    const int r = threadIdx.x & 127;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const TcLayout &L = E.L;
    tc_fence_before();
    wg_sync(E.bar);
    if (r == 0) {
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < 2; ++k)
            tc_mma(E.tmem, tc_desc(s0 + L.x + k * 256, 128, 512), tc_desc(s0 + L.w1 + k * 256, 128, 512), k > 0);
        tc_commit(s0 + L.mbar);
    }
}

static __device__ __forceinline__ void tc_stage2(TcEval &E)
{
    const int r = threadIdx.x & 127, wq = r >> 5;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const TcLayout &L = E.L;
    if (!mbar_wait(s0 + L.mbar, E.phase1, E.timeout_ns)) tc_timeout(E);
    E.phase1 ^= 1;
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint32_t v[32];
        tc_ld32(E.tmem + lane_base + 32 * half, v);
        tc_wait_ld(v);
#pragma unroll
        for (int kc = 0; kc < 4; ++kc) {
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                w[u] = pack_bf16(silu_of_half(__uint_as_float(v[8 * kc + 2 * u])),
                                 silu_of_half(__uint_as_float(v[8 * kc + 2 * u + 1])));
            *(uint4 *)(g_smem + L.h + tc_off80(r, 4 * half + kc)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    fence_async_smem();
    tc_fence_before();
    wg_sync(E.bar);
    if (r == 0) {
        tc_fence_after();
#pragma unroll
        for (int k = 0; k < kTcK2 / 16; ++k)
            tc_mma(E.tmem + 64, tc_desc(s0 + L.h + k * 256, 128, 1280), tc_desc(s0 + L.w2 + k * 256, 128, 1280),
                   k > 0);
        tc_commit(s0 + L.mbar + 8);
    }
}

static __device__ __forceinline__ float tc_finish(TcEval &E)
{
    const int r = threadIdx.x & 127, wq = r >> 5;
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    const TcLayout &L = E.L;
    if (!mbar_wait(s0 + L.mbar + 8, E.phase2, E.timeout_ns)) tc_timeout(E);
    E.phase2 ^= 1;
    tc_fence_after();
    const uint32_t lane_base = (uint32_t)(32 * wq) << 16;
    const float4 *w3 = (const float4 *)(g_smem + L.w3);
    float acc = 0.f;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        uint32_t v[32];
        tc_ld32(E.tmem + lane_base + 64 + 32 * half, v);
        tc_wait_ld(v);
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
            const float4 w = w3[8 * half + j4];
            acc = fmaf(w.x, silu_of_half(__uint_as_float(v[4 * j4])), acc);
            acc = fmaf(w.y, silu_of_half(__uint_as_float(v[4 * j4 + 1])), acc);
            acc = fmaf(w.z, silu_of_half(__uint_as_float(v[4 * j4 + 2])), acc);
            acc = fmaf(w.w, silu_of_half(__uint_as_float(v[4 * j4 + 3])), acc);
        }
    }
    tc_fence_before();
    return *(const float *)(g_smem + L.b3) + acc;
}

// f of row (threadIdx.x mod 128) of the warpgroup's X tile, unpipelined.
static __device__ __forceinline__ float tc_eval(TcEval &E)
{
    tc_issue1(E);
    tc_stage2(E);
    return tc_finish(E);
}

}  // namespace smc
