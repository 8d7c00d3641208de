// pair_fixed.cuh -- dE of a pair-model swap trial in exact fixed point, from
// per-shell species histograms (Algorithm 1 with pair site energies).
//
// For a trial a <-> b with species A = s_a, B = s_b and
// D_m[q] = V_m(B, q) - V_m(A, q),
//   dE = sum_m sum_q c_m[q] D_m[q],
//   c_m[q] = #{j in N_m(a) \ b : s_j = q} - #{j in N_m(b) \ a : s_j = q}.
// Each shell holds as many neighbours of a (without b) as of b (without a),
// so sum_q c_m[q] = 0 and the reference species R = S - 1 drops out:
//   dE = sum_m sum_{q < R} c_m[q] D'_m[q],  D'_m[q] = D_m[q] - D_m[R].
// The coefficients are taken in fixed point, Q_m[q] = round(D'_m[q] 2^sigma)
// (integer models: sigma = 0 and Q = D' exactly), and the counts live in
// 8-bit fields of 32-bit words, biased by b_m (8 for shells 1-2, whose
// |c| <= 7, and 16 for shell 3, |c| <= 12): word w of shell m holds
// c_m[4w + j] + b_m in byte j.  Then
//   dE_fix = sum_m sum_w dot4(H_m^w, Q_m^w) - sum_m b_m sum_q Q_m[q]
// where dot4 is a four-byte dot product.  Q is split into four byte planes,
// Q = P0 + 2^8 P1 + 2^16 P2 + 2^24 P3 (P3 signed), so that every dot4 is one
// dp4a instruction; all of it is int32 arithmetic modulo 2^32, which is exact
// because the true dE_fix lies in (-2^31, 2^31) (sigma is chosen so).  The
// result dE_fix 2^-sigma differs from the exact dE of the FP32 coefficients
// by at most sum_q |c_m[q]| 2^-(sigma+1) <= 13 * 2^-sigma for two shells.
//
// A site of species s adds 1 << (8 s) to the low word (zero for s >= 4: the
// shift amount is clamped, not wrapped) and 1 << (8 s - 32) to the high word
// (species 4..7; zero for s < 4).  The sweep kernels keep species multiplied
// by 8 in memory during a launch, so the shift amount is the stored byte.
#pragma once

#include "sweep_common.cuh"

namespace smc {

// Words of a table row (A, B): shells x species words x 4 byte planes, then
// the bias word, padded to a multiple of 4 words (16-byte loads).
__host__ __device__ constexpr int qrow_words(int NSH, int SW) { return (NSH * SW * 4 + 1 + 3) / 4 * 4; }
constexpr int kQRows = kMaxSpecies * kMaxSpecies;  // row A * 8 + B
constexpr int kMaxQRowWords = 28;                  // three shells, two species words
static_assert(qrow_words(3, 2) == kMaxQRowWords, "row size");
constexpr float kAcceptBias = 30.0f;               // 2^30 = twice the range of the acceptance word r

__device__ __forceinline__ uint32_t nib8(uint32_t v8)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(v8));  // clamped: 0 for v8 >= 32
    return r;
}
__device__ __forceinline__ uint32_t nib8hi(uint32_t v8)
{
    uint32_t r;
    asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(1u), "r"(v8 - 32u));  // 0 for v8 < 32 (huge shift)
    return r;
}
__device__ __forceinline__ uint32_t dp4a_uu(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t dp4a_us(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Histogram words of one shell (SW words of four 8-bit fields).
template <int SW>
__device__ __forceinline__ void hadd(uint32_t (&h)[SW], uint32_t v8)
{
    h[0] += nib8(v8);
    if constexpr (SW == 2) h[1] += nib8hi(v8);
}
template <int SW>
__device__ __forceinline__ void hsub(uint32_t (&h)[SW], uint32_t v8)
{
    h[0] -= nib8(v8);
    if constexpr (SW == 2) h[1] -= nib8hi(v8);
}

// Histogram words of one neighbour (SW words of four 8-bit fields), summed
// as values so that the counts of a shell form short add trees instead of
// one chain of dependent adds.
template <int SW>
struct HV {
    uint32_t w[SW];
};
template <int SW>
__device__ __forceinline__ HV<SW> hv(uint32_t v8)
{
    HV<SW> h;
    h.w[0] = nib8(v8);
    if constexpr (SW == 2) h.w[1] = nib8hi(v8);
    return h;
}
template <int SW>
__device__ __forceinline__ HV<SW> hconst(uint32_t c)
{
    HV<SW> h;
#pragma unroll
    for (int w = 0; w < SW; ++w) h.w[w] = c;
    return h;
}
template <int SW>
__device__ __forceinline__ HV<SW> operator+(const HV<SW> &a, const HV<SW> &b)
{
    HV<SW> h;
#pragma unroll
    for (int w = 0; w < SW; ++w) h.w[w] = a.w[w] + b.w[w];
    return h;
}
template <int SW>
__device__ __forceinline__ HV<SW> operator-(const HV<SW> &a, const HV<SW> &b)
{
    HV<SW> h;
#pragma unroll
    for (int w = 0; w < SW; ++w) h.w[w] = a.w[w] - b.w[w];
    return h;
}

// dE_fix of the histogram words H[m][w] against table row `row` (smem or
// global, 16-byte aligned).
template <int NSH, int SW>
__device__ __forceinline__ int32_t dot_fixed(const uint32_t (&H)[NSH][SW], const uint32_t *row)
{
    constexpr int NB = NSH * SW * 4;
    uint32_t p0 = row[NB], p1 = 0u, p2 = 0u, p3 = 0u;
#pragma unroll
    for (int m = 0; m < NSH; ++m)
#pragma unroll
        for (int w = 0; w < SW; ++w) {
            const uint4 q = *(const uint4 *)(row + (m * SW + w) * 4);
            p0 = dp4a_uu(H[m][w], q.x, p0);
            p1 = dp4a_uu(H[m][w], q.y, p1);
            p2 = dp4a_uu(H[m][w], q.z, p2);
            p3 = dp4a_us(H[m][w], q.w, p3);
        }
    return (int32_t)(p0 + (p1 << 8) + (p2 << 16) + (p3 << 24));
}

// Metropolis decision on dE_fix.  Integer models (sigma = 0): dE <= 0 or
// r < T[dE] (host FP64 table).  Floating-point models: dE <= 0 or
// r + 1/2 < 2^29 exp(-dE / kT).  With 2^30 exp(-dE / kT) = 2^x,
// x = dE_fix cx + 30 and cx = -log2(e) 2^-sigma / kT (host FP64, rounded to
// FP32), u = 2^x from ex2.approx, the test is 2r + 1 < u, and since 2r + 1 is
// an integer this is exactly 2r + 1 < ceil(u) in integers.
template <bool IS_INT>
__device__ __forceinline__ bool accept_fixed(int32_t dE, uint32_t r, float cx, const uint32_t *tab, int2 ti)
{
    if constexpr (IS_INT) {
        if (dE <= 0) return true;
        return dE < ti.y && r < __ldg(tab + ti.x + dE);
    } else {
        const float u = ex2_approx(fmaf((float)dE, cx, kAcceptBias));
        const int thr = __float2int_ru(u);  // saturates for u >= 2^31 (then dE < 0)
        return (dE <= 0) | ((int)(2u * r + 1u) < thr);
    }
}

// Replicated table (two shells, one species word: at most 4 + 1 species): for shell m and row A * 5 + B, eight copies of
// the row's four plane words side by side (128 bytes), copy j read by the
// lanes j, j + 8, ... -- the 8 lanes that a 16-byte shared load serves at
// once then read 8 different bank groups, whatever their rows.  No bias
// word: the counts are biased by 128 per field and turned into signed bytes
// (c + 128) ^ 0x80 = c for dp4a with signed first operands.
constexpr int kRTabRows = 25;
constexpr int kRTabBytes = 2 * kRTabRows * 128;

__device__ __forceinline__ uint32_t dp4a_su(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t dp4a_ss(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm("dp4a.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

// dE_fix from two shells' count words biased by 128 per field and the
// replicated table's row for (A, B) (absolute offset `row`, shell 1 at
// + kRTabRows * 128): sum over shells of dot4(c, Q) with signed c.
__device__ __forceinline__ int32_t dot_fixed_rtab(uint32_t h0, uint32_t h1, uint32_t row)
{
    const uint4 q0 = *(const uint4 *)(g_smem + row);
    const uint4 q1 = *(const uint4 *)(g_smem + row + kRTabRows * 128);
    const uint32_t c0 = h0 ^ 0x80808080u, c1 = h1 ^ 0x80808080u;
    const uint32_t p0 = dp4a_su(c1, q1.x, dp4a_su(c0, q0.x, 0u));
    const uint32_t p1 = dp4a_su(c1, q1.y, dp4a_su(c0, q0.y, 0u));
    const uint32_t p2 = dp4a_su(c1, q1.z, dp4a_su(c0, q0.z, 0u));
    const uint32_t p3 = dp4a_ss(c1, q1.w, dp4a_ss(c0, q0.w, 0u));
    return (int32_t)(p0 + (p1 << 8) + (p2 << 16) + (p3 << 24));
}

// Writes the replicated table at shared offset 0: word i of (shell m, row
// A * 5 + B, copy j) is plane word i of shell m in row A * 8 + B of the
// plain table (qrow words per row).
__device__ __forceinline__ void fill_rtab(const uint32_t *qtab, int qrow, int tid, int nthr)
{
    for (int e = tid; e < 2 * kRTabRows * 8 * 4; e += nthr) {
        const int i = e & 3, row = (e >> 5) % kRTabRows, m = (e >> 5) / kRTabRows;
        const int A = row / 5, B = row % 5;
        ((uint32_t *)g_smem)[e] = qtab[(A * 8 + B) * qrow + m * 4 + i];
    }
}

// Host: fixed-point table of a pair model (rows A * 8 + B, A, B < 8; rows of
// species >= S are zero).  Returns false if a coefficient is not finite.
struct PairTable {
    int nsh = 2, sw = 1, rw = 12, sigma = 0;
    double scale = 1.0;  // eV (or units) per dE_fix unit: 2^-sigma
    std::vector<uint32_t> rows;
};
bool build_pair_table(const smc_model *m, int S, PairTable &t);

// The resident sweep (sweep_resident.cu) of R replicas: SMC_ERR_UNSUPPORTED,
// with nothing enqueued, when a replica does not fit it.
smc_status launch_pair_sweep_resident(int R, const smc_lattice *lats, const smc_model *m, const PairTable &pt,
                                      int8_t *const *occ, uint64_t seed, uint32_t replica0, uint64_t sweep0,
                                      int nsweeps, const double *kT, double *e_acc, int64_t *n_acc,
                                      cudaStream_t stream);
int debug_resident();

}  // namespace smc
