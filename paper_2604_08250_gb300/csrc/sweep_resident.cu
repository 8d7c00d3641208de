// sweep_resident.cu -- the pair-model sweep with the lattice resident in
// shared memory, for lattices whose rows fit in the SMs' shared memory
// (128^3 cells: 4.2 MB of 34 MB).
//
// The same schedule and arithmetic as the streaming kernel of sweep_pair.cu
// (groups of four mini-steps, one column of link cells per warp, the exact
// fixed-point dE of pair_fixed.cuh), so the trajectories are the same bit for
// bit.  What changes is where the rows live.  Each CTA owns a rectangular
// block of columns and keeps in shared memory every row its columns ever
// touch (a window of 4 b + 7 rows per axis and sublattice), for the whole
// launch.  Rows that another CTA also touches travel as versions:
//
//   after group g, a CTA publishes each row its columns wrote at g that
//   another CTA reads before the row's next write: 64-bit words of 4
//   species bytes (x 8) and the tag g + 1 (g counted from the launch);
//   before group g, it fetches the rows its columns read at g whose last
//   write is another CTA's and whose version it has not read since, polling
//   each word until it carries the expected tag.
//
// A word is single-copy atomic, so a matching tag means matching bytes; no
// fence or flag sits between a write and its readers, only the data's own
// latency.  Versions live in two copies (by sweep parity) of one slot per
// (group of the write, row): the copy a write overwrites was last read 33
// groups earlier, and the CTA's exchange warps make sure its neighbours have
// finished that group (their progress flags, released by each CTA's release
// warp) before READY -- a check that in practice never waits.  The host
// builds the lists from the groups' row-level read and write sets.
//
// Roles in a CTA: warps 0..nc-1 run the trials of one column each and
// publish the rows they wrote; the exchange warps fetch the next group's
// versions (with their periodic x-halos) while the current group runs and
// arrive on READY; the release warp releases the CTA's progress flag once
// every compute warp has counted a group as done.  The exchange warps fetch
// for group g + 2 once the compute warps finished g - 1, so a fetch may land
// while group g or g + 1 runs.  A fetched row is not written by this CTA in
// either (its last writer before g + 2 is another CTA), and if one of them
// reads it, it reads the same bytes: a newer version would be a write by a
// neighbour at g + 1 of a row this CTA touches at g (excluded by the lag-2
// rule when g + 1 has dy >= 1, and impossible when it has dy = 0, since the
// neighbour then waits for this CTA's g) or at g + 1 (same-group
// disjointness).  The READY barriers cycle through four named barriers so
// that the exchange warps' arrivals for different groups never meet in one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <vector>

#include "pair_fixed.cuh"

namespace smc {

namespace {

// Block descriptor (ints): [0..3] first column (cy, cz) and columns per axis,
// [4..7] window origin y (sublattice 0, 1) and z (0, 1), [8..9] list offset
// and size, [10] replica (index into P.rep), [11] block index within the
// replica, [12..13] blocks per axis of the replica, [14] global index of the
// replica's first block (its progress flags), [15..16] window rows per axis,
// [17] row pitch, [18] offset of the replica's lattice copy (bytes),
// [19] offset of its version slots (words), [20] its version slots.
constexpr int kResDesc = 24;
constexpr int kResCols = 8;  // compute warps per CTA (columns per block at most)

// The exchange warps prepare group g once the compute warps finished group
// g - kAhead - 1, so while groups g - kAhead .. g - 1 may still wait for
// their compute warps.  READY barriers cycle through kBars > kAhead named
// barriers by group, so that arrivals for different groups never meet in one.
constexpr int kAhead = 2, kBars = 4;
__device__ __forceinline__ int bar_ready(int gs) { return 1 + (gs & (kBars - 1)); }

// bar.sync / bar.arrive are the warp-aligned barrier forms: every lane of
// the warp must execute them together, so the warp reconverges first.
__device__ __forceinline__ void named_sync(int id, int n)
{
    __syncwarp();
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n)
{
    __syncwarp();
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

#define RD8(off) ((uint32_t)g_smem[(off)])

// dE_fix of the trial at a (ya = shared offset of a, own row) with pa = the
// partner row (y0 + s_off, z0 + s_off) at x + s_off; rows are rb apart in y
// and RZ apart in z on both sublattices.  XB: the replicated table at shared
// offset 0 (qt = this lane's copy offset), counts biased by 128 per field;
// else the plain table.
template <int NSH, int SW, bool XB = false>
__device__ __forceinline__ int32_t res_dE(uint32_t ya, uint32_t pa, uint32_t rb, uint32_t RZ, uint32_t w,
                                          uint32_t qt, uint32_t &a8, uint32_t &b8, uint32_t &pb)
{
    static_assert(!XB || (NSH == 2 && SW == 1), "replicated table: two shells, one species word");
    // partner direction = w >> 29 = (kx, ky, kz): b = pa + ky rb + kz RZ + kx,
    // and b's own-sublattice neighbours start (ky - 1, kz - 1, kx - 1) from a
    const uint32_t offb = ((w >> 30) & 1u) * rb + ((w >> 29) & 1u) * RZ + (w >> 31);
    a8 = RD8(ya);
    pb = pa + offb;
    b8 = RD8(pb);
    using HW = HV<SW>;
    constexpr uint32_t B12 = XB ? 0x80808080u : 0x08080808u;
    const uint32_t ob = ya + offb - rb - RZ - 1u;
    // shell 1: a's 8 partner-sublattice neighbours minus b, minus b's 8
    // trial-sublattice neighbours plus a (short add trees)
    const HW a0 = hconst<SW>(B12) + hv<SW>(a8) + hv<SW>(RD8(pa));
    const HW a1 = hv<SW>(RD8(pa + 1)) + hv<SW>(RD8(pa + rb)) + hv<SW>(RD8(pa + rb + 1));
    const HW a2 = hv<SW>(RD8(pa + RZ)) + hv<SW>(RD8(pa + RZ + 1)) + hv<SW>(RD8(pa + RZ + rb));
    const HW a3 = hv<SW>(RD8(pa + RZ + rb + 1));
    const HW b0 = hv<SW>(b8) + hv<SW>(RD8(ob)) + hv<SW>(RD8(ob + 1));
    const HW b1 = hv<SW>(RD8(ob + rb)) + hv<SW>(RD8(ob + rb + 1)) + hv<SW>(RD8(ob + RZ));
    const HW b2 = hv<SW>(RD8(ob + RZ + 1)) + hv<SW>(RD8(ob + RZ + rb)) + hv<SW>(RD8(ob + RZ + rb + 1));
    const HW h0 = (a0 + a1) + (a2 + a3) - ((b0 + b1) + b2);
    // shell 2: a's 6 trial-sublattice neighbours, b's 6 partner-sublattice ones
    const HW c0 = hconst<SW>(B12) + hv<SW>(RD8(ya - 1)) + hv<SW>(RD8(ya + 1));
    const HW c1 = hv<SW>(RD8(ya - rb)) + hv<SW>(RD8(ya + rb)) + hv<SW>(RD8(ya - RZ));
    const HW c2 = hv<SW>(RD8(ya + RZ));
    const HW d0 = hv<SW>(RD8(pb - 1)) + hv<SW>(RD8(pb + 1)) + hv<SW>(RD8(pb - rb));
    const HW d1 = hv<SW>(RD8(pb + rb)) + hv<SW>(RD8(pb - RZ)) + hv<SW>(RD8(pb + RZ));
    const HW h1 = ((c0 + c1) + c2) - (d0 + d1);
    uint32_t H[NSH][SW];
#pragma unroll
    for (int w = 0; w < SW; ++w) {
        H[0][w] = h0.w[w];
        H[1][w] = h1.w[w];
    }
    if constexpr (NSH >= 3) {
        // shell 3: a's 12 trial-sublattice neighbours, b's 12
        // partner-sublattice ones (biased by 16 per field)
        const HW e0 = hconst<SW>(0x10101010u) + hv<SW>(RD8(ya - rb - RZ)) + hv<SW>(RD8(ya + rb - RZ));
        const HW e1 = hv<SW>(RD8(ya - rb + RZ)) + hv<SW>(RD8(ya + rb + RZ)) + hv<SW>(RD8(ya - rb - 1));
        const HW e2 = hv<SW>(RD8(ya - rb + 1)) + hv<SW>(RD8(ya + rb - 1)) + hv<SW>(RD8(ya + rb + 1));
        const HW e3 = hv<SW>(RD8(ya - RZ - 1)) + hv<SW>(RD8(ya - RZ + 1)) + hv<SW>(RD8(ya + RZ - 1));
        const HW e4 = hv<SW>(RD8(ya + RZ + 1));
        const HW f0 = hv<SW>(RD8(pb - rb - RZ)) + hv<SW>(RD8(pb + rb - RZ)) + hv<SW>(RD8(pb - rb + RZ));
        const HW f1 = hv<SW>(RD8(pb + rb + RZ)) + hv<SW>(RD8(pb - rb - 1)) + hv<SW>(RD8(pb - rb + 1));
        const HW f2 = hv<SW>(RD8(pb + rb - 1)) + hv<SW>(RD8(pb + rb + 1)) + hv<SW>(RD8(pb - RZ - 1));
        const HW f3 = hv<SW>(RD8(pb - RZ + 1)) + hv<SW>(RD8(pb + RZ - 1)) + hv<SW>(RD8(pb + RZ + 1));
        const HW h2 = ((e0 + e1) + (e2 + e3) + e4) - ((f0 + f1) + (f2 + f3));
#pragma unroll
        for (int w = 0; w < SW; ++w) H[2][w] = h2.w[w];
    }
    if constexpr (XB) {
        return dot_fixed_rtab(H[0][0], H[1][0], qt + (a8 * 5u + b8) * 16u);
    } else {
        constexpr uint32_t half_row = (uint32_t)qrow_words(NSH, SW) / 2;  // (A * 8 + B) rows = (8 a8 + b8) / 8
        return dot_fixed<NSH, SW>(H, (const uint32_t *)(g_smem + (8u * a8 + b8) * half_row));
    }
}

// Shared-memory body offset of window row (s, y, z) of a block whose window
// on sublattice s starts at (ylo, zlo).
__device__ __forceinline__ uint32_t res_body(int ylo, int zlo, int s, int y, int z, int ny, int nz, int Wy, int Wz,
                                             uint32_t rows, uint32_t rb)
{
    int yy = y - ylo, zz = z - zlo;
    yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
    zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
    return rows + (uint32_t)((s * Wz + zz) * Wy + yy) * rb + 16u;
}

// The progress flag of neighbour lane (lanes 0..8 but 4: (dy, dz) = (lane % 3
// - 1, lane / 3 - 1)); nullptr for the other lanes.
__device__ __forceinline__ const uint32_t *res_flag(const SweepParams &P, const int *d, int lane)
{
    if (lane >= 9 || lane == 4) return nullptr;
    const int NBy = d[12], NBz = d[13];
    int nby = d[11] % NBy + (lane % 3) - 1, nbz = d[11] / NBy + (lane / 3) - 1;
    nby = nby < 0 ? nby + NBy : (nby >= NBy ? nby - NBy : nby);
    nbz = nbz < 0 ? nbz + NBz : (nbz >= NBz ? nbz - NBz : nbz);
    return P.flags + d[14] + nbz * NBy + nby;
}

// Gives up a wait: records a timeout (unless another block aborted first)
// and raises the block's and the launch's abort flags.
__device__ __forceinline__ void res_give_up(const SweepParams &P, volatile int *s_abort, bool timed_out)
{
    if (timed_out) {
        atomicCAS(P.status, 0, (int)SMC_ERR_TIMEOUT);
        atomicExch(P.abort_flag, 1);
    }
    *s_abort = 1;
}

// Bounded wait (whole warp) until the 8 neighbouring blocks' progress flags
// are >= need; false once the launch or the block aborts or the time runs out.
// *seen receives the smallest flag read by the successful look.
__device__ bool res_wait(const SweepParams &P, const uint32_t *fp, uint32_t need, volatile int *s_abort, int lane,
                         uint32_t *seen)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        const uint32_t v = fp == nullptr ? 0xffffffffu : ld_acquire_u32(fp);
        if (__all_sync(0xffffffffu, v >= need)) {
            *seen = __reduce_min_sync(0xffffffffu, v);
            return true;
        }
        int stop = 0;
        if (lane == 0) {
            const bool late = (long long)(global_ns() - t0) > P.timeout_ns;
            if (late || *s_abort || ld_volatile_i32(P.abort_flag)) {
                res_give_up(P, s_abort, late);
                stop = 1;
            }
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) return false;
    }
}

// Bounded wait (whole warp) until the block's count of finished
// (compute warp, group) pairs is >= need; acquires the compute warps' writes.
__device__ bool res_wait_count(const SweepParams &P, const volatile unsigned *cnt, unsigned need,
                               volatile int *s_abort, int lane)
{
    const uint64_t t0 = global_ns();
    int stop = 0;
    if (lane == 0) {
        while (*cnt < need) {
            const bool late = (long long)(global_ns() - t0) > P.timeout_ns;
            if (late || *s_abort || ld_volatile_i32(P.abort_flag)) {
                res_give_up(P, s_abort, late);
                stop = 1;
                break;
            }
        }
        __threadfence_block();
    }
    return __shfl_sync(0xffffffffu, stop, 0) == 0;
}

// Row versions.  Every row a block writes in group g and another block
// reads before its next write is published as a version: (nx + 7) / 8
// 16-byte chunks of two words (4 species bytes | tag << 32) (when nx is
// 4 mod 8 the last word carries no species), tag = global group of the write + 1, in
// copy (global group >> 5) & 1 of its version slot.  A reader knows the
// tag it needs, so it polls the words themselves: a word with that tag holds
// that version's bytes (each 64-bit word is single-copy atomic), and no fence
// or flag stands between the write and the read.
__device__ __forceinline__ uint32_t ver_word(int nver, int gw, uint32_t vid, int nx)
{
    return ((uint32_t)((gw >> 5) & 1) * (uint32_t)nver + vid) * (uint32_t)(((nx + 7) >> 3) * 2);
}

// Fetches the versions of list entries ent[0, n) ({smem slot | d << 16,
// version slot}) that group G reads, written in group G - d (entries with
// G - d < 0 predate the launch and are already in the window).  The nxw
// exchange warps share the 16-byte chunks (chunk q to warp (q / 32) % nxw),
// K chunks per lane per round, each chunk polled until both its words carry
// the tag.  False on timeout or abort.
template <int K>
__device__ bool res_fetch_versions(const SweepParams &P, const unsigned long long *xver, int nver, const uint2 *ent,
                                   int n, uint32_t rows, uint32_t rb, int nx, int G, int xw, int nxw,
                                   volatile int *s_abort, int lane)
{
    const int cpr = (nx + 7) >> 3;  // the last chunk holds 4 species when nx % 8 == 4
    const bool half = (nx & 7) != 0;
    const int tot = n * cpr, step = 32 * nxw, de = step / cpr, dc = step - de * cpr;
    const uint64_t t0 = global_ns();
    for (int base = 0; base < tot; base += step * K) {
        uint32_t src[K], dst[K], tag[K];  // word offset in xver, shared address, tag
        uint32_t todo = 0u, first = 0u, last = 0u;  // chunks that also fill the right / left x-halo
        {
            const int q0 = base + 32 * xw + lane;
            int e = q0 / cpr, c = q0 - e * cpr;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                src[k] = 0u;
                dst[k] = 0u;
                tag[k] = 0u;
                if (e < n) {
                    const uint2 en = ent[e];
                    const int gw = G - (int)(en.x >> 16);
                    if (gw >= 0) {
                        src[k] = ver_word(nver, gw, en.y, nx) + 2u * (uint32_t)c;
                        dst[k] = rows + (en.x & 0xffffu) * rb + 16u + 8u * (uint32_t)c;
                        tag[k] = (uint32_t)gw + 1u;
                        todo |= 1u << k;
                        if (c == 0) first |= 1u << k;
                        if (c == cpr - 1) last |= 1u << k;
                    }
                }
                e += de;
                c += dc;
                if (c >= cpr) {
                    c -= cpr;
                    ++e;
                }
            }
        }
        while (__any_sync(0xffffffffu, todo != 0u)) {
            ulonglong2 v[K];
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (todo & (1u << k)) v[k] = ld_relaxed_v2u64(xver + src[k]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if ((todo & (1u << k)) && (uint32_t)(v[k].x >> 32) == tag[k] && (uint32_t)(v[k].y >> 32) == tag[k]) {
                    const bool lk = (last >> k) & 1u;
                    if (half && lk) {
                        *(uint32_t *)(g_smem + dst[k]) = (uint32_t)v[k].x;
                    } else {
                        *(uint2 *)(g_smem + dst[k]) = make_uint2((uint32_t)v[k].x, (uint32_t)v[k].y);
                    }
                    // periodic x-halos: body[0..4) after the row, body[nx-4..nx) before it
                    if (first & (1u << k)) *(uint32_t *)(g_smem + dst[k] + nx) = (uint32_t)v[k].x;
                    if (lk)
                        *(uint32_t *)(g_smem + dst[k] + (half ? 0 : 4) - nx) =
                            half ? (uint32_t)v[k].x : (uint32_t)v[k].y;
                    todo &= ~(1u << k);
                }
            }
            const bool pending = __any_sync(0xffffffffu, todo != 0u);
            int stop = 0;
            if (pending && lane == 0) {
                const bool late = (long long)(global_ns() - t0) > P.timeout_ns;
                if (late || *s_abort || ld_volatile_i32(P.abort_flag)) {
                    res_give_up(P, s_abort, late);
                    stop = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) return false;
        }
    }
    return true;
}

// RB, WY: the row pitch and window rows per y of every block, when known at
// compile time (0: read from the descriptor), so that the trial's row offsets
// are immediates.  Those kernels (two shells, one species word) also take
// the replicated pair table (res_xb_table).
template <bool IS_INT, int NSH, int SW, int RB, int WY>
__global__ void __launch_bounds__(416, 1) k_sweep_resident(const __grid_constant__ SweepParams P)
{
    constexpr bool XB = RB != 0 && WY != 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    // compute warps, then P.rxw exchange warps, then the release warp
    const int nxw = P.rxw, nc = nwarp - nxw - 1, nbar = (nc + nxw) * 32;
    const int blk = blockIdx.x;
    const int *d = P.rdesc + blk * kResDesc;
    const int rep = d[10];
    const RepDesc &RD = P.rep[rep];
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NLx = RD.NLx;
    const int Wy = WY ? WY : d[15], Wz = d[16];
    const uint32_t rb = RB ? (uint32_t)RB : (uint32_t)d[17], RZ = (uint32_t)Wy * rb;
    const int8_t *exch = P.exch + (uint32_t)d[18];
    unsigned long long *xver = P.xver + (uint32_t)d[19];
    const int nver = d[20];
    const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    __shared__ volatile int s_abort;  // a wait gave up: stop
    __shared__ volatile int s_stop;   // the group at which the compute warps stop (set by the exchange warp)
    __shared__ unsigned s_cnt;        // (compute warp, group) pairs finished and published
    // shared memory: [table][rows][lists][Philox words per compute warp]
    const int qwords = kQRows * P.qrow;
    const uint32_t rows = XB ? (uint32_t)kRTabBytes : (uint32_t)qwords * 4u;
    const int nslots = 2 * Wy * Wz;
    const uint32_t lists = rows + (uint32_t)nslots * rb;
    const int nk = (NLx + 31) >> 5;
    const uint32_t wsm0 = lists + (uint32_t)P.rblob * 4u;
    if constexpr (XB)
        fill_rtab(P.qtab, P.qrow, tid, blockDim.x);
    else
        for (int i = tid; i < qwords; i += blockDim.x) ((uint32_t *)g_smem)[i] = P.qtab[i];
    const uint32_t qt = (uint32_t)(lane & 7) * 16u;
    const uint32_t *gl = P.rlists + d[8];
    uint32_t *L = (uint32_t *)(g_smem + lists);
    for (int i = tid; i < d[9]; i += blockDim.x) L[i] = gl[i];
    if (tid == 0) {
        s_abort = 0;
        s_stop = 0x7fffffff;
        s_cnt = 0u;
    }
    // the window's rows from the exchange copy (species x 8)
    {
        const bool v16 = (nx & 15) == 0;
        const int cb = v16 ? 16 : 4, cpr = nx / cb;
        for (int q = tid; q < nslots * cpr; q += blockDim.x) {
            const int slot = q / cpr, c = q - slot * cpr;
            const int s = slot / (Wy * Wz), yy = slot % Wy, zz = (slot / Wy) % Wz;
            int y = d[4 + s] + yy, z = d[6 + s] + zz;
            y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
            z = z < 0 ? z + nz : (z >= nz ? z - nz : z);
            const int8_t *src = exch + ((size_t)((s * nz + z) * ny + y)) * nx + cb * c;
            const uint32_t dst = smem0 + rows + (uint32_t)slot * rb + 16u + (uint32_t)(cb * c);
            if (v16)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
            else
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        for (int q = tid; q < 2 * nslots; q += blockDim.x) {
            const uint32_t body = rows + (uint32_t)(q >> 1) * rb + 16u;
            if (q & 1)
                *(unsigned *)(g_smem + body + nx) = *(const unsigned *)(g_smem + body);
            else
                *(unsigned *)(g_smem + body - 4) = *(const unsigned *)(g_smem + body + nx - 4);
        }
        __syncthreads();
    }
    const int total = P.nsweeps * 32;
    // list header (offsets in words): fetch lists per group [0..33), publish
    // lists per (group, compute warp) [33 .. 33 + 32 nc + 1), then the final
    // rows' offset and count; fetch and publish entries are word pairs
    const uint32_t *fo = L, *po = L + 33;
    const uint32_t fin0 = L[33 + 32 * nc + 1], fin1 = L[33 + 32 * nc + 2];

    if (warp >= nc && warp < nc + nxw) {
        // ---------------- exchange warps ----------------
        // Prepare group gs + 1 while the compute warps run group gs: the
        // versions of the rows it reads that another block wrote (with their
        // x-halos), shared between the exchange warps, then READY.
        const int xw = warp - nc;
        named_arrive(bar_ready(0), nbar);  // group 0: the window was loaded from the lattice copy
        const uint32_t *fp = res_flag(P, d, lane);
        uint32_t nbmin = 0u;  // a lower bound of the neighbours' progress flags
        bool ok = true;
        int gs = 0;
        for (; gs + 1 < total; ++gs) {
            const int nxt = gs + 1, gn = nxt & 31;
            // never more than kAhead groups ahead: the compute warps finished
            // nxt - kAhead - 1
            ok = res_wait_count(P, &s_cnt, (unsigned)(max(nxt - kAhead, 0) * nc), &s_abort, lane);
            // Group nxt's versions overwrite those of nxt - 64, which readers
            // fetch up to group nxt - 33: the neighbours must have finished it
            // (READY of nxt waits for this warp).
            if (ok && xw == 0 && nxt >= 64 && nbmin < (uint32_t)(nxt - 32))
                ok = res_wait(P, fp, (uint32_t)(nxt - 32), &s_abort, lane, &nbmin);
            if (ok)
                ok = res_fetch_versions<8>(P, xver, nver, (const uint2 *)(L + fo[gn]), (int)(fo[gn + 1] - fo[gn]) >> 1,
                                           rows, rb, nx, nxt, xw, nxw, &s_abort, lane);
            if (!ok) break;
            named_arrive(bar_ready(nxt), nbar);
        }
        if (!ok) {
            // The compute warps stop at READY of the smallest group an
            // exchange warp gave up before (s_stop, lowered before that
            // barrier's arrival).  If that is gs + 1, they pass the READYs
            // already given without waiting and finish group gs + 1 - kBars
            // in bounded time; only then is the barrier of gs + 1 free of
            // that group's arrivals.  If another exchange warp gave up at an
            // earlier group, the compute warps never reach gs + 1.
            int arrive = 0;
            if (lane == 0 && s_stop > gs) {
                atomicMin((int *)&s_stop, gs + 1);
                const uint64_t t0 = global_ns();
                while (*(volatile unsigned *)&s_cnt < (unsigned)(max(gs + 2 - kBars, 0) * nc) &&
                       (long long)(global_ns() - t0) < P.timeout_ns) {
                }
                arrive = 1;
            }
            if (__shfl_sync(0xffffffffu, arrive, 0)) named_arrive(bar_ready(gs + 1), nbar);
        }
    } else if (warp == nc + nxw) {
        // ---------------- release warp ----------------
        // Releases the block's progress flag once every compute warp finished
        // a group: the neighbours' exchange warps wait for it before their
        // versions overwrite the slots this block may still have to read
        // (st.release orders this block's reads before the flag).
        for (int gs = 0; gs < total; ++gs) {
            if (!res_wait_count(P, &s_cnt, (unsigned)((gs + 1) * nc), &s_abort, lane)) break;
            if (lane == 0 && blk != P.skip_tile) st_release_u32(P.flags + blk, (uint32_t)gs + 1);
        }
    } else {
        // ---------------- compute warps ----------------
        const bool active = warp < d[2] * d[3];
        const int cy = d[0] + warp % max(d[2], 1), cz = d[1] + warp / max(d[2], 1);
        const uint32_t wsm = wsm0 + (uint32_t)warp * (uint32_t)nk * 512u;
        const int ylo0 = d[4], ylo1 = d[5], zlo0 = d[6], zlo1 = d[7];
        // publish chunks: (nx + 7) / 8 per row (a last half chunk carries 4
        // bytes of the halo, not read); this lane's first chunk and the step
        const int cpr = (nx + 7) >> 3;
        const int pub_e0 = lane / cpr, pub_c0 = lane - pub_e0 * cpr, pub_de = 32 / cpr, pub_dc = 32 - pub_de * cpr;
        long long accE = 0, accN = 0;
        for (int gs = 0; gs < total; ++gs) {
            const int t = gs >> 5, g = gs & 31;
            const int dy = g & 3, dz = (g >> 2) & 3, sub = g >> 4, soff = sub == 0 ? -1 : 0;
            const int y0 = 4 * cy + dy, z0 = 4 * cz + dz;
            const uint64_t sweep = P.sweep0 + (uint64_t)t;
            U4 w4{0u, 0u, 0u, 0u};
            if (active) {
                // Philox words of this column's link cells for this group
                const uint32_t rowsite = (uint32_t)(((sub * nz + z0) * ny + y0) * nx);
                const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
                uint32_t *wp = (uint32_t *)(g_smem + wsm);
                if (nk == 1 && NLx == 32) {
                    w4 = philox10(U4{(rowsite >> 2) + (uint32_t)lane, RD.rep, (uint32_t)sweep, (uint32_t)(sweep >> 32)},
                                  k0, k1);
                } else {
#pragma unroll 1
                    for (int k = 0; k < nk; ++k) {
                        const int i = lane + 32 * k;
                        if (i < NLx) {
                            const U4 w = philox10(U4{(rowsite >> 2) + (uint32_t)i, RD.rep, (uint32_t)sweep,
                                                     (uint32_t)(sweep >> 32)},
                                                  k0, k1);
                            wp[(k * 4 + 0) * 32 + lane] = w.x;
                            wp[(k * 4 + 1) * 32 + lane] = w.y;
                            wp[(k * 4 + 2) * 32 + lane] = w.z;
                            wp[(k * 4 + 3) * 32 + lane] = w.w;
                        }
                    }
                }
            }
            float cx = 0.f;
            int2 ti = make_int2(0, 0);
            if constexpr (IS_INT)
                ti = P.temp.tabinfo[P.beta_stride ? rep * P.beta_stride + t : rep];
            else
                cx = P.temp.beta[P.beta_stride ? rep * P.beta_stride + t : rep];
            const uint32_t ownb = res_body(sub ? ylo1 : ylo0, sub ? zlo1 : zlo0, sub, y0, z0, ny, nz, Wy, Wz, rows, rb);
            const uint32_t parb = res_body(sub ? ylo0 : ylo1, sub ? zlo0 : zlo1, 1 - sub, y0 + soff, z0 + soff, ny, nz,
                                           Wy, Wz, rows, rb);
            named_sync(bar_ready(gs), nbar);
            if (gs >= s_stop) break;
            if (active) {
                auto trial = [&](int x, uint32_t w) {
                    uint32_t a8, b8, pb;
                    const uint32_t ya = ownb + (uint32_t)x;
                    const int32_t dE =
                        res_dE<NSH, SW, XB>(ya, parb + (uint32_t)(x + soff), rb, RZ, w, qt, a8, b8, pb);
                    if (accept_fixed<IS_INT>(dE, w & kRMask, cx, P.tab, ti)) {
                        int xb = x + soff + (int)(w >> 31);
                        const int wrap = xb < 0 ? nx : (xb >= nx ? -nx : 0);
                        pb += (uint32_t)wrap;
                        xb += wrap;
                        // the cell and, within 4 of a row end, its periodic
                        // x-halo copy (no halo pass between mini-steps)
                        g_smem[ya] = (unsigned char)b8;
                        if (x < 4) g_smem[ya + nx] = (unsigned char)b8;
                        if (x >= nx - 4) g_smem[ya - nx] = (unsigned char)b8;
                        g_smem[pb] = (unsigned char)a8;
                        if (xb < 4) g_smem[pb + nx] = (unsigned char)a8;
                        if (xb >= nx - 4) g_smem[pb - nx] = (unsigned char)a8;
                        accE += dE;
                        accN += 1;
                    }
                };
                if (nk == 1 && NLx == 32) {
                    // one link cell per lane: its four words stay in registers
                    trial(4 * lane + 0, w4.x);
                    __syncwarp();  // the next mini-step reads what this one wrote
                    trial(4 * lane + 1, w4.y);
                    __syncwarp();  // the next mini-step reads what this one wrote
                    trial(4 * lane + 2, w4.z);
                    __syncwarp();  // the next mini-step reads what this one wrote
                    trial(4 * lane + 3, w4.w);
                    __syncwarp();  // the next mini-step reads what this one wrote
                } else {
                    for (int dx = 0; dx < 4; ++dx) {
#pragma unroll 1
                        for (int k = 0; k < nk; ++k) {
                            const int i = lane + 32 * k;
                            if (i < NLx)
                                trial(4 * i + dx, *(const uint32_t *)(g_smem + wsm +
                                                                      (uint32_t)(((k * 4 + dx) * 32 + lane) * 4)));
                        }
                        __syncwarp();  // the next mini-step reads what this one wrote
                    }
                }
                // publish the versions of the rows this column wrote that other
                // blocks read ({smem slot, version slot} entries)
                if (blk != P.skip_tile) {
                    const uint2 *pe = (const uint2 *)(L + po[g * nc + warp]);
                    const int np = (int)(po[g * nc + warp + 1] - po[g * nc + warp]) >> 1;
                    const unsigned long long tag = (unsigned long long)(gs + 1) << 32;
                    // chunk q = lane + 32 i of entry e = q / cpr, chunk c = q % cpr,
                    // stepped without divisions
                    int e = pub_e0, c = pub_c0;
                    for (int q = lane; q < np * cpr; q += 32) {
                        const uint2 en = pe[e];
                        const uint2 w = *(const uint2 *)(g_smem + rows + en.x * rb + 16u + 8u * c);
                        st_relaxed_v2u64(xver + ver_word(nver, gs, en.y, nx) + 2 * c, tag | w.x, tag | w.y);
                        e += pub_de;
                        c += pub_dc;
                        if (c >= cpr) {
                            c -= cpr;
                            ++e;
                        }
                    }
                }
            }
            // count this warp's group as done (release at CTA scope: the
            // stores above are ordered before the count)
            __syncwarp();
            if (lane == 0) {
                __threadfence_block();
                atomicAdd(&s_cnt, 1u);
            }
        }
        const long long e_w = warp_sum<long long>(accE), n_w = warp_sum<long long>(accN);
        if (lane == 0) {
            P.part_e[blk * nc + warp] = (double)e_w;
            P.part_n[blk * nc + warp] = n_w;
        }
    }
    __syncthreads();
    if (s_abort) return;
    // final rows, back to plain species in the caller's array
    if ((nx & 15) == 0) {
        for (int q = tid; q < (int)(fin1 * (uint32_t)(nx >> 4)); q += blockDim.x) {
            const int cpr = nx >> 4, e = q / cpr, c = q - e * cpr;
            const uint32_t v = L[fin0 + e], slot = v >> 21, row = v & 0x1FFFFFu;
            const int4 w = *((const int4 *)(g_smem + rows + slot * rb + 16u) + c);
            int4 o;
            o.x = (int)(((uint32_t)w.x >> 3) & 0x07070707u);
            o.y = (int)(((uint32_t)w.y >> 3) & 0x07070707u);
            o.z = (int)(((uint32_t)w.z >> 3) & 0x07070707u);
            o.w = (int)(((uint32_t)w.w >> 3) & 0x07070707u);
            *((int4 *)(RD.occ + (size_t)row * nx) + c) = o;
        }
    } else {
        for (int q = tid; q < (int)(fin1 * (uint32_t)(nx >> 2)); q += blockDim.x) {
            const int cpr = nx >> 2, e = q / cpr, c = q - e * cpr;
            const uint32_t v = L[fin0 + e], slot = v >> 21, row = v & 0x1FFFFFu;
            const uint32_t w = *((const uint32_t *)(g_smem + rows + slot * rb + 16u) + c);
            *((uint32_t *)(RD.occ + (size_t)row * nx) + c) = (w >> 3) & 0x07070707u;
        }
    }
    // per-warp partial sums; the last CTA reduces them in order
    __shared__ int s_last;
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(P.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || tid >= P.R) return;
    // thread r: replica r's blocks in order
    __threadfence();
    double se = 0.0;
    long long sn = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        if (__ldcg(P.rdesc + b * kResDesc + 10) != tid) continue;
        for (int k = b * nc; k < (b + 1) * nc; ++k) {
            se += __ldcg(P.part_e + k);
            sn += __ldcg(P.part_n + k);
        }
    }
    const RepDesc &RR = P.rep[tid];
    if (RR.e_acc) *RR.e_acc += se * P.escale;
    if (RR.n_acc) *RR.n_acc += sn;
}

// ---------------------------------------------------------------------------
// Host: block shape, windows and exchange lists.
// ---------------------------------------------------------------------------
struct ResPlan {
    int ok = 0, by = 0, bz = 0, NBy = 0, NBz = 0, nblocks = 0, nc = 0, Wy = 0, Wz = 0, rowB = 0, blob = 0;
    int nver = 0;  // version slots (rows written in one group and read by another block)
    int per_sm = 0;  // CTAs per SM
    int nxw = 4;   // exchange warps
    size_t smem = 0;
    std::vector<int> desc;
    std::vector<uint32_t> lists;
    const void *kernel = nullptr;
};

// Rows (sub, y, z) -> id (sub * nz + z) * ny + y read and written by column
// (cy, cz) in group g (the same sets as the streaming kernel stages).
void column_rows(int cy, int cz, int g, int ny, int nz, int nsh, std::vector<int> &R, std::vector<int> &W)
{
    const int dy = g & 3, dz = (g >> 2) & 3, sub = g >> 4, soff = sub == 0 ? -1 : 0;
    const int y0 = 4 * cy + dy, z0 = 4 * cz + dz;
    auto id = [&](int s, int y, int z) {
        y = ((y % ny) + ny) % ny;
        z = ((z % nz) + nz) % nz;
        return (s * nz + z) * ny + y;
    };
    R.clear();
    W.clear();
    for (int b = -1; b <= 1; ++b)
        for (int a = -1; a <= 1; ++a) R.push_back(id(sub, y0 + a, z0 + b));
    for (int sz = 0; sz < 4; ++sz)
        for (int sy = 0; sy < 4; ++sy) {
            if (nsh < 3 && (sy == 0 || sy == 3) && (sz == 0 || sz == 3)) continue;
            R.push_back(id(1 - sub, y0 + soff - 1 + sy, z0 + soff - 1 + sz));
        }
    W.push_back(id(sub, y0, z0));
    for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) W.push_back(id(1 - sub, y0 + soff + a, z0 + soff + b));
}

// Window slot of row r for a block with descriptor dd, or -1 outside.
int res_slot_of(const int *dd, int r, int ny, int nz, int Wy, int Wz)
{
    const int s = r / (ny * nz), z = (r / ny) % nz, y = r % ny;
    int yy = y - dd[4 + s], zz = z - dd[6 + s];
    yy = ((yy % ny) + ny) % ny;
    zz = ((zz % nz) + nz) % nz;
    if (yy >= Wy || zz >= Wz) return -1;
    return (s * Wz + zz) * Wy + yy;
}

template <bool IS_INT>
const void *pick_resident(int nsh, int sw)
{
    if (nsh >= 3)
        return sw == 2 ? (const void *)k_sweep_resident<IS_INT, 3, 2, 0, 0>
                       : (const void *)k_sweep_resident<IS_INT, 3, 1, 0, 0>;
    return sw == 2 ? (const void *)k_sweep_resident<IS_INT, 2, 2, 0, 0> : (const void *)k_sweep_resident<IS_INT, 2, 1, 0, 0>;
}
// the specialisation for blocks of 2 x 4 columns on 128-cell rows (pitch 256
// bytes, 15 window rows per y), when every block of a launch has them
template <bool IS_INT>
const void *pick_resident_fixed(int nsh, int sw, int rowB, int Wy)
{
    if (nsh == 2 && sw == 1 && rowB == 256 && Wy == 15) return (const void *)k_sweep_resident<IS_INT, 2, 1, 256, 15>;
    return nullptr;
}

// Builds the plan for one lattice, or leaves ok = 0 when the lattice does not
// fit (the streaming kernel then runs).
template <bool IS_INT>
smc_status build_res_plan(const smc_lattice &lat, const PairTable &pt, Workspace *ws, bool few_blocks, ResPlan &rp)
{
    rp = ResPlan();
    const int nx = lat.nx, ny = lat.ny, nz = lat.nz;
    const int NLy = ny / 4, NLz = nz / 4, nsh = pt.nsh;
    // row pitch: a multiple of 128 bytes when the windows fit with it, so that
    // the same x of every row falls in the same bank (the lanes' partner rows
    // differ per lane; their x do not), else the 16-byte halos only
    int rowB = (nx + 32 + 127) / 128 * 128;
    const void *kern = pick_resident<IS_INT>(pt.nsh, pt.sw);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    // block shapes with at most 8 columns, at most one CTA per SM and at
    // least 3 blocks per axis; the fewest columns per block (the shortest
    // group; with few_blocks, for replicas sharing a launch, the most), then
    // the fewest rows held.  A tuned tile shape (tile_y, tile_z) selects the
    // block shape.
    const int shapes[][2] = {{1, 1}, {1, 2}, {2, 1}, {2, 2}, {1, 4}, {4, 1}, {2, 3}, {3, 2}, {2, 4}, {4, 2}, {1, 8}, {8, 1}};
    const Tuning tu = current_tuning();
    int best = -1, best_nc = 1 << 30, best_rows = 1 << 30;
    for (int i = 0; i < (int)(sizeof shapes / sizeof shapes[0]); ++i) {
        const int by = shapes[i][0], bz = shapes[i][1];
        if (tu.tile_y > 0 && tu.tile_z > 0 && (by != tu.tile_y || bz != tu.tile_z)) continue;
        const int NBy = (NLy + by - 1) / by, NBz = (NLz + bz - 1) / bz;
        if (NBy < 3 || NBz < 3 || NBy * NBz > ws->num_sms) continue;
        const int Wy = 4 * by + 7, Wz = 4 * bz + 7;
        if (Wy >= ny || Wz >= nz) continue;
        const int nrows = 2 * Wy * Wz, nc = by * bz;
        const bool better_nc = few_blocks ? (best < 0 || nc > best_nc) : nc < best_nc;
        if (better_nc || (nc == best_nc && nrows < best_rows)) {
            best = i;
            best_nc = nc;
            best_rows = nrows;
        }
    }
    if (best < 0 || nx % 4 != 0) return SMC_OK;
    const int by = shapes[best][0], bz = shapes[best][1];
    rp.by = by;
    rp.bz = bz;
    rp.NBy = (NLy + by - 1) / by;
    rp.NBz = (NLz + bz - 1) / bz;
    rp.nblocks = rp.NBy * rp.NBz;
    rp.nc = by * bz;
    rp.Wy = 4 * by + 7;
    rp.Wz = 4 * bz + 7;
    rp.rowB = rowB;
    const int nrows_lat = 2 * ny * nz;
    auto block_of = [&](int cy, int cz) { return (cz / bz) * rp.NBy + (cy / by); };
    // per row: writer block at every group (-1 = none)
    std::vector<int> wblk((size_t)nrows_lat * 32, -1);
    std::vector<int> R, W;
    for (int g = 0; g < 32; ++g)
        for (int cz = 0; cz < NLz; ++cz)
            for (int cy = 0; cy < NLy; ++cy) {
                column_rows(cy, cz, g, ny, nz, nsh, R, W);
                for (int r : W) wblk[(size_t)r * 32 + g] = block_of(cy, cz);
            }
    // last write of row r before group g (cyclic over the sweep): writer
    // block and distance d in groups (1..32), or (-1, 0) if never written
    auto last_write = [&](int r, int g, int &d) {
        for (d = 1; d <= 32; ++d) {
            const int b = wblk[(size_t)r * 32 + ((g - d + 64) & 31)];
            if (b >= 0) return b;
        }
        d = 0;
        return -1;
    };
    rp.desc.assign((size_t)rp.nblocks * kResDesc, 0);
    rp.lists.clear();
    const int nc = kResCols;  // compute warps of the kernel (some idle for smaller blocks)
    std::vector<int> vslot((size_t)32 * nrows_lat, -1);  // (group of the write, row) -> version slot
    int nver = 0;
    struct Blk {
        std::vector<uint32_t> hdr, body;
    };
    std::vector<Blk> blks(rp.nblocks);
    bool fits = true;
    for (int blk = 0; blk < rp.nblocks; ++blk) {
        const int bky = blk % rp.NBy, bkz = blk / rp.NBy;
        const int cy0 = bky * by, cz0 = bkz * bz;
        const int ncy = std::min(by, NLy - cy0), ncz = std::min(bz, NLz - cz0);
        int *dd = &rp.desc[(size_t)blk * kResDesc];
        dd[0] = cy0;
        dd[1] = cz0;
        dd[2] = ncy;
        dd[3] = ncz;
        dd[4] = 4 * cy0 - 1;  // sublattice 0 rows y in [4 cy0 - 1, 4 cy0 + 4 by + 5]
        dd[5] = 4 * cy0 - 2;  // sublattice 1 rows y in [4 cy0 - 2, 4 cy0 + 4 by + 4]
        dd[6] = 4 * cz0 - 1;
        dd[7] = 4 * cz0 - 2;
        dd[11] = blk;
        dd[12] = rp.NBy;
        dd[13] = rp.NBz;
        dd[15] = rp.Wy;
        dd[16] = rp.Wz;
        // rows the block reads in each group
        std::vector<std::vector<int>> reads(32);
        for (int g = 0; g < 32; ++g) {
            for (int k = 0; k < ncy * ncz; ++k) {
                column_rows(cy0 + k % ncy, cz0 + k / ncy, g, ny, nz, nsh, R, W);
                reads[g].insert(reads[g].end(), R.begin(), R.end());
            }
            std::sort(reads[g].begin(), reads[g].end());
            reads[g].erase(std::unique(reads[g].begin(), reads[g].end()), reads[g].end());
        }
        auto reads_at = [&](int g, int r) {
            const auto &v = reads[(g + 64) & 31];
            return std::binary_search(v.begin(), v.end(), r);
        };
        Blk &B = blks[blk];
        B.hdr.assign(33 + 32 * nc + 3, 0);  // an even size: the entry pairs stay 8-byte aligned
        // fetch lists per group: rows read at g whose last write is another
        // block's and whose version the block has not read since (the window
        // keeps it): {smem slot | d << 16, version slot}
        for (int g = 0; g < 32; ++g) {
            B.hdr[g] = (uint32_t)(B.hdr.size() + B.body.size());
            std::vector<std::pair<int, std::pair<uint32_t, uint32_t>>> ents;  // (-d, entry)
            for (int r : reads[g]) {
                int d = 0;
                const int wb = last_write(r, g, d);
                if (wb < 0 || wb == blk) continue;
                bool seen = false;
                for (int h = g - d + 1; h < g && !seen; ++h) seen = reads_at(h, r);
                if (seen) continue;
                const int sl = res_slot_of(dd, r, ny, nz, rp.Wy, rp.Wz);
                if (sl < 0) {
                    fits = false;
                    continue;
                }
                int &v = vslot[(size_t)((g - d + 64) & 31) * nrows_lat + r];
                if (v < 0) v = nver++;
                ents.push_back({-d, {(uint32_t)sl | ((uint32_t)d << 16), (uint32_t)v}});
            }
            // oldest versions first: they are ready at once, and the rows
            // written in the previous group (the ones that may still have to
            // be waited for) come last, in as few polling rounds as possible
            std::stable_sort(ents.begin(), ents.end(),
                             [](const auto &a, const auto &b) { return a.first < b.first; });
            for (const auto &en : ents) {
                B.body.push_back(en.second.first);
                B.body.push_back(en.second.second);
            }
        }
        B.hdr[32] = (uint32_t)(B.hdr.size() + B.body.size());
    }
    // publish lists per (group, compute warp): the rows a column writes whose
    // version another block reads ({smem slot, version slot}); final rows:
    // those whose last write in the sweep is this block's
    for (int blk = 0; blk < rp.nblocks && fits; ++blk) {
        const int *dd = &rp.desc[(size_t)blk * kResDesc];
        const int cy0 = dd[0], cz0 = dd[1], ncy = dd[2], ncz = dd[3];
        Blk &B = blks[blk];
        for (int g = 0; g < 32; ++g)
            for (int k = 0; k < nc; ++k) {
                B.hdr[33 + g * nc + k] = (uint32_t)(B.hdr.size() + B.body.size());
                if (k >= ncy * ncz) continue;
                column_rows(cy0 + k % ncy, cz0 + k / ncy, g, ny, nz, nsh, R, W);
                for (int r : W) {
                    const int v = vslot[(size_t)g * nrows_lat + r];
                    if (v < 0) continue;
                    const int sl = res_slot_of(dd, r, ny, nz, rp.Wy, rp.Wz);
                    if (sl < 0) fits = false;
                    B.body.push_back((uint32_t)sl);
                    B.body.push_back((uint32_t)v);
                }
            }
        B.hdr[33 + 32 * nc] = (uint32_t)(B.hdr.size() + B.body.size());
        B.hdr[33 + 32 * nc + 1] = (uint32_t)(B.hdr.size() + B.body.size());
        uint32_t nfin = 0;
        for (int r = 0; r < nrows_lat; ++r) {
            int d = 0;
            if (last_write(r, 32, d) == blk) {
                const int sl = res_slot_of(dd, r, ny, nz, rp.Wy, rp.Wz);
                if (sl < 0) fits = false;
                B.body.push_back(((uint32_t)sl << 21) | (uint32_t)r);
                ++nfin;
            }
        }
        B.hdr[33 + 32 * nc + 2] = nfin;
        rp.desc[(size_t)blk * kResDesc + 8] = (int)rp.lists.size();
        rp.desc[(size_t)blk * kResDesc + 9] = (int)(B.hdr.size() + B.body.size());
        rp.blob = std::max(rp.blob, (int)(B.hdr.size() + B.body.size()));
        rp.lists.insert(rp.lists.end(), B.hdr.begin(), B.hdr.end());
        rp.lists.insert(rp.lists.end(), B.body.begin(), B.body.end());
        if (rp.lists.size() & 1) rp.lists.push_back(0u);  // next block's lists 8-byte aligned
    }
    if (!fits) return SMC_OK;  // a row outside the window (not expected)
    rp.nver = std::max(nver, 1);
    const int nk = (nx / 4 + 31) / 32;
    auto smem_of = [&](int pitch) {
        return (size_t)kQRows * pt.rw * 4 + 64 + (size_t)2 * rp.Wy * rp.Wz * pitch +
               ((size_t)rp.blob * 4 + 15) / 16 * 16 + (size_t)nc * nk * 512;
    };
    if (smem_of(rowB) > dyn_max) rowB = nx + 32;
    rp.rowB = rowB;
    const size_t smem = smem_of(rowB);
    if (smem > dyn_max) return SMC_OK;
    for (int blk = 0; blk < rp.nblocks; ++blk) {
        rp.desc[(size_t)blk * kResDesc + 17] = rowB;
        rp.desc[(size_t)blk * kResDesc + 20] = rp.nver;
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (kResCols + rp.nxw + 1) * 32, smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1 || rp.nblocks > per_sm * ws->num_sms) return SMC_OK;
    rp.per_sm = per_sm;
    rp.smem = smem;
    rp.kernel = kern;
    rp.ok = 1;
    return SMC_OK;
}

__global__ void k_occ_to_exch(const int8_t *occ, int8_t *exch, long long n, int S, int *status)
{
    const long long nw = n >> 2;
    const uint32_t *s4 = (const uint32_t *)occ;
    uint32_t *d4 = (uint32_t *)exch;
    const uint32_t lim = (uint32_t)(0x80 - S) * 0x01010101u;
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t v = s4[i];
        bad |= ((v | (v + lim)) & 0x80808080u) != 0u;
        d4[i] = (v & 0x07070707u) << 3;
    }
    if (bad) atomicCAS(status, 0, (int)SMC_ERR_ARG);
}

}  // namespace

// The resident sweep for R replicas, when every replica fits (four-cell link
// cells on every axis, rows of a multiple of 16 bytes, windows within shared
// memory).  Replicas run in waves: one cooperative launch per wave of
// replicas whose blocks are resident at once (each block waits only for
// blocks of its own replica).  Returns SMC_ERR_UNSUPPORTED, having enqueued
// nothing, when one replica does not fit.
namespace {

struct ResWave {
    std::vector<int> reps;       // replicas of the wave, in order
    int nblocks = 0, blob = 0;   // CTAs; largest list blob of a block (words)
    size_t smem = 0;             // dynamic shared memory per CTA
    size_t exch_bytes = 0, ver_words = 0;
    void *dev = nullptr;         // [descriptors | lists], uploaded once
    size_t lists_off = 0;
};

struct ResMulti {
    bool ok = false;
    const void *kernel = nullptr;
    std::vector<ResPlan> rp;
    std::vector<ResWave> waves;
};

void free_waves(ResMulti &mp)
{
    for (auto &w : mp.waves)
        if (w.dev) cudaFree(w.dev);
    mp.waves.clear();
}

template <bool IS_INT>
smc_status build_res_multi(int R, const smc_lattice *lats, const PairTable &pt, Workspace *ws, ResMulti &mp)
{
    mp = ResMulti();
    for (int r = 0; r < R; ++r) {
        ResPlan rp;
        const smc_status st = build_res_plan<IS_INT>(lats[r], pt, ws, R > 1, rp);
        if (st != SMC_OK) return st;
        if (!rp.ok) return SMC_OK;
        mp.kernel = rp.kernel;
        mp.rp.push_back(std::move(rp));
    }
    bool same = true;
    for (const auto &rp : mp.rp) same = same && rp.rowB == mp.rp[0].rowB && rp.Wy == mp.rp[0].Wy;
    const void *fixed = same ? pick_resident_fixed<IS_INT>(pt.nsh, pt.sw, mp.rp[0].rowB, mp.rp[0].Wy) : nullptr;
    cudaFuncAttributes fa;
    cudaError_t e;
    if (fixed) {
        // the compile-time-pitch kernel keeps the replicated table (larger
        // than the plain one): taken when every block still fits as before
        const size_t plain = (size_t)kQRows * pt.rw * 4;
        const size_t extra = (size_t)kRTabBytes > plain ? (size_t)kRTabBytes - plain : 0;
        e = cudaFuncGetAttributes(&fa, fixed);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
        const size_t fdyn = ws->smem_optin - fa.sharedSizeBytes;
        e = cudaFuncSetAttribute(fixed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fdyn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        // (largest CTA: any block with the largest list blob of a wave)
        auto pad = [](int blob) { return ((size_t)blob * 4 + 15) / 16 * 16; };
        size_t base = 0;
        int maxblob = 0, need_sm = 0;
        for (const auto &rp : mp.rp) {
            base = std::max(base, rp.smem + extra - pad(rp.blob));
            maxblob = std::max(maxblob, rp.blob);
            need_sm = std::max(need_sm, rp.per_sm);
        }
        const size_t smax = base + pad(maxblob);
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fixed, (kResCols + mp.rp[0].nxw + 1) * 32, smax);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (smax <= fdyn && per_sm >= need_sm) {
            mp.kernel = fixed;
            for (auto &rp : mp.rp) {
                rp.smem += extra;
                rp.per_sm = std::min(rp.per_sm, per_sm);
            }
        }
    }
    e = cudaFuncGetAttributes(&fa, mp.kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    // waves: first-fit decreasing by block count (every wave's blocks
    // resident at once, at most kMaxReplicas replicas per wave)
    auto smem_with_blob = [&](const ResPlan &rp, int blob) {
        return rp.smem - ((size_t)rp.blob * 4 + 15) / 16 * 16 + ((size_t)blob * 4 + 15) / 16 * 16;
    };
    std::vector<int> order(R);
    for (int r = 0; r < R; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return mp.rp[a].nblocks > mp.rp[b].nblocks; });
    std::vector<ResWave> bins;
    std::vector<int> bin_ps;
    for (int r : order) {
        const ResPlan &rp = mp.rp[r];
        bool placed = false;
        for (size_t i = 0; i < bins.size() && !placed; ++i) {
            ResWave &w = bins[i];
            const int ps = std::min(bin_ps[i], rp.per_sm), blob = std::max(w.blob, rp.blob);
            size_t smem = smem_with_blob(rp, blob);
            for (int q : w.reps) smem = std::max(smem, smem_with_blob(mp.rp[q], blob));
            if ((int)w.reps.size() >= kMaxReplicas || w.nblocks + rp.nblocks > ps * ws->num_sms || smem > dyn_max)
                continue;
            w.reps.push_back(r);
            w.nblocks += rp.nblocks;
            w.blob = blob;
            w.smem = smem;
            bin_ps[i] = ps;
            placed = true;
        }
        if (!placed) {
            if (smem_with_blob(rp, rp.blob) > dyn_max || rp.nblocks > rp.per_sm * ws->num_sms) return SMC_OK;
            ResWave w;
            w.reps.push_back(r);
            w.nblocks = rp.nblocks;
            w.blob = rp.blob;
            w.smem = smem_with_blob(rp, rp.blob);
            bins.push_back(w);
            bin_ps.push_back(rp.per_sm);
        }
    }
    for (auto &w : bins) {
        std::sort(w.reps.begin(), w.reps.end());
        // descriptors and lists of the wave's blocks
        std::vector<int> desc;
        std::vector<uint32_t> lists;
        int flag0 = 0;
        for (int lr = 0; lr < (int)w.reps.size(); ++lr) {
            const ResPlan &rp = mp.rp[w.reps[lr]];
            const smc_lattice &l = lats[w.reps[lr]];
            for (int b = 0; b < rp.nblocks; ++b) {
                const int *src = &rp.desc[(size_t)b * kResDesc];
                const size_t at = desc.size();
                desc.insert(desc.end(), src, src + kResDesc);
                desc[at + 8] += (int)lists.size();
                desc[at + 10] = lr;
                desc[at + 14] = flag0;
                desc[at + 18] = (int)w.exch_bytes;
                desc[at + 19] = (int)w.ver_words;
            }
            lists.insert(lists.end(), rp.lists.begin(), rp.lists.end());
            if (lists.size() & 1) lists.push_back(0u);
            flag0 += rp.nblocks;
            w.exch_bytes += ((size_t)2 * l.nx * l.ny * l.nz + 255) / 256 * 256;
            w.ver_words += (size_t)2 * rp.nver * (size_t)(((l.nx + 7) / 8) * 2);
        }
        w.lists_off = (desc.size() * 4 + 15) / 16 * 16;
        e = cudaMalloc(&w.dev, w.lists_off + lists.size() * 4);
        if (e == cudaSuccess) e = cudaMemcpy(w.dev, desc.data(), desc.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy((unsigned char *)w.dev + w.lists_off, lists.data(), lists.size() * 4,
                           cudaMemcpyHostToDevice);
        mp.waves.push_back(w);
        if (e != cudaSuccess) return cuda_fail(e, "resident plan upload");
    }
    mp.ok = true;
    return SMC_OK;
}

}  // namespace

smc_status launch_pair_sweep_resident(int R, const smc_lattice *lats, const smc_model *m, const PairTable &pt,
                                      int8_t *const *occ, uint64_t seed, uint32_t replica0, uint64_t sweep0,
                                      int nsweeps, const double *kT, double *e_acc, int64_t *n_acc,
                                      cudaStream_t stream)
{
    if (R < 1 || R > kMaxReplicas) return SMC_ERR_UNSUPPORTED;
    for (int r = 0; r < R; ++r) {
        const smc_lattice &l = lats[r];
        if (lc_edge(l.nx) != 4 || lc_edge(l.ny) != 4 || lc_edge(l.nz) != 4 || (uintptr_t)occ[r] % 4 ||
            l.nx > 1024 || l.nspecies != lats[0].nspecies)
            return SMC_ERR_UNSUPPORTED;
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    const bool is_int = m->kind == SMC_PAIR_I32;
    static std::vector<long long> key_cached;
    static ResMulti plan_cached;
    const Tuning tu = current_tuning();
    std::vector<long long> key = {R, pt.nsh, pt.sw, is_int, ws->device, ws->num_sms, tu.tile_y, tu.tile_z};
    for (int r = 0; r < R; ++r) key.insert(key.end(), {lats[r].nx, lats[r].ny, lats[r].nz});
    if (key != key_cached) {
        free_waves(plan_cached);
        key_cached.clear();
        ResMulti mp;
        st = is_int ? build_res_multi<true>(R, lats, pt, ws, mp) : build_res_multi<false>(R, lats, pt, ws, mp);
        plan_cached = std::move(mp);
        if (st != SMC_OK) {
            free_waves(plan_cached);
            plan_cached.ok = false;
            return st;
        }
        key_cached = key;
    }
    const ResMulti &mp = plan_cached;
    if (!mp.ok) return SMC_ERR_UNSUPPORTED;

    // per-sweep temperatures: one launch per kMaxBeta / (replicas of the wave) sweeps
    bool constant = true;
    for (int r = 0; r < R && constant; ++r)
        for (int t = 1; t < nsweeps; ++t)
            if (kT[(size_t)r * nsweeps + t] != kT[(size_t)r * nsweeps]) {
                constant = false;
                break;
            }
    const int cap = is_int ? kMaxBeta / 2 : kMaxBeta;
    for (const auto &w : mp.waves)
        if (!constant && (int)w.reps.size() > cap) return SMC_ERR_UNSUPPORTED;
    std::vector<uint32_t> tabs;
    std::vector<std::pair<double, int2>> tindex;
    auto table_of = [&](double kt) -> int2 {
        for (auto &p : tindex)
            if (p.first == kt) return p.second;
        std::vector<uint32_t> t = int_table(m->unit_ev, kt);
        int2 ti = make_int2((int)tabs.size(), (int)t.size());
        tabs.insert(tabs.end(), t.begin(), t.end());
        tindex.push_back({kt, ti});
        return ti;
    };
    if (is_int)
        for (int r = 0; r < R; ++r)
            for (int t = 0; t < nsweeps; ++t) table_of(kT[(size_t)r * nsweeps + t]);

    // workspace: [flags | part_e | part_n | ticket, abort | tables | lattice copies | versions], sized for
    // the largest wave
    size_t nbmax = 0, exmax = 0, vwmax = 0;
    for (const auto &w : mp.waves) {
        nbmax = std::max(nbmax, (size_t)w.nblocks);
        exmax = std::max(exmax, w.exch_bytes);
        vwmax = std::max(vwmax, w.ver_words);
    }
    const size_t np = nbmax * kResCols;
    const size_t off_flags = 0, off_pe = ((nbmax * 4 + 15) / 16) * 16, off_pn = off_pe + np * 8;
    const size_t off_misc = off_pn + np * 8, off_tab = off_misc + 16;
    const size_t off_exch = off_tab + ((tabs.size() * 4 + 255) / 256) * 256;
    const size_t off_ver = off_exch + exmax;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_ver + vwmax * 8, &st);
    if (!scr) return st;
    cudaError_t e = cudaSuccess;
    if (!tabs.empty()) {
        e = cudaMemcpyAsync(scr + off_tab, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(acceptance tables)");
    }
    static SweepParams P;
    for (const auto &w : mp.waves) {
        memset(&P, 0, sizeof P);
        const int Rw = (int)w.reps.size();
        P.R = Rw;
        P.G = 32;
        P.Lx = P.Ly = P.Lz = 4;
        P.nshells = m->nshells;
        P.S = lats[0].nspecies;
        P.seed = seed;
        P.timeout_ns = debug_timeout_ns();
        P.skip_tile = (int)debug_skip_tile();
        P.rblob = w.blob;
        P.rxw = mp.rp[w.reps[0]].nxw;
        P.qrow = pt.rw;
        P.escale = pt.scale;
        memcpy(P.qtab, pt.rows.data(), pt.rows.size() * 4);
        P.flags = (uint32_t *)(scr + off_flags);
        P.part_e = (double *)(scr + off_pe);
        P.part_n = (long long *)(scr + off_pn);
        P.ticket = (unsigned *)(scr + off_misc);
        P.abort_flag = (int *)(scr + off_misc + 4);
        P.status = ws->status;
        P.rdesc = (const int *)w.dev;
        P.rlists = (const uint32_t *)((const unsigned char *)w.dev + w.lists_off);
        P.tab = (const uint32_t *)(scr + off_tab);
        P.exch = (int8_t *)(scr + off_exch);
        P.xver = (unsigned long long *)(scr + off_ver);
        for (int lr = 0; lr < Rw; ++lr) {
            const int r = w.reps[lr];
            RepDesc &d = P.rep[lr];
            d.occ = occ[r];
            d.e_acc = e_acc ? e_acc + r : nullptr;
            d.n_acc = n_acc ? (long long *)n_acc + r : nullptr;
            d.nx = lats[r].nx;
            d.ny = lats[r].ny;
            d.nz = lats[r].nz;
            d.NLx = d.nx / 4;
            d.NLy = d.ny / 4;
            d.NLz = d.nz / 4;
            d.rep = replica0 + (uint32_t)r;
        }
        const int chunk = constant ? nsweeps : std::max(1, cap / Rw);
        for (int t0 = 0; t0 < nsweeps; t0 += chunk) {
            const int nc = std::min(chunk, nsweeps - t0);
            P.sweep0 = sweep0 + (uint64_t)t0;
            P.nsweeps = nc;
            P.beta_stride = constant ? 0 : nc;
            for (int lr = 0; lr < Rw; ++lr)
                for (int t = 0; t < (constant ? 1 : nc); ++t) {
                    const double kt = kT[(size_t)w.reps[lr] * nsweeps + t0 + t];
                    const int idx = constant ? lr : lr * nc + t;
                    if (is_int)
                        P.temp.tabinfo[idx] = table_of(kt);
                    else
                        P.temp.beta[idx] = (float)(-1.4426950408889634 * pt.scale / kt);
                }
            // flags, sums and tags from zero: a tag (group + 1 >= 1) only ever
            // matches a version written in this launch
            e = cudaMemsetAsync(scr, 0, off_tab, stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(scr + off_ver, 0, w.ver_words * 8, stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(resident scratch)");
            size_t xo = 0;
            for (int lr = 0; lr < Rw; ++lr) {
                const smc_lattice &l = lats[w.reps[lr]];
                const size_t N = 2 * (size_t)l.nx * l.ny * l.nz;
                const long long nw = (long long)(N / 4);
                const int grid =
                    (int)std::max<long long>(1, std::min<long long>((nw + 255) / 256, (long long)ws->num_sms * 8));
                k_occ_to_exch<<<grid, 256, 0, stream>>>(occ[w.reps[lr]], P.exch + xo, (long long)N, l.nspecies,
                                                        P.status);
                xo += (N + 255) / 256 * 256;
            }
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "k_occ_to_exch");
            void *args[] = {(void *)&P};
            e = cudaLaunchCooperativeKernel(mp.kernel, dim3(w.nblocks), dim3((kResCols + P.rxw + 1) * 32), args,
                                            w.smem, stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(resident sweep)");
        }
    }
    return SMC_OK;
}

}  // namespace smc
