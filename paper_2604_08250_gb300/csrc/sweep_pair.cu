// sweep_pair.cu -- persistent swap-MC sweep kernels for pair models.
//
// Algorithm 1 of the paper runs n_A sequential mini-steps per sweep; in each,
// every link cell (LC) tries to swap its site at the mini-step's offset with
// a random nearest neighbour, all LCs in parallel (Sec. II-A, III-A).
//
// GPU organisation.  With mini-step k = ((sub*Lz + dz)*Ly + dy)*Lx + dx, the
// Lx consecutive mini-steps that share (sub, dy, dz) form a "group".  Within a
// group, the trials of one x-row of LCs (a "column", fixed (cy, cz)) read and
// write only that row's neighbourhood: rows y0-2..y0+2, z0-2..z0+2 of the two
// sublattices, where y0 = cy*Ly + dy, z0 = cz*Lz + dz.  Distinct columns of a
// group touch disjoint rows, so a column's Lx mini-steps run in lock-step on
// a copy of those rows in shared memory.  Columns are grouped into
// rectangular tiles; a tile may start group G only after its 8 neighbouring
// tiles have finished group G - lag (per-tile progress flags in global
// memory, bounded waits).  Trials in the same mini-step are independent, and
// a column's dependencies reach only the adjacent columns, so this reproduces
// the sequential mini-step order exactly.
//
// dE of a trial (a -> b) is the pair-model energy change written through the
// first-neighbour histograms: with D_m[q] = V_m(s_b, q) - V_m(s_a, q),
//   dE = sum_m [ sum_{j in N_m(a)\b} D_m[s_j] - sum_{j in N_m(b)\a} D_m[s_j] ],
// which equals the Omega-reduced local-energy difference of Algorithm 1 for
// pair site energies e_i = 1/2 sum_v V(s_i, s_{i+v}).  Every kernel here
// evaluates it in the exact fixed point of pair_fixed.cuh, so the sweep
// kernels and the lock-step trace agree bit for bit.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "pair_fixed.cuh"

namespace smc {

static_assert(kPairQWords == kQRows * kMaxQRowWords, "table size");

// Slot of row y0 + delta inside a window [lo, lo + W) along an axis of n cells.
// For n >= W the window rows are distinct and slot = delta - lo; otherwise the
// window holds the whole axis and slot = (y0 + delta) mod n.
struct Win {
    int big;   // n >= W
    int cnt;   // rows held
    int base;  // global row of slot 0
    int lo, y0, n;
    __device__ __forceinline__ int slot(int delta) const
    {
        if (big) return delta - lo;
        int v = (y0 + delta) % n;
        return v < 0 ? v + n : v;
    }
    __device__ __forceinline__ int row(int k) const
    {
        int v = (base + k) % n;
        return v < 0 ? v + n : v;
    }
};

__device__ __forceinline__ Win make_win(int n, int W, int lo, int y0)
{
    Win w;
    w.n = n;
    w.lo = lo;
    w.y0 = y0;
    w.big = n >= W;
    w.cnt = w.big ? W : n;
    w.base = w.big ? (y0 + lo) : 0;
    return w;
}

// Rows of one column held in shared memory: the trial sublattice ("own",
// window [-1, 1] per axis) and the partner sublattice ("oth", window
// [s_off-1, s_off+2], s_off = -1 for sub 0 and 0 for sub 1).
struct ColView {
    unsigned char *own, *oth;
    Win oy, oz, ty, tz;
    int rowB;
    __device__ __forceinline__ unsigned char *O(int dy, int dz) const
    {
        return own + (oz.slot(dz) * oy.cnt + oy.slot(dy)) * rowB;
    }
    __device__ __forceinline__ unsigned char *T(int dy, int dz) const
    {
        return oth + (tz.slot(dz) * ty.cnt + ty.slot(dy)) * rowB;
    }
};

// dE_fix of swapping the trial site a (own sublattice, x) with its partner
// in direction `dir` (bits kx, ky, kz -> vector 2k-1 in half units), from raw
// species read through a view.  Returns the species A, B and the partner's
// offsets through references.
template <int NSH, int SW, class View>
__device__ __forceinline__ int32_t trial_dE_hist(const View &cv, int x, int nx, int s_off, int dir,
                                                 const uint32_t *qt, int qrow, int &A, int &B, int &ex, int &ey,
                                                 int &ez)
{
    const int kx = (dir >> 2) & 1, ky = (dir >> 1) & 1, kz = dir & 1;
    ex = kx + s_off;
    ey = ky + s_off;
    ez = kz + s_off;
    const int xm2 = wrapc(x - 2, nx), xm1 = wrapc(x - 1, nx), xp1 = wrapc(x + 1, nx), xp2 = wrapc(x + 2, nx);
    auto xo = [&](int d) { return d == -2 ? xm2 : (d == -1 ? xm1 : (d == 0 ? x : (d == 1 ? xp1 : xp2))); };
    A = cv.O(0, 0)[x] & 7;
    const int bx = xo(ex);
    B = cv.T(ey, ez)[bx] & 7;
    if (A == B) return 0;
    auto sp = [](const unsigned char *row, int xx) { return (uint32_t)(row[xx] & 7) << 3; };
    uint32_t H[NSH][SW];
#pragma unroll
    for (int m = 0; m < NSH; ++m)
#pragma unroll
        for (int w = 0; w < SW; ++w) H[m][w] = m < 2 ? 0x08080808u : 0x10101010u;
    // shell 1 of a (partner sublattice), all but b
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (u == dir) continue;
        const int fx = ((u >> 2) & 1) + s_off, fy = ((u >> 1) & 1) + s_off, fz = (u & 1) + s_off;
        hadd<SW>(H[0], sp(cv.T(fy, fz), xo(fx)));
    }
    // shell 1 of b (trial sublattice), all but a
    const int sb = -1 - s_off;
    const int nd = 7 - dir;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (u == nd) continue;
        const int gx = ex + ((u >> 2) & 1) + sb, gy = ey + ((u >> 1) & 1) + sb, gz = ez + (u & 1) + sb;
        hsub<SW>(H[0], sp(cv.O(gy, gz), xo(gx)));
    }
    {
        const unsigned char *o00 = cv.O(0, 0);
        hadd<SW>(H[1], sp(o00, xm1));
        hadd<SW>(H[1], sp(o00, xp1));
        hadd<SW>(H[1], sp(cv.O(-1, 0), x));
        hadd<SW>(H[1], sp(cv.O(1, 0), x));
        hadd<SW>(H[1], sp(cv.O(0, -1), x));
        hadd<SW>(H[1], sp(cv.O(0, 1), x));
        const unsigned char *tb = cv.T(ey, ez);
        hsub<SW>(H[1], sp(tb, xo(ex - 1)));
        hsub<SW>(H[1], sp(tb, xo(ex + 1)));
        hsub<SW>(H[1], sp(cv.T(ey - 1, ez), bx));
        hsub<SW>(H[1], sp(cv.T(ey + 1, ez), bx));
        hsub<SW>(H[1], sp(cv.T(ey, ez - 1), bx));
        hsub<SW>(H[1], sp(cv.T(ey, ez + 1), bx));
    }
    if constexpr (NSH >= 3) {
#pragma unroll
        for (int p = -1; p <= 1; p += 2)
#pragma unroll
            for (int q = -1; q <= 1; q += 2) {
                hadd<SW>(H[2], sp(cv.O(p, q), x));      // (0, +-1, +-1)
                hadd<SW>(H[2], sp(cv.O(p, 0), xo(q)));  // (+-1, +-1, 0)
                hadd<SW>(H[2], sp(cv.O(0, p), xo(q)));  // (+-1, 0, +-1)
                hsub<SW>(H[2], sp(cv.T(ey + p, ez + q), bx));
                hsub<SW>(H[2], sp(cv.T(ey + p, ez), xo(ex + q)));
                hsub<SW>(H[2], sp(cv.T(ey, ez + p), xo(ex + q)));
            }
    }
    return dot_fixed<NSH, SW>(H, qt + (A * 8 + B) * qrow);
}

// Waits until the 8 neighbouring tiles of (ty, tz) have completed `need`
// groups.  Bounded: on timeout the status word and the abort flag are set.
__device__ bool wait_tile(const SweepParams &P, const RepDesc &D, int ty, int tz, uint32_t need, int *s_stop)
{
    if (threadIdx.x < 32) {
        const int k = threadIdx.x;
        const uint32_t *fp = nullptr;
        if (k < 9 && k != 4) {
            int nty = ty + (k % 3) - 1, ntz = tz + (k / 3) - 1;
            nty = nty < 0 ? nty + D.NTy : (nty >= D.NTy ? nty - D.NTy : nty);
            ntz = ntz < 0 ? ntz + D.NTz : (ntz >= D.NTz ? ntz - D.NTz : ntz);
            fp = P.flags + D.tile0 + ntz * D.NTy + nty;
        }
        const uint64_t t0 = global_ns();
        int stop = 0;
        for (;;) {
            const bool ok = (fp == nullptr) || ld_acquire_u32(fp) >= need;
            if (__all_sync(0xffffffffu, ok)) break;
            if (k == 0) {
                if (ld_volatile_i32(P.abort_flag)) {
                    stop = 1;
                } else if ((long long)(global_ns() - t0) > P.timeout_ns) {
                    atomicCAS(P.status, 0, (int)SMC_ERR_TIMEOUT);
                    atomicExch(P.abort_flag, 1);
                    stop = 1;
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
            __nanosleep(40);
        }
        if (k == 0) *s_stop = stop;
    }
    __syncthreads();
    return *s_stop == 0;
}

// General path: any lattice (link-cell edges 4 or the whole axis).  A CTA
// owns tiles of columns, stages CB columns' rows into shared memory at a
// time and runs their mini-steps with CTA barriers between them.  Species
// are read raw (this path does not use the scaled storage of the fast path).
template <bool IS_INT, int NSH, int SW>
__global__ void __launch_bounds__(512) k_sweep_pair(const __grid_constant__ SweepParams P)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_stop;
    __shared__ int s_last;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;

    uint32_t *Qt = (uint32_t *)smem;
    double *slot_e = (double *)(smem + (size_t)kQRows * P.qrow * 4);
    long long *slot_n = (long long *)(slot_e + P.tpc * nwarp);
    unsigned char *colbuf = (unsigned char *)(slot_n + P.tpc * nwarp);

    for (int i = tid; i < kQRows * P.qrow; i += nthr) Qt[i] = P.qtab[i];
    for (int i = tid; i < P.tpc * nwarp; i += nthr) {
        slot_e[i] = 0.0;
        slot_n[i] = 0;
    }
    if (tid == 0) s_stop = 0;
    __syncthreads();

    bool aborted = false;
    for (int t = 0; t < P.nsweeps && !aborted; ++t) {
        const uint64_t sweep = P.sweep0 + (uint64_t)t;
        for (int g = 0; g < P.G && !aborted; ++g) {
            const uint32_t gstep = (uint32_t)(t * P.G + g);
            const int dy = g % P.Ly, dz = (g / P.Ly) % P.Lz, sub = g / (P.Ly * P.Lz);
            const int s_off = sub == 0 ? -1 : 0;
            int slotk = 0;
            for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++slotk) {
                int r = 0;
                while (r + 1 < P.R && P.rep[r + 1].tile0 <= tile) ++r;
                const RepDesc &RD = P.rep[r];
                const int lt = tile - RD.tile0, ty = lt % RD.NTy, tz = lt / RD.NTy;
                if (!wait_tile(P, RD, ty, tz, gstep, &s_stop)) {
                    aborted = true;
                    break;
                }
                float cx = 0.f;
                int2 ti = make_int2(0, 0);
                if constexpr (IS_INT)
                    ti = P.temp.tabinfo[P.beta_stride ? r * P.beta_stride + t : r];
                else
                    cx = P.temp.beta[P.beta_stride ? r * P.beta_stride + t : r];

                const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NLx = RD.NLx;
                const int rowB = (nx + 15) & ~15;
                const int j0 = ty * P.TY, j1 = min(j0 + P.TY, RD.NLy);
                const int l0 = tz * P.TZ, l1 = min(l0 + P.TZ, RD.NLz);
                const int nj = j1 - j0, ncols = nj * (l1 - l0);
                // window shapes are the same for every column of the tile
                const Win oy0 = make_win(ny, 3, -1, dy), oz0 = make_win(nz, 3, -1, dz);
                const Win ty0 = make_win(ny, 4, s_off - 1, dy), tz0 = make_win(nz, 4, s_off - 1, dz);
                const int rows_own = oy0.cnt * oz0.cnt, rows_oth = ty0.cnt * tz0.cnt;
                const int rows_col = rows_own + rows_oth;
                const int col_bytes = rows_col * rowB;
                long long accE = 0, accN = 0;

                for (int cb = 0; cb < ncols; cb += P.CB) {
                    const int nc = min(P.CB, ncols - cb);
                    // ---- stage the rows of nc columns into shared memory ----
                    const int chunks_row = rowB >> 4;
                    const bool vec = RD.vec != 0;
                    const int total = vec ? nc * rows_col * chunks_row : nc * rows_col * nx;
                    for (int q = tid; q < total; q += nthr) {
                        int c, rw, off;
                        if (vec) {
                            c = q / (rows_col * chunks_row);
                            int rem = q - c * rows_col * chunks_row;
                            rw = rem / chunks_row;
                            off = (rem - rw * chunks_row) << 4;
                        } else {
                            c = q / (rows_col * nx);
                            int rem = q - c * rows_col * nx;
                            rw = rem / nx;
                            off = rem - rw * nx;
                        }
                        const int cc = cb + c, j = j0 + cc % nj, l = l0 + cc / nj;
                        const int y0 = j * P.Ly + dy, z0 = l * P.Lz + dz;
                        int gsub, gy, gz;
                        if (rw < rows_own) {
                            const Win wy = make_win(ny, 3, -1, y0), wz = make_win(nz, 3, -1, z0);
                            gsub = sub;
                            gy = wy.row(rw % wy.cnt);
                            gz = wz.row(rw / wy.cnt);
                        } else {
                            const int k2 = rw - rows_own;
                            const Win wy = make_win(ny, 4, s_off - 1, y0), wz = make_win(nz, 4, s_off - 1, z0);
                            gsub = 1 - sub;
                            gy = wy.row(k2 % wy.cnt);
                            gz = wz.row(k2 / wy.cnt);
                        }
                        const int8_t *src = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx + off;
                        unsigned char *dst = colbuf + (size_t)c * col_bytes + rw * rowB + off;
                        if (vec) {
                            const unsigned saddr = (unsigned)__cvta_generic_to_shared(dst);
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(src)
                                         : "memory");
                        } else {
                            *dst = (unsigned char)__ldcg(src);
                        }
                    }
                    asm volatile("cp.async.wait_all;" ::: "memory");
                    __syncthreads();

                    // ---- the Lx mini-steps of this group, in lock-step ----
                    const int items = nc * NLx;
                    for (int dx = 0; dx < P.Lx; ++dx) {
                        for (int it = tid; it < items; it += nthr) {
                            const int c = it / NLx, i = it - c * NLx;
                            const int cc = cb + c, j = j0 + cc % nj, l = l0 + cc / nj;
                            const int y0 = j * P.Ly + dy, z0 = l * P.Lz + dz;
                            ColView cv;
                            cv.own = colbuf + (size_t)c * col_bytes;
                            cv.oth = cv.own + rows_own * rowB;
                            cv.rowB = rowB;
                            cv.oy = make_win(ny, 3, -1, y0);
                            cv.oz = make_win(nz, 3, -1, z0);
                            cv.ty = make_win(ny, 4, s_off - 1, y0);
                            cv.tz = make_win(nz, 4, s_off - 1, z0);
                            const int x = i * P.Lx + dx;
                            const uint32_t s = (uint32_t)(((sub * nz + z0) * ny + y0) * nx + x);
                            const uint32_t w = site_word(P.seed, RD.rep, sweep, s);
                            int A, B, ex, ey, ez;
                            const int32_t dE = trial_dE_hist<NSH, SW, ColView>(cv, x, nx, s_off, (int)(w >> kRBits),
                                                                               Qt, P.qrow, A, B, ex, ey, ez);
                            if (accept_fixed<IS_INT>(dE, w & kRMask, cx, P.tab, ti)) {
                                if (A != B) {
                                    cv.O(0, 0)[x] = (unsigned char)B;
                                    cv.T(ey, ez)[wrapc(x + ex, nx)] = (unsigned char)A;
                                }
                                accE += dE;
                                accN += 1;
                            }
                        }
                        __syncthreads();
                    }

                    // ---- write back the rows this group may have changed ----
                    // trial row (0, 0) and partner rows (s_off .. s_off+1)^2
                    for (int q = tid; q < nc * 5 * chunks_row * (vec ? 1 : 16); q += nthr) {
                        int c, wr, off;
                        if (vec) {
                            c = q / (5 * chunks_row);
                            int rem = q - c * 5 * chunks_row;
                            wr = rem / chunks_row;
                            off = (rem - wr * chunks_row) << 4;
                        } else {
                            c = q / (5 * chunks_row * 16);
                            int rem = q - c * 5 * chunks_row * 16;
                            wr = rem / (chunks_row * 16);
                            off = rem - wr * chunks_row * 16;
                            if (off >= nx) continue;
                        }
                        const int cc = cb + c, j = j0 + cc % nj, l = l0 + cc / nj;
                        const int y0 = j * P.Ly + dy, z0 = l * P.Lz + dz;
                        int gsub, gy, gz, srow;
                        if (wr == 0) {
                            const Win wy = make_win(ny, 3, -1, y0), wz = make_win(nz, 3, -1, z0);
                            gsub = sub;
                            gy = y0;
                            gz = z0;
                            srow = wz.slot(0) * wy.cnt + wy.slot(0);
                        } else {
                            const int ddy = s_off + ((wr - 1) & 1), ddz = s_off + ((wr - 1) >> 1);
                            const Win wy = make_win(ny, 4, s_off - 1, y0), wz = make_win(nz, 4, s_off - 1, z0);
                            gsub = 1 - sub;
                            gy = wrapc(y0 + ddy, ny);
                            gz = wrapc(z0 + ddz, nz);
                            srow = rows_own + wz.slot(ddz) * wy.cnt + wy.slot(ddy);
                        }
                        int8_t *dstg = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx + off;
                        const unsigned char *srcs = colbuf + (size_t)c * col_bytes + srow * rowB + off;
                        if (vec)
                            *(int4 *)dstg = *(const int4 *)srcs;
                        else
                            *dstg = (int8_t)*srcs;
                    }
                    __syncthreads();
                }

                // ---- per-tile accumulation (fixed order) and publication ----
                const double e_w = (double)warp_sum<long long>(accE);
                const long long n_w = warp_sum<long long>(accN);
                if (lane == 0) {
                    slot_e[slotk * nwarp + warp] += e_w;
                    slot_n[slotk * nwarp + warp] += n_w;
                }
                __syncthreads();
                if (tid == 0 && tile != P.skip_tile) {
                    __threadfence();
                    st_release_u32(P.flags + tile, gstep + 1);
                }
            }
        }
    }

    // ---- per-tile partial sums, then the last CTA reduces them in order ----
    __syncthreads();
    if (s_stop) return;
    {
        int k = 0;
        for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++k) {
            if (tid == 0) {
                double se = 0.0;
                long long sn = 0;
                for (int w = 0; w < nwarp; ++w) {
                    se += slot_e[k * nwarp + w];
                    sn += slot_n[k * nwarp + w];
                }
                P.part_e[tile] = se;
                P.part_n[tile] = sn;
            }
        }
    }
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(P.ticket, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int r = tid; r < P.R; r += nthr) {
        const RepDesc &RD = P.rep[r];
        double se = 0.0;
        long long sn = 0;
        const int nt = RD.NTy * RD.NTz;
        for (int k = 0; k < nt; ++k) {
            se += __ldcg(P.part_e + RD.tile0 + k);
            sn += __ldcg(P.part_n + RD.tile0 + k);
        }
        if (RD.e_acc) *RD.e_acc += se * P.escale;
        if (RD.n_acc) *RD.n_acc += sn;
    }
}

// ---------------------------------------------------------------------------
// Fast path: every axis holds >= 2 four-cell link cells (Lx = Ly = Lz = 4).
// One warp owns tiles of columns and runs them without CTA barriers: for
// each column it waits for the tile's neighbours, stages the column's rows
// in its own shared memory, runs the 4 mini-steps of the group (lane i
// handles link cells i, i+32, ...), writes back the 5 rows the group may
// change and, after the tile's last column, publishes its progress.
//
// Staging is one bulk copy per row (cp.async.bulk, completing on an
// mbarrier), and a warp keeps two column buffers: while it runs the trials
// of one column, the rows of the next are in flight.  The next column is
// fetched early only when that cannot read stale rows: a column of the same
// tile and group (distinct columns of a group touch disjoint rows), or a
// column of another tile whose neighbours have already published the group
// it needs.  Philox runs once per link cell and group: the four trial sites
// of a link cell's x-row, x = 4i .. 4i+3, share the counter s >> 2.
//
// During a launch every species byte holds 8 s (the shift of its histogram
// field; a pass before and after the launch converts), so a neighbour adds
// nib8(byte) to its shell's word.
//
// Shared-memory rows of a column (stride rb): the row body starts 16 bytes
// in and is framed by a 4-byte periodic halo on each side, so x-2 .. x+2
// need no wrap.  Trial-sublattice rows (dy, dz) in [-1, 1]^2 are at index
// (dz+1)*3 + (dy+1); partner-sublattice rows (sy, sz) in [0, 4)^2, i.e.
// (dy, dz) = (s_off-1+sy, s_off-1+sz), at pslot(sy, sz).  Two-shell models
// never read the four partner corner rows (not loaded).
// ---------------------------------------------------------------------------
template <int NSH>
__host__ __device__ __forceinline__ constexpr int pslot(int sy, int sz)
{
    return NSH >= 3 ? 9 + sz * 4 + sy : 9 + (sz == 0 ? sy - 1 : (sz == 1 ? 2 + sy : (sz == 2 ? 6 + sy : 9 + sy)));
}
template <int NSH>
__host__ __device__ constexpr int fast_nrows()
{
    return NSH >= 3 ? 25 : 21;
}

#define LD8(off) ((uint32_t)g_smem[(off)])

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// Bounded wait for a buffer's bulk copies (parity of the phase to complete).
// Every copy waited for was issued by this warp, so the wait ends unless the
// hardware fails; past the time limit the status word and the abort flag are
// set.
__device__ __forceinline__ bool mbar_wait(const SweepParams &P, uint32_t a, uint32_t parity)
{
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(a, parity)) return true;
        if ((long long)(global_ns() - t0) > P.timeout_ns) {
            atomicCAS(P.status, 0, (int)SMC_ERR_TIMEOUT);
            atomicExch(P.abort_flag, 1);
            return false;
        }
    }
}

// One non-blocking look at the 8 neighbouring tiles' progress.
__device__ __forceinline__ bool deps_ready(const SweepParams &P, const RepDesc &D, int ty, int tz, uint32_t need,
                                           int lane)
{
    bool ok = true;
    if (lane < 9 && lane != 4) {
        int nty = ty + (lane % 3) - 1, ntz = tz + (lane / 3) - 1;
        nty = nty < 0 ? nty + D.NTy : (nty >= D.NTy ? nty - D.NTy : nty);
        ntz = ntz < 0 ? ntz + D.NTz : (ntz >= D.NTz ? ntz - D.NTz : ntz);
        ok = ld_acquire_u32(P.flags + D.tile0 + ntz * D.NTy + nty) >= need;
    }
    return __all_sync(0xffffffffu, ok);
}

// Row r of a column: sublattice (relative: 0 own, 1 partner) and offsets.
template <int NSH>
__device__ __forceinline__ void fast_row(int r, int soff, int &part, int &dy, int &dz)
{
    if (r < 9) {
        dy = r % 3 - 1;
        dz = r / 3 - 1;
        part = 0;
    } else {
        const int k = r - 9;
        int sy, sz;
        if (NSH >= 3) {
            sy = k & 3;
            sz = k >> 2;
        } else {
            sz = k < 2 ? 0 : (k < 6 ? 1 : (k < 10 ? 2 : 3));
            sy = k < 2 ? k + 1 : (k < 6 ? k - 2 : (k < 10 ? k - 6 : k - 9));
        }
        dy = sy - 1 + soff;
        dz = sz - 1 + soff;
        part = 1;
    }
}

// Geometry of a work item (sweep t of the launch, group g, tile, column c).
struct FastGeo {
    int r, ty, tz, j, l, y0, z0, dy, dz, sub, soff, ncols, nj;
    uint32_t gstep, need;
};

__device__ __forceinline__ FastGeo fast_geo(const SweepParams &P, int t, int g, int tile, int c)
{
    FastGeo q;
    int r = 0;
    while (r + 1 < P.R && P.rep[r + 1].tile0 <= tile) ++r;
    const RepDesc &RD = P.rep[r];
    q.r = r;
    const int lt = tile - RD.tile0;
    q.ty = lt % RD.NTy;
    q.tz = lt / RD.NTy;
    const int j0 = q.ty * P.TY, j1 = min(j0 + P.TY, RD.NLy);
    const int l0 = q.tz * P.TZ, l1 = min(l0 + P.TZ, RD.NLz);
    q.nj = j1 - j0;
    q.ncols = q.nj * (l1 - l0);
    q.j = j0 + c % q.nj;
    q.l = l0 + c / q.nj;
    q.dy = g & 3;
    q.dz = (g >> 2) & 3;
    q.sub = g >> 4;
    q.soff = q.sub == 0 ? -1 : 0;
    q.y0 = 4 * q.j + q.dy;
    q.z0 = 4 * q.l + q.dz;
    q.gstep = (uint32_t)(t * P.G + g);
    const int lagv = P.lag[g];
    q.need = q.gstep + 1 >= (uint32_t)lagv ? q.gstep + 1 - lagv : 0;
    return q;
}

// Stages the rows of column geometry q into the buffer at g_smem offset buf.
// Rows of a multiple of 16 bytes, 16-byte aligned: mode 0, one cp.async.bulk
// per row, completing on mbarrier `mbar` (absolute shared address); mode 1,
// 16-byte cp.async per lane in one commit group (the issuing warp waits with
// cp.async.wait_group).  Otherwise the warp copies 4-byte words and returns
// with the rows in place.
template <int NSH>
__device__ __forceinline__ void fast_stage(const RepDesc &RD, const FastGeo &q, uint32_t smem0, uint32_t buf,
                                           uint32_t rb, uint32_t mbar, int lane, int mode)
{
    constexpr int NROWS = fast_nrows<NSH>();
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz;
    const int8_t *src = RD.occ;
    if (lane < NROWS) {
        int part, dy, dz;
        fast_row<NSH>(lane, q.soff, part, dy, dz);
        const int gsub = part ? 1 - q.sub : q.sub;
        const int gy = wrapc(q.y0 + dy, ny), gz = wrapc(q.z0 + dz, nz);
        src = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx;
    }
    if (RD.vec && mode == 0) {
        // order this warp's earlier generic accesses of the buffer, and the
        // rows other warps published (seen through the acquire loads), before
        // the async-proxy copies
        __syncwarp();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_expect_tx(mbar, (uint32_t)(NROWS * nx));
        __syncwarp();
        if (lane < NROWS) bulk_g2s(smem0 + buf + (uint32_t)lane * rb + 16, src, (uint32_t)nx, mbar);
    } else if (RD.vec) {
        // 16-byte cp.async (L2 only: never a stale L1 line), one commit group
        const int cpr = nx >> 4;
        int lr = 0, lc = lane, rstep = 1, cstep = 32;
        if (cpr < 32) {
            rstep = 32 / cpr;
            lr = lane / cpr;
            lc = lane - lr * cpr;
            cstep = cpr;
        }
        for (int it = 0; it < (NROWS + rstep - 1) / rstep; ++it) {
            const int rr = lr + it * rstep;
            const int rsel = rr < NROWS ? rr : 0;
            const int8_t *s = (const int8_t *)__shfl_sync(0xffffffffu, (unsigned long long)src, rsel);
            if (lr < rstep && rr < NROWS) {
                const uint32_t d = smem0 + buf + (uint32_t)rr * rb + 16;
                for (int c = lc; c < cpr; c += cstep)
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16 * c), "l"(s + 16 * c)
                                 : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
        const int cpr = nx >> 2;
        int lr = 0, lc = lane, rstep = 1, cstep = 32;
        if (cpr < 32) {
            rstep = 32 / cpr;
            lr = lane / cpr;
            lc = lane - lr * cpr;
            cstep = cpr;
        }
        for (int it = 0; it < (NROWS + rstep - 1) / rstep; ++it) {
            const int rr = lr + it * rstep;
            const int rsel = rr < NROWS ? rr : 0;
            const unsigned *s4 = (const unsigned *)__shfl_sync(0xffffffffu, (unsigned long long)src, rsel);
            if (lr < rstep && rr < NROWS) {
                unsigned *d4 = (unsigned *)(g_smem + buf + (uint32_t)rr * rb + 16);
                for (int c = lc; c < cpr; c += cstep) d4[c] = __ldcg(s4 + c);
            }
        }
        __syncwarp();
    }
}

// dE_fix of the trial at a = own row (0, 0), x, with ya = row-0 body + x and
// pa = ya + s_off, partner direction dir; the species a8, b8 (x 8) and b's
// shared-memory offset through references.
template <int NSH, int SW, int RB>
__device__ __forceinline__ int32_t fast_dE(uint32_t ya, uint32_t pa, uint32_t rbr, uint32_t dir, uint32_t lut,
                                           uint32_t qt, uint32_t &a8, uint32_t &b8, uint32_t &pb)
{
    using H = HV<SW>;
    constexpr uint32_t B12 = 0x08080808u;
    const uint32_t rb = RB ? (uint32_t)RB : rbr;
    constexpr uint32_t S11 = pslot<NSH>(1, 1), S21 = pslot<NSH>(2, 1), S12 = pslot<NSH>(1, 2), S22 = pslot<NSH>(2, 2);
    const int4 L = *(const int4 *)(g_smem + lut + dir * 16u);
    a8 = LD8(ya + 4 * rb);
    pb = pa + (uint32_t)L.x;
    b8 = LD8(pb);
    const uint32_t ob = ya + (uint32_t)L.y;
    // shell 1: a's 8 partner-sublattice neighbours minus b, minus b's 8
    // trial-sublattice neighbours plus a (biased by 8 per field)
    const H a0 = hconst<SW>(B12) + hv<SW>(a8) + hv<SW>(LD8(pa + S11 * rb));
    const H a1 = hv<SW>(LD8(pa + S11 * rb + 1)) + hv<SW>(LD8(pa + S21 * rb)) + hv<SW>(LD8(pa + S21 * rb + 1));
    const H a2 = hv<SW>(LD8(pa + S12 * rb)) + hv<SW>(LD8(pa + S12 * rb + 1)) + hv<SW>(LD8(pa + S22 * rb));
    const H a3 = hv<SW>(LD8(pa + S22 * rb + 1));
    const H b0 = hv<SW>(b8) + hv<SW>(LD8(ob)) + hv<SW>(LD8(ob + 1));
    const H b1 = hv<SW>(LD8(ob + rb)) + hv<SW>(LD8(ob + rb + 1)) + hv<SW>(LD8(ob + 3 * rb));
    const H b2 = hv<SW>(LD8(ob + 3 * rb + 1)) + hv<SW>(LD8(ob + 4 * rb)) + hv<SW>(LD8(ob + 4 * rb + 1));
    const H h0 = (a0 + a1) + (a2 + a3) - ((b0 + b1) + b2);
    // shell 2: a's 6 trial-sublattice neighbours, b's 6 partner-sublattice ones
    const H c0 = hconst<SW>(B12) + hv<SW>(LD8(ya + 4 * rb - 1)) + hv<SW>(LD8(ya + 4 * rb + 1));
    const H c1 = hv<SW>(LD8(ya + 3 * rb)) + hv<SW>(LD8(ya + 5 * rb)) + hv<SW>(LD8(ya + rb));
    const H c2 = hv<SW>(LD8(ya + 7 * rb));
    const H d0 = hv<SW>(LD8(pb - 1)) + hv<SW>(LD8(pb + 1)) + hv<SW>(LD8(pb - rb));
    const H d1 = hv<SW>(LD8(pb + rb)) + hv<SW>(LD8(pb - (uint32_t)L.z)) + hv<SW>(LD8(pb + (uint32_t)L.w));
    const H h1 = ((c0 + c1) + c2) - (d0 + d1);
    uint32_t Hw[NSH][SW];
#pragma unroll
    for (int w = 0; w < SW; ++w) {
        Hw[0][w] = h0.w[w];
        Hw[1][w] = h1.w[w];
    }
    if constexpr (NSH >= 3) {
        // shell 3: a's 12 trial-sublattice neighbours, b's 12
        // partner-sublattice ones (biased by 16 per field)
        const H e0 = hconst<SW>(0x10101010u) + hv<SW>(LD8(ya)) + hv<SW>(LD8(ya + 2 * rb));
        const H e1 = hv<SW>(LD8(ya + 6 * rb)) + hv<SW>(LD8(ya + 8 * rb)) + hv<SW>(LD8(ya + 3 * rb - 1));
        const H e2 = hv<SW>(LD8(ya + 3 * rb + 1)) + hv<SW>(LD8(ya + 5 * rb - 1)) + hv<SW>(LD8(ya + 5 * rb + 1));
        const H e3 = hv<SW>(LD8(ya + rb - 1)) + hv<SW>(LD8(ya + rb + 1)) + hv<SW>(LD8(ya + 7 * rb - 1));
        const H e4 = hv<SW>(LD8(ya + 7 * rb + 1));
        const H f0 = hv<SW>(LD8(pb - 5 * rb)) + hv<SW>(LD8(pb - 3 * rb)) + hv<SW>(LD8(pb + 3 * rb));
        const H f1 = hv<SW>(LD8(pb + 5 * rb)) + hv<SW>(LD8(pb - rb - 1)) + hv<SW>(LD8(pb - rb + 1));
        const H f2 = hv<SW>(LD8(pb + rb - 1)) + hv<SW>(LD8(pb + rb + 1)) + hv<SW>(LD8(pb - 4 * rb - 1));
        const H f3 = hv<SW>(LD8(pb - 4 * rb + 1)) + hv<SW>(LD8(pb + 4 * rb - 1)) + hv<SW>(LD8(pb + 4 * rb + 1));
        const H h2 = ((e0 + e1) + (e2 + e3) + e4) - ((f0 + f1) + (f2 + f3));
#pragma unroll
        for (int w = 0; w < SW; ++w) Hw[2][w] = h2.w[w];
    }
    constexpr uint32_t half_row = (uint32_t)qrow_words(NSH, SW) / 2;  // (A * 8 + B) rows = (8 a8 + b8) / 8
    const uint32_t *row = (const uint32_t *)(g_smem + qt + (8u * a8 + b8) * half_row);
    return dot_fixed<NSH, SW>(Hw, row);
}

// Team synchronisation: the tw warps that share a column meet at named
// barrier tb (1 + team index in the CTA); one warp needs only __syncwarp.
// team_and also returns the AND of the threads' predicates.
// (bar.sync and bar.red are warp-aligned: the warp reconverges first.)
__device__ __forceinline__ void team_sync(int tw, int tb)
{
    __syncwarp();
    if (tw > 1) asm volatile("bar.sync %0, %1;" ::"r"(tb), "r"(tw * 32) : "memory");
}
__device__ __forceinline__ bool team_and(int tw, int tb, bool p)
{
    if (tw == 1) return __all_sync(0xffffffffu, p);
    __syncwarp();
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred q, d;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.and.pred d, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, d;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)p), "r"(tb), "r"(tw * 32)
        : "memory");
    return r != 0;
}

// KU trials of mini-step dx per lane: link cells i = ib + is * (k0 + u),
// u < KU (ib = lane + 32 * warp-in-team, is = 32 * team size).
template <bool IS_INT, int NSH, int SW, int RB, int KU, bool GUARD>
__device__ __forceinline__ void fast_trials(const SweepParams &P, uint32_t body, int soff, uint32_t rbr,
                                            uint32_t wsm, int k0, int nk, int ib, int is, int NLx, int nx, int dx,
                                            int lane, float cx, int2 ti, uint32_t lut, uint32_t qt, long long &accE,
                                            long long &accN)
{
    const uint32_t rb = RB ? (uint32_t)RB : rbr;
    int32_t dE[KU];
    uint32_t a8[KU], b8[KU], pb[KU], ya[KU];
    bool acc[KU];
#pragma unroll
    for (int u = 0; u < KU; ++u) {
        const int k = k0 + u, i = ib + is * k;
        acc[u] = false;
        if (!GUARD || (k < nk && i < NLx)) {
            const int x = 4 * i + dx;
            ya[u] = body + (uint32_t)x;
            const uint32_t w = *(const uint32_t *)(g_smem + wsm + (uint32_t)(((k * 4 + dx) * 32 + lane) * 4));
            dE[u] = fast_dE<NSH, SW, RB>(ya[u], ya[u] + soff, rbr, w >> kRBits, lut, qt, a8[u], b8[u], pb[u]);
            acc[u] = accept_fixed<IS_INT>(dE[u], w & kRMask, cx, P.tab, ti);
            // b's store address wraps along x (the load may read a halo copy)
            const int xb = x + soff + (int)(w >> 31);
            pb[u] += xb < 0 ? (uint32_t)nx : (xb >= nx ? (uint32_t)(-nx) : 0u);
        }
    }
#pragma unroll
    for (int u = 0; u < KU; ++u) {
        if (acc[u]) {
            g_smem[ya[u] + 4 * rb] = (unsigned char)b8[u];
            g_smem[pb[u]] = (unsigned char)a8[u];
            accE += dE[u];
            accN += 1;
        }
    }
}

// The fast kernel.  A team of tw warps (1, 2 or 4) shares one column at a
// time: the team's first warp ("leader") polls the neighbours' progress,
// issues the row copies into the team's two buffers and publishes the
// tile's progress; every warp of the team runs its own link cells (lane +
// 32 w + 32 tw k) and waits for the copies on the buffer's mbarrier.
// Shared memory: [table][8 direction offsets][team regions: barriers, two
// buffers][warp regions: accumulator slots, Philox words].
template <bool IS_INT, int NSH, int SW, int RB>
__global__ void __launch_bounds__(256) k_sweep_fast(const __grid_constant__ SweepParams P)
{
    constexpr int NROWS = fast_nrows<NSH>();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int tw = P.team, wi = warp % tw, tix = warp / tw, tpb = nwarp / tw;
    const int gteam = blockIdx.x * tpb + tix, NT = gridDim.x * tpb, NW = gridDim.x * nwarp;
    const int tb = 1 + tix;
    const bool leader = wi == 0;
    const uint32_t rb = RB ? (uint32_t)RB : (uint32_t)P.rowB;
    const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    // fixed-point table and the per-direction offsets of b and its rows
    const uint32_t qt = 0u;
    const int qwords = kQRows * P.qrow;
    for (int i = tid; i < qwords; i += blockDim.x) ((uint32_t *)g_smem)[i] = P.qtab[i];
    const uint32_t lut = (uint32_t)qwords * 4u;
    if (tid < 8) {
        const int kx = (tid >> 2) & 1, ky = (tid >> 1) & 1, kz = tid & 1;
        int4 e;
        e.x = pslot<NSH>(ky + 1, kz + 1) * (int)rb + kx;
        e.y = (3 * kz + ky) * (int)rb + kx - 1;
        e.z = NSH >= 3 ? 4 * (int)rb : (3 + kz) * (int)rb;
        e.w = NSH >= 3 ? 4 * (int)rb : (4 - kz) * (int)rb;
        *(int4 *)(g_smem + lut + (uint32_t)tid * 16u) = e;
    }
    const uint32_t tbase = lut + 128u + (uint32_t)tix * (uint32_t)P.team_bytes;
    const uint32_t mbar0 = tbase, buf0 = tbase + 16u, bufsz = (uint32_t)NROWS * rb;
    const int nbuf = P.nbuf;  // 1: no prefetch, the next column reuses the buffer
    const uint32_t wbase = lut + 128u + (uint32_t)tpb * (uint32_t)P.team_bytes + (uint32_t)warp * (uint32_t)P.warp_bytes;
    // per-tile sums of dE_fix and accepted counts: exact integers
    long long *slot_e = (long long *)(g_smem + wbase);
    long long *slot_n = slot_e + P.tpc;
    const uint32_t wsm = wbase + (uint32_t)P.tpc * 16u;
    const int is = 32 * tw, ib = lane + 32 * wi;
    const int nkw = (P.maxNLx + is - 1) / is;
    for (int i = lane; i < P.tpc; i += 32) {
        slot_e[i] = 0;
        slot_n[i] = 0;
    }
    if (leader && lane == 0) {
        mbar_init(smem0 + mbar0, 1);
        mbar_init(smem0 + mbar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool aborted = false;
    // per buffer b: bit b of par = parity of its barrier's next phase; bit b
    // of inflight (leader) = copies issued and not yet waited for
    uint32_t par = 0u, inflight = 0u;
    if (gteam < P.ntiles) {
        int t = 0, g = 0, tile = gteam, c = 0, nb = 0, slotk = 0;
        long long accE = 0, accN = 0;
        FastGeo q = fast_geo(P, t, g, tile, c);
        bool ok = true;
        if (leader) {
            ok = wait_tile_warp(P, P.rep[q.r], q.ty, q.tz, q.need, lane);
            if (ok) {
                fast_stage<NSH>(P.rep[q.r], q, smem0, buf0, rb, smem0 + mbar0, lane, P.stage);
                if (P.rep[q.r].vec && P.stage == 0) inflight = 1u;
            }
        }
        if (!team_and(tw, tb, ok)) aborted = true;
        while (!aborted) {
            const RepDesc &RD = P.rep[q.r];
            const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NLx = RD.NLx;
            // the next item
            int t2 = t, g2 = g, tile2 = tile, c2 = c + 1, slot2 = slotk;
            if (c2 >= q.ncols) {
                c2 = 0;
                tile2 += NT;
                ++slot2;
                if (tile2 >= P.ntiles) {
                    tile2 = gteam;
                    slot2 = 0;
                    if (++g2 == P.G) {
                        g2 = 0;
                        ++t2;
                    }
                }
            }
            const bool has_next = t2 < P.nsweeps;
            FastGeo q2;
            if (has_next) q2 = fast_geo(P, t2, g2, tile2, c2);
            const bool next_vec = has_next && P.rep[q2.r].vec != 0;
            auto can_prefetch = [&]() -> bool {
                if (!next_vec || nbuf < 2) return false;
                if (c2 > 0) return true;
                if (tile2 == tile) return false;
                return deps_ready(P, P.rep[q2.r], q2.ty, q2.tz, q2.need, lane);
            };
            const int nbn = nbuf == 2 ? nb ^ 1 : nb;
            const uint32_t bcur = buf0 + (uint32_t)nb * bufsz, bnext = buf0 + (uint32_t)nbn * bufsz;
            const uint32_t mcur = smem0 + mbar0 + 8u * (uint32_t)nb, mnext = smem0 + mbar0 + 8u * (uint32_t)nbn;
            bool pre = false;
            if (leader && can_prefetch()) {
                fast_stage<NSH>(P.rep[q2.r], q2, smem0, bnext, rb, mnext, lane, P.stage);
                if (P.stage == 0) inflight |= 1u << nbn;
                pre = true;
            }
            // Philox words of this warp's link cells (while the rows land)
            const uint64_t sweep = P.sweep0 + (uint64_t)t;
            {
                const uint32_t rowsite = (uint32_t)(((q.sub * nz + q.z0) * ny + q.y0) * nx);
                const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
                uint32_t *wp = (uint32_t *)(g_smem + wsm);
#pragma unroll 1
                for (int k = 0; k < nkw; ++k) {
                    const int i = ib + is * k;
                    if (i < NLx) {
                        const U4 w = philox10(
                            U4{(rowsite >> 2) + (uint32_t)i, RD.rep, (uint32_t)sweep, (uint32_t)(sweep >> 32)}, k0, k1);
                        wp[(k * 4 + 0) * 32 + lane] = w.x;
                        wp[(k * 4 + 1) * 32 + lane] = w.y;
                        wp[(k * 4 + 2) * 32 + lane] = w.z;
                        wp[(k * 4 + 3) * 32 + lane] = w.w;
                    }
                }
            }
            ok = true;
            if (RD.vec && P.stage == 0) {
                ok = mbar_wait(P, mcur, (par >> nb) & 1u);
                par ^= 1u << nb;
                if (ok) inflight &= ~(1u << nb);
            } else if (RD.vec && leader) {
                // this item's group is the newest unless the next one was just issued
                if (pre)
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                else
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                __syncwarp();
            }
            // periodic halos: 4 bytes before and after each row body
            if (leader && lane < NROWS) {
                const uint32_t bd = bcur + (uint32_t)lane * rb + 16u;
                *(unsigned *)(g_smem + bd - 4) = *(const unsigned *)(g_smem + bd + nx - 4);
                *(unsigned *)(g_smem + bd + nx) = *(const unsigned *)(g_smem + bd);
            }
            if (!team_and(tw, tb, ok)) {
                aborted = true;
                break;
            }
            float cx = 0.f;
            int2 ti = make_int2(0, 0);
            if constexpr (IS_INT)
                ti = P.temp.tabinfo[P.beta_stride ? q.r * P.beta_stride + t : q.r];
            else
                cx = P.temp.beta[P.beta_stride ? q.r * P.beta_stride + t : q.r];
            const uint32_t body = bcur + 16u;
            // halo refresh of the 5 rows a mini-step writes: leader lane l < 10
            // takes row l / 2 (own (0,0), then partner (1,1), (2,1), (1,2),
            // (2,2)) and side l % 2
            uint32_t hrow = 0;
            if (lane < 10) {
                const int r5 = lane >> 1;
                const int sl = r5 == 0 ? 4 : pslot<NSH>(1 + ((r5 - 1) & 1), 1 + ((r5 - 1) >> 1));
                hrow = body + (uint32_t)sl * rb;
            }
            for (int dx = 0; dx < 4; ++dx) {
                if (NLx == is * nkw && (nkw & 3) == 0) {
#pragma unroll 1
                    for (int kk = 0; kk < nkw; kk += 4)
                        fast_trials<IS_INT, NSH, SW, RB, 4, false>(P, body, q.soff, rb, wsm, kk, nkw, ib, is, NLx, nx,
                                                                   dx, lane, cx, ti, lut, qt, accE, accN);
                } else if (NLx == is * nkw && (nkw & 1) == 0) {
#pragma unroll 1
                    for (int kk = 0; kk < nkw; kk += 2)
                        fast_trials<IS_INT, NSH, SW, RB, 2, false>(P, body, q.soff, rb, wsm, kk, nkw, ib, is, NLx, nx,
                                                                   dx, lane, cx, ti, lut, qt, accE, accN);
                } else if (NLx == is * nkw) {
#pragma unroll 1
                    for (int kk = 0; kk < nkw; ++kk)
                        fast_trials<IS_INT, NSH, SW, RB, 1, false>(P, body, q.soff, rb, wsm, kk, nkw, ib, is, NLx, nx,
                                                                   dx, lane, cx, ti, lut, qt, accE, accN);
                } else {
#pragma unroll 1
                    for (int kk = 0; kk < nkw; ++kk)
                        fast_trials<IS_INT, NSH, SW, RB, 1, true>(P, body, q.soff, rb, wsm, kk, nkw, ib, is, NLx, nx,
                                                                  dx, lane, cx, ti, lut, qt, accE, accN);
                }
                team_sync(tw, tb);
                if (leader && lane < 10) {
                    if (lane & 1)
                        *(unsigned *)(g_smem + hrow + nx) = *(const unsigned *)(g_smem + hrow);
                    else
                        *(unsigned *)(g_smem + hrow - 4) = *(const unsigned *)(g_smem + hrow + nx - 4);
                }
                team_sync(tw, tb);
                if (leader && !pre && dx < 3 && can_prefetch()) {
                    fast_stage<NSH>(P.rep[q2.r], q2, smem0, bnext, rb, mnext, lane, P.stage);
                    if (P.stage == 0) inflight |= 1u << nbn;
                    pre = true;
                }
            }
            // ---- write back trial row (0,0) and partner rows (s_off..s_off+1)^2,
            // row by row, the team's threads over the row's chunks ----
            {
                const bool vec = RD.vec != 0;
                const int cpr = vec ? (nx >> 4) : (nx >> 2);
#pragma unroll 1
                for (int wrow = 0; wrow < 5; ++wrow) {
                    int slot, gsub, gy, gz;
                    if (wrow == 0) {
                        slot = 4;
                        gsub = q.sub;
                        gy = q.y0;
                        gz = q.z0;
                    } else {
                        const int sy = 1 + ((wrow - 1) & 1), sz = 1 + ((wrow - 1) >> 1);
                        slot = pslot<NSH>(sy, sz);
                        gsub = 1 - q.sub;
                        gy = wrapc(q.y0 + sy - 1 + q.soff, ny);
                        gz = wrapc(q.z0 + sz - 1 + q.soff, nz);
                    }
                    int8_t *dstg = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx;
                    const unsigned char *srcs = g_smem + body + (uint32_t)slot * rb;
                    for (int cc = lane + 32 * wi; cc < cpr; cc += is) {
                        if (vec)
                            *((int4 *)dstg + cc) = *((const int4 *)srcs + cc);
                        else
                            *((unsigned *)dstg + cc) = *((const unsigned *)srcs + cc);
                    }
                }
            }
            // every thread's row stores, then one release by the leader's lane 0
            // (the barrier orders the team's stores before it)
            team_sync(tw, tb);
            if (c + 1 >= q.ncols) {
                // the tile's last column: accumulate in fixed order and publish
                const long long e_w = warp_sum<long long>(accE);
                const long long n_w = warp_sum<long long>(accN);
                if (lane == 0) {
                    slot_e[slotk] += e_w;
                    slot_n[slotk] += n_w;
                }
                accE = 0;
                accN = 0;
                if (leader && lane == 0 && tile != P.skip_tile) st_release_u32(P.flags + tile, q.gstep + 1);
            }
            if (!has_next) break;
            ok = true;
            if (leader && !pre) {
                if (c2 == 0) ok = wait_tile_warp(P, P.rep[q2.r], q2.ty, q2.tz, q2.need, lane);
                if (ok) {
                    fast_stage<NSH>(P.rep[q2.r], q2, smem0, bnext, rb, mnext, lane, P.stage);
                    if (next_vec && P.stage == 0) inflight |= 1u << nbn;
                }
            }
            if (!team_and(tw, tb, ok)) {
                aborted = true;
                break;
            }
            t = t2;
            g = g2;
            tile = tile2;
            c = c2;
            slotk = slot2;
            q = q2;
            nb = nbn;
        }
    }
    if (aborted) {
        // let the team's copies in flight land before the CTA ends
        if (leader) asm volatile("cp.async.wait_all;" ::: "memory");
        if (leader)
            for (int b = 0; b < 2; ++b)
                if (inflight & (1u << b)) mbar_wait(P, smem0 + mbar0 + 8u * (uint32_t)b, (par >> b) & 1u);
        return;
    }
    // ---- per-tile partial sums (one per warp of the team); the last warp to
    // finish reduces them, all its lanes at once: the partial sums are
    // integers (dE_fix, counts), so their int64 sum is exact in any order ----
    if (lane == 0) {
        int k = 0;
        for (int tl = gteam; tl < P.ntiles; tl += NT, ++k) {
            P.part_e[(size_t)tl * tw + wi] = (double)slot_e[k];
            P.part_n[(size_t)tl * tw + wi] = slot_n[k];
        }
    }
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicAdd(P.ticket, 1u) == (unsigned)NW - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    for (int r = 0; r < P.R; ++r) {
        const RepDesc &RD = P.rep[r];
        const int np = RD.NTy * RD.NTz * tw;
        const double *pe = P.part_e + (size_t)RD.tile0 * tw;
        const long long *pn = P.part_n + (size_t)RD.tile0 * tw;
        long long se = 0, sn = 0;
        for (int k = lane; k < np; k += 32) {
            se += (long long)__ldcg(pe + k);
            sn += __ldcg(pn + k);
        }
        se = warp_sum<long long>(se);
        sn = warp_sum<long long>(sn);
        if (lane == 0) {
            if (RD.e_acc) *RD.e_acc += (double)se * P.escale;
            if (RD.n_acc) *RD.n_acc += sn;
        }
    }
}

// ---------------------------------------------------------------------------
// Paired-group streaming sweep (rows of 128, 256 or 512 cells, one lattice,
// two shells, at most 4 + 1 species).  The groups of a column come in pairs
// (dy, dy + 1) with dy = 0 or 2: group dy + 1 reads no row that a
// neighbouring column writes in group dy, nor the other way round (the
// lag-2 rule of groups with dy >= 1), so once the 8 neighbouring columns
// have finished the previous pair, one warp stages the union of the pair's
// rows (28 rows instead of 2 x 21), runs both groups' 4 mini-steps in it,
// writes back the union of the rows they change (8 instead of 2 x 5) and
// publishes the pair.  Rows in shared memory (relative to the pair's first
// group, y0 = 4 cy + dy, z0 = 4 cz + dz):
//   slots 0..11:  own sublattice, (y0 - 1 + oy, z0 - 1 + oz) at 4 oz + oy,
//                 oy < 4, oz < 3;
//   slots 12..27: partner sublattice, (y0 + s_off - 1 + sy, z0 + s_off - 1
//                 + sz) for sy in 1..3 (sz = 0, 3) or 0..4 (sz = 1, 2), at
//                 pslot2(sy, sz).
// Group h (0 or 1) of the pair sees its own rows shifted by h in y.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pslot2(int sy, int sz)
{
    return sz == 0 ? 11 + sy : (sz == 1 ? 15 + sy : (sz == 2 ? 20 + sy : 24 + sy));
}
constexpr int kPairRows = 28;

// dE_fix of the trial at a (ya = slot-0 body + x, pa = ya + s_off) of group
// H of the pair, direction dir; a8, b8 and b's offset through references.
template <int RB, int H>
__device__ __forceinline__ int32_t pair2_dE(uint32_t ya, uint32_t pa, uint32_t dir, uint32_t lut, uint32_t qt,
                                            uint32_t &a8, uint32_t &b8, uint32_t &pb)
{
    using HW = HV<1>;
    constexpr uint32_t rb = (uint32_t)RB;
    constexpr uint32_t A0 = 5 + H;  // own (0, 0)
    constexpr uint32_t S11 = pslot2(1 + H, 1), S21 = pslot2(2 + H, 1), S12 = pslot2(1 + H, 2),
                       S22 = pslot2(2 + H, 2);
    // b's partner row and x (L.x), b's own 2 x 2 rows (L.y): one 8-byte load
    // (16 lanes of 8 directions per phase); b's partner rows z -/+ 1 are
    // (4 + kz) and (5 - kz) rows away
    const int2 L = *(const int2 *)(g_smem + lut + (uint32_t)H * 64u + dir * 8u);
    const uint32_t kz = dir & 1u;
    const uint32_t Lz = (4u + kz) * rb, Lw = (5u - kz) * rb;
    a8 = LD8(ya + A0 * rb);
    pb = pa + (uint32_t)L.x;
    b8 = LD8(pb);
    const uint32_t ob = ya + (uint32_t)L.y;
    // shell 1: a's 8 partner-sublattice neighbours minus b, minus b's 8
    // trial-sublattice neighbours plus a (counts biased by 128 per field)
    const HW a0 = hconst<1>(0x80808080u) + hv<1>(a8) + hv<1>(LD8(pa + S11 * rb));
    const HW a1 = hv<1>(LD8(pa + S11 * rb + 1)) + hv<1>(LD8(pa + S21 * rb)) + hv<1>(LD8(pa + S21 * rb + 1));
    const HW a2 = hv<1>(LD8(pa + S12 * rb)) + hv<1>(LD8(pa + S12 * rb + 1)) + hv<1>(LD8(pa + S22 * rb));
    const HW a3 = hv<1>(LD8(pa + S22 * rb + 1));
    const HW b0 = hv<1>(b8) + hv<1>(LD8(ob)) + hv<1>(LD8(ob + 1));
    const HW b1 = hv<1>(LD8(ob + rb)) + hv<1>(LD8(ob + rb + 1)) + hv<1>(LD8(ob + 4 * rb));
    const HW b2 = hv<1>(LD8(ob + 4 * rb + 1)) + hv<1>(LD8(ob + 5 * rb)) + hv<1>(LD8(ob + 5 * rb + 1));
    const HW h0 = (a0 + a1) + (a2 + a3) - ((b0 + b1) + b2);
    // shell 2: a's 6 trial-sublattice neighbours, b's 6 partner-sublattice ones
    const HW c0 = hconst<1>(0x80808080u) + hv<1>(LD8(ya + A0 * rb - 1)) + hv<1>(LD8(ya + A0 * rb + 1));
    const HW c1 = hv<1>(LD8(ya + (A0 - 1) * rb)) + hv<1>(LD8(ya + (A0 + 1) * rb)) + hv<1>(LD8(ya + (A0 - 4) * rb));
    const HW c2 = hv<1>(LD8(ya + (A0 + 4) * rb));
    const HW d0 = hv<1>(LD8(pb - 1)) + hv<1>(LD8(pb + 1)) + hv<1>(LD8(pb - rb));
    const HW d1 = hv<1>(LD8(pb + rb)) + hv<1>(LD8(pb - Lz)) + hv<1>(LD8(pb + Lw));
    const HW h1 = ((c0 + c1) + c2) - (d0 + d1);
    return dot_fixed_rtab(h0.w[0], h1.w[0], qt + (a8 * 5u + b8) * 16u);
}

// The trials of mini-step dx of group H for this lane's NKW link cells
// i = lane + 32 k, with the random words wv[k].  b's store address wraps
// along x only for the row's first cell (lane 0, k = 0, dx = 0, s_off = -1,
// kx = 0: x = -1) and its last (lane 31, k = NKW - 1, dx = 3, s_off = 0,
// kx = 1: x = nx); its loads may read the halo copies.
template <bool IS_INT, int RB, int NKW, int H>
__device__ __forceinline__ void pair2_trials(const SweepParams &P, uint32_t body, int soff, int nx, int dx, int lane,
                                             float cx, int2 ti, uint32_t lut, uint32_t qt, const uint32_t (&wv)[NKW],
                                             long long &accE, uint32_t &accN)
{
    const bool lo_edge = lane == 0 && dx == 0 && soff < 0, hi_edge = lane == 31 && dx == 3 && soff == 0;
    constexpr uint32_t A0 = 5 + H;
    int32_t dE[NKW];
    uint32_t a8[NKW], b8[NKW], pb[NKW], ya[NKW];
    bool acc[NKW];
#pragma unroll
    for (int u = 0; u < NKW; ++u) {
        const int x = 4 * (lane + 32 * u) + dx;
        ya[u] = body + (uint32_t)x;
        const uint32_t w = wv[u];
        dE[u] = pair2_dE<RB, H>(ya[u], ya[u] + soff, w >> kRBits, lut, qt, a8[u], b8[u], pb[u]);
        acc[u] = accept_fixed<IS_INT>(dE[u], w & kRMask, cx, P.tab, ti);
        const bool kx = (w >> 31) != 0;
        if (u == 0 && lo_edge && !kx) pb[u] += (uint32_t)nx;
        if (u == NKW - 1 && hi_edge && kx) pb[u] -= (uint32_t)nx;
    }
#pragma unroll
    for (int u = 0; u < NKW; ++u) {
        if (acc[u]) {
            g_smem[ya[u] + A0 * (uint32_t)RB] = (unsigned char)b8[u];
            g_smem[pb[u]] = (unsigned char)a8[u];
            accE += dE[u];
            accN += 1u;
        }
    }
}

// Global row of slot `slot` of the pair at (sub, y0, z0, s_off).
__device__ __forceinline__ const int8_t *pair2_row(const RepDesc &RD, int slot, int sub, int y0, int z0, int soff)
{
    int s, y, z;
    if (slot < 12) {
        s = sub;
        y = y0 - 1 + (slot & 3);
        z = z0 - 1 + (slot >> 2);
    } else {
        const int k = slot - 12;
        const int sz = k < 3 ? 0 : (k < 8 ? 1 : (k < 13 ? 2 : 3));
        const int sy = k - (sz == 0 ? -1 : (sz == 1 ? 3 : (sz == 2 ? 8 : 12)));
        s = 1 - sub;
        y = y0 + soff - 1 + sy;
        z = z0 + soff - 1 + sz;
    }
    return RD.occ + ((size_t)((s * RD.nz + wrapc(z, RD.nz)) * RD.ny + wrapc(y, RD.ny))) * RD.nx;
}

// Stages the pair's 28 rows into the warp's buffer (bulk copies completing on
// the buffer's mbarrier).
__device__ __forceinline__ void pair2_stage(const RepDesc &RD, int sub, int y0, int z0, int soff, uint32_t dst,
                                            uint32_t rb, uint32_t mbar, int lane)
{
    const int8_t *src = lane < kPairRows ? pair2_row(RD, lane, sub, y0, z0, soff) : RD.occ;
    // order this warp's earlier accesses of the buffer, and the rows other
    // warps published (seen through the acquire loads), before the copies
    __syncwarp();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_expect_tx(mbar, (uint32_t)(kPairRows * RD.nx));
    __syncwarp();
    if (lane < kPairRows) bulk_g2s(dst + (uint32_t)lane * rb + 16u, src, (uint32_t)RD.nx, mbar);
}

// Pair item geometry: sweep t, pair index pp (0..15), tile (ty, tz).
struct Pair2Geo {
    int sub, soff, y0, z0;
    uint32_t gstep, need;  // the pair's first group; neighbours' progress needed
};
__device__ __forceinline__ Pair2Geo pair2_geo(int t, int pp, int ty, int tz)
{
    Pair2Geo q;
    const int g = 2 * pp;
    q.sub = g >> 4;
    q.soff = q.sub == 0 ? -1 : 0;
    q.y0 = 4 * ty + (g & 3);
    q.z0 = 4 * tz + ((g >> 2) & 3);
    q.gstep = (uint32_t)(t * 32 + g);
    q.need = q.gstep;  // the neighbours finished group gstep - 1 (their previous pair)
    return q;
}

// One warp per column-pair item, the tiles of one column each, gteam + k NT.
// Shared memory: [replicated table][LUT: 2 groups x 8 directions][per warp:
// mbarrier (16 bytes), 28 rows of RB bytes].
template <bool IS_INT, int NKW>
__global__ void __launch_bounds__(512, 1) k_sweep_pairs(const __grid_constant__ SweepParams P)
{
    constexpr int RB = 128 * NKW + 128;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int gteam = blockIdx.x * nwarp + warp, NT = gridDim.x * nwarp, NW = NT;
    const uint32_t rb = (uint32_t)RB;
    const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(g_smem);
    fill_rtab(P.qtab, P.qrow, tid, blockDim.x);
    const uint32_t qt = (uint32_t)(lane & 7) * 16u, lut = (uint32_t)kRTabBytes;
    if (tid < 16) {
        const int H = tid >> 3, kx = (tid >> 2) & 1, ky = (tid >> 1) & 1, kz = tid & 1;
        int2 e;
        e.x = pslot2(ky + 1 + H, kz + 1) * RB + kx;  // b: partner row (ky + 1 + H, kz + 1), x + s_off + kx
        e.y = (kz * 4 + H + ky) * RB + kx - 1;       // b's own 2 x 2 rows from (H + ky, kz), x + kx - 1
        *(int2 *)(g_smem + lut + (uint32_t)tid * 8u) = e;
    }
    const uint32_t wbase = lut + 256u + (uint32_t)warp * (uint32_t)P.warp_bytes;
    const uint32_t mbar = smem0 + wbase, buf = wbase + 16u;
    if (lane == 0) {
        mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const RepDesc &RD = P.rep[0];
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NTy = RD.NTy;
    const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
    bool aborted = false, inflight = false;
    uint32_t par = 0u;
    long long accE = 0, accN = 0;
    if (gteam < P.ntiles) {
        const int dty = NT % NTy, dtz = NT / NTy, ty0 = gteam % NTy, tz0 = gteam / NTy;
        int t = 0, pp = 0, tile = gteam, ty = ty0, tz = tz0;
        Pair2Geo q = pair2_geo(t, pp, ty, tz);
        bool ok = wait_tile_warp(P, RD, ty, tz, q.need, lane);
        if (ok) {
            pair2_stage(RD, q.sub, q.y0, q.z0, q.soff, smem0 + buf, rb, mbar, lane);
            inflight = true;
        }
        if (!__all_sync(0xffffffffu, ok)) aborted = true;
        while (!aborted) {
            // the next item
            int t2 = t, pp2 = pp, tile2 = tile + NT, ty2 = ty + dty, tz2 = tz + dtz;
            if (ty2 >= NTy) {
                ty2 -= NTy;
                ++tz2;
            }
            if (tile2 >= P.ntiles) {
                tile2 = gteam;
                ty2 = ty0;
                tz2 = tz0;
                if (++pp2 == 16) {
                    pp2 = 0;
                    ++t2;
                }
            }
            const bool has_next = t2 < P.nsweeps;
            const uint64_t sweep = P.sweep0 + (uint64_t)t;
            float cx = 0.f;
            int2 ti = make_int2(0, 0);
            if constexpr (IS_INT)
                ti = P.temp.tabinfo[P.beta_stride ? t : 0];
            else
                cx = P.temp.beta[P.beta_stride ? t : 0];
            const uint32_t body = buf + 16u;
            // Philox words of the pair's first group (while the rows land)
            uint32_t wr[NKW][4];
            auto philox_group = [&](int h) {
                const uint32_t rowsite = (uint32_t)(((q.sub * nz + q.z0) * ny + q.y0 + h) * nx);
#pragma unroll
                for (int k = 0; k < NKW; ++k) {
                    const U4 w = philox10(U4{(rowsite >> 2) + (uint32_t)(lane + 32 * k), RD.rep, (uint32_t)sweep,
                                             (uint32_t)(sweep >> 32)},
                                          k0, k1);
                    wr[k][0] = w.x;
                    wr[k][1] = w.y;
                    wr[k][2] = w.z;
                    wr[k][3] = w.w;
                }
            };
            philox_group(0);
            ok = mbar_wait(P, mbar, par);
            par ^= 1u;
            if (ok) inflight = false;
            if (!__all_sync(0xffffffffu, ok)) {
                aborted = true;
                break;
            }
            // periodic halos: 4 bytes before and after each row body
            if (lane < kPairRows) {
                const uint32_t bd = body + (uint32_t)lane * rb;
                *(unsigned *)(g_smem + bd - 4) = *(const unsigned *)(g_smem + bd + nx - 4);
                *(unsigned *)(g_smem + bd + nx) = *(const unsigned *)(g_smem + bd);
            }
            __syncwarp();
            // the two groups; after each mini-step the halos of the 5 rows it
            // may change (lane l < 10: row l / 2, side l % 2)
            uint32_t accN32 = 0;  // this pair's accepted trials (at most 8 NKW per lane)
            auto run_group = [&](auto Hc) {
                constexpr int H = decltype(Hc)::value;
                uint32_t hrow = 0;
                if (lane < 10) {
                    const int r5 = lane >> 1;
                    const int sl = r5 == 0 ? 5 + H : pslot2(1 + H + ((r5 - 1) & 1), 1 + ((r5 - 1) >> 1));
                    hrow = body + (uint32_t)sl * rb;
                }
#pragma unroll 1
                for (int dx = 0; dx < 4; ++dx) {
                    uint32_t wv[NKW];
#pragma unroll
                    for (int k = 0; k < NKW; ++k) {
                        wv[k] = wr[k][0];
                        wr[k][0] = wr[k][1];
                        wr[k][1] = wr[k][2];
                        wr[k][2] = wr[k][3];
                    }
                    pair2_trials<IS_INT, RB, NKW, H>(P, body, q.soff, nx, dx, lane, cx, ti, lut, qt, wv, accE, accN32);
                    __syncwarp();
                    if (lane < 10) {
                        if (lane & 1)
                            *(unsigned *)(g_smem + hrow + nx) = *(const unsigned *)(g_smem + hrow);
                        else
                            *(unsigned *)(g_smem + hrow - 4) = *(const unsigned *)(g_smem + hrow + nx - 4);
                    }
                    __syncwarp();
                }
            };
            run_group(std::integral_constant<int, 0>());
            philox_group(1);
            run_group(std::integral_constant<int, 1>());
            accN += accN32;
            // write back the rows the pair changed: own (0, 0) of both groups
            // (slots 5, 6) and partner slots 16-18 and 21-23
#pragma unroll 1
            for (int wrow = 0; wrow < 8; ++wrow) {
                const int slot = wrow < 2 ? 5 + wrow : (wrow < 5 ? 14 + wrow : 16 + wrow);
                int8_t *dstg = (int8_t *)pair2_row(RD, slot, q.sub, q.y0, q.z0, q.soff);
                const int4 *srcs = (const int4 *)(g_smem + body + (uint32_t)slot * rb);
                for (int cc = lane; cc < (nx >> 4); cc += 32) *((int4 *)dstg + cc) = srcs[cc];
            }
            // the rows' stores, then the release (the pair's second group)
            __syncwarp();
            if (lane == 0 && tile != P.skip_tile) st_release_u32(P.flags + tile, q.gstep + 2);
            if (!has_next) break;
            const Pair2Geo q2 = pair2_geo(t2, pp2, ty2, tz2);
            ok = wait_tile_warp(P, RD, ty2, tz2, q2.need, lane);
            if (ok) {
                pair2_stage(RD, q2.sub, q2.y0, q2.z0, q2.soff, smem0 + buf, rb, mbar, lane);
                inflight = true;
            }
            if (!__all_sync(0xffffffffu, ok)) {
                aborted = true;
                break;
            }
            t = t2;
            pp = pp2;
            tile = tile2;
            ty = ty2;
            tz = tz2;
            q = q2;
        }
    }
    if (aborted) {
        // let the copies in flight land before the CTA ends
        if (inflight) mbar_wait(P, mbar, par);
        return;
    }
    // per-warp sums (exact integers); the last warp reduces them
    const long long e_w = warp_sum<long long>(accE), n_w = warp_sum<long long>(accN);
    if (lane == 0 && gteam < P.ntiles) {
        ((long long *)P.part_e)[gteam] = e_w;
        P.part_n[gteam] = n_w;
    }
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicAdd(P.ticket, 1u) == (unsigned)NW - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    const int np = P.ntiles;
    long long se = 0, sn = 0;
    for (int k = lane; k < np; k += 32) {
        se += __ldcg((const long long *)P.part_e + k);
        sn += __ldcg(P.part_n + k);
    }
    se = warp_sum<long long>(se);
    sn = warp_sum<long long>(sn);
    if (lane == 0) {
        if (RD.e_acc) *RD.e_acc += (double)se * P.escale;
        if (RD.n_acc) *RD.n_acc += sn;
    }
}

// Species byte conversion around a fast-path launch: up (s -> 8 s, with a
// check that 0 <= s < S; a byte outside sets SMC_ERR_ARG in the status word
// and is taken mod 8) or down (8 s -> s).
__global__ void k_occ_scale(int8_t *occ, long long n, int up, int S, int *status)
{
    const long long nw = n >> 2;
    uint32_t *w4 = (uint32_t *)occ;
    const uint32_t lim = (uint32_t)(0x80 - S) * 0x01010101u;
    bool bad = false;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nw; i += (long long)gridDim.x * blockDim.x) {
        const uint32_t v = w4[i];
        if (up) {
            bad |= ((v | (v + lim)) & 0x80808080u) != 0u;
            w4[i] = (v & 0x07070707u) << 3;
        } else {
            w4[i] = (v >> 3) & 0x07070707u;
        }
    }
    for (long long i = (nw << 2) + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = occ[i];
        if (up) {
            bad |= v < 0 || v >= S;
            occ[i] = (int8_t)((v & 7) << 3);
        } else {
            occ[i] = (int8_t)((v >> 3) & 7);
        }
    }
    if (bad) atomicCAS(status, 0, (int)SMC_ERR_ARG);
}

// ---------------------------------------------------------------------------
// Lock-step trace of one mini-step: one thread per trial, reading rows
// straight from global memory through the same dE arithmetic.  Phase 1
// evaluates every trial (read-only), phase 2 applies the accepted swaps.
// ---------------------------------------------------------------------------
struct GView {
    const unsigned char *occ;
    int nx, ny, nz, sub, y0, z0;
    __device__ __forceinline__ const unsigned char *O(int dy, int dz) const
    {
        return occ + ((size_t)((sub * nz + wrapc(z0 + dz, nz)) * ny + wrapc(y0 + dy, ny))) * nx;
    }
    __device__ __forceinline__ const unsigned char *T(int dy, int dz) const
    {
        return occ + ((size_t)(((1 - sub) * nz + wrapc(z0 + dz, nz)) * ny + wrapc(y0 + dy, ny))) * nx;
    }
};

template <bool IS_INT, int NSH, int SW>
__global__ void k_ministep_eval(const __grid_constant__ SweepParams P, int k, float *dE_out, uint8_t *acc_out,
                                int *swap_a, int *swap_b)
{
    __shared__ __align__(16) uint32_t Qt[kPairQWords];
    for (int i = threadIdx.x; i < kQRows * P.qrow; i += blockDim.x) Qt[i] = P.qtab[i];
    __syncthreads();
    const RepDesc &RD = P.rep[0];
    const int ntr = RD.NLx * RD.NLy * RD.NLz;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ntr) return;
    const int dx = k % P.Lx, dy = (k / P.Lx) % P.Ly, dz = (k / (P.Lx * P.Ly)) % P.Lz;
    const int sub = k / (P.Lx * P.Ly * P.Lz);
    const int s_off = sub == 0 ? -1 : 0;
    const int cx_ = c % RD.NLx, cy = (c / RD.NLx) % RD.NLy, cz = c / (RD.NLx * RD.NLy);
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz;
    const int x = cx_ * P.Lx + dx, y0 = cy * P.Ly + dy, z0 = cz * P.Lz + dz;
    const GView gv{(const unsigned char *)RD.occ, nx, ny, nz, sub, y0, z0};
    const uint32_t s = (uint32_t)(((sub * nz + z0) * ny + y0) * nx + x);
    const uint32_t w = site_word(P.seed, RD.rep, P.sweep0, s);
    int A, B, ex, ey, ez;
    const int32_t dE =
        trial_dE_hist<NSH, SW, GView>(gv, x, nx, s_off, (int)(w >> kRBits), Qt, P.qrow, A, B, ex, ey, ez);
    float cxp = 0.f;
    int2 ti = make_int2(0, 0);
    if constexpr (IS_INT)
        ti = P.temp.tabinfo[0];
    else
        cxp = P.temp.beta[0];
    const bool acc = accept_fixed<IS_INT>(dE, w & kRMask, cxp, P.tab, ti);
    if (dE_out) dE_out[c] = (float)dE * (float)P.escale;
    if (acc_out) acc_out[c] = acc ? 1 : 0;
    const int by = wrapc(y0 + ey, ny), bz = wrapc(z0 + ez, nz), bx = wrapc(x + ex, nx);
    swap_a[c] = (acc && A != B) ? (int)s : -1;
    swap_b[c] = ((1 - sub) * nz + bz) * ny * nx + by * nx + bx;
}

__global__ void k_ministep_apply(int8_t *occ, int ntr, const int *swap_a, const int *swap_b)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ntr) return;
    const int a = swap_a[c];
    if (a < 0) return;
    const int b = swap_b[c];
    const int8_t t = occ[a];
    occ[a] = occ[b];
    occ[b] = t;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
bool build_pair_table(const smc_model *m, int S, PairTable &t)
{
    const bool is_int = m->kind == SMC_PAIR_I32;
    t.nsh = m->nshells >= 3 ? 3 : 2;
    t.sw = S <= 5 ? 1 : 2;
    t.rw = qrow_words(t.nsh, t.sw);
    const int R = S - 1, nf = 4 * t.sw;
    auto V = [&](int mm, int p, int q) -> double {
        return is_int ? (double)m->v_i32[(mm * S + p) * S + q] : (double)m->v_f32[(mm * S + p) * S + q];
    };
    if (is_int) {
        t.sigma = 0;
    } else {
        // |dE_fix| <= 2^sigma sum_m 2 (z_m - 1) max|D'_m| with |D'_m| <= 4 max|V_m|;
        // keep it below 2^30
        static const int z[3] = {8, 6, 12};
        double bound = 0.0;
        for (int mm = 0; mm < m->nshells; ++mm) {
            double M = 0.0;
            for (int p = 0; p < S; ++p)
                for (int q = 0; q < S; ++q) {
                    const double v = V(mm, p, q);
                    if (!std::isfinite(v)) return false;
                    M = std::max(M, std::fabs(v));
                }
            bound += 8.0 * (z[mm] - 1) * M;
        }
        t.sigma = bound > 0.0 ? (int)std::floor(std::log2(1073741824.0 / bound)) : 40;
        t.sigma = std::max(-60, std::min(t.sigma, 60));
    }
    t.scale = std::ldexp(1.0, -t.sigma);
    t.rows.assign((size_t)kQRows * t.rw, 0u);
    for (int A = 0; A < S; ++A)
        for (int B = 0; B < S; ++B) {
            uint32_t *row = &t.rows[(size_t)(A * 8 + B) * t.rw];
            uint32_t kb = 0u;
            for (int mm = 0; mm < t.nsh; ++mm) {
                int64_t Q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                if (mm < m->nshells && A != B)
                    for (int q = 0; q < R && q < nf; ++q) {
                        const double d = (V(mm, B, q) - V(mm, A, q)) - (V(mm, B, R) - V(mm, A, R));
                        Q[q] = is_int ? (int64_t)d : (int64_t)std::llrint(std::ldexp(d, t.sigma));
                    }
                const uint32_t bias = mm < 2 ? 8u : 16u;
                for (int q = 0; q < nf; ++q) kb -= bias * (uint32_t)Q[q];
                for (int w = 0; w < t.sw; ++w)
                    for (int k = 0; k < 4; ++k) {
                        uint32_t word = 0u;
                        for (int j = 0; j < 4; ++j) word |= (((uint32_t)Q[4 * w + j] >> (8 * k)) & 0xFFu) << (8 * j);
                        row[(mm * t.sw + w) * 4 + k] = word;
                    }
            }
            row[t.nsh * t.sw * 4] = kb;
        }
    return true;
}

// Exponent factor of the FP Metropolis test: -log2(e) 2^-sigma / kT.
static float accept_cx(double scale, double kT)
{
    return (float)(-1.4426950408889634 * scale / kT);
}

static void load_table(SweepParams &P, const PairTable &pt)
{
    P.qrow = pt.rw;
    P.escale = pt.scale;
    memcpy(P.qtab, pt.rows.data(), pt.rows.size() * 4);
}

// Warp count of a warp-per-tile kernel.  Warp w owns tiles w, w + NW, ...
// and CTA b lands on SM b mod num_sms (then b + num_sms, ...), so an SM's
// time is the sum of its warps' tile counts.  Among all CTA counts that fit
// at once, take the one with the smallest busiest-SM load (ties: more warps,
// which hide latency better): e.g. 16384 tiles on 152 SMs x 2 CTAs x 8 warps
// are best served by all 2432 warps (busiest SM 112 tiles), not by 2048
// (128 tiles, 48 SMs half idle).
long long balanced_warps(long long ntiles, int nwarps, int per_sm, int num_sms)
{
    // SM 0 is always the busiest: it holds the most CTAs, and its k-th CTA
    // (index k num_sms) has the lowest index, i.e. the most extra tiles,
    // among the SMs' k-th CTAs.
    const long long max_ctas = std::min<long long>((long long)per_sm * num_sms, (ntiles + nwarps - 1) / nwarps);
    long long best = nwarps, best_load = -1;
    for (long long ctas = 1; ctas <= max_ctas; ++ctas) {
        const long long nw = ctas * nwarps, q = ntiles / nw, rmd = ntiles % nw;
        long long worst = 0;
        for (long long b = 0; b < ctas; b += num_sms)
            worst += q * nwarps + std::max<long long>(0, std::min<long long>(rmd - b * nwarps, nwarps));
        if (best_load < 0 || worst <= best_load) {
            best_load = worst;
            best = nw;
        }
    }
    return best;
}

namespace {

struct Plan {
    int Lx, Ly, Lz, G;
    int threads, CB, TY, TZ, ntiles, grid, tpc, warp_bytes = 0, nap_cap = 128, rowB = 0, maxNLx = 1;
    int team = 1, team_bytes = 0, nbuf = 2;
    size_t smem;
    const void *kernel = nullptr;
};

int col_bytes_of(const smc_lattice &l)
{
    const int rowB = (l.nx + 15) & ~15;
    const int oy = l.ny >= 3 ? 3 : l.ny, oz = l.nz >= 3 ? 3 : l.nz;
    const int ty = l.ny >= 4 ? 4 : l.ny, tz = l.nz >= 4 ? 4 : l.nz;
    return (oy * oz + ty * tz) * rowB;
}

template <bool IS_INT>
const void *pick_slow(int nsh, int sw)
{
    if (nsh >= 3) return sw == 2 ? (const void *)k_sweep_pair<IS_INT, 3, 2> : (const void *)k_sweep_pair<IS_INT, 3, 1>;
    return sw == 2 ? (const void *)k_sweep_pair<IS_INT, 2, 2> : (const void *)k_sweep_pair<IS_INT, 2, 1>;
}

template <bool IS_INT>
smc_status make_plan(int R, const smc_lattice *lats, Workspace *ws, const PairTable &pt, Plan &pl)
{
    const Tuning tu = current_tuning();
    pl.Lx = lc_edge(lats[0].nx);
    pl.Ly = lc_edge(lats[0].ny);
    pl.Lz = lc_edge(lats[0].nz);
    pl.G = 2 * pl.Ly * pl.Lz;
    int maxNLx = 1, maxcol = 0;
    for (int r = 0; r < R; ++r) {
        maxNLx = std::max(maxNLx, lats[r].nx / pl.Lx);
        maxcol = std::max(maxcol, col_bytes_of(lats[r]));
    }
    pl.threads = tu.threads ? tu.threads : (maxNLx <= 128 ? 128 : 256);
    if (pl.threads % 32 || pl.threads < 32 || pl.threads > 512) {
        set_error("tuning.threads must be a multiple of 32 in [32, 512]");
        return SMC_ERR_ARG;
    }
    pl.CB = std::max(1, pl.threads / maxNLx);
    pl.TY = tu.tile_y;
    pl.TZ = tu.tile_z;
    if (pl.TY <= 0) pl.TY = pl.CB;
    if (pl.TZ <= 0) pl.TZ = std::max(1, pl.CB / pl.TY);
    pl.ntiles = 0;
    for (int r = 0; r < R; ++r) {
        const int NLy = lats[r].ny / pl.Ly, NLz = lats[r].nz / pl.Lz;
        pl.ntiles += ((NLy + pl.TY - 1) / pl.TY) * ((NLz + pl.TZ - 1) / pl.TZ);
    }
    pl.CB = std::min(pl.CB, pl.TY * pl.TZ);
    const int nwarps = pl.threads / 32;
    const size_t base = (size_t)kQRows * pt.rw * 4;
    auto smem_for = [&](int cb, int tpc) { return base + (size_t)tpc * nwarps * 16 + (size_t)cb * maxcol; };
    const void *kern = pick_slow<IS_INT>(pt.nsh, pt.sw);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    while (pl.CB > 1 && smem_for(pl.CB, 64) > dyn_max) pl.CB /= 2;
    if (smem_for(pl.CB, 1) > dyn_max) {
        set_error("lattice rows too long for shared memory (nx = %d)", lats[0].nx);
        return SMC_ERR_UNSUPPORTED;
    }
    size_t smem = smem_for(pl.CB, 64);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    // resident CTAs with the accumulator slots sized for the worst case
    int per_sm = 0;
    for (int tpc_guess = 1;; tpc_guess *= 2) {
        smem = smem_for(pl.CB, tpc_guess);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, pl.threads, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (per_sm < 1) {
            set_error("sweep kernel does not fit on an SM (threads %d, smem %zu)", pl.threads, smem);
            return SMC_ERR_UNSUPPORTED;
        }
        if (tu.ctas_per_sm > 0) per_sm = std::min(per_sm, tu.ctas_per_sm);
        pl.grid = std::min(pl.ntiles, per_sm * ws->num_sms);
        pl.tpc = (pl.ntiles + pl.grid - 1) / pl.grid;
        if (pl.tpc <= tpc_guess) break;
        if (smem_for(pl.CB, tpc_guess * 2) > dyn_max) {
            set_error("too many tiles per CTA for shared memory");
            return SMC_ERR_UNSUPPORTED;
        }
        if (tpc_guess > 4096) {
            set_error("too many tiles per CTA");
            return SMC_ERR_UNSUPPORTED;
        }
    }
    pl.smem = smem;
    pl.kernel = kern;
    return SMC_OK;
}

// Rows of 128, 256 or 512 cells of one lattice with a two-shell model of at
// most 4 + 1 species, one-column tiles: rows of nx + 128 bytes (a multiple of
// 128) and random words in registers (kernels with a compile-time row stride).
bool fast_wide(int R, const smc_lattice *lats, int nsh, int sw)
{
    const int nx = lats[0].nx;
    const Tuning tu = current_tuning();
    return R == 1 && nsh == 2 && sw == 1 && (nx == 128 || nx == 256 || nx == 512) && tu.tile_y <= 1 &&
           tu.tile_z <= 1;
}

template <bool IS_INT>
const void *pick_fast(int nsh, int sw)
{
    if (nsh >= 3)
        return sw == 2 ? (const void *)k_sweep_fast<IS_INT, 3, 2, 0> : (const void *)k_sweep_fast<IS_INT, 3, 1, 0>;
    return sw == 2 ? (const void *)k_sweep_fast<IS_INT, 2, 2, 0> : (const void *)k_sweep_fast<IS_INT, 2, 1, 0>;
}

// Plan of the warp-per-tile kernel: tiles of TY x TZ columns, one warp each
// (a warp owns ceil(ntiles / warps) tiles), shared memory = table + offsets
// + per warp (accumulator slots, barriers, Philox words, two row buffers).
template <bool IS_INT>
smc_status make_fast_plan_uncached(int R, const smc_lattice *lats, Workspace *ws, const PairTable &pt, int rowB,
                                   Plan &pl);

// The plan depends only on the shapes, the model's shell and species
// counts, the tuning and the device, so repeated calls (short chunks of a
// long run, one call per sample) reuse it instead of searching again.
template <bool IS_INT>
smc_status make_fast_plan(int R, const smc_lattice *lats, Workspace *ws, const PairTable &pt, int rowB, Plan &pl)
{
    static std::vector<long long> key_cached;
    static Plan plan_cached;
    const Tuning tu = current_tuning();
    std::vector<long long> key = {R,        pt.nsh,     pt.sw,      rowB,     lats[0].nspecies, ws->device,
                                  ws->num_sms, (long long)ws->smem_optin, tu.tile_y, tu.tile_z, tu.threads,
                                  tu.ctas_per_sm, debug_fast_team(), debug_fast_nbuf()};
    for (int r = 0; r < R; ++r) {
        key.push_back(lats[r].nx);
        key.push_back(lats[r].ny);
        key.push_back(lats[r].nz);
    }
    if (key == key_cached) {
        pl = plan_cached;
        return SMC_OK;
    }
    const smc_status st = make_fast_plan_uncached<IS_INT>(R, lats, ws, pt, rowB, pl);
    if (st == SMC_OK) {
        key_cached = key;
        plan_cached = pl;
    }
    return st;
}

template <bool IS_INT>
smc_status make_fast_plan_uncached(int R, const smc_lattice *lats, Workspace *ws, const PairTable &pt, int rowB,
                                   Plan &pl)
{
    const Tuning tu = current_tuning();
    pl.Lx = pl.Ly = pl.Lz = 4;
    pl.G = 32;
    pl.kernel = pick_fast<IS_INT>(pt.nsh, pt.sw);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, pl.kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(pl.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    int nkmax = 1, maxNLx = 1;
    for (int r = 0; r < R; ++r) {
        nkmax = std::max(nkmax, (lats[r].nx / 4 + 31) / 32);
        maxNLx = std::max(maxNLx, lats[r].nx / 4);
    }
    pl.maxNLx = maxNLx;
    // one column per tile unless tuned: the smallest unit of work keeps the
    // neighbour pipeline fullest
    pl.TY = tu.tile_y > 0 ? tu.tile_y : 1;
    pl.TZ = tu.tile_z > 0 ? tu.tile_z : 1;
    pl.ntiles = 0;
    for (int r = 0; r < R; ++r)
        pl.ntiles += ((lats[r].ny / 4 + pl.TY - 1) / pl.TY) * ((lats[r].nz / 4 + pl.TZ - 1) / pl.TZ);
    const size_t head = (size_t)kQRows * pt.rw * 4 + 128;
    const int nrows = pt.nsh >= 3 ? 25 : 21;
    // A team of tw warps shares a column (two row buffers per team); every
    // warp keeps its accumulator slots and Philox words.  Total warps: all
    // resident at once (cooperative launch), teams preferably a divisor of the
    // tile count so that every team owns as many tiles as the others (an
    // unevenly loaded team makes its neighbours wait).  The most resident
    // warps win (latency hiding); then the smaller team (fewer barriers);
    // then CTAs that spread evenly over the SMs.
    const int cand[4] = {64, 128, 192, 256};
    long long best_w = 0;
    int best_tw = 0, best_nb = 0;
    pl.threads = 0;
    bool best_even = false;
    // Measured on GB300 (512^3 and 128^3, two-shell quinary model): one warp
    // per column with one buffer runs fastest (16 resident warps hide the
    // staging latency better than 8 warps with two buffers each, and teams
    // pay a barrier per mini-step), so those are the defaults; the hooks can
    // still select the others.
    const int force_tw = debug_fast_team(), force_nb = debug_fast_nbuf();
    for (int nbuf = 2; nbuf >= 1; --nbuf) {
        if (force_nb ? nbuf != force_nb : nbuf != 1) continue;
        for (int tw = 1; tw <= 4; tw *= 2) {
            if (force_tw ? tw != force_tw : tw != 1) continue;
            const int nkw = (maxNLx + 32 * tw - 1) / (32 * tw);
            const size_t team_bytes = 16 + (size_t)nbuf * nrows * rowB;
            for (int ci = 0; ci < 4; ++ci) {
                const int threads = tu.threads ? std::min(tu.threads, 256) : cand[ci];  // launch bound is 256
                if (tu.threads && ci > 0) break;
                const int nwarps = threads / 32;
                if (nwarps % tw) continue;
                const int tpb = nwarps / tw;
                for (int tpc_guess = 1;; tpc_guess *= 2) {
                    const size_t wb = ((size_t)16 * tpc_guess + (size_t)512 * nkw + 15) / 16 * 16;
                    const size_t smem = head + (size_t)tpb * team_bytes + (size_t)nwarps * wb;
                    if (smem > dyn_max) break;
                    int per_sm = 0;
                    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.kernel, threads, smem);
                    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
                    if (tu.ctas_per_sm > 0) per_sm = std::min(per_sm, tu.ctas_per_sm);
                    if (per_sm < 1) break;
                    const long long nt = balanced_warps(pl.ntiles, tpb, per_sm, ws->num_sms);  // teams
                    const int tpc = (int)((pl.ntiles + nt - 1) / nt);
                    if (tpc <= tpc_guess) {
                        const long long grid = nt / tpb, nw = nt * tw;
                        const bool even = grid <= ws->num_sms || grid % ws->num_sms == 0;
                        // the most resident warps; then the smaller team (fewer
                        // barriers); then two buffers; then even CTAs; then
                        // larger CTAs (at 128^3 and 512^3 CTAs of 8 warps ran
                        // 5-20 % faster than smaller ones with as many warps)
                        const bool same = nw == best_w && tw == best_tw && nbuf == best_nb;
                        const bool better = nw > best_w || (nw == best_w && tw < best_tw) ||
                                            (nw == best_w && tw == best_tw && nbuf > best_nb) ||
                                            (same && even && !best_even) ||
                                            (same && even == best_even && threads > pl.threads);
                        if (better) {
                            best_w = nw;
                            best_tw = tw;
                            best_nb = nbuf;
                            best_even = even;
                            pl.threads = threads;
                            pl.grid = (int)grid;
                            pl.tpc = tpc_guess;
                            pl.smem = smem;
                            pl.warp_bytes = (int)wb;
                            pl.team = tw;
                            pl.team_bytes = (int)team_bytes;
                            pl.nbuf = nbuf;
                            pl.rowB = rowB;
                        }
                        break;
                    }
                }
            }
        }
    }
    if (best_w == 0) {
        set_error("fast sweep kernel does not fit on an SM (rows of %d bytes)", rowB);
        return SMC_ERR_UNSUPPORTED;
    }
    // sleep between progress polls: short for small columns (latency-bound),
    // longer for long ones (a tile-group takes tens of microseconds)
    pl.nap_cap = maxNLx >= 64 ? 1024 : 32;
    pl.CB = 1;
    return SMC_OK;
}

// Plan of the paired-group kernel (fast_wide lattices): one CTA per SM with
// as many warps as shared memory and registers allow (at most 16), CTAs
// spread so that the busiest SM has the fewest tiles.
template <bool IS_INT>
smc_status make_pairs_plan(const smc_lattice &lat, Workspace *ws, Plan &pl)
{
    static long long key_cached[5] = {-1, -1, -1, -1, -1};
    static Plan plan_cached;
    const long long key[5] = {lat.nx, lat.ny, lat.nz, ws->device, (long long)ws->smem_optin};
    if (std::equal(key, key + 5, key_cached)) {
        pl = plan_cached;
        return SMC_OK;
    }
    const int nkw = lat.nx / 128;
    pl.kernel = nkw == 1 ? (const void *)k_sweep_pairs<IS_INT, 1>
                         : (nkw == 2 ? (const void *)k_sweep_pairs<IS_INT, 2> : (const void *)k_sweep_pairs<IS_INT, 4>);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, pl.kernel);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const size_t dyn_max = ws->smem_optin - fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(pl.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    pl.Lx = pl.Ly = pl.Lz = 4;
    pl.G = 32;
    pl.TY = pl.TZ = 1;
    pl.CB = 1;
    pl.ntiles = (lat.ny / 4) * (lat.nz / 4);
    pl.maxNLx = lat.nx / 4;
    pl.rowB = lat.nx + 128;
    pl.team = 1;
    pl.nbuf = 1;
    pl.team_bytes = 0;
    pl.tpc = 1;
    pl.nap_cap = 1024;
    pl.warp_bytes = 16 + kPairRows * pl.rowB;
    const size_t head = (size_t)kRTabBytes + 256;
    int wpc = 0;
    for (int w = 16; w >= 1 && !wpc; --w) {
        const size_t smem = head + (size_t)w * pl.warp_bytes;
        if (smem > dyn_max) continue;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.kernel, 32 * w, smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (per_sm >= 1) wpc = w;
    }
    if (!wpc) {
        set_error("paired sweep kernel does not fit on an SM (rows of %d bytes)", pl.rowB);
        return SMC_ERR_UNSUPPORTED;
    }
    pl.threads = 32 * wpc;
    pl.smem = head + (size_t)wpc * pl.warp_bytes;
    pl.grid = (int)(balanced_warps(pl.ntiles, wpc, 1, ws->num_sms) / wpc);
    std::copy(key, key + 5, key_cached);
    plan_cached = pl;
    return SMC_OK;
}

// Fast path: 4-cell link cells on every axis, rows of at most 1024 cells,
// 4-byte aligned occupancy.
bool fast_ok(int R, const smc_lattice *lats, int8_t *const *occ, int &rowB)
{
    bool fast = true;
    rowB = 0;
    for (int r = 0; r < R; ++r) {
        const smc_lattice &l = lats[r];
        fast = fast && lc_edge(l.nx) == 4 && lc_edge(l.ny) == 4 && lc_edge(l.nz) == 4 && l.nx <= 1024 &&
               ((uintptr_t)occ[r] % 4 == 0);
        rowB = std::max(rowB, ((l.nx + 15) & ~15) + 32);  // body at +16, 4-byte halos, 16-byte rows
    }
    const Tuning tu = current_tuning();
    if (tu.threads && tu.threads % 32) fast = false;
    return fast;
}

// Shared parameter-block setup of the sweep launches (tiles, replicas,
// table, schedule lags).
void fill_params(SweepParams &P, const Plan &pl, bool fast, int R, const smc_lattice *lats, int8_t *const *occ,
                 uint32_t replica0, double *e_acc, int64_t *n_acc, const smc_model *m, const PairTable &pt,
                 uint64_t seed)
{
    memset(&P, 0, sizeof P);
    P.R = R;
    P.G = pl.G;
    P.Lx = pl.Lx;
    P.Ly = pl.Ly;
    P.Lz = pl.Lz;
    P.TY = pl.TY;
    P.TZ = pl.TZ;
    P.CB = std::min(pl.CB, pl.TY * pl.TZ);
    P.nshells = m->nshells;
    P.S = lats[0].nspecies;
    P.tpc = pl.tpc;
    P.warp_bytes = pl.warp_bytes;
    P.nap_cap = pl.nap_cap;
    P.rowB = pl.rowB;
    P.maxNLx = pl.maxNLx;
    P.team = pl.team;
    P.team_bytes = pl.team_bytes;
    P.nbuf = pl.nbuf;
    // bulk copies for long rows (512^3: 3.36 against 3.56 ms per sweep),
    // 16-byte cp.async for short ones (128^3: 0.218 against 0.249 ms)
    P.stage = debug_fast_stage() == 1 ? 0 : (debug_fast_stage() == 2 ? 1 : (pl.maxNLx >= 64 ? 0 : 1));
    for (int g = 0; g < kMaxGroups; ++g) P.lag[g] = 1;
    if (fast) {
        // Groups with dy >= 1 conflict with neighbouring columns only two
        // groups back (pair models with up to three shells), so they may
        // start once the neighbours have finished the group before last.
        for (int g = 0; g < pl.G; ++g) P.lag[g] = (g % pl.Ly) == 0 ? 1 : 2;
    }
    P.skip_tile = (int)debug_skip_tile();
    P.seed = seed;
    P.timeout_ns = debug_timeout_ns();
    int tile0 = 0;
    for (int r = 0; r < R; ++r) {
        RepDesc &d = P.rep[r];
        d.occ = occ[r];
        d.e_acc = e_acc ? e_acc + r : nullptr;
        d.n_acc = n_acc ? (long long *)n_acc + r : nullptr;
        d.nx = lats[r].nx;
        d.ny = lats[r].ny;
        d.nz = lats[r].nz;
        d.NLx = d.nx / pl.Lx;
        d.NLy = d.ny / pl.Ly;
        d.NLz = d.nz / pl.Lz;
        d.NTy = (d.NLy + pl.TY - 1) / pl.TY;  // a tile wider than the grid is clipped
        d.NTz = (d.NLz + pl.TZ - 1) / pl.TZ;
        d.tile0 = tile0;
        d.rep = replica0 + (uint32_t)r;
        d.vec = (d.nx % 16 == 0) && ((uintptr_t)occ[r] % 16 == 0);
        tile0 += d.NTy * d.NTz;
    }
    P.ntiles = tile0;
    load_table(P, pt);
}

// Species byte conversion around fast-path launches.
smc_status scale_occ(int R, const smc_lattice *lats, int8_t *const *occ, bool up, int *status, int num_sms,
                     cudaStream_t stream)
{
    for (int r = 0; r < R; ++r) {
        const long long n = 2LL * lats[r].nx * lats[r].ny * lats[r].nz;
        const long long nw = (n + 3) / 4;
        const int grid = (int)std::max<long long>(1, std::min<long long>((nw + 255) / 256, (long long)num_sms * 8));
        k_occ_scale<<<grid, 256, 0, stream>>>(occ[r], n, up ? 1 : 0, lats[r].nspecies, status);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "k_occ_scale");
    }
    return SMC_OK;
}

}  // namespace

// Integer acceptance table T[d] = floor(2^29 exp(-d unit / kT)) for d = 0 ..
// len-1 (T[len] = 0), in FP64 on the host.
std::vector<uint32_t> int_table(double unit_ev, double kT)
{
    std::vector<uint32_t> t;
    for (int64_t d = 0;; ++d) {
        const double v = floor(536870912.0 * exp(-(double)d * unit_ev / kT));
        if (v <= 0.0 || d > (1 << 24)) break;
        t.push_back((uint32_t)v);
    }
    return t;
}

template <bool IS_INT>
static smc_status sweep_impl(int R, const smc_lattice *lats, const smc_model *m, int8_t *const *occ, uint64_t seed,
                             uint32_t replica0, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                             int64_t *n_acc, cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    PairTable pt;
    if (!build_pair_table(m, lats[0].nspecies, pt)) {
        set_error("pair coefficients must be finite");
        return SMC_ERR_ARG;
    }
    if (debug_resident() == 0) {
        // lattices that fit in the SMs' shared memory stay there
        st = launch_pair_sweep_resident(R, lats, m, pt, occ, seed, replica0, sweep0, nsweeps, kT, e_acc, n_acc,
                                        stream);
        if (st != SMC_ERR_UNSUPPORTED) return st;
    }
    int rowB = 0;
    const bool fast = fast_ok(R, lats, occ, rowB);
    // (paired kernel: bulk row copies, so 16-byte aligned rows)
    const bool wide = fast && fast_wide(R, lats, pt.nsh, pt.sw) && (uintptr_t)occ[0] % 16 == 0;
    Plan pl;
    if (wide)
        st = make_pairs_plan<IS_INT>(lats[0], ws, pl);
    else
        st = fast ? make_fast_plan<IS_INT>(R, lats, ws, pt, rowB, pl) : make_plan<IS_INT>(R, lats, ws, pt, pl);
    if (st != SMC_OK) return st;
    if (!fast) pl.rowB = rowB;

    static SweepParams P;  // large: keep off the stack (host-only, guarded by the API lock)
    fill_params(P, pl, fast, R, lats, occ, replica0, e_acc, n_acc, m, pt, seed);

    // temperature schedule: constant per replica over the call, or per sweep
    bool constant = true;
    for (int r = 0; r < R && constant; ++r)
        for (int t = 1; t < nsweeps; ++t)
            if (kT[(size_t)r * nsweeps + t] != kT[(size_t)r * nsweeps]) {
                constant = false;
                break;
            }
    const int cap = IS_INT ? kMaxBeta / 2 : kMaxBeta;
    const int chunk = constant ? nsweeps : std::max(1, cap / R);
    if (!constant && R > cap) {
        set_error("per-sweep temperatures for more than %d replicas", cap);
        return SMC_ERR_UNSUPPORTED;
    }

    // integer path: one acceptance table per distinct kT
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
    if (IS_INT) {
        for (int r = 0; r < R; ++r)
            for (int t = 0; t < nsweeps; ++t) table_of(kT[(size_t)r * nsweeps + t]);
    }

    // workspace: [flags | part_e | part_n | ticket, abort | tables]; the fast
    // kernel keeps one partial sum per tile and warp of its team
    const size_t nt = (size_t)P.ntiles, np = nt * (size_t)std::max(1, P.team);
    const size_t off_flags = 0, off_pe = ((nt * 4 + 15) / 16) * 16, off_pn = off_pe + np * 8;
    const size_t off_misc = off_pn + np * 8, off_tab = off_misc + 16;
    const size_t need = off_tab + tabs.size() * 4;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, need, &st);
    if (!scr) return st;
    P.flags = (uint32_t *)(scr + off_flags);
    P.part_e = (double *)(scr + off_pe);
    P.part_n = (long long *)(scr + off_pn);
    P.ticket = (unsigned *)(scr + off_misc);
    P.abort_flag = (int *)(scr + off_misc + 4);
    P.status = ws->status;
    P.tab = (const uint32_t *)(scr + off_tab);
    cudaError_t e;
    if (!tabs.empty()) {
        e = cudaMemcpyAsync(scr + off_tab, tabs.data(), tabs.size() * 4, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(acceptance tables)");
    }
    if (fast) {
        st = scale_occ(R, lats, occ, true, P.status, ws->num_sms, stream);
        if (st != SMC_OK) return st;
    }
    smc_status run = SMC_OK;
    for (int t0 = 0; t0 < nsweeps && run == SMC_OK; t0 += chunk) {
        const int nc = std::min(chunk, nsweeps - t0);
        P.sweep0 = sweep0 + (uint64_t)t0;
        P.nsweeps = nc;
        P.beta_stride = constant ? 0 : nc;
        for (int r = 0; r < R; ++r)
            for (int t = 0; t < (constant ? 1 : nc); ++t) {
                const double kt = kT[(size_t)r * nsweeps + t0 + t];
                const int idx = constant ? r : r * nc + t;
                if (IS_INT)
                    P.temp.tabinfo[idx] = table_of(kt);
                else
                    P.temp.beta[idx] = accept_cx(pt.scale, kt);
            }
        e = cudaMemsetAsync(scr, 0, off_tab, stream);
        if (e != cudaSuccess) {
            run = cuda_fail(e, "cudaMemsetAsync(sweep scratch)");
            break;
        }
        void *args[] = {(void *)&P};
        e = cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream);
        if (e != cudaSuccess) run = cuda_fail(e, "cudaLaunchCooperativeKernel(sweep)");
    }
    if (fast) {
        // the species go back to plain indices even when a launch failed
        st = scale_occ(R, lats, occ, false, P.status, ws->num_sms, stream);
        if (run == SMC_OK && st != SMC_OK) run = st;
    }
    return run;
}

smc_status launch_pair_sweep(int R, const smc_lattice *lats, const smc_model *m, int8_t *const *occ, uint64_t seed,
                             uint32_t replica0, uint64_t sweep0, int nsweeps, const double *kT, double *e_acc,
                             int64_t *n_acc, cudaStream_t stream)
{
    for (int r = 1; r < R; ++r) {
        if (lc_edge(lats[r].nx) != lc_edge(lats[0].nx) || lc_edge(lats[r].ny) != lc_edge(lats[0].ny) ||
            lc_edge(lats[r].nz) != lc_edge(lats[0].nz) || lats[r].nspecies != lats[0].nspecies) {
            set_error("batched replicas must share link-cell edges and species count (replica %d)", r);
            return SMC_ERR_UNSUPPORTED;
        }
    }
    if (m->kind == SMC_PAIR_I32)
        return sweep_impl<true>(R, lats, m, occ, seed, replica0, sweep0, nsweeps, kT, e_acc, n_acc, stream);
    return sweep_impl<false>(R, lats, m, occ, seed, replica0, sweep0, nsweeps, kT, e_acc, n_acc, stream);
}

// ---------------------------------------------------------------------------
// One mini-step on one x-slab (Sec. III-B, 1D slab decomposition).  The
// window holds cells [x0 - g, x0 + w + g) of every row, laid out as the box
// with x restricted to it: [sub][z][y][w + 2 g].  The trials of the slab's
// link cells run as in the whole box, each with the random word of its
// global site id, and apply their swaps in place (the trials of a mini-step
// touch disjoint cells).  part 1 runs the first and last link cell of every
// x-row of the slab -- the trials that change cells within g <= 3 of the
// slab's edges, the cells the ghost exchange sends -- part 2 the others,
// whose reads and writes stay inside the slab, and part 0 all of them.
// ---------------------------------------------------------------------------
struct SlabView {
    unsigned char *occ;
    int W, ny, nz, sub, y0, z0;
    __device__ __forceinline__ unsigned char *O(int dy, int dz) const
    {
        return occ + ((size_t)((sub * nz + wrapc(z0 + dz, nz)) * ny + wrapc(y0 + dy, ny))) * W;
    }
    __device__ __forceinline__ unsigned char *T(int dy, int dz) const
    {
        return occ + ((size_t)(((1 - sub) * nz + wrapc(z0 + dz, nz)) * ny + wrapc(y0 + dy, ny))) * W;
    }
};

template <bool IS_INT, int NSH, int SW>
__global__ void __launch_bounds__(128) k_slab_ministep(const __grid_constant__ SweepParams P, int k, int x0, int w,
                                                       int g, int part, long long *sums)
{
    __shared__ __align__(16) uint32_t Qt[kPairQWords];
    __shared__ long long s_e[4], s_n[4];
    for (int i = threadIdx.x; i < kQRows * P.qrow; i += blockDim.x) Qt[i] = P.qtab[i];
    __syncthreads();
    const RepDesc &RD = P.rep[0];
    const int ncx = w / 4;
    const int ncp = part == 0 ? ncx : (part == 1 ? min(ncx, 2) : max(ncx - 2, 0));
    const int ntr = ncp * RD.NLy * RD.NLz;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    long long e = 0, n = 0;
    if (c < ntr) {
        const int ci = c % ncp, cy = (c / ncp) % RD.NLy, cz = c / (ncp * RD.NLy);
        const int cx = part == 2 ? 1 + ci : (part == 1 && ci == 1 ? ncx - 1 : ci);
        const int dx = k % 4, dy = (k / 4) % P.Ly, dz = (k / (4 * P.Ly)) % P.Lz;
        const int sub = k / (4 * P.Ly * P.Lz);
        const int s_off = sub == 0 ? -1 : 0;
        const int nx = RD.nx, ny = RD.ny, nz = RD.nz, W = w + 2 * g;
        const int xg = x0 + 4 * cx + dx, xl = xg - x0 + g;
        const int y0 = cy * P.Ly + dy, z0 = cz * P.Lz + dz;
        const SlabView sv{(unsigned char *)RD.occ, W, ny, nz, sub, y0, z0};
        const uint32_t site = (uint32_t)(((sub * nz + z0) * ny + y0) * nx + xg);
        const uint32_t wd = site_word(P.seed, RD.rep, P.sweep0, site);
        int A, B, ex, ey, ez;
        const int32_t dE =
            trial_dE_hist<NSH, SW, SlabView>(sv, xl, W, s_off, (int)(wd >> kRBits), Qt, P.qrow, A, B, ex, ey, ez);
        float cxp = 0.f;
        int2 ti = make_int2(0, 0);
        if constexpr (IS_INT)
            ti = P.temp.tabinfo[0];
        else
            cxp = P.temp.beta[0];
        if (accept_fixed<IS_INT>(dE, wd & kRMask, cxp, P.tab, ti)) {
            if (A != B) {
                sv.O(0, 0)[xl] = (unsigned char)B;
                sv.T(ey, ez)[xl + ex] = (unsigned char)A;
            }
            e = dE;
            n = 1;
        }
    }
    e = warp_sum<long long>(e);
    n = warp_sum<long long>(n);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) {
        s_e[wp] = e;
        s_n[wp] = n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long te = 0, tn = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            te += s_e[i];
            tn += s_n[i];
        }
        if (te) atomicAdd((unsigned long long *)sums, (unsigned long long)te);
        if (tn) atomicAdd((unsigned long long *)sums + 1, (unsigned long long)tn);
    }
}

// e_acc += sum dE_fix * escale; n_acc += count (one thread).
__global__ void k_slab_finish(const long long *sums, double escale, double *e_acc, int64_t *n_acc)
{
    if (e_acc) *e_acc += (double)sums[0] * escale;
    if (n_acc) *n_acc += sums[1];
}

template <bool IS_INT>
static smc_status slab_impl(const smc_lattice *lat, const smc_model *m, int8_t *win, int x0, int w, int g,
                            uint64_t seed, uint32_t replica, uint64_t sweep, int k, double kT, double *e_acc,
                            int64_t *n_acc, int part, cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    PairTable pt;
    if (!build_pair_table(m, lat->nspecies, pt)) {
        set_error("pair coefficients must be finite");
        return SMC_ERR_ARG;
    }
    static SweepParams P;
    memset(&P, 0, sizeof P);
    P.R = 1;
    P.Lx = 4;
    P.Ly = lc_edge(lat->ny);
    P.Lz = lc_edge(lat->nz);
    P.nshells = m->nshells;
    P.S = lat->nspecies;
    P.seed = seed;
    P.sweep0 = sweep;
    RepDesc &d = P.rep[0];
    d.occ = win;
    d.nx = lat->nx;
    d.ny = lat->ny;
    d.nz = lat->nz;
    d.NLx = d.nx / 4;
    d.NLy = d.ny / P.Ly;
    d.NLz = d.nz / P.Lz;
    d.rep = replica;
    load_table(P, pt);
    std::vector<uint32_t> tab;
    if (IS_INT) {
        tab = int_table(m->unit_ev, kT);
        P.temp.tabinfo[0] = make_int2(0, (int)tab.size());
    } else {
        P.temp.beta[0] = accept_cx(pt.scale, kT);
    }
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, 16 + tab.size() * 4 + 16, &st);
    if (!scr) return st;
    long long *sums = (long long *)scr;
    P.tab = (const uint32_t *)(scr + 16);
    cudaError_t e = cudaMemsetAsync(sums, 0, 16, stream);
    if (e == cudaSuccess && !tab.empty())
        e = cudaMemcpyAsync(scr + 16, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "slab mini-step setup");
    const int ncx = w / 4;
    const int ncp = part == 0 ? ncx : (part == 1 ? std::min(ncx, 2) : std::max(ncx - 2, 0));
    const int ntr = ncp * d.NLy * d.NLz;
    const int threads = 128, blocks = std::max(1, (ntr + threads - 1) / threads);
    if (pt.nsh >= 3) {
        if (pt.sw == 2)
            k_slab_ministep<IS_INT, 3, 2><<<blocks, threads, 0, stream>>>(P, k, x0, w, g, part, sums);
        else
            k_slab_ministep<IS_INT, 3, 1><<<blocks, threads, 0, stream>>>(P, k, x0, w, g, part, sums);
    } else {
        if (pt.sw == 2)
            k_slab_ministep<IS_INT, 2, 2><<<blocks, threads, 0, stream>>>(P, k, x0, w, g, part, sums);
        else
            k_slab_ministep<IS_INT, 2, 1><<<blocks, threads, 0, stream>>>(P, k, x0, w, g, part, sums);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_slab_ministep");
    k_slab_finish<<<1, 1, 0, stream>>>(sums, pt.scale, e_acc, n_acc);
    e = cudaGetLastError();
    return e == cudaSuccess ? SMC_OK : cuda_fail(e, "k_slab_finish");
}

smc_status launch_slab_ministep(const smc_lattice *lat, const smc_model *m, int8_t *win, int x0, int w, int g,
                                uint64_t seed, uint32_t replica, uint64_t sweep, int k, double kT, double *e_acc,
                                int64_t *n_acc, int part, cudaStream_t stream)
{
    if (m->kind == SMC_PAIR_I32)
        return slab_impl<true>(lat, m, win, x0, w, g, seed, replica, sweep, k, kT, e_acc, n_acc, part, stream);
    return slab_impl<false>(lat, m, win, x0, w, g, seed, replica, sweep, k, kT, e_acc, n_acc, part, stream);
}

template <bool IS_INT>
static smc_status trace_impl(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                             uint32_t replica, uint64_t sweep, int k, double kT, float *dE, uint8_t *acc,
                             cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    PairTable pt;
    if (!build_pair_table(m, lat->nspecies, pt)) {
        set_error("pair coefficients must be finite");
        return SMC_ERR_ARG;
    }
    static SweepParams P;
    memset(&P, 0, sizeof P);
    P.R = 1;
    P.Lx = lc_edge(lat->nx);
    P.Ly = lc_edge(lat->ny);
    P.Lz = lc_edge(lat->nz);
    P.nshells = m->nshells;
    P.S = lat->nspecies;
    P.seed = seed;
    P.sweep0 = sweep;
    RepDesc &d = P.rep[0];
    d.occ = occ;
    d.nx = lat->nx;
    d.ny = lat->ny;
    d.nz = lat->nz;
    d.NLx = d.nx / P.Lx;
    d.NLy = d.ny / P.Ly;
    d.NLz = d.nz / P.Lz;
    d.rep = replica;
    load_table(P, pt);
    const int ntr = d.NLx * d.NLy * d.NLz;
    std::vector<uint32_t> tab;
    if (IS_INT) {
        tab = int_table(m->unit_ev, kT);
        P.temp.tabinfo[0] = make_int2(0, (int)tab.size());
    } else {
        P.temp.beta[0] = accept_cx(pt.scale, kT);
    }
    const size_t off_tab = ((size_t)ntr * 8 + 15) / 16 * 16;
    unsigned char *scr = (unsigned char *)workspace_scratch(ws, off_tab + tab.size() * 4 + 16, &st);
    if (!scr) return st;
    int *swap_a = (int *)scr, *swap_b = swap_a + ntr;
    P.tab = (const uint32_t *)(scr + off_tab);
    cudaError_t e;
    if (!tab.empty()) {
        e = cudaMemcpyAsync(scr + off_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(acceptance table)");
    }
    const int threads = 128, blocks = (ntr + threads - 1) / threads;
    if (pt.nsh >= 3) {
        if (pt.sw == 2)
            k_ministep_eval<IS_INT, 3, 2><<<blocks, threads, 0, stream>>>(P, k, dE, acc, swap_a, swap_b);
        else
            k_ministep_eval<IS_INT, 3, 1><<<blocks, threads, 0, stream>>>(P, k, dE, acc, swap_a, swap_b);
    } else {
        if (pt.sw == 2)
            k_ministep_eval<IS_INT, 2, 2><<<blocks, threads, 0, stream>>>(P, k, dE, acc, swap_a, swap_b);
        else
            k_ministep_eval<IS_INT, 2, 1><<<blocks, threads, 0, stream>>>(P, k, dE, acc, swap_a, swap_b);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_ministep_eval");
    k_ministep_apply<<<blocks, threads, 0, stream>>>(occ, ntr, swap_a, swap_b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_ministep_apply");
    return SMC_OK;
}

smc_status launch_ministep_trace(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                                 uint32_t replica, uint64_t sweep, int k, double kT, float *dE, uint8_t *acc,
                                 cudaStream_t stream)
{
    if (m->kind == SMC_PAIR_I32)
        return trace_impl<true>(lat, m, occ, seed, replica, sweep, k, kT, dE, acc, stream);
    return trace_impl<false>(lat, m, occ, seed, replica, sweep, k, kT, dE, acc, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free sweep (smc_sweep_noalloc).  Some callers cannot call
// cudaMalloc -- code that runs while a CUDA graph is being captured, or hosts
// whose memory is owned by their own pool and must not see the library
// allocate behind its back -- so this entry point keeps its scratch (progress
// flags, per-tile partial sums, ticket and abort words) in the file-scope
// array below instead of the library workspace, and reports device-side
// failures in the caller's status word.  Every GPU that loads the library
// holds the array until the process exits.  Host code must not use the
// array's name as a device address: the address is looked up with
// cudaGetSymbolAddress on every call, with the caller's device current (the
// lookup allocates nothing once the module is loaded, and stays valid after
// the context is re-created).
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxTiles = 16384;
constexpr size_t kNoAllocFlagsOff = 256;
constexpr size_t kNoAllocPartEOff = kNoAllocFlagsOff + (size_t)kNoAllocMaxTiles * 4;
constexpr size_t kNoAllocPartNOff = kNoAllocPartEOff + (size_t)kNoAllocMaxTiles * 8;
constexpr size_t kNoAllocBytes = kNoAllocPartNOff + (size_t)kNoAllocMaxTiles * 8;  // 320 KB + 256 B

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

smc_status launch_pair_sweep_noalloc(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                                     uint32_t replica, uint64_t sweep0, int nsweeps, const double *kT,
                                     double *e_acc, int64_t *n_acc, int32_t *status, cudaStream_t stream)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    void *sym = nullptr;
    e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    unsigned char *scr = (unsigned char *)sym;
    // Device attributes the plans need, queried directly (no workspace).
    Workspace ws;
    int sms = 0, optin = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    ws.device = dev;
    ws.num_sms = sms;
    ws.smem_optin = (size_t)optin;

    PairTable pt;
    if (!build_pair_table(m, lat->nspecies, pt)) {
        set_error("pair coefficients must be finite");
        return SMC_ERR_ARG;
    }
    int8_t *occs[1] = {occ};
    int rowB = 0;
    const bool fast = fast_ok(1, lat, occs, rowB);
    Plan pl;
    smc_status st = fast ? make_fast_plan<false>(1, lat, &ws, pt, rowB, pl) : make_plan<false>(1, lat, &ws, pt, pl);
    if (st != SMC_OK) return st;
    if (!fast) pl.rowB = rowB;
    if ((long long)pl.ntiles * std::max(1, pl.team) > kNoAllocMaxTiles) {
        set_error("smc_sweep_noalloc: %d link-cell tiles exceed the scratch limit of %d (use a larger tile_y/tile_z "
                  "tuning or smc_sweep)", pl.ntiles, kNoAllocMaxTiles);
        return SMC_ERR_UNSUPPORTED;
    }

    static SweepParams P;
    fill_params(P, pl, fast, 1, lat, occs, replica, e_acc, n_acc, m, pt, seed);
    bool constant = true;
    for (int t = 1; t < nsweeps; ++t)
        if (kT[t] != kT[0]) constant = false;
    const int chunk = constant ? nsweeps : kMaxBeta;
    P.flags = (uint32_t *)(scr + kNoAllocFlagsOff);
    P.part_e = (double *)(scr + kNoAllocPartEOff);
    P.part_n = (long long *)(scr + kNoAllocPartNOff);
    P.ticket = (unsigned *)(scr + 0);
    P.abort_flag = (int *)(scr + 4);
    P.status = (int *)status;
    P.tab = nullptr;
    e = cudaMemsetAsync(status, 0, sizeof(int32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    if (fast) {
        st = scale_occ(1, lat, occs, true, P.status, sms, stream);
        if (st != SMC_OK) return st;
    }
    smc_status run = SMC_OK;
    for (int t0 = 0; t0 < nsweeps && run == SMC_OK; t0 += chunk) {
        const int nc = std::min(chunk, nsweeps - t0);
        P.sweep0 = sweep0 + (uint64_t)t0;
        P.nsweeps = nc;
        P.beta_stride = constant ? 0 : nc;
        for (int t = 0; t < (constant ? 1 : nc); ++t) P.temp.beta[t] = accept_cx(pt.scale, kT[t0 + t]);
        // the array keeps the last call's contents: zero what must start at
        // zero (ticket, abort word, flags and partial sums of this call's tiles)
        e = cudaMemsetAsync(scr, 0, kNoAllocFlagsOff + (size_t)P.ntiles * 4, stream);
        const size_t np = (size_t)P.ntiles * (size_t)std::max(1, P.team);
        if (e == cudaSuccess) e = cudaMemsetAsync(scr + kNoAllocPartEOff, 0, np * 8, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(scr + kNoAllocPartNOff, 0, np * 8, stream);
        if (e != cudaSuccess) {
            run = cuda_fail(e, "cudaMemsetAsync(no-alloc scratch)");
            break;
        }
        void *args[] = {(void *)&P};
        e = cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream);
        if (e != cudaSuccess) run = cuda_fail(e, "cudaLaunchCooperativeKernel(no-alloc sweep)");
    }
    if (fast) {
        st = scale_occ(1, lat, occs, false, P.status, sms, stream);
        if (run == SMC_OK && st != SMC_OK) run = st;
    }
    return run;
}

}  // namespace smc
