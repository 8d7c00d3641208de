// sweep_pair.cu -- persistent swap-MC sweep kernel for pair models.
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
// group touch disjoint rows, so a column's Lx mini-steps run inside one CTA
// in lock-step with only CTA-level barriers, on a copy of those rows in
// shared memory.  Columns are grouped into rectangular tiles; a tile may start
// group G only after its 8 neighbouring tiles have finished group G-1
// (per-tile progress flags in global memory, bounded waits).  Trials in the
// same mini-step are independent, and a column's dependencies reach only the
// adjacent columns, so this reproduces the sequential mini-step order exactly.
//
// dE of a trial (a -> b) is the pair-model energy change written through the
// first-neighbour histograms: with D_m[q] = V_m(s_b, q) - V_m(s_a, q),
//   dE = sum_m [ sum_{j in N_m(a)\b} D_m[s_j] - sum_{j in N_m(b)\a} D_m[s_j] ],
// which equals the Omega-reduced local-energy difference of Algorithm 1
// lines 4-8 for pair site energies e_i = 1/2 sum_v V(s_i, s_{i+v}).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "sweep_common.cuh"

namespace smc {

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

// dE of swapping the trial site a (own sublattice, x) with its partner in
// direction `dir` (bits kx, ky, kz -> vector 2k-1 in half units).
// Returns the species A, B and the partner's coordinates through pointers.
template <bool IS_INT, class View>
__device__ __forceinline__ typename Acc<IS_INT>::T trial_dE(const View &cv, int x, int nx, int s_off,
                                                            int dir, int nshells, int S, const void *Dtab,
                                                            int &A, int &B, int &ex, int &ey, int &ez)
{
    using T = typename Acc<IS_INT>::T;
    const int kx = (dir >> 2) & 1, ky = (dir >> 1) & 1, kz = dir & 1;
    ex = kx + s_off;
    ey = ky + s_off;
    ez = kz + s_off;
    const int xm2 = wrapc(x - 2, nx), xm1 = wrapc(x - 1, nx), xp1 = wrapc(x + 1, nx), xp2 = wrapc(x + 2, nx);
    auto xo = [&](int d) { return d == -2 ? xm2 : (d == -1 ? xm1 : (d == 0 ? x : (d == 1 ? xp1 : xp2))); };
    A = cv.O(0, 0)[x] & 7;
    const int bx = xo(ex);
    B = cv.T(ey, ez)[bx] & 7;
    if (A == B) return T(0);
    const T *D = (const T *)Dtab;
    const T *D1 = D + ((0 * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
    T dE = T(0);
    // shell 1 of a (partner sublattice), all but b
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (u == dir) continue;
        const int fx = ((u >> 2) & 1) + s_off, fy = ((u >> 1) & 1) + s_off, fz = (u & 1) + s_off;
        dE += D1[cv.T(fy, fz)[xo(fx)] & 7];
    }
    // shell 1 of b (trial sublattice), all but a
    const int sb = -1 - s_off;
    const int nd = 7 - dir;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (u == nd) continue;
        const int gx = ex + ((u >> 2) & 1) + sb, gy = ey + ((u >> 1) & 1) + sb, gz = ez + (u & 1) + sb;
        dE -= D1[cv.O(gy, gz)[xo(gx)] & 7];
    }
    if (nshells >= 2) {
        const T *D2 = D + ((1 * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
        const unsigned char *o00 = cv.O(0, 0);
        dE += D2[o00[xm1] & 7] + D2[o00[xp1] & 7] + D2[cv.O(-1, 0)[x] & 7] + D2[cv.O(1, 0)[x] & 7] +
              D2[cv.O(0, -1)[x] & 7] + D2[cv.O(0, 1)[x] & 7];
        const unsigned char *tb = cv.T(ey, ez);
        dE -= D2[tb[xo(ex - 1)] & 7] + D2[tb[xo(ex + 1)] & 7] + D2[cv.T(ey - 1, ez)[bx] & 7] +
              D2[cv.T(ey + 1, ez)[bx] & 7] + D2[cv.T(ey, ez - 1)[bx] & 7] + D2[cv.T(ey, ez + 1)[bx] & 7];
    }
    if (nshells >= 3) {
        const T *D3 = D + ((2 * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
#pragma unroll
        for (int p = -1; p <= 1; p += 2)
#pragma unroll
            for (int q = -1; q <= 1; q += 2) {
                dE += D3[cv.O(p, q)[x] & 7];           // (0, +-1, +-1)
                dE += D3[cv.O(p, 0)[xo(q)] & 7];       // (+-1, +-1, 0)
                dE += D3[cv.O(0, p)[xo(q)] & 7];       // (+-1, 0, +-1)
                dE -= D3[cv.T(ey + p, ez + q)[bx] & 7];
                dE -= D3[cv.T(ey + p, ez)[xo(ex + q)] & 7];
                dE -= D3[cv.T(ey, ez + p)[xo(ex + q)] & 7];
            }
    }
    return dE;
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

template <bool IS_INT>
__global__ void __launch_bounds__(512) k_sweep_pair(const __grid_constant__ SweepParams P)
{
    using T = typename Acc<IS_INT>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_stop;
    __shared__ int s_last;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;

    T *Dt = (T *)smem;
    double *slot_e = (double *)(smem + kDEntries * 4);
    long long *slot_n = (long long *)(slot_e + P.tpc * nwarp);
    unsigned char *colbuf = (unsigned char *)(slot_n + P.tpc * nwarp);

    for (int i = tid; i < kDEntries; i += nthr) {
        if constexpr (IS_INT)
            Dt[i] = P.D.di[i];
        else
            Dt[i] = P.D.df[i];
    }
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
                float beta = 0.f;
                int2 ti = make_int2(0, 0);
                if constexpr (IS_INT)
                    ti = P.temp.tabinfo[P.beta_stride ? r * P.beta_stride + t : r];
                else
                    beta = P.temp.beta[P.beta_stride ? r * P.beta_stride + t : r];

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
                T accE = T(0);
                double accE_d = 0.0;
                long long accN = 0;

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
                            const T dE = trial_dE<IS_INT, ColView>(cv, x, nx, s_off, (int)(w >> kRBits),
                                                                   P.nshells, P.S, Dt, A, B, ex, ey, ez);
                            if (metropolis<IS_INT>(dE, w & kRMask, beta, P.tab, ti)) {
                                if (A != B) {
                                    cv.O(0, 0)[x] = (unsigned char)B;
                                    cv.T(ey, ez)[wrapc(x + ex, nx)] = (unsigned char)A;
                                }
                                if constexpr (IS_INT)
                                    accE += dE;
                                else
                                    accE_d += (double)dE;
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
                double e_w;
                if constexpr (IS_INT)
                    e_w = (double)warp_sum<long long>((long long)accE);
                else
                    e_w = warp_sum<double>(accE_d);
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
        if (RD.e_acc) *RD.e_acc += se;
        if (RD.n_acc) *RD.n_acc += sn;
    }
}

// ---------------------------------------------------------------------------
// Fast path: every axis holds >= 2 four-cell link cells (Lx = Ly = Lz = 4).
// One warp owns a tile of columns and runs it without CTA barriers: it waits
// for its tile's neighbours, stages the column's rows in its own shared
// memory, runs the 4 mini-steps of the group (lane i handles link cells
// i, i+32, ...), writes back the 5 rows the group may change and publishes
// its progress.  Philox is evaluated once per link cell and group: the four
// trial sites of a link cell's x-row, x = 4i .. 4i+3, share the counter
// s >> 2 and use its four output words.
//
// Shared-memory rows of a column (stride rb = padded nx + 32): the row body
// starts 16 bytes in and is framed by a 4-byte periodic halo on each side,
// so x-2 .. x+2 need no wrap.  Trial-sublattice rows (dy, dz) in [-1, 1]^2
// are at index (dz+1)*3 + (dy+1); partner-sublattice rows (sy, sz) in
// [0, 4)^2, i.e. (dy, dz) = (s_off-1+sy, s_off-1+sz), at 9 + sz*4 + sy.
// Two-shell models never read the four partner corner rows (not loaded).
// A neighbour of species q adds 1 << (4q) to a histogram of 4-bit counts.
//
// dE through the histograms: with c_m[q] = #{j in N_m(a)\b: s_j = q} -
// #{j in N_m(b)\a: s_j = q} and D_m[q] = V_m(s_b, q) - V_m(s_a, q),
// dE = sum_m sum_q c_m[q] D_m[q].  For shells 1 and 2, c + 8 lies in [1, 15]
// and one biased word holds all of c_m; shell 3 keeps the two counts apart.
// ---------------------------------------------------------------------------
// Sum over the first S-1 species only: every shell holds the same number of
// neighbours of a (without b) as of b (without a), so sum_q c[q] = 0 and
// c[S-1] = -sum_{q<S-1} c[q].  The kernel's table row for (m, A, B) holds
// D'[q] = D[q] - D[S-1] for q < S-1 and, in entry 7, -8 sum_q D'[q] (the
// 4-bit fields of shells 1 and 2 carry a bias of 8).
// In shared memory the fast kernel keeps the table rows (m, A, B) of its
// species template ST compactly, RS = fast_rs(ST) words each: D'[0..ST-2],
// then the bias.  An odd stride for ST = 2 and 5 sends the rows of the up
// to 25 (A, B) pairs a warp reads at once to distinct banks.
__host__ __device__ constexpr int fast_rs(int ST) { return ST == 8 ? 8 : (ST | 1); }
__host__ __device__ constexpr int fast_d_bytes(int NSH, int ST)
{
    return ((NSH >= 3 ? 3 : 2) * ST * ST * fast_rs(ST) * 4 + 15) / 16 * 16;
}

template <bool IS_INT, int S>
__device__ __forceinline__ typename Acc<IS_INT>::T dot_biased(uint32_t H, const typename Acc<IS_INT>::T *D)
{
    using T = typename Acc<IS_INT>::T;
    T acc = D[S - 1];
#pragma unroll
    for (int q = 0; q < S - 1; ++q) {
        const int f = (int)((H >> (4 * q)) & 15u);
        if constexpr (IS_INT)
            acc += f * D[q];
        else
            acc = fmaf((float)f, D[q], acc);
    }
    return acc;
}

template <bool IS_INT, int S>
__device__ __forceinline__ typename Acc<IS_INT>::T dot_diff(uint32_t Ha, uint32_t Hb, const typename Acc<IS_INT>::T *D)
{
    using T = typename Acc<IS_INT>::T;
    T acc = T(0);
#pragma unroll
    for (int q = 0; q < S - 1; ++q) {
        const int f = (int)((Ha >> (4 * q)) & 15u) - (int)((Hb >> (4 * q)) & 15u);
        if constexpr (IS_INT)
            acc += f * D[q];
        else
            acc = fmaf((float)f, D[q], acc);
    }
    return acc;
}

#define NIB(v) (1u << ((v) << 2))

// po: byte offsets (in g_smem) of the 9 trial-sublattice row bodies; pt: of
// the partner block (row index 0).  Returns dE; A, B and the partner's
// row offset and x through references.
// Shared-memory row index of partner-sublattice slot (sy, sz).  Two-shell
// models store the 12 slots they can read (the 4x4 window without its
// corners) compactly; three-shell models store all 16.
template <int NSH>
__host__ __device__ __forceinline__ int pslot(int sy, int sz)
{
    if (NSH >= 3) return 9 + sz * 4 + sy;
    return 9 + (sz == 0 ? sy - 1 : (sz == 1 ? 2 + sy : (sz == 2 ? 6 + sy : 9 + sy)));
}

// po: byte offsets (in g_smem) of the 9 trial-sublattice row bodies; col0:
// offset of row 0's body.  Returns dE (exactly 0 when a and b hold the same
// species: the table rows D'(A, A) vanish); A, B and the partner's row
// offset and x through references.
template <bool IS_INT, int NSH, int S, int SOFF>
__device__ __forceinline__ typename Acc<IS_INT>::T fast_dE(const uint32_t *po, uint32_t col0, uint32_t rb, int x,
                                                           int dir, uint32_t dt, int &A, int &B, uint32_t &brow,
                                                           int &xb)
{
    using T = typename Acc<IS_INT>::T;
    const int kx = (dir >> 2) & 1, ky = (dir >> 1) & 1, kz = dir & 1;
    A = (int)(SM8(po[4] + x) & 7u);
    // partner's row: slot (ky+1, kz+1) = 12 + 4 kz + ky (two shells) or 14 + 4 kz + ky
    const uint32_t rbp = col0 + (uint32_t)((NSH >= 3 ? 14 : 12) + 4 * kz + ky) * rb;
    xb = x + SOFF + kx;
    B = (int)(SM8(rbp + xb) & 7u);
    brow = rbp;
    // shell 1: a's 8 partner-sublattice neighbours minus b, minus b's 8
    // trial-sublattice neighbours plus a.  A species >= 8 (invalid input)
    // shifts the 1 out of the word and is ignored.
    uint32_t H1 = 0x88888888u - NIB(B) + NIB(A);
    {
        const uint32_t xa = col0 + x + SOFF;
        const uint32_t r11 = xa + pslot<NSH>(1, 1) * rb, r21 = xa + pslot<NSH>(2, 1) * rb;
        const uint32_t r12 = xa + pslot<NSH>(1, 2) * rb, r22 = xa + pslot<NSH>(2, 2) * rb;
        H1 += NIB(SM8(r11)) + NIB(SM8(r11 + 1)) + NIB(SM8(r21)) + NIB(SM8(r21 + 1)) + NIB(SM8(r12)) +
              NIB(SM8(r12 + 1)) + NIB(SM8(r22)) + NIB(SM8(r22 + 1));
        const uint32_t ob = po[0] + (uint32_t)(kz * 3 + ky) * rb + x + kx - 1;
        H1 -= NIB(SM8(ob)) + NIB(SM8(ob + 1)) + NIB(SM8(ob + rb)) + NIB(SM8(ob + rb + 1)) + NIB(SM8(ob + 3 * rb)) +
              NIB(SM8(ob + 3 * rb + 1)) + NIB(SM8(ob + 4 * rb)) + NIB(SM8(ob + 4 * rb + 1));
    }
    constexpr int RS = fast_rs(S), SH = S * S * RS;
    const T *Dt = (const T *)(g_smem + dt);
    const T *D1 = Dt + (A * S + B) * RS;
    T dE = dot_biased<IS_INT, S>(H1, D1);
    const uint32_t bx = rbp + xb;
    // partner rows one slot down / up in z (compact layout: 3 or 4 rows apart)
    const uint32_t zdn = NSH >= 3 ? 4 * rb : 3 * rb + (uint32_t)kz * rb;
    const uint32_t zup = NSH >= 3 ? 4 * rb : 4 * rb - (uint32_t)kz * rb;
    if (NSH >= 2) {
        const uint32_t ax = po[4] + x;
        uint32_t H2 = 0x88888888u;
        H2 += NIB(SM8(ax - 1)) + NIB(SM8(ax + 1)) + NIB(SM8(po[3] + x)) + NIB(SM8(po[5] + x)) + NIB(SM8(po[1] + x)) +
              NIB(SM8(po[7] + x));
        H2 -= NIB(SM8(bx - 1)) + NIB(SM8(bx + 1)) + NIB(SM8(bx - rb)) + NIB(SM8(bx + rb)) + NIB(SM8(bx - zdn)) +
              NIB(SM8(bx + zup));
        dE += dot_biased<IS_INT, S>(H2, D1 + SH);
    }
    if (NSH >= 3) {
        const uint32_t Ha = NIB(SM8(po[0] + x)) + NIB(SM8(po[2] + x)) + NIB(SM8(po[6] + x)) + NIB(SM8(po[8] + x)) +
                            NIB(SM8(po[3] + x - 1)) + NIB(SM8(po[3] + x + 1)) + NIB(SM8(po[5] + x - 1)) +
                            NIB(SM8(po[5] + x + 1)) + NIB(SM8(po[1] + x - 1)) + NIB(SM8(po[1] + x + 1)) +
                            NIB(SM8(po[7] + x - 1)) + NIB(SM8(po[7] + x + 1));
        const uint32_t Hb = NIB(SM8(bx - 5 * rb)) + NIB(SM8(bx - 3 * rb)) + NIB(SM8(bx + 3 * rb)) +
                            NIB(SM8(bx + 5 * rb)) + NIB(SM8(bx - rb - 1)) + NIB(SM8(bx - rb + 1)) +
                            NIB(SM8(bx + rb - 1)) + NIB(SM8(bx + rb + 1)) + NIB(SM8(bx - 4 * rb - 1)) +
                            NIB(SM8(bx - 4 * rb + 1)) + NIB(SM8(bx + 4 * rb - 1)) + NIB(SM8(bx + 4 * rb + 1));
        dE += dot_diff<IS_INT, S>(Ha, Hb, D1 + 2 * SH);
    }
    return dE;
}
#undef NIB

template <bool IS_INT, int NSH, int S, int SOFF, int KU, bool GUARD>
__device__ __forceinline__ void fast_trials(const SweepParams &P, const uint32_t *po, uint32_t col0, uint32_t rb,
                                            const uint32_t *wsm, int k0, int nk, int NLx, int nx, int dx, int lane,
                                            float beta, int2 ti, uint32_t dt, typename Acc<IS_INT>::T &colE,
                                            long long &accN)
{
    using T = typename Acc<IS_INT>::T;
    T dE[KU];
    int A[KU], B[KU], xb[KU], xs[KU];
    uint32_t brow[KU];
    bool acc[KU];
#pragma unroll
    for (int u = 0; u < KU; ++u) {
        const int k = k0 + u, i = lane + 32 * k;
        acc[u] = false;
        if (!GUARD || (k < nk && i < NLx)) {
            const int x = 4 * i + dx;
            xs[u] = x;
            const uint32_t w = wsm[(k * 4 + dx) * 32 + lane];
            dE[u] = fast_dE<IS_INT, NSH, S, SOFF>(po, col0, rb, x, (int)(w >> kRBits), dt, A[u], B[u], brow[u], xb[u]);
            acc[u] = metropolis<IS_INT>(dE[u], w & kRMask, beta, P.tab, ti);
        }
    }
#pragma unroll
    for (int u = 0; u < KU; ++u) {
        if (acc[u]) {
            halo_store(po[4], xs[u], nx, (unsigned char)B[u]);
            halo_store(brow[u], xb[u], nx, (unsigned char)A[u]);
            colE += dE[u];
            accN += 1;
        }
    }
}

template <bool IS_INT, int NSH, int S, int SOFF>
__device__ __forceinline__ void fast_column(const SweepParams &P, const RepDesc &RD, uint32_t col, int y0, int z0,
                                            uint64_t sweep, float beta, int2 ti, uint32_t dt, int lane,
                                            typename Acc<IS_INT>::T &accE, double &accEd, long long &accN)
{
    using T = typename Acc<IS_INT>::T;
    constexpr int sub = SOFF == -1 ? 0 : 1;
    constexpr int rows = NSH >= 3 ? 25 : 21;
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz, NLx = RD.NLx;
    const uint32_t rb = (uint32_t)P.rowB;
    const bool vec = RD.vec != 0;
    // ---- per-row source (global) and destination (shared) of this column:
    // lane r computes row r once; the others read it by shuffle ----
    const int8_t *my_src = RD.occ;
    uint32_t my_dst = 0;
    if (lane < rows) {
        int gsub, dy, dz;
        if (lane < 9) {
            dy = lane % 3 - 1;
            dz = lane / 3 - 1;
            gsub = sub;
        } else {
            const int k = lane - 9;
            int sy, sz;
            if (NSH >= 3) {
                sy = k & 3;
                sz = k >> 2;
            } else {
                sz = k < 2 ? 0 : (k < 6 ? 1 : (k < 10 ? 2 : 3));
                sy = k < 2 ? k + 1 : (k < 6 ? k - 2 : (k < 10 ? k - 6 : k - 9));
            }
            dy = sy - 1 + SOFF;
            dz = sz - 1 + SOFF;
            gsub = 1 - sub;
        }
        const int gy = wrapc(y0 + dy, ny), gz = wrapc(z0 + dz, nz);
        my_src = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx;
        my_dst = col + (uint32_t)lane * rb + 16;
    }
    // ---- stage the rows (L2-only copies: never a stale L1 line) ----
    {
        const int cpr = vec ? (nx >> 4) : (nx >> 2);
        int lr = 0, lc = lane, rstep = 1, cstep = 32;
        if (cpr < 32) {
            rstep = 32 / cpr;
            lr = lane / cpr;
            lc = lane - lr * cpr;
            cstep = cpr;
        }
        const int iters = (rows + rstep - 1) / rstep;
        const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(g_smem);
        for (int it = 0; it < iters; ++it) {
            const int rr = lr + it * rstep;
            const int rsel = rr < rows ? rr : 0;
            const int8_t *src = (const int8_t *)__shfl_sync(0xffffffffu, (unsigned long long)my_src, rsel);
            const uint32_t dst = __shfl_sync(0xffffffffu, my_dst, rsel);
            if (lr < rstep && rr < rows) {
                if (vec) {
                    for (int c = lc; c < cpr; c += cstep)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem0 + dst + 16 * c),
                                     "l"(src + 16 * c)
                                     : "memory");
                } else {
                    const unsigned *s4 = (const unsigned *)src;
                    unsigned *d4 = (unsigned *)(g_smem + dst);
                    for (int c = lc; c < cpr; c += 4 * cstep) {
                        const int c1 = c + cstep, c2 = c + 2 * cstep, c3 = c + 3 * cstep;
                        const unsigned v0 = __ldcg(s4 + c);
                        const unsigned v1 = c1 < cpr ? __ldcg(s4 + c1) : 0u;
                        const unsigned v2 = c2 < cpr ? __ldcg(s4 + c2) : 0u;
                        const unsigned v3 = c3 < cpr ? __ldcg(s4 + c3) : 0u;
                        d4[c] = v0;
                        if (c1 < cpr) d4[c1] = v1;
                        if (c2 < cpr) d4[c2] = v2;
                        if (c3 < cpr) d4[c3] = v3;
                    }
                }
            }
        }
    }
    // ---- Philox words of this lane's link cells, kept in shared memory
    // (computed while the row copies are in flight) ----
    uint32_t *wsm = (uint32_t *)(g_smem + col + (uint32_t)rows * rb + 16);  // [k][dx][lane]
    const int nk = (NLx + 31) >> 5;
    {
        const uint32_t rowsite = (uint32_t)(((sub * nz + z0) * ny + y0) * nx);
        const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
#pragma unroll 1
        for (int k = 0; k < nk; ++k) {
            const int i = lane + 32 * k;
            if (i < NLx) {
                const U4 w =
                    philox10(U4{(rowsite >> 2) + (uint32_t)i, RD.rep, (uint32_t)sweep, (uint32_t)(sweep >> 32)}, k0, k1);
                wsm[(k * 4 + 0) * 32 + lane] = w.x;
                wsm[(k * 4 + 1) * 32 + lane] = w.y;
                wsm[(k * 4 + 2) * 32 + lane] = w.z;
                wsm[(k * 4 + 3) * 32 + lane] = w.w;
            }
        }
    }
    if (vec) asm volatile("cp.async.wait_all;" ::: "memory");
    __syncwarp();
    // periodic halos: 4 bytes before and after each row body
    if (lane < rows) {
        *(unsigned *)(g_smem + my_dst - 4) = *(const unsigned *)(g_smem + my_dst + nx - 4);
        *(unsigned *)(g_smem + my_dst + nx) = *(const unsigned *)(g_smem + my_dst);
    }
    __syncwarp();
    uint32_t po[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) po[r] = col + (uint32_t)r * rb + 16;
    const uint32_t col0 = col + 16;
    // ---- the four mini-steps of the group ----
    // accepted dE of this lane's trials in the column (at most nx / 8 of
    // them), in the kernel's type; widened to FP64 once per column
    T colE = T(0);
#pragma unroll 1
    for (int dx = 0; dx < 4; ++dx) {
        if (NLx == 32 * nk && (nk & 3) == 0) {
#pragma unroll 1
            for (int kk = 0; kk < nk; kk += 4)
                fast_trials<IS_INT, NSH, S, SOFF, 4, false>(P, po, col0, rb, wsm, kk, nk, NLx, nx, dx, lane, beta, ti,
                                                            dt, colE, accN);
        } else if (NLx == 32 * nk) {
#pragma unroll 1
            for (int kk = 0; kk < nk; ++kk)
                fast_trials<IS_INT, NSH, S, SOFF, 1, false>(P, po, col0, rb, wsm, kk, nk, NLx, nx, dx, lane, beta, ti,
                                                            dt, colE, accN);
        } else {
#pragma unroll 1
            for (int kk = 0; kk < nk; ++kk)
                fast_trials<IS_INT, NSH, S, SOFF, 1, true>(P, po, col0, rb, wsm, kk, nk, NLx, nx, dx, lane, beta, ti,
                                                           dt, colE, accN);
        }
        __syncwarp();
    }
    if constexpr (IS_INT)
        accE += colE;
    else
        accEd += (double)colE;
    // ---- write back trial row (0,0) and partner rows (s_off..s_off+1)^2 ----
    {
        const int cpr = vec ? (nx >> 4) : (nx >> 2);
        int lr = 0, lc = lane, rstep = 1, cstep = 32;
        if (cpr < 32) {
            rstep = 32 / cpr;
            lr = lane / cpr;
            lc = lane - lr * cpr;
            cstep = cpr;
        }
        if (lr < rstep) {
            for (int wr = lr; wr < 5; wr += rstep) {
                int slot, gsub, gy, gz;
                if (wr == 0) {
                    slot = 4;
                    gsub = sub;
                    gy = y0;
                    gz = z0;
                } else {
                    const int sy = 1 + ((wr - 1) & 1), sz = 1 + ((wr - 1) >> 1);
                    slot = pslot<NSH>(sy, sz);
                    gsub = 1 - sub;
                    gy = wrapc(y0 + sy - 1 + SOFF, ny);
                    gz = wrapc(z0 + sz - 1 + SOFF, nz);
                }
                int8_t *dstg = RD.occ + ((size_t)((gsub * nz + gz) * ny + gy)) * nx;
                const unsigned char *srcs = g_smem + col + (uint32_t)slot * rb + 16;
                if (vec) {
                    for (int c = lc; c < cpr; c += cstep) *((int4 *)dstg + c) = *((const int4 *)srcs + c);
                } else {
                    for (int c = lc; c < cpr; c += cstep) *((unsigned *)dstg + c) = *((const unsigned *)srcs + c);
                }
            }
        }
    }
    __syncwarp();
}

template <bool IS_INT, int NSH, int S>
__global__ void __launch_bounds__(256, 2) k_sweep_fast(const __grid_constant__ SweepParams P)
{
    using T = typename Acc<IS_INT>::T;
    unsigned char *smem = g_smem;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const int gw = blockIdx.x * nwarp + warp, NW = gridDim.x * nwarp;
    // compact table: row (m, A, B) of RS words = D'[0..S-2], bias
    constexpr int RS = fast_rs(S), NDE = (NSH >= 3 ? 3 : 2) * S * S * RS;
    T *Dt = (T *)smem;
    for (int i = tid; i < NDE; i += blockDim.x) {
        const int q = i % RS, row = i / RS, mm = row / (S * S), A = (row / S) % S, B = row % S;
        const int src = ((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies + (q == S - 1 ? 7 : q);
        if constexpr (IS_INT)
            Dt[i] = q < S ? P.D.di[src] : 0;
        else
            Dt[i] = q < S ? P.D.df[src] : 0.f;
    }
    __syncthreads();
    unsigned char *wbase = smem + fast_d_bytes(NSH, S) + (size_t)warp * P.warp_bytes;
    double *slot_e = (double *)wbase;
    long long *slot_n = (long long *)(slot_e + P.tpc);
    const uint32_t col = (uint32_t)((unsigned char *)(slot_n + P.tpc) - smem);
    for (int i = lane; i < P.tpc; i += 32) {
        slot_e[i] = 0.0;
        slot_n[i] = 0;
    }
    __syncwarp();

    bool aborted = false;
    for (int t = 0; t < P.nsweeps && !aborted; ++t) {
        const uint64_t sweep = P.sweep0 + (uint64_t)t;
        for (int g = 0; g < P.G && !aborted; ++g) {
            const uint32_t gstep = (uint32_t)(t * P.G + g);
            const int dy = g & 3, dz = (g >> 2) & 3, sub = g >> 4;
            const int lagv = P.lag[g];
            const uint32_t need = gstep + 1 >= (uint32_t)lagv ? gstep + 1 - lagv : 0;
            int slotk = 0;
            for (int tile = gw; tile < P.ntiles; tile += NW, ++slotk) {
                int r = 0;
                while (r + 1 < P.R && P.rep[r + 1].tile0 <= tile) ++r;
                const RepDesc &RD = P.rep[r];
                const int lt = tile - RD.tile0, ty = lt % RD.NTy, tz = lt / RD.NTy;
                if (!wait_tile_warp(P, RD, ty, tz, need, lane)) {
                    aborted = true;
                    break;
                }
                float beta = 0.f;
                int2 ti = make_int2(0, 0);
                if constexpr (IS_INT)
                    ti = P.temp.tabinfo[P.beta_stride ? r * P.beta_stride + t : r];
                else
                    beta = P.temp.beta[P.beta_stride ? r * P.beta_stride + t : r];
                T accE = T(0);
                double accEd = 0.0;
                long long accN = 0;
                const int j0 = ty * P.TY, j1 = min(j0 + P.TY, RD.NLy);
                const int l0 = tz * P.TZ, l1 = min(l0 + P.TZ, RD.NLz);
                for (int l = l0; l < l1; ++l)
                    for (int j = j0; j < j1; ++j) {
                        const int y0 = 4 * j + dy, z0 = 4 * l + dz;
                        if (sub == 0)
                            fast_column<IS_INT, NSH, S, -1>(P, RD, col, y0, z0, sweep, beta, ti, 0u, lane, accE,
                                                            accEd, accN);
                        else
                            fast_column<IS_INT, NSH, S, 0>(P, RD, col, y0, z0, sweep, beta, ti, 0u, lane, accE,
                                                           accEd, accN);
                    }
                double e_w;
                if constexpr (IS_INT)
                    e_w = (double)warp_sum<long long>((long long)accE);
                else
                    e_w = warp_sum<double>(accEd);
                const long long n_w = warp_sum<long long>(accN);
                if (lane == 0) {
                    slot_e[slotk] += e_w;
                    slot_n[slotk] += n_w;
                }
                // every lane's row stores, then one release by lane 0 (the warp
                // barrier orders the other lanes' stores before it)
                __syncwarp();
                if (lane == 0 && tile != P.skip_tile) st_release_u32(P.flags + tile, gstep + 1);
            }
        }
    }
    // ---- per-tile partial sums; the last warp to finish reduces them in order ----
    if (aborted) return;
    if (lane == 0) {
        int k = 0;
        for (int tile = gw; tile < P.ntiles; tile += NW, ++k) {
            P.part_e[tile] = slot_e[k];
            P.part_n[tile] = slot_n[k];
        }
    }
    __threadfence();
    __syncwarp();
    unsigned last = 0;
    if (lane == 0) last = (atomicAdd(P.ticket, 1u) == (unsigned)NW - 1) ? 1u : 0u;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    for (int r = lane; r < P.R; r += 32) {
        const RepDesc &RD = P.rep[r];
        double se = 0.0;
        long long sn = 0;
        const int nt = RD.NTy * RD.NTz;
        for (int k = 0; k < nt; ++k) {
            se += __ldcg(P.part_e + RD.tile0 + k);
            sn += __ldcg(P.part_n + RD.tile0 + k);
        }
        if (RD.e_acc) *RD.e_acc += se;
        if (RD.n_acc) *RD.n_acc += sn;
    }
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

template <bool IS_INT>
__global__ void k_ministep_eval(const __grid_constant__ SweepParams P, int k, float *dE_out, uint8_t *acc_out,
                                int *swap_a, int *swap_b)
{
    using T = typename Acc<IS_INT>::T;
    __shared__ T Dt[kDEntries];
    for (int i = threadIdx.x; i < kDEntries; i += blockDim.x) {
        if constexpr (IS_INT)
            Dt[i] = P.D.di[i];
        else
            Dt[i] = P.D.df[i];
    }
    __syncthreads();
    const RepDesc &RD = P.rep[0];
    const int ntr = RD.NLx * RD.NLy * RD.NLz;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ntr) return;
    const int dx = k % P.Lx, dy = (k / P.Lx) % P.Ly, dz = (k / (P.Lx * P.Ly)) % P.Lz;
    const int sub = k / (P.Lx * P.Ly * P.Lz);
    const int s_off = sub == 0 ? -1 : 0;
    const int cx = c % RD.NLx, cy = (c / RD.NLx) % RD.NLy, cz = c / (RD.NLx * RD.NLy);
    const int nx = RD.nx, ny = RD.ny, nz = RD.nz;
    const int x = cx * P.Lx + dx, y0 = cy * P.Ly + dy, z0 = cz * P.Lz + dz;
    const GView gv{(const unsigned char *)RD.occ, nx, ny, nz, sub, y0, z0};
    const uint32_t s = (uint32_t)(((sub * nz + z0) * ny + y0) * nx + x);
    const uint32_t w = site_word(P.seed, RD.rep, P.sweep0, s);
    int A, B, ex, ey, ez;
    const T dE = trial_dE<IS_INT, GView>(gv, x, nx, s_off, (int)(w >> kRBits), P.nshells, P.S, Dt, A, B, ex, ey, ez);
    float beta = 0.f;
    int2 ti = make_int2(0, 0);
    if constexpr (IS_INT)
        ti = P.temp.tabinfo[0];
    else
        beta = P.temp.beta[0];
    const bool acc = metropolis<IS_INT>(dE, w & kRMask, beta, P.tab, ti);
    if (dE_out) dE_out[c] = (float)dE;
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
// Warp count of the warp-per-tile kernel.  Warp w owns tiles w, w + NW, ...
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
    int threads, CB, TY, TZ, ntiles, grid, tpc, warp_bytes = 0, nap_cap = 128, rowB = 0;
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
smc_status make_plan(int R, const smc_lattice *lats, Workspace *ws, Plan &pl)
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
    const size_t base = (size_t)kDEntries * 4;
    auto smem_for = [&](int cb, int tpc) { return base + (size_t)tpc * nwarps * 16 + (size_t)cb * maxcol; };
    while (pl.CB > 1 && smem_for(pl.CB, 64) > ws->smem_optin) pl.CB /= 2;
    if (smem_for(pl.CB, 1) > ws->smem_optin) {
        set_error("lattice rows too long for shared memory (nx = %d)", lats[0].nx);
        return SMC_ERR_UNSUPPORTED;
    }
    auto kern = k_sweep_pair<IS_INT>;
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
    pl.kernel = (const void *)k_sweep_pair<IS_INT>;
    return SMC_OK;
}

template <bool IS_INT, int NSH>
const void *pick_fast(int S)
{
    switch (S) {
    case 2: return (const void *)k_sweep_fast<IS_INT, NSH, 2>;
    case 5: return (const void *)k_sweep_fast<IS_INT, NSH, 5>;
    default: return (const void *)k_sweep_fast<IS_INT, NSH, 8>;
    }
}

// Plan of the warp-per-tile kernel: tiles of TY x TZ columns, one warp each
// (a warp owns ceil(ntiles / warps) tiles), shared memory = D table + per warp
// (accumulator slots + 25 rows).
template <bool IS_INT>
smc_status make_fast_plan_uncached(int R, const smc_lattice *lats, int8_t *const *occ, Workspace *ws, int nshells,
                                   int rowB, int same_nx, Plan &pl);

// The plan depends only on the shapes, the model's shell and species
// counts, the tuning and the device, so repeated calls (short chunks of a
// long run, one call per sample) reuse it instead of searching again.
template <bool IS_INT>
smc_status make_fast_plan(int R, const smc_lattice *lats, int8_t *const *occ, Workspace *ws, int nshells,
                          int rowB, int same_nx, Plan &pl)
{
    static std::vector<long long> key_cached;
    static Plan plan_cached;
    const Tuning tu = current_tuning();
    std::vector<long long> key = {R, nshells, rowB, same_nx, lats[0].nspecies, ws->device, ws->num_sms,
                                  (long long)ws->smem_optin, tu.tile_y, tu.tile_z, tu.threads, tu.ctas_per_sm};
    for (int r = 0; r < R; ++r) {
        key.push_back(lats[r].nx);
        key.push_back(lats[r].ny);
        key.push_back(lats[r].nz);
    }
    if (key == key_cached) {
        pl = plan_cached;
        return SMC_OK;
    }
    const smc_status st = make_fast_plan_uncached<IS_INT>(R, lats, occ, ws, nshells, rowB, same_nx, pl);
    if (st == SMC_OK) {
        key_cached = key;
        plan_cached = pl;
    }
    return st;
}

template <bool IS_INT>
smc_status make_fast_plan_uncached(int R, const smc_lattice *lats, int8_t *const *occ, Workspace *ws, int nshells,
                                   int rowB, int same_nx, Plan &pl)
{
    const Tuning tu = current_tuning();
    pl.Lx = pl.Ly = pl.Lz = 4;
    pl.G = 32;
    (void)same_nx;
    (void)occ;
    const int S = lats[0].nspecies;
    const int ST = S == 2 ? 2 : (S == 5 ? 5 : 8);
    const int nsh_t = nshells >= 3 ? 3 : 2;
    pl.kernel = nsh_t == 3 ? pick_fast<IS_INT, 3>(S) : pick_fast<IS_INT, 2>(S);
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
    // one column per tile unless tuned: the smallest unit of work keeps the
    // neighbour pipeline fullest
    pl.TY = tu.tile_y > 0 ? tu.tile_y : 1;
    pl.TZ = tu.tile_z > 0 ? tu.tile_z : 1;
    pl.ntiles = 0;
    for (int r = 0; r < R; ++r)
        pl.ntiles += ((lats[r].ny / 4 + pl.TY - 1) / pl.TY) * ((lats[r].nz / 4 + pl.TZ - 1) / pl.TZ);
    const size_t dbytes = (size_t)fast_d_bytes(nsh_t, ST);
    // Total warps NW: all resident at once (cooperative launch); preferably a
    // divisor of the tile count so that every warp owns as many tiles as the
    // others (an unevenly loaded warp makes its neighbours wait).  Between
    // CTA sizes giving as many warps, the one whose CTAs spread evenly over
    // the SMs (at most one per SM, or a multiple of the SM count) wins: a
    // warp that shares its scheduler with more warps than the others runs
    // slower and its neighbours wait for it (128^3: 1,024 warps as 128 CTAs
    // of 8 run a sweep in 199 us, as 256 CTAs of 4 in 226 us).
    auto search = [&](int rb, Plan &out) -> long long {
        const size_t rows_bytes = (size_t)(nsh_t >= 3 ? 25 : 21) * rb + 16 + (size_t)512 * nkmax;
        const int cand[2] = {128, 256};
        long long best_nw = 0;
        bool best_even = false;
        for (int ci = 0; ci < 2; ++ci) {
            const int threads = tu.threads ? std::min(tu.threads, 256) : cand[ci];  // launch bound is 256
            if (tu.threads && ci > 0) break;
            const int nwarps = threads / 32;
            for (int tpc_guess = 1;; tpc_guess *= 2) {
                const size_t wb = ((size_t)16 * tpc_guess + rows_bytes + 15) / 16 * 16;
                const size_t smem = dbytes + (size_t)nwarps * wb;
                if (smem > dyn_max) break;
                int per_sm = 0;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pl.kernel, threads, smem) != cudaSuccess)
                    return -1;
                if (tu.ctas_per_sm > 0) per_sm = std::min(per_sm, tu.ctas_per_sm);
                if (per_sm < 1) break;
                const long long res = (long long)per_sm * ws->num_sms * nwarps;
                const long long nw = balanced_warps(pl.ntiles, nwarps, per_sm, ws->num_sms);
                (void)res;
                const int tpc = (int)((pl.ntiles + nw - 1) / nw);
                if (tpc <= tpc_guess) {
                    const long long grid = nw / nwarps;
                    const bool even = grid <= ws->num_sms || grid % ws->num_sms == 0;
                    if (nw > best_nw || (nw == best_nw && even && !best_even)) {
                        best_nw = nw;
                        best_even = even;
                        out.threads = threads;
                        out.grid = (int)(nw / nwarps);
                        out.tpc = tpc_guess;
                        out.smem = smem;
                        out.warp_bytes = (int)wb;
                        out.rowB = rb;
                    }
                    break;
                }
            }
        }
        return best_nw;
    };
    const long long nw = search(rowB, pl);
    if (nw < 0) return cuda_fail(cudaGetLastError(), "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (nw == 0) {
        set_error("fast sweep kernel does not fit on an SM (rows of %d bytes)", rowB);
        return SMC_ERR_UNSUPPORTED;
    }
    // sleep between progress polls: short for small columns (latency-bound;
    // at 128^3 a cap of 32 ns measured 1 % faster than 128 ns), longer for
    // long ones (a tile-group takes tens of microseconds)
    pl.nap_cap = maxNLx >= 64 ? 1024 : 32;
    pl.CB = 1;
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
    // Fast path: 4-cell link cells on every axis, rows of at most 1024 cells,
    // 4-byte aligned occupancy.
    bool fast = true;
    int rowB_fast = 0, same_nx = lats[0].nx;
    for (int r = 0; r < R; ++r) {
        const smc_lattice &l = lats[r];
        fast = fast && lc_edge(l.nx) == 4 && lc_edge(l.ny) == 4 && lc_edge(l.nz) == 4 && l.nx <= 1024 &&
               ((uintptr_t)occ[r] % 4 == 0);
        rowB_fast = std::max(rowB_fast, ((l.nx + 15) & ~15) + 16);  // body at +16, 4-byte halos
        if (l.nx != same_nx) same_nx = -1;
    }
    if (current_tuning().threads && current_tuning().threads % 32) fast = false;
    Plan pl;
    if (fast) {
        st = make_fast_plan<IS_INT>(R, lats, occ, ws, m->nshells, rowB_fast, same_nx, pl);
        if (st != SMC_OK) return st;
    } else {
        st = make_plan<IS_INT>(R, lats, ws, pl);
        if (st != SMC_OK) return st;
    }

    static SweepParams P;  // large: keep off the stack (host-only, guarded by the API lock)
    memset(&P, 0, sizeof P);
    P.R = R;
    P.G = pl.G;
    P.Lx = pl.Lx;
    P.Ly = pl.Ly;
    P.Lz = pl.Lz;
    P.TY = pl.TY;
    P.TZ = pl.TZ;
    P.CB = pl.CB;
    P.nshells = m->nshells;
    P.S = lats[0].nspecies;
    P.tpc = pl.tpc;
    P.warp_bytes = pl.warp_bytes;
    P.nap_cap = pl.nap_cap;
    P.rowB = fast ? pl.rowB : rowB_fast;
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
    P.CB = std::min(P.CB, P.TY * P.TZ);
    P.ntiles = tile0;

    // D[m][A][B][q] = V_m(B, q) - V_m(A, q), padded to 8 species.  The fast
    // kernel reads D'[q] = D[q] - D[ST-1] for q < ST-1 (ST = its species
    // template: 2, 5 or 8) and, in entry 7 of shells 1 and 2, -8 sum D'.
    const int S = P.S;
    if (fast) {
        const int ST = S == 2 ? 2 : (S == 5 ? 5 : 8);
        for (int mm = 0; mm < m->nshells; ++mm)
            for (int A = 0; A < S; ++A)
                for (int B = 0; B < S; ++B) {
                    auto Dv = [&](int q) -> double {
                        if (q >= S) return 0.0;
                        if (IS_INT) return (double)m->v_i32[(mm * S + B) * S + q] - m->v_i32[(mm * S + A) * S + q];
                        return (double)m->v_f32[(mm * S + B) * S + q] - (double)m->v_f32[(mm * S + A) * S + q];
                    };
                    const int base = ((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
                    double bias = 0.0;
                    for (int q = 0; q < ST - 1; ++q) {
                        const double d = Dv(q) - Dv(ST - 1);
                        if (IS_INT)
                            P.D.di[base + q] = (int)d;
                        else
                            P.D.df[base + q] = (float)d;
                        bias += d;
                    }
                    if (mm < 2) {
                        if (IS_INT)
                            P.D.di[base + 7] = (int)(-8.0 * bias);
                        else
                            P.D.df[base + 7] = (float)(-8.0 * bias);
                    }
                }
    }
    for (int mm = 0; mm < (fast ? 0 : m->nshells); ++mm)
        for (int A = 0; A < S; ++A)
            for (int B = 0; B < S; ++B)
                for (int q = 0; q < S; ++q) {
                    const int idx = ((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies + q;
                    if (IS_INT)
                        P.D.di[idx] = m->v_i32[(mm * S + B) * S + q] - m->v_i32[(mm * S + A) * S + q];
                    else
                        P.D.df[idx] = (float)((double)m->v_f32[(mm * S + B) * S + q] -
                                              (double)m->v_f32[(mm * S + A) * S + q]);
                }

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

    // workspace: [flags | part_e | part_n | ticket, abort | tables]
    const size_t nt = (size_t)P.ntiles;
    const size_t off_flags = 0, off_pe = ((nt * 4 + 15) / 16) * 16, off_pn = off_pe + nt * 8;
    const size_t off_misc = off_pn + nt * 8, off_tab = off_misc + 16;
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

    for (int t0 = 0; t0 < nsweeps; t0 += chunk) {
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
                    P.temp.beta[idx] = (float)(1.0 / kt);
            }
        e = cudaMemsetAsync(scr, 0, off_tab, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sweep scratch)");
        void *args[] = {(void *)&P};
        e = cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(sweep)");
    }
    return SMC_OK;
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

template <bool IS_INT>
static smc_status trace_impl(const smc_lattice *lat, const smc_model *m, int8_t *occ, uint64_t seed,
                             uint32_t replica, uint64_t sweep, int k, double kT, float *dE, uint8_t *acc,
                             cudaStream_t stream)
{
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
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
    const int S = P.S;
    for (int mm = 0; mm < m->nshells; ++mm)
        for (int A = 0; A < S; ++A)
            for (int B = 0; B < S; ++B)
                for (int q = 0; q < S; ++q) {
                    const int idx = ((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies + q;
                    if (IS_INT)
                        P.D.di[idx] = m->v_i32[(mm * S + B) * S + q] - m->v_i32[(mm * S + A) * S + q];
                    else
                        P.D.df[idx] = (float)((double)m->v_f32[(mm * S + B) * S + q] -
                                              (double)m->v_f32[(mm * S + A) * S + q]);
                }
    const int ntr = d.NLx * d.NLy * d.NLz;
    std::vector<uint32_t> tab;
    if (IS_INT) {
        tab = int_table(m->unit_ev, kT);
        P.temp.tabinfo[0] = make_int2(0, (int)tab.size());
    } else {
        P.temp.beta[0] = (float)(1.0 / kT);
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
    k_ministep_eval<IS_INT><<<blocks, threads, 0, stream>>>(P, k, dE, acc, swap_a, swap_b);
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

    const int R = 1;
    const smc_lattice *lats = lat;
    int8_t *occs[1] = {occ};
    const bool fast = lc_edge(lat->nx) == 4 && lc_edge(lat->ny) == 4 && lc_edge(lat->nz) == 4 && lat->nx <= 1024 &&
                      ((uintptr_t)occ % 4 == 0);
    const int rowB_fast = ((lat->nx + 15) & ~15) + 16;
    Plan pl;
    smc_status st = fast ? make_fast_plan<false>(R, lats, occs, &ws, m->nshells, rowB_fast, lat->nx, pl)
                         : make_plan<false>(R, lats, &ws, pl);
    if (st != SMC_OK) return st;
    if (pl.ntiles > kNoAllocMaxTiles) {
        set_error("smc_sweep_noalloc: %d link-cell tiles exceed the scratch limit of %d (use a larger tile_y/tile_z "
                  "tuning or smc_sweep)", pl.ntiles, kNoAllocMaxTiles);
        return SMC_ERR_UNSUPPORTED;
    }

    static SweepParams P;
    memset(&P, 0, sizeof P);
    P.R = 1;
    P.G = pl.G;
    P.Lx = pl.Lx;
    P.Ly = pl.Ly;
    P.Lz = pl.Lz;
    P.TY = pl.TY;
    P.TZ = pl.TZ;
    P.CB = std::min(pl.CB, pl.TY * pl.TZ);
    P.nshells = m->nshells;
    P.S = lat->nspecies;
    P.tpc = pl.tpc;
    P.warp_bytes = pl.warp_bytes;
    P.nap_cap = pl.nap_cap;
    P.rowB = fast ? pl.rowB : rowB_fast;
    for (int g = 0; g < kMaxGroups; ++g) P.lag[g] = 1;
    if (fast)
        for (int g = 0; g < pl.G; ++g) P.lag[g] = (g % pl.Ly) == 0 ? 1 : 2;
    P.skip_tile = (int)debug_skip_tile();
    P.seed = seed;
    P.timeout_ns = debug_timeout_ns();
    RepDesc &d = P.rep[0];
    d.occ = occ;
    d.e_acc = e_acc;
    d.n_acc = (long long *)n_acc;
    d.nx = lat->nx;
    d.ny = lat->ny;
    d.nz = lat->nz;
    d.NLx = d.nx / pl.Lx;
    d.NLy = d.ny / pl.Ly;
    d.NLz = d.nz / pl.Lz;
    d.NTy = (d.NLy + pl.TY - 1) / pl.TY;
    d.NTz = (d.NLz + pl.TZ - 1) / pl.TZ;
    d.tile0 = 0;
    d.rep = replica;
    d.vec = (d.nx % 16 == 0) && ((uintptr_t)occ % 16 == 0);
    P.ntiles = d.NTy * d.NTz;
    const int S = P.S;
    if (fast) {
        const int ST = S == 2 ? 2 : (S == 5 ? 5 : 8);
        for (int mm = 0; mm < m->nshells; ++mm)
            for (int A = 0; A < S; ++A)
                for (int B = 0; B < S; ++B) {
                    auto Dv = [&](int q) -> double {
                        if (q >= S) return 0.0;
                        return (double)m->v_f32[(mm * S + B) * S + q] - (double)m->v_f32[(mm * S + A) * S + q];
                    };
                    const int base = ((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies;
                    double bias = 0.0;
                    for (int q = 0; q < ST - 1; ++q) {
                        const double dq = Dv(q) - Dv(ST - 1);
                        P.D.df[base + q] = (float)dq;
                        bias += dq;
                    }
                    if (mm < 2) P.D.df[base + 7] = (float)(-8.0 * bias);
                }
    } else {
        for (int mm = 0; mm < m->nshells; ++mm)
            for (int A = 0; A < S; ++A)
                for (int B = 0; B < S; ++B)
                    for (int q = 0; q < S; ++q)
                        P.D.df[((mm * kMaxSpecies + A) * kMaxSpecies + B) * kMaxSpecies + q] =
                            (float)((double)m->v_f32[(mm * S + B) * S + q] - (double)m->v_f32[(mm * S + A) * S + q]);
    }
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
    for (int t0 = 0; t0 < nsweeps; t0 += chunk) {
        const int nc = std::min(chunk, nsweeps - t0);
        P.sweep0 = sweep0 + (uint64_t)t0;
        P.nsweeps = nc;
        P.beta_stride = constant ? 0 : nc;
        for (int t = 0; t < (constant ? 1 : nc); ++t) P.temp.beta[t] = (float)(1.0 / kT[t0 + t]);
        // the array keeps the last call's contents: zero what must start at
        // zero (ticket, abort word, flags and partial sums of this call's tiles)
        e = cudaMemsetAsync(scr, 0, kNoAllocFlagsOff + (size_t)P.ntiles * 4, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(scr + kNoAllocPartEOff, 0, (size_t)P.ntiles * 8, stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(scr + kNoAllocPartNOff, 0, (size_t)P.ntiles * 8, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(no-alloc scratch)");
        void *args[] = {(void *)&P};
        e = cudaLaunchCooperativeKernel(pl.kernel, dim3(pl.grid), dim3(pl.threads), args, pl.smem, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(no-alloc sweep)");
    }
    return SMC_OK;
}

}  // namespace smc
