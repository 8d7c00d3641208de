/*
 * smc_oracle.c -- serial CPU oracle (TEST INFRASTRUCTURE ONLY; see header).
 *
 * Every function follows the definition it names, in FP64 / int64, with no
 * blocking, fusion or reordering beyond what that definition states.  The
 * paper passages followed are cited per function.
 */
#include "smc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplications and */
/* a key-dependent xor/permutation; the key is bumped by two Weyl constants   */
/* between rounds.  The paper's GPU code draws from cuRAND (Sec. III-B); a    */
/* counter-based generator keyed by (seed, sweep, site) replaces it here.     */
/* ------------------------------------------------------------------------ */
#define PH_M0 0xD2511F53u
#define PH_M1 0xCD9E8D57u
#define PH_W0 0x9E3779B9u
#define PH_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PH_W0;
            k1 += PH_W1;
        }
        uint64_t prod0 = (uint64_t)PH_M0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)PH_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random word of site s for sweep `sweep` (counter = (s>>2, replica, sweep)). */
static uint32_t site_word(uint64_t seed, uint32_t replica, uint64_t sweep, int64_t s)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)(s >> 2), replica, (uint32_t)sweep, (uint32_t)(sweep >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[s & 3];
}

/* ------------------------------------------------------------------------ */
/* Geometry of the BCC lattice.                                              */
/* ------------------------------------------------------------------------ */
static int64_t floor_mod(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

int64_t orc_nsites(const orc_lattice *lat)
{
    return 2LL * lat->nx * lat->ny * lat->nz;
}

static void site_coords(const orc_lattice *lat, int64_t s, int *sub, int *x, int *y, int *z)
{
    *x = (int)(s % lat->nx);
    s /= lat->nx;
    *y = (int)(s % lat->ny);
    s /= lat->ny;
    *z = (int)(s % lat->nz);
    *sub = (int)(s / lat->nz);
}

static int64_t site_id(const orc_lattice *lat, int sub, int x, int y, int z)
{
    return (((int64_t)sub * lat->nz + z) * lat->ny + y) * lat->nx + x;
}

/* Site reached from s by vector v (half-lattice units): the position in
 * half units is 2*cell + sub + v; its parity gives the sublattice. */
int64_t orc_neighbor(const orc_lattice *lat, int64_t s, int vx, int vy, int vz)
{
    int sub, x, y, z;
    site_coords(lat, s, &sub, &x, &y, &z);
    int64_t px = 2LL * x + sub + vx, py = 2LL * y + sub + vy, pz = 2LL * z + sub + vz;
    int nsub = (int)floor_mod(px, 2);
    if (floor_mod(py, 2) != nsub || floor_mod(pz, 2) != nsub) return -1; /* not a BCC vector */
    int64_t cx = floor_mod((px - nsub) / 2, lat->nx);
    int64_t cy = floor_mod((py - nsub) / 2, lat->ny);
    int64_t cz = floor_mod((pz - nsub) / 2, lat->nz);
    return site_id(lat, nsub, (int)cx, (int)cy, (int)cz);
}

/* Shell vectors, each shell in lexicographic order with - before +. */
int orc_shell_vectors(int shell, int out[][3])
{
    int n = 0;
    for (int a = -2; a <= 2; ++a)
        for (int b = -2; b <= 2; ++b)
            for (int c = -2; c <= 2; ++c) {
                int ok = 0;
                if (shell == 1)
                    ok = (a == -1 || a == 1) && (b == -1 || b == 1) && (c == -1 || c == 1);
                else {
                    int even = (a % 2 == 0) && (b % 2 == 0) && (c % 2 == 0);
                    int nz = (a != 0) + (b != 0) + (c != 0);
                    if (shell == 2) ok = even && nz == 1;
                    if (shell == 3) ok = even && nz == 2;
                }
                if (ok) {
                    out[n][0] = a;
                    out[n][1] = b;
                    out[n][2] = c;
                    ++n;
                }
            }
    return n;
}

static int g_shell_n[4];
static int g_shell_v[4][12][3];
static int g_geom_ready = 0;

static void geom_init(void)
{
    if (g_geom_ready) return;
    for (int m = 1; m <= 3; ++m) g_shell_n[m] = orc_shell_vectors(m, g_shell_v[m]);
    g_geom_ready = 1;
}

/* Link-cell edge per axis (Sec. II-A; the paper's fcc runs use 4x4x4 cells). */
static int lc_edge(int n)
{
    return (n >= 8 && n % 4 == 0) ? 4 : n;
}

int orc_schedule(const orc_lattice *lat, int32_t L[3])
{
    L[0] = lc_edge(lat->nx);
    L[1] = lc_edge(lat->ny);
    L[2] = lc_edge(lat->nz);
    return 2 * L[0] * L[1] * L[2];
}

static int lattice_ok(const orc_lattice *lat)
{
    if (lat->nx < 2 || lat->ny < 2 || lat->nz < 2) return 0;
    if (lat->nspecies < 1 || lat->nspecies > ORC_MAX_SPECIES) return 0;
    if (orc_nsites(lat) >= (1LL << 31)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* Initial configuration: sites sorted by (64-bit Philox key, site id); the  */
/* first counts[0] sorted sites take species 0, the next counts[1] species 1 */
/* and so on.                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    int64_t s;
} keyrec;

static int keyrec_cmp(const void *pa, const void *pb)
{
    const keyrec *a = (const keyrec *)pa, *b = (const keyrec *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->s != b->s) return a->s < b->s ? -1 : 1;
    return 0;
}

int orc_init_lattice(const orc_lattice *lat, const int64_t *counts, uint64_t seed,
                     uint32_t replica, int8_t *occ)
{
    if (!lattice_ok(lat)) return -1;
    int64_t N = orc_nsites(lat), tot = 0;
    for (int p = 0; p < lat->nspecies; ++p) {
        if (counts[p] < 0) return -1;
        tot += counts[p];
    }
    if (tot != N) return -1;
    keyrec *rec = (keyrec *)malloc(sizeof(keyrec) * (size_t)N);
    if (!rec) return -1;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t s = 0; s < N; ++s) {
        uint32_t hi[4], lo[4];
        uint32_t ca[4] = {(uint32_t)(s >> 2), replica, 0xFFFFFFFEu, 0xFFFFFFFFu};
        uint32_t cb[4] = {(uint32_t)(s >> 2), replica, 0xFFFFFFFFu, 0xFFFFFFFFu};
        orc_philox4x32_10(ca, key, hi);
        orc_philox4x32_10(cb, key, lo);
        rec[s].key = ((uint64_t)hi[s & 3] << 32) | (uint64_t)lo[s & 3];
        rec[s].s = s;
    }
    qsort(rec, (size_t)N, sizeof(keyrec), keyrec_cmp);
    int64_t pos = 0;
    for (int p = 0; p < lat->nspecies; ++p)
        for (int64_t c = 0; c < counts[p]; ++c) occ[rec[pos++].s] = (int8_t)p;
    free(rec);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Site energies.                                                            */
/*  pair:  e_i = 1/2 sum_{m} sum_{v in shell m} V_m(sigma_i, sigma_{i+v})    */
/*         (effective pair interactions, Sec. IV-B; E = sum_i e_i counts     */
/*          every bond once);                                               */
/*  MLP:   e_i = f(x_i), x_i = [onehot(sigma_i) | shell-1 counts | shell-2  */
/*         counts | shell-3 counts] (5 each), f = W3 silu(W2 silu(W1 x + b1) */
/*         + b2) + b3 (MLPNet, Sec. IV-B, with SiLU and widths 20-64-64-1).  */
/* ------------------------------------------------------------------------ */
static double silu(double z)
{
    return z / (1.0 + exp(-z));
}

double orc_mlp_eval(const orc_model *m, const double x[ORC_MLP_IN])
{
    double h1[ORC_MLP_HID], h2[ORC_MLP_HID];
    for (int j = 0; j < ORC_MLP_HID; ++j) {
        double z = m->b1[j];
        for (int i = 0; i < ORC_MLP_IN; ++i) z += m->w1[j * ORC_MLP_IN + i] * x[i];
        h1[j] = silu(z);
    }
    for (int k = 0; k < ORC_MLP_HID; ++k) {
        double z = m->b2[k];
        for (int j = 0; j < ORC_MLP_HID; ++j) z += m->w2[k * ORC_MLP_HID + j] * h1[j];
        h2[k] = silu(z);
    }
    double f = m->b3;
    for (int k = 0; k < ORC_MLP_HID; ++k) f += m->w3[k] * h2[k];
    return f;
}

/* MLPNet (Sec. IV-B): an input layer and two hidden layers of 96 units,
 * each followed by ReLU, then a linear regression layer:
 *   h1 = relu(W0 x + b0), h2 = relu(W1 h1 + b1), h3 = relu(W2 h2 + b2),
 *   f = W3 h3 + b3. */
static double relu(double z)
{
    return z > 0.0 ? z : 0.0;
}

double orc_mlpnet_eval(const orc_model *m, const double x[ORC_MLP_IN])
{
    double h1[ORC_NET_HID], h2[ORC_NET_HID], h3[ORC_NET_HID];
    for (int j = 0; j < ORC_NET_HID; ++j) {
        double z = m->net_b0[j];
        for (int i = 0; i < ORC_MLP_IN; ++i) z += m->net_w0[j * ORC_MLP_IN + i] * x[i];
        h1[j] = relu(z);
    }
    for (int k = 0; k < ORC_NET_HID; ++k) {
        double z = m->net_b1[k];
        for (int j = 0; j < ORC_NET_HID; ++j) z += m->net_w1[k * ORC_NET_HID + j] * h1[j];
        h2[k] = relu(z);
    }
    for (int k = 0; k < ORC_NET_HID; ++k) {
        double z = m->net_b2[k];
        for (int j = 0; j < ORC_NET_HID; ++j) z += m->net_w2[k * ORC_NET_HID + j] * h2[j];
        h3[k] = relu(z);
    }
    double f = m->net_b3;
    for (int k = 0; k < ORC_NET_HID; ++k) f += m->net_w3[k] * h3[k];
    return f;
}

static void mlp_features(const orc_lattice *lat, const int8_t *occ, int64_t i, double x[ORC_MLP_IN])
{
    for (int t = 0; t < ORC_MLP_IN; ++t) x[t] = 0.0;
    x[occ[i]] = 1.0;
    for (int m = 1; m <= 3; ++m)
        for (int t = 0; t < g_shell_n[m]; ++t) {
            const int *v = g_shell_v[m][t];
            int64_t j = orc_neighbor(lat, i, v[0], v[1], v[2]);
            x[ORC_MLP_SPECIES * m + occ[j]] += 1.0;
        }
}

static int has_pair(const orc_model *m)
{
    return m->kind == ORC_PAIR_I32 || m->kind == ORC_PAIR_F32 || m->kind == ORC_PAIR_F32_MLP;
}

static int has_mlp(const orc_model *m)
{
    return m->kind == ORC_MLP || m->kind == ORC_PAIR_F32_MLP;
}

#define ORC_MAX_NEIGH 24 /* largest shell of either lattice (FCC shell 3) */

/* Local energy of the qSRO model (Sec. IV-B, Eq. quadratic_local_SRO):
 *   E_i = sum_{m, p' <= p} V_m^{pp'} pi_m^{pp'} + sum_{m, p} W_m^p (pi_m^{pp})^2 + C,
 *   pi_m^{pp'} = n_m^{pp'} / sum_{pp'} n_m^{pp'},
 * with n_m^{pp'} the number of pairs (i, j), j in shell m of i, whose two
 * species are {p, p'} (counted once per unordered pair, p' <= p).  The
 * linear sum runs over p' <= p, same-element pairs included; the constant
 * lambda sum W^2 (a training regulariser) is left out.
 * qsro_shell_terms: the shell-sh part of E_i from the species q[0..z-1] of
 * the z shell-sh neighbours of a site of species si (any lattice). */
static double qsro_shell_terms(const orc_model *m, int S, int sh, int si, const int *q, int z)
{
    double n[ORC_MAX_SPECIES][ORC_MAX_SPECIES];
    memset(n, 0, sizeof n);
    double total = 0.0;
    for (int t = 0; t < z; ++t) {
        int p = si, r = q[t];
        if (r > p) {
            int tmp = p;
            p = r;
            r = tmp;
        }
        n[p][r] += 1.0;
        total += 1.0;
    }
    double e = 0.0;
    for (int p = 0; p < S; ++p)
        for (int r = 0; r <= p; ++r) e += (double)m->v_f32[((sh - 1) * S + p) * S + r] * (n[p][r] / total);
    for (int p = 0; p < S; ++p) {
        double pi = n[p][p] / total;
        e += (double)m->qsro_w[(sh - 1) * S + p] * pi * pi;
    }
    return e;
}

static double qsro_site_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ, int64_t i)
{
    double e = m->qsro_c;
    int q[ORC_MAX_NEIGH];
    for (int sh = 1; sh <= m->nshells; ++sh) {
        for (int t = 0; t < g_shell_n[sh]; ++t) {
            const int *v = g_shell_v[sh][t];
            q[t] = occ[orc_neighbor(lat, i, v[0], v[1], v[2])];
        }
        e += qsro_shell_terms(m, lat->nspecies, sh, occ[i], q, g_shell_n[sh]);
    }
    return e;
}

/* Twice the pair site energy of an integer model (an integer). */
static int64_t site_energy2_i64(const orc_lattice *lat, const orc_model *m, const int8_t *occ, int64_t i)
{
    int S = lat->nspecies;
    int64_t e2 = 0;
    for (int sh = 1; sh <= m->nshells; ++sh)
        for (int t = 0; t < g_shell_n[sh]; ++t) {
            const int *v = g_shell_v[sh][t];
            int64_t j = orc_neighbor(lat, i, v[0], v[1], v[2]);
            e2 += m->v_i32[((sh - 1) * S + occ[i]) * S + occ[j]];
        }
    return e2;
}

double orc_site_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ, int64_t i)
{
    geom_init();
    int S = lat->nspecies;
    double e = 0.0;
    if (m->kind == ORC_PAIR_I32) return 0.5 * (double)site_energy2_i64(lat, m, occ, i);
    if (m->kind == ORC_QSRO) return qsro_site_energy(lat, m, occ, i);
    if (m->kind == ORC_MLPNET) {
        double x[ORC_MLP_IN];
        mlp_features(lat, occ, i, x);
        return orc_mlpnet_eval(m, x);
    }
    if (has_pair(m)) {
        double sum = 0.0;
        for (int sh = 1; sh <= m->nshells; ++sh)
            for (int t = 0; t < g_shell_n[sh]; ++t) {
                const int *v = g_shell_v[sh][t];
                int64_t j = orc_neighbor(lat, i, v[0], v[1], v[2]);
                sum += (double)m->v_f32[((sh - 1) * S + occ[i]) * S + occ[j]];
            }
        e += 0.5 * sum;
    }
    if (has_mlp(m)) {
        double x[ORC_MLP_IN];
        mlp_features(lat, occ, i, x);
        e += orc_mlp_eval(m, x);
    }
    return e;
}

double orc_total_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ)
{
    geom_init();
    if (m->kind == ORC_PAIR_I32) return (double)orc_total_energy_i64(lat, m, occ);
    double e = 0.0;
    int64_t N = orc_nsites(lat);
    for (int64_t i = 0; i < N; ++i) e += orc_site_energy(lat, m, occ, i);
    return e;
}

int64_t orc_total_energy_i64(const orc_lattice *lat, const orc_model *m, const int8_t *occ)
{
    geom_init();
    int64_t N = orc_nsites(lat), e2 = 0;
    for (int64_t i = 0; i < N; ++i) e2 += site_energy2_i64(lat, m, occ, i);
    return e2 / 2; /* every bond is counted from both ends, so e2 is even */
}

/* Reach of the model in shells: a site energy depends on the sites this many
 * shells away. */
static int model_reach(const orc_model *m)
{
    int r = (has_pair(m) || m->kind == ORC_QSRO) ? m->nshells : 0;
    if ((has_mlp(m) || m->kind == ORC_MLPNET) && r < 3) r = 3;
    return r;
}

static int cmp_i64(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Omega(a, b): the sites whose local energy can change when a and b swap --
 * a, b and every site within the model's reach of either (the local
 * interaction zone of Sec. II-A), without duplicates. */
static int build_omega(const orc_lattice *lat, const orc_model *m, int64_t a, int64_t b, int64_t *om)
{
    int n = 0, reach = model_reach(m);
    om[n++] = a;
    om[n++] = b;
    for (int sh = 1; sh <= reach; ++sh)
        for (int t = 0; t < g_shell_n[sh]; ++t) {
            const int *v = g_shell_v[sh][t];
            om[n++] = orc_neighbor(lat, a, v[0], v[1], v[2]);
            om[n++] = orc_neighbor(lat, b, v[0], v[1], v[2]);
        }
    qsort(om, (size_t)n, sizeof(int64_t), cmp_i64);
    int u = 0;
    for (int t = 0; t < n; ++t)
        if (u == 0 || om[t] != om[u - 1]) om[u++] = om[t];
    return u;
}

/* dE of swapping a and b, by Algorithm 1: local energies of Omega
 * before (E0) and after (E1) the swap, reduced over Omega. */
double orc_delta_e(const orc_lattice *lat, const orc_model *m, int8_t *occ, int64_t a, int64_t b)
{
    geom_init();
    int64_t om[2 + 4 * 26];
    int n = build_omega(lat, m, a, b, om);
    int8_t sa = occ[a], sb = occ[b];
    if (m->kind == ORC_PAIR_I32) {
        int64_t e0 = 0, e1 = 0;
        for (int t = 0; t < n; ++t) e0 += site_energy2_i64(lat, m, occ, om[t]);
        occ[a] = sb;
        occ[b] = sa;
        for (int t = 0; t < n; ++t) e1 += site_energy2_i64(lat, m, occ, om[t]);
        occ[a] = sa;
        occ[b] = sb;
        return (double)((e1 - e0) / 2);
    }
    double e0 = 0.0, e1 = 0.0;
    for (int t = 0; t < n; ++t) e0 += orc_site_energy(lat, m, occ, om[t]);
    occ[a] = sb;
    occ[b] = sa;
    for (int t = 0; t < n; ++t) e1 += orc_site_energy(lat, m, occ, om[t]);
    occ[a] = sa;
    occ[b] = sb;
    return e1 - e0;
}

/* ------------------------------------------------------------------------ */
/* Pair counts and Warren-Cowley SRO.  n_m^{pq} = #{(i, v in shell m):      */
/* sigma_i = p, sigma_{i+v} = q} (the pair numbers behind pi_m^{pp'} of     */
/* Eq. 2); alpha_m^{pq} = 1 - n_m^{pq} / (N c_p z_m c_q).                    */
/* ------------------------------------------------------------------------ */
void orc_pair_counts(const orc_lattice *lat, int nshells, const int8_t *occ, int64_t *counts)
{
    geom_init();
    int S = lat->nspecies;
    memset(counts, 0, sizeof(int64_t) * (size_t)(nshells * S * S));
    int64_t N = orc_nsites(lat);
    for (int64_t i = 0; i < N; ++i)
        for (int sh = 1; sh <= nshells; ++sh)
            for (int t = 0; t < g_shell_n[sh]; ++t) {
                const int *v = g_shell_v[sh][t];
                int64_t j = orc_neighbor(lat, i, v[0], v[1], v[2]);
                counts[((sh - 1) * S + occ[i]) * S + occ[j]] += 1;
            }
}

void orc_sro(const orc_lattice *lat, int nshells, const int8_t *occ, double *alpha)
{
    geom_init();
    int S = lat->nspecies;
    int64_t N = orc_nsites(lat);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nshells * S * S));
    int64_t Np[ORC_MAX_SPECIES] = {0};
    for (int64_t i = 0; i < N; ++i) Np[occ[i]] += 1;
    orc_pair_counts(lat, nshells, occ, cnt);
    for (int sh = 1; sh <= nshells; ++sh)
        for (int p = 0; p < S; ++p)
            for (int q = 0; q < S; ++q) {
                int idx = ((sh - 1) * S + p) * S + q;
                if (Np[p] == 0 || Np[q] == 0) {
                    alpha[idx] = NAN;
                    continue;
                }
                double cp = (double)Np[p] / (double)N, cq = (double)Np[q] / (double)N;
                alpha[idx] = 1.0 - (double)cnt[idx] / ((double)N * cp * (double)g_shell_n[sh] * cq);
            }
    free(cnt);
}

/* ------------------------------------------------------------------------ */
/* Metropolis criterion (Algorithm 1).                                */
/* ------------------------------------------------------------------------ */
#define R_BITS 29
#define R_SCALE 536870912.0 /* 2^29 */

int64_t orc_accept_table(double unit_ev, double kT, uint32_t *table, int64_t cap)
{
    int64_t d = 0;
    for (;;) {
        double t = floor(R_SCALE * exp(-(double)d * unit_ev / kT));
        if (t <= 0.0) return d;
        if (d < cap) table[d] = (uint32_t)t;
        ++d;
        if (d > (1LL << 26)) return -1;
    }
}

static int accept_fp(double dE, uint32_t r, double kT)
{
    if (dE <= 0.0) return 1;
    double u = ((double)r + 0.5) / R_SCALE;
    return u < exp(-dE / kT);
}

static int accept_int(int64_t dE, uint32_t r, const uint32_t *T, int64_t len)
{
    if (dE <= 0) return 1;
    return dE < len && r < T[dE];
}

/* ------------------------------------------------------------------------ */
/* Sweeps (Algorithm 1): n_A sequential mini-steps; in mini-step k every    */
/* link cell tries to swap its site at offset o_k with a random nearest      */
/* neighbour.                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L[3], NL[3], nA;
} sched;

static void make_sched(const orc_lattice *lat, sched *sc)
{
    sc->nA = orc_schedule(lat, sc->L);
    sc->NL[0] = lat->nx / sc->L[0];
    sc->NL[1] = lat->ny / sc->L[1];
    sc->NL[2] = lat->nz / sc->L[2];
}

/* Site a of link cell c in mini-step k. */
static int64_t trial_site(const orc_lattice *lat, const sched *sc, int k, int64_t c)
{
    int dx = k % sc->L[0];
    int r = k / sc->L[0];
    int dy = r % sc->L[1];
    r /= sc->L[1];
    int dz = r % sc->L[2];
    int sub = r / sc->L[2];
    int cx = (int)(c % sc->NL[0]);
    int64_t rc = c / sc->NL[0];
    int cy = (int)(rc % sc->NL[1]);
    int cz = (int)(rc / sc->NL[1]);
    return site_id(lat, sub, cx * sc->L[0] + dx, cy * sc->L[1] + dy, cz * sc->L[2] + dz);
}

typedef struct {
    uint32_t *T;
    int64_t len;
} acc_tab;

static int make_table(const orc_model *m, double kT, acc_tab *at)
{
    at->T = NULL;
    at->len = 0;
    if (m->kind != ORC_PAIR_I32) return 0;
    if (!(kT > 0.0) || isinf(kT)) return -1;
    int64_t len = orc_accept_table(m->unit_ev, kT, NULL, 0);
    if (len < 0) return -1;
    at->T = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(len > 0 ? len : 1));
    orc_accept_table(m->unit_ev, kT, at->T, len);
    at->len = len;
    return 0;
}

/* One trial at site a of `lat` whose random word is that of site id `a_rng`
 * (the same site in the whole box; a_rng = a unless `lat` is one slab of it).
 * Returns 1 if accepted; *dE_out gets dE. */
static int one_trial_at(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
                        uint32_t replica, uint64_t sweep, int64_t a, int64_t a_rng, double kT,
                        const acc_tab *at, double *dE_out, int64_t *b_out)
{
    uint32_t w = site_word(seed, replica, sweep, a_rng);
    int dir = (int)(w >> R_BITS);
    uint32_t r = w & ((1u << R_BITS) - 1u);
    const int *v = g_shell_v[1][dir];
    int64_t b = orc_neighbor(lat, a, v[0], v[1], v[2]);
    double dE = orc_delta_e(lat, m, occ, a, b);
    int acc;
    if (m->kind == ORC_PAIR_I32)
        acc = accept_int((int64_t)dE, r, at->T, at->len);
    else
        acc = accept_fp(dE, r, kT);
    if (acc) {
        int8_t t = occ[a];
        occ[a] = occ[b];
        occ[b] = t;
    }
    *dE_out = dE;
    if (b_out) *b_out = b;
    return acc;
}

static int one_trial(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
                     uint32_t replica, uint64_t sweep, int64_t a, double kT, const acc_tab *at,
                     double *dE_out, int64_t *b_out)
{
    return one_trial_at(lat, m, occ, seed, replica, sweep, a, a, kT, at, dE_out, b_out);
}

/* The steps of Algorithm 1 in its order, for one mini-step: sigma1 = sigma0, every trial
 * swapped in sigma1, local energies E0 (sigma0) and E1 (sigma1) of all sites,
 * reduction over each Omega, Metropolis, accepted sites copied to sigma0. */
static void ministep_literal(const orc_lattice *lat, const orc_model *m, int8_t *occ,
                             const sched *sc, int k, uint64_t seed, uint32_t replica,
                             uint64_t sweep, double kT, const acc_tab *at, double *e_acc,
                             int64_t *n_acc)
{
    int64_t N = orc_nsites(lat), NC = N / sc->nA;
    int8_t *s1 = (int8_t *)malloc((size_t)N);
    double *E0 = (double *)malloc(sizeof(double) * (size_t)N);
    double *E1 = (double *)malloc(sizeof(double) * (size_t)N);
    int64_t *A = (int64_t *)malloc(sizeof(int64_t) * (size_t)NC);
    int64_t *B = (int64_t *)malloc(sizeof(int64_t) * (size_t)NC);
    uint32_t *R = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)NC);
    memcpy(s1, occ, (size_t)N); /* the auxiliary copy sigma1 */
    for (int64_t c = 0; c < NC; ++c) {
        int64_t a = trial_site(lat, sc, k, c);
        uint32_t w = site_word(seed, replica, sweep, a);
        const int *v = g_shell_v[1][w >> R_BITS];
        A[c] = a;
        B[c] = orc_neighbor(lat, a, v[0], v[1], v[2]);
        R[c] = w & ((1u << R_BITS) - 1u);
    }
    for (int64_t c = 0; c < NC; ++c) { /* every trial swap made in sigma1 */
        int8_t t = s1[A[c]];
        s1[A[c]] = s1[B[c]];
        s1[B[c]] = t;
    }
    for (int64_t i = 0; i < N; ++i) { /* local energies E0 of sigma0, E1 of sigma1 */
        if (m->kind == ORC_PAIR_I32) {
            E0[i] = (double)site_energy2_i64(lat, m, occ, i);
            E1[i] = (double)site_energy2_i64(lat, m, s1, i);
        } else {
            E0[i] = orc_site_energy(lat, m, occ, i);
            E1[i] = orc_site_energy(lat, m, s1, i);
        }
    }
    int64_t om[2 + 4 * 26];
    for (int64_t c = 0; c < NC; ++c) {
        int n = build_omega(lat, m, A[c], B[c], om);
        double eb0 = 0.0, eb1 = 0.0; /* the reductions over Omega */
        for (int t = 0; t < n; ++t) {
            eb0 += E0[om[t]];
            eb1 += E1[om[t]];
        }
        double dE = eb1 - eb0;
        int acc;
        if (m->kind == ORC_PAIR_I32) {
            dE = dE / 2.0; /* doubled integer site energies */
            acc = accept_int((int64_t)dE, R[c], at->T, at->len);
        } else {
            acc = accept_fp(dE, R[c], kT);
        }
        if (acc) { /* an accepted swap is copied back to sigma0 */
            occ[A[c]] = s1[A[c]];
            occ[B[c]] = s1[B[c]];
            if (e_acc) *e_acc += dE;
            if (n_acc) *n_acc += 1;
        }
    }
    free(s1);
    free(E0);
    free(E1);
    free(A);
    free(B);
    free(R);
}

static int model_ok(const orc_lattice *lat, const orc_model *m)
{
    if (m->kind < ORC_PAIR_I32 || m->kind > ORC_MLPNET) return 0;
    if (m->kind == ORC_MLPNET && (!m->net_w0 || !m->net_w1 || !m->net_w2 || !m->net_w3 || !m->net_b0 ||
                                  !m->net_b1 || !m->net_b2 || lat->nspecies > ORC_MLP_SPECIES))
        return 0;
    if ((has_pair(m) || m->kind == ORC_QSRO) && (m->nshells < 1 || m->nshells > 3)) return 0;
    if (m->kind == ORC_QSRO && (!m->v_f32 || !m->qsro_w)) return 0;
    if (m->kind == ORC_PAIR_I32 && (!m->v_i32 || !(m->unit_ev > 0.0))) return 0;
    if ((m->kind == ORC_PAIR_F32 || m->kind == ORC_PAIR_F32_MLP) && !m->v_f32) return 0;
    if (has_mlp(m) && (!m->w1 || !m->w2 || !m->w3 || !m->b1 || !m->b2)) return 0;
    if (has_mlp(m) && lat->nspecies > ORC_MLP_SPECIES) return 0;
    return 1;
}

int orc_sweep(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
              uint32_t replica, uint64_t sweep0, int32_t nsweeps, const double *kT,
              double *e_acc, int64_t *n_acc, int mode)
{
    geom_init();
    if (!lattice_ok(lat) || !model_ok(lat, m) || nsweeps < 0) return -1;
    sched sc;
    make_sched(lat, &sc);
    int64_t NC = orc_nsites(lat) / sc.nA;
    for (int32_t t = 0; t < nsweeps; ++t) {
        uint64_t sweep = sweep0 + (uint64_t)t;
        acc_tab at;
        if (make_table(m, kT[t], &at) != 0) return -1;
        for (int k = 0; k < sc.nA; ++k) {
            if (mode == 1) {
                ministep_literal(lat, m, occ, &sc, k, seed, replica, sweep, kT[t], &at, e_acc, n_acc);
                continue;
            }
            for (int64_t c = 0; c < NC; ++c) {
                int64_t a = trial_site(lat, &sc, k, c);
                double dE;
                if (one_trial(lat, m, occ, seed, replica, sweep, a, kT[t], &at, &dE, NULL)) {
                    if (e_acc) *e_acc += dE;
                    if (n_acc) *n_acc += 1;
                }
            }
        }
        free(at.T);
    }
    return 0;
}

int64_t orc_ministep_trace(const orc_lattice *lat, const orc_model *m, int8_t *occ,
                           uint64_t seed, uint32_t replica, uint64_t sweep, int32_t k,
                           double kT, double *dE, uint8_t *acc, int64_t *site_a,
                           int64_t *site_b)
{
    geom_init();
    if (!lattice_ok(lat) || !model_ok(lat, m)) return -1;
    sched sc;
    make_sched(lat, &sc);
    if (k < 0 || k >= sc.nA) return -1;
    acc_tab at;
    if (make_table(m, kT, &at) != 0) return -1;
    int64_t NC = orc_nsites(lat) / sc.nA;
    for (int64_t c = 0; c < NC; ++c) {
        int64_t a = trial_site(lat, &sc, k, c), b;
        double d;
        int ac = one_trial(lat, m, occ, seed, replica, sweep, a, kT, &at, &d, &b);
        if (dE) dE[c] = d;
        if (acc) acc[c] = (uint8_t)ac;
        if (site_a) site_a[c] = a;
        if (site_b) site_b[c] = b;
    }
    free(at.T);
    return NC;
}

/* ------------------------------------------------------------------------ */
/* One x-slab of the box (Sec. III-B, 1D slab decomposition).  A slab owns   */
/* the cells x0 <= x < x0 + w of every sublattice, y and z, and holds g more */
/* cells on each side (ghosts, x taken modulo nx) in occ_loc, laid out as a  */
/* box of w + 2g cells along x: [sub][z][y][x - x0 + g].  The trials of      */
/* mini-step k whose site lies in the slab run exactly as in the whole box:  */
/* same link cells in the same order, random words of the global site ids.   */
/* Reads reach g cells past the slab at most, so the local box never wraps.  */
/* ------------------------------------------------------------------------ */

/* Cells a trial reads beyond its own cell along x.  Positions along x are
 * integers (sublattice 0) or half-integers (sublattice 1) in units of the
 * cell edge.  The partner b sits 1/2 away; every shell-1..3 vector moves x
 * by 1 at most.  Pair models read the shells of a and b: 1.5 from a, which
 * is 2 cells.  MLP and qSRO models change the energies of Omega (a, b and
 * their shell neighbours, 1.5 from a), and each of those reads its own
 * shells: 2.5 from a, which is 3 cells. */
int orc_slab_ghost_cells(const orc_model *m)
{
    return (has_mlp(m) || m->kind == ORC_QSRO || m->kind == ORC_MLPNET) ? 3 : 2;
}

int64_t orc_slab_ministep(const orc_lattice *glat, const orc_model *m, int8_t *occ_loc,
                          int32_t x0, int32_t w, int32_t g, uint64_t seed, uint32_t replica,
                          uint64_t sweep, int32_t k, double kT, double *e_acc, int64_t *n_acc)
{
    geom_init();
    if (!lattice_ok(glat) || !model_ok(glat, m)) return -1;
    sched sc;
    make_sched(glat, &sc);
    if (glat->nx < 8 || sc.L[0] != 4 || k < 0 || k >= sc.nA) return -1;
    if (x0 < 0 || w < 4 || x0 % 4 != 0 || w % 4 != 0 || x0 + w > glat->nx) return -1;
    if (g < orc_slab_ghost_cells(m) || g > w) return -1;
    orc_lattice loc = *glat;
    loc.nx = w + 2 * g;
    if (!lattice_ok(&loc)) return -1;
    acc_tab at;
    if (make_table(m, kT, &at) != 0) return -1;
    int dx = k % 4, r = k / 4;
    int dy = r % sc.L[1];
    r /= sc.L[1];
    int dz = r % sc.L[2];
    int sub = r / sc.L[2];
    int64_t nt = 0;
    for (int cz = 0; cz < sc.NL[2]; ++cz)
        for (int cy = 0; cy < sc.NL[1]; ++cy)
            for (int cx = x0 / 4; cx < (x0 + w) / 4; ++cx) {
                int x = cx * 4 + dx, y = cy * sc.L[1] + dy, z = cz * sc.L[2] + dz;
                int64_t a_glob = site_id(glat, sub, x, y, z);
                int64_t a_loc = site_id(&loc, sub, x - x0 + g, y, z);
                double dE;
                if (one_trial_at(&loc, m, occ_loc, seed, replica, sweep, a_loc, a_glob, kT, &at, &dE, NULL)) {
                    if (e_acc) *e_acc += dE;
                    if (n_acc) *n_acc += 1;
                }
                ++nt;
            }
    free(at.T);
    return nt;
}

/* ------------------------------------------------------------------------ */
/* dE/dtheta.  Pair parameters V_m(p, q) = V_m(q, p), one per unordered      */
/* {p, q}: the derivative of E = sum_i 1/2 sum_v V(sigma_i, sigma_{i+v}) is  */
/* accumulated term by term.  MLP parameters: back-propagation of every     */
/* site function f(x_i), summed over sites.                                  */
/* ------------------------------------------------------------------------ */
#define MLP_NPARAM (ORC_MLP_HID * ORC_MLP_IN + ORC_MLP_HID + ORC_MLP_HID * ORC_MLP_HID + ORC_MLP_HID + ORC_MLP_HID + 1)

static int pair_param_index(int S, int p, int q)
{
    if (p > q) {
        int t = p;
        p = q;
        q = t;
    }
    /* rows p = 0..S-1 with q = p..S-1 */
    return p * S - p * (p - 1) / 2 + (q - p);
}

int64_t orc_grad_size(const orc_lattice *lat, const orc_model *m)
{
    int S = lat->nspecies;
    int64_t n = 0;
    if (has_pair(m)) n += (int64_t)m->nshells * S * (S + 1) / 2;
    if (has_mlp(m)) n += MLP_NPARAM;
    if (m->kind == ORC_QSRO) n += (int64_t)m->nshells * S * (S + 1) / 2 + (int64_t)m->nshells * S + 1;
    return n;
}

/* dE/dtheta of the qSRO energy (Eq. quadratic_local_SRO), term by term:
 * dE/dV_m^{pp'} = sum_i pi_m^{pp'}(i) (one parameter per unordered pair),
 * dE/dW_m^p = sum_i pi_m^{pp}(i)^2, dE/dC = N. */
static void qsro_grad(const orc_lattice *lat, const orc_model *m, const int8_t *occ, double *grad)
{
    int S = lat->nspecies, per = S * (S + 1) / 2;
    int64_t N = orc_nsites(lat);
    double *gV = grad, *gW = grad + (int64_t)m->nshells * per, *gC = gW + (int64_t)m->nshells * S;
    for (int64_t i = 0; i < N; ++i)
        for (int sh = 1; sh <= m->nshells; ++sh) {
            double n[ORC_MAX_SPECIES][ORC_MAX_SPECIES];
            memset(n, 0, sizeof n);
            double total = 0.0;
            for (int t = 0; t < g_shell_n[sh]; ++t) {
                const int *v = g_shell_v[sh][t];
                int64_t j = orc_neighbor(lat, i, v[0], v[1], v[2]);
                int p = occ[i], q = occ[j];
                if (q > p) {
                    int tmp = p;
                    p = q;
                    q = tmp;
                }
                n[p][q] += 1.0;
                total += 1.0;
            }
            for (int p = 0; p < S; ++p)
                for (int q = 0; q <= p; ++q) gV[(sh - 1) * per + pair_param_index(S, p, q)] += n[p][q] / total;
            for (int p = 0; p < S; ++p) {
                double pi = n[p][p] / total;
                gW[(sh - 1) * S + p] += pi * pi;
            }
        }
    *gC = (double)N;
}

static double dsilu(double z)
{
    double sg = 1.0 / (1.0 + exp(-z));
    return sg * (1.0 + z * (1.0 - sg));
}

/* Adds d f(x)/d theta to g (layout W1, b1, W2, b2, W3, b3). */
static void mlp_backprop(const orc_model *m, const double x[ORC_MLP_IN], double *g)
{
    double z1[ORC_MLP_HID], h1[ORC_MLP_HID], z2[ORC_MLP_HID], h2[ORC_MLP_HID];
    double d2[ORC_MLP_HID], d1[ORC_MLP_HID];
    for (int j = 0; j < ORC_MLP_HID; ++j) {
        double z = m->b1[j];
        for (int i = 0; i < ORC_MLP_IN; ++i) z += m->w1[j * ORC_MLP_IN + i] * x[i];
        z1[j] = z;
        h1[j] = silu(z);
    }
    for (int k = 0; k < ORC_MLP_HID; ++k) {
        double z = m->b2[k];
        for (int j = 0; j < ORC_MLP_HID; ++j) z += m->w2[k * ORC_MLP_HID + j] * h1[j];
        z2[k] = z;
        h2[k] = silu(z);
    }
    double *gW1 = g, *gb1 = gW1 + ORC_MLP_HID * ORC_MLP_IN, *gW2 = gb1 + ORC_MLP_HID;
    double *gb2 = gW2 + ORC_MLP_HID * ORC_MLP_HID, *gW3 = gb2 + ORC_MLP_HID, *gb3 = gW3 + ORC_MLP_HID;
    gb3[0] += 1.0;
    for (int k = 0; k < ORC_MLP_HID; ++k) {
        gW3[k] += h2[k];
        d2[k] = m->w3[k] * dsilu(z2[k]);
        gb2[k] += d2[k];
        for (int j = 0; j < ORC_MLP_HID; ++j) gW2[k * ORC_MLP_HID + j] += d2[k] * h1[j];
    }
    for (int j = 0; j < ORC_MLP_HID; ++j) {
        double s = 0.0;
        for (int k = 0; k < ORC_MLP_HID; ++k) s += m->w2[k * ORC_MLP_HID + j] * d2[k];
        d1[j] = s * dsilu(z1[j]);
        gb1[j] += d1[j];
        for (int i = 0; i < ORC_MLP_IN; ++i) gW1[j * ORC_MLP_IN + i] += d1[j] * x[i];
    }
}

int orc_energy_grad(const orc_lattice *lat, const orc_model *m, const int8_t *occ, double *grad)
{
    geom_init();
    if (!lattice_ok(lat) || !model_ok(lat, m) || m->kind == ORC_MLPNET) return -1;
    int S = lat->nspecies;
    int64_t n = orc_grad_size(lat, m), N = orc_nsites(lat);
    for (int64_t t = 0; t < n; ++t) grad[t] = 0.0;
    if (m->kind == ORC_QSRO) {
        qsro_grad(lat, m, occ, grad);
        return 0;
    }
    double *gm = grad;
    if (has_pair(m)) {
        int per = S * (S + 1) / 2;
        for (int64_t i = 0; i < N; ++i)
            for (int sh = 1; sh <= m->nshells; ++sh)
                for (int t = 0; t < g_shell_n[sh]; ++t) {
                    const int *v = g_shell_v[sh][t];
                    int64_t j = orc_neighbor(lat, i, v[0], v[1], v[2]);
                    grad[(sh - 1) * per + pair_param_index(S, occ[i], occ[j])] += 0.5;
                }
        gm = grad + (int64_t)m->nshells * per;
    }
    if (has_mlp(m)) {
        double x[ORC_MLP_IN];
        for (int64_t i = 0; i < N; ++i) {
            mlp_features(lat, occ, i, x);
            mlp_backprop(m, x, gm);
        }
    }
    return 0;
}

/* ======================================================================== */
/* FCC lattice (the paper's lattice, Sec. IV-C and Sec. V-C), pair and qSRO */
/* models.                                                                   */
/* nx x ny x nz cubic cells (each >= 1), 4 sites per cell at the half-unit   */
/* offsets (0,0,0), (1,1,0), (1,0,1), (0,1,1) (sublattices 0-3); site id     */
/* s = ((sub*nz + z)*ny + y)*nx + x, N = 4 nx ny nz.  Shells 1-3: 12 vectors */
/* of squared half-unit length 2, 6 of length 4, 24 of length 6, each in     */
/* lexicographic order of (vx, vy, vz).  Link cells as for BCC (edge 4 along */
/* an axis of n >= 8 cells, n % 4 == 0, else the whole axis); a sweep is     */
/* n_A = 4 Lx Ly Lz mini-steps, k = ((sub Lz + dz) Ly + dy) Lx + dx.         */
/* Random numbers: Philox4x32-10 with key seed and counter (s, replica,      */
/* sweep lo, sweep hi) per trial site s: r = word 0 & (2^29 - 1) for the     */
/* Metropolis test, partner index floor(12 word 1 / 2^32).                   */
/* ======================================================================== */
static const int g_fcc_basis[4][3] = {{0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
static int g_fcc_n[4];
static int g_fcc_v[4][24][3];
static int g_fcc_ready = 0;

int orc_fcc_shell_vectors(int shell, int out[][3])
{
    if (shell < 1 || shell > 3) return 0;
    int n = 0, want = 2 * shell;
    for (int x = -2; x <= 2; ++x)
        for (int y = -2; y <= 2; ++y)
            for (int z = -2; z <= 2; ++z)
                if (x * x + y * y + z * z == want && ((x + y + z) & 1) == 0) {
                    out[n][0] = x;
                    out[n][1] = y;
                    out[n][2] = z;
                    ++n;
                }
    return n;
}

static void fcc_init(void)
{
    if (g_fcc_ready) return;
    for (int m = 1; m <= 3; ++m) g_fcc_n[m] = orc_fcc_shell_vectors(m, g_fcc_v[m]);
    g_fcc_ready = 1;
}

int64_t orc_fcc_nsites(const orc_lattice *lat)
{
    return 4LL * lat->nx * lat->ny * lat->nz;
}

static int fcc_lattice_ok(const orc_lattice *lat)
{
    if (lat->nx < 1 || lat->ny < 1 || lat->nz < 1) return 0;
    if (lat->nspecies < 1 || lat->nspecies > ORC_MAX_SPECIES) return 0;
    return orc_fcc_nsites(lat) < (1LL << 31);
}

static int64_t fcc_site_id(const orc_lattice *lat, int sub, int x, int y, int z)
{
    return (((int64_t)sub * lat->nz + z) * lat->ny + y) * lat->nx + x;
}

/* Site reached from s by v (half units): position 2 cell + basis + v; its
 * parities name the sublattice. */
int64_t orc_fcc_neighbor(const orc_lattice *lat, int64_t s, int vx, int vy, int vz)
{
    int64_t t = s;
    int x = (int)(t % lat->nx);
    t /= lat->nx;
    int y = (int)(t % lat->ny);
    t /= lat->ny;
    int z = (int)(t % lat->nz);
    int sub = (int)(t / lat->nz);
    int64_t p[3] = {2LL * x + g_fcc_basis[sub][0] + vx, 2LL * y + g_fcc_basis[sub][1] + vy,
                    2LL * z + g_fcc_basis[sub][2] + vz};
    int par = (int)(((p[0] & 1) << 2) | ((p[1] & 1) << 1) | (p[2] & 1));
    int nsub;
    switch (par) {
    case 0: nsub = 0; break;
    case 6: nsub = 1; break;  /* (1,1,0) */
    case 5: nsub = 2; break;  /* (1,0,1) */
    case 3: nsub = 3; break;  /* (0,1,1) */
    default: return -1;
    }
    int64_t c[3];
    for (int d = 0; d < 3; ++d) c[d] = (p[d] - (p[d] & 1)) / 2;
    return fcc_site_id(lat, nsub, (int)floor_mod(c[0], lat->nx), (int)floor_mod(c[1], lat->ny),
                       (int)floor_mod(c[2], lat->nz));
}

int orc_fcc_schedule(const orc_lattice *lat, int32_t L[3])
{
    L[0] = lc_edge(lat->nx);
    L[1] = lc_edge(lat->ny);
    L[2] = lc_edge(lat->nz);
    return 4 * L[0] * L[1] * L[2];
}

static int fcc_model_ok(const orc_model *m)
{
    if (m->kind != ORC_PAIR_I32 && m->kind != ORC_PAIR_F32 && m->kind != ORC_QSRO) return 0;
    if (m->nshells < 1 || m->nshells > 3) return 0;
    if (m->kind == ORC_PAIR_I32) return m->v_i32 && m->unit_ev > 0.0;
    if (m->kind == ORC_QSRO) return m->v_f32 && m->qsro_w;
    return m->v_f32 != NULL;
}

/* qSRO local energy (Eq. quadratic_local_SRO) with the FCC shells (12, 6, 24
 * neighbours). */
static double fcc_qsro_site_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ, int64_t i)
{
    double e = m->qsro_c;
    int q[ORC_MAX_NEIGH];
    for (int sh = 1; sh <= m->nshells; ++sh) {
        for (int t = 0; t < g_fcc_n[sh]; ++t) {
            const int *v = g_fcc_v[sh][t];
            q[t] = occ[orc_fcc_neighbor(lat, i, v[0], v[1], v[2])];
        }
        e += qsro_shell_terms(m, lat->nspecies, sh, occ[i], q, g_fcc_n[sh]);
    }
    return e;
}

/* Pair models: the site energy, and twice it exactly for integer models
 * (e2).  qSRO: the local energy E_i. */
static double fcc_site_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ, int64_t i,
                              int64_t *e2)
{
    if (m->kind == ORC_QSRO) {
        if (e2) *e2 = 0;
        return fcc_qsro_site_energy(lat, m, occ, i);
    }
    int S = lat->nspecies;
    int64_t acc2 = 0;
    double acc = 0.0;
    for (int sh = 1; sh <= m->nshells; ++sh)
        for (int t = 0; t < g_fcc_n[sh]; ++t) {
            const int *v = g_fcc_v[sh][t];
            int64_t j = orc_fcc_neighbor(lat, i, v[0], v[1], v[2]);
            int idx = ((sh - 1) * S + occ[i]) * S + occ[j];
            if (m->kind == ORC_PAIR_I32)
                acc2 += m->v_i32[idx];
            else
                acc += (double)m->v_f32[idx];
        }
    if (e2) *e2 = acc2;
    return m->kind == ORC_PAIR_I32 ? 0.5 * (double)acc2 : 0.5 * acc;
}

double orc_fcc_total_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ)
{
    fcc_init();
    double e = 0.0;
    int64_t N = orc_fcc_nsites(lat);
    for (int64_t i = 0; i < N; ++i) e += fcc_site_energy(lat, m, occ, i, NULL);
    return e;
}

int64_t orc_fcc_total_energy_i64(const orc_lattice *lat, const orc_model *m, const int8_t *occ)
{
    fcc_init();
    int64_t N = orc_fcc_nsites(lat), tot = 0, e2;
    for (int64_t i = 0; i < N; ++i) {
        fcc_site_energy(lat, m, occ, i, &e2);
        tot += e2;
    }
    return tot / 2;
}

/* dE of swapping a and b: the local energies of a, b and every site within
 * the model's shells of either, before and after (Algorithm 1). */
double orc_fcc_delta_e(const orc_lattice *lat, const orc_model *m, int8_t *occ, int64_t a, int64_t b)
{
    fcc_init();
    int64_t om[2 + 2 * (12 + 6 + 24)];
    int n = 0;
    om[n++] = a;
    om[n++] = b;
    for (int sh = 1; sh <= m->nshells; ++sh)
        for (int t = 0; t < g_fcc_n[sh]; ++t) {
            const int *v = g_fcc_v[sh][t];
            om[n++] = orc_fcc_neighbor(lat, a, v[0], v[1], v[2]);
            om[n++] = orc_fcc_neighbor(lat, b, v[0], v[1], v[2]);
        }
    qsort(om, (size_t)n, sizeof(int64_t), cmp_i64);
    int u = 0;
    for (int t = 0; t < n; ++t)
        if (u == 0 || om[t] != om[u - 1]) om[u++] = om[t];
    int8_t sa = occ[a], sb = occ[b];
    int64_t e0i = 0, e1i = 0, e2;
    double e0 = 0.0, e1 = 0.0;
    for (int t = 0; t < u; ++t) {
        e0 += fcc_site_energy(lat, m, occ, om[t], &e2);
        e0i += e2;
    }
    occ[a] = sb;
    occ[b] = sa;
    for (int t = 0; t < u; ++t) {
        e1 += fcc_site_energy(lat, m, occ, om[t], &e2);
        e1i += e2;
    }
    occ[a] = sa;
    occ[b] = sb;
    if (m->kind == ORC_PAIR_I32) return (double)((e1i - e0i) / 2);
    return e1 - e0;
}

static void fcc_words(uint64_t seed, uint32_t replica, uint64_t sweep, int64_t s, uint32_t *r, int *dir)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)s, replica, (uint32_t)sweep, (uint32_t)(sweep >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    *r = out[0] & ((1u << R_BITS) - 1u);
    *dir = (int)(((uint64_t)out[1] * 12u) >> 32);
}

/* Mini-step k: every link cell's trial, in increasing link-cell order. */
static int64_t fcc_ministep(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
                            uint32_t replica, uint64_t sweep, int k, double kT, const acc_tab *at, double *dE_out,
                            uint8_t *acc_out, int64_t *a_out, int64_t *b_out, double *e_acc, int64_t *n_acc)
{
    int32_t L[3];
    int nA = orc_fcc_schedule(lat, L);
    (void)nA;
    int NL[3] = {lat->nx / L[0], lat->ny / L[1], lat->nz / L[2]};
    int dx = k % L[0], r = k / L[0];
    int dy = r % L[1];
    r /= L[1];
    int dz = r % L[2];
    int sub = r / L[2];
    int64_t c = 0;
    for (int cz = 0; cz < NL[2]; ++cz)
        for (int cy = 0; cy < NL[1]; ++cy)
            for (int cx = 0; cx < NL[0]; ++cx, ++c) {
                int64_t a = fcc_site_id(lat, sub, cx * L[0] + dx, cy * L[1] + dy, cz * L[2] + dz);
                uint32_t rr;
                int dir;
                fcc_words(seed, replica, sweep, a, &rr, &dir);
                const int *v = g_fcc_v[1][dir];
                int64_t b = orc_fcc_neighbor(lat, a, v[0], v[1], v[2]);
                double dE = orc_fcc_delta_e(lat, m, occ, a, b);
                int acc = m->kind == ORC_PAIR_I32 ? accept_int((int64_t)dE, rr, at->T, at->len)
                                                  : accept_fp(dE, rr, kT);
                if (acc) {
                    int8_t t = occ[a];
                    occ[a] = occ[b];
                    occ[b] = t;
                    if (e_acc) *e_acc += dE;
                    if (n_acc) *n_acc += 1;
                }
                if (dE_out) dE_out[c] = dE;
                if (acc_out) acc_out[c] = (uint8_t)acc;
                if (a_out) a_out[c] = a;
                if (b_out) b_out[c] = b;
            }
    return c;
}

int orc_fcc_sweep(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed, uint32_t replica,
                  uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc, int64_t *n_acc)
{
    fcc_init();
    if (!fcc_lattice_ok(lat) || !fcc_model_ok(m) || nsweeps < 0) return -1;
    int32_t L[3];
    int nA = orc_fcc_schedule(lat, L);
    for (int32_t t = 0; t < nsweeps; ++t) {
        acc_tab at;
        if (make_table(m, kT[t], &at) != 0) return -1;
        for (int k = 0; k < nA; ++k)
            fcc_ministep(lat, m, occ, seed, replica, sweep0 + (uint64_t)t, k, kT[t], &at, NULL, NULL, NULL, NULL,
                         e_acc, n_acc);
        free(at.T);
    }
    return 0;
}

int64_t orc_fcc_ministep_trace(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
                               uint32_t replica, uint64_t sweep, int32_t k, double kT, double *dE, uint8_t *acc,
                               int64_t *site_a, int64_t *site_b)
{
    fcc_init();
    if (!fcc_lattice_ok(lat) || !fcc_model_ok(m)) return -1;
    int32_t L[3];
    if (k < 0 || k >= orc_fcc_schedule(lat, L)) return -1;
    acc_tab at;
    if (make_table(m, kT, &at) != 0) return -1;
    int64_t n = fcc_ministep(lat, m, occ, seed, replica, sweep, k, kT, &at, dE, acc, site_a, site_b, NULL, NULL);
    free(at.T);
    return n;
}
