/*
 * smc_oracle.h -- serial CPU oracle for canonical swap Monte Carlo on a BCC
 * alloy lattice (SMC-X / SMC-AI, Sec. II-A and Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the parity reference for the
 * CUDA path.  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the CUDA library: geometry, Philox, acceptance tables, energies and
 * gradients are all written here again, from their definitions.
 *
 * Arithmetic: integers are exact (int64); floating point is FP64.  Model
 * parameters given in FP32 or BF16 are widened to FP64 without rounding.
 *
 * Conventions (the readings of the paper this oracle follows):
 *   - BCC site (sub, x, y, z), position (x + sub/2, y + sub/2, z + sub/2) a.
 *     Canonical id s = ((sub*nz + z)*ny + y)*nx + x.
 *   - Neighbour vectors in half-lattice-constant units h = a/2:
 *       shell 1 (8):  (+-1,+-1,+-1), ordered lexicographically, - before +;
 *       shell 2 (6):  (+-2,0,0), (0,+-2,0), (0,0,+-2);
 *       shell 3 (12): two non-zero components, each +-2.
 *   - Link cells (Sec. II-A, Algorithm 1): edge L = 4 cells along an
 *     axis whose length n is >= 8 and a multiple of 4, else L = n (one cell
 *     along that axis).  n_A = 2*Lx*Ly*Lz mini-steps per sweep; mini-step k
 *     visits offset (sub, dx, dy, dz) with k = ((sub*Lz + dz)*Ly + dy)*Lx + dx.
 *   - RNG: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo, seed hi),
 *     counter = (s >> 2, replica, sweep lo, sweep hi); site s uses output
 *     word s & 3.  Partner direction = word >> 29 (index into shell 1),
 *     acceptance number r = word & (2^29 - 1).
 *   - Metropolis (Algorithm 1): integer models accept iff dE <= 0 or
 *     r < T[dE], T[d] = floor(2^29 exp(-d*unit/kT)); floating-point models
 *     accept iff dE <= 0 or (r + 1/2) 2^-29 < exp(-dE/kT).
 */
#ifndef SMC_ORACLE_H
#define SMC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SPECIES 8
#define ORC_MLP_IN 20
#define ORC_MLP_HID 64
#define ORC_MLP_SPECIES 5
#define ORC_NET_HID 96

enum { ORC_PAIR_I32 = 0, ORC_PAIR_F32 = 1, ORC_MLP = 2, ORC_PAIR_F32_MLP = 3, ORC_QSRO = 4, ORC_MLPNET = 5 };

typedef struct {
    int32_t nx, ny, nz;   /* cells per axis, each >= 2 */
    int32_t nspecies;     /* 1 .. 8 (MLP models: <= 5) */
} orc_lattice;

/* MLP parameters in FP64 (the wrapper widens the BF16 weights and FP32
 * biases exactly).  Layouts: w1[64][20], w2[64][64], w3[64] (row = output
 * unit). */
typedef struct {
    int32_t kind;            /* ORC_PAIR_I32 .. ORC_QSRO */
    int32_t nshells;         /* pair shells used, 1..3 */
    const int32_t *v_i32;    /* [nshells][S][S], integer units */
    const float *v_f32;      /* [nshells][S][S], eV (qSRO: V_m^{pp'}) */
    double unit_ev;          /* eV per integer unit (integer model) */
    const double *w1, *w2, *w3;
    const double *b1, *b2;
    double b3;
    const float *qsro_w;     /* qSRO: W_m^p, [nshells][S], eV */
    double qsro_c;           /* qSRO: C, eV per site */
    /* MLPNet (Sec. IV-B): W0 [96][20], W1 [96][96], W2 [96][96], W3 [96],
     * b0, b1, b2 [96], b3 (row = output unit), FP64 */
    const double *net_w0, *net_w1, *net_w2, *net_w3;
    const double *net_b0, *net_b1, *net_b2;
    double net_b3;
} orc_model;

/* Philox4x32-10 block function: out = Philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Geometry. */
int64_t orc_nsites(const orc_lattice *lat);
int64_t orc_neighbor(const orc_lattice *lat, int64_t s, int vx, int vy, int vz);
int orc_shell_vectors(int shell, int out[][3]);   /* returns count */
int orc_schedule(const orc_lattice *lat, int32_t L[3]);  /* returns n_A */

/* Composition-conserving random initial configuration. */
int orc_init_lattice(const orc_lattice *lat, const int64_t *counts, uint64_t seed,
                     uint32_t replica, int8_t *occ);

/* Energies. */
double orc_site_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ, int64_t i);
double orc_total_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ);
int64_t orc_total_energy_i64(const orc_lattice *lat, const orc_model *m, const int8_t *occ);
double orc_delta_e(const orc_lattice *lat, const orc_model *m, int8_t *occ, int64_t a, int64_t b);

/* Ordered pair counts n_m^{pq} and Warren-Cowley SRO alpha_m^{pq}. */
void orc_pair_counts(const orc_lattice *lat, int nshells, const int8_t *occ, int64_t *counts);
void orc_sro(const orc_lattice *lat, int nshells, const int8_t *occ, double *alpha);

/* Acceptance table of the integer path. Returns its length (first zero entry
 * index), writing at most cap entries. */
int64_t orc_accept_table(double unit_ev, double kT, uint32_t *table, int64_t cap);

/* Sweeps.  mode 0: trials of a mini-step applied one by one in increasing
 * link-cell order (valid because they are independent); mode 1: Algorithm 1
 * as printed (auxiliary lattice, local energies of every site before and
 * after, reduction over Omega, masked copy back). */
int orc_sweep(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
              uint32_t replica, uint64_t sweep0, int32_t nsweeps, const double *kT,
              double *e_acc, int64_t *n_acc, int mode);

/* One mini-step k of sweep `sweep`, recording every trial's dE and decision
 * (trial order = increasing link-cell index).  Returns the number of trials. */
int64_t orc_ministep_trace(const orc_lattice *lat, const orc_model *m, int8_t *occ,
                           uint64_t seed, uint32_t replica, uint64_t sweep, int32_t k,
                           double kT, double *dE, uint8_t *acc, int64_t *site_a,
                           int64_t *site_b);

/* 1D slab decomposition along x (Sec. III-B).  orc_slab_ghost_cells: the
 * cells a trial reads past its own along x (2 for pair models, 3 with the
 * MLP).  orc_slab_ministep: the trials of mini-step k whose sites lie in
 * cells [x0, x0 + w) of the box `glat`, on occ_loc = that slab plus g ghost
 * cells per side ([sub][z][y][x - x0 + g], w + 2g cells along x, x modulo
 * nx).  Needs nx >= 8 with nx % 4 == 0, x0 and w multiples of 4 and
 * ghost cells <= g <= w.  Returns the number of trials, or -1. */
int orc_slab_ghost_cells(const orc_model *m);
int64_t orc_slab_ministep(const orc_lattice *glat, const orc_model *m, int8_t *occ_loc,
                          int32_t x0, int32_t w, int32_t g, uint64_t seed, uint32_t replica,
                          uint64_t sweep, int32_t k, double kT, double *e_acc, int64_t *n_acc);

/* dE/dtheta: pair part [nshells][S(S+1)/2] (p <= q), then (MLP models) the
 * 5569 MLP parameters in the order W1, b1, W2, b2, W3, b3. */
int64_t orc_grad_size(const orc_lattice *lat, const orc_model *m);
int orc_energy_grad(const orc_lattice *lat, const orc_model *m, const int8_t *occ, double *grad);

/* MLP site function on an explicit feature vector (for tests). */
double orc_mlp_eval(const orc_model *m, const double x[ORC_MLP_IN]);
/* MLPNet site function on an explicit feature vector (for tests). */
double orc_mlpnet_eval(const orc_model *m, const double x[ORC_MLP_IN]);

/* FCC lattice (pair models): nx x ny x nz cubic cells of 4 sites (half-unit
 * offsets (0,0,0), (1,1,0), (1,0,1), (0,1,1)); shells of 12, 6 and 24
 * half-unit vectors in lexicographic order; n_A = 4 Lx Ly Lz mini-steps;
 * per trial site s, Philox(counter (s, replica, sweep lo, sweep hi)):
 * r = word 0 & (2^29 - 1), partner index floor(12 word 1 / 2^32). */
int64_t orc_fcc_nsites(const orc_lattice *lat);
int64_t orc_fcc_neighbor(const orc_lattice *lat, int64_t s, int vx, int vy, int vz);
int orc_fcc_shell_vectors(int shell, int out[][3]);
int orc_fcc_schedule(const orc_lattice *lat, int32_t L[3]);
double orc_fcc_total_energy(const orc_lattice *lat, const orc_model *m, const int8_t *occ);
int64_t orc_fcc_total_energy_i64(const orc_lattice *lat, const orc_model *m, const int8_t *occ);
double orc_fcc_delta_e(const orc_lattice *lat, const orc_model *m, int8_t *occ, int64_t a, int64_t b);
int orc_fcc_sweep(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed, uint32_t replica,
                  uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc, int64_t *n_acc);
int64_t orc_fcc_ministep_trace(const orc_lattice *lat, const orc_model *m, int8_t *occ, uint64_t seed,
                               uint32_t replica, uint64_t sweep, int32_t k, double kT, double *dE, uint8_t *acc,
                               int64_t *site_a, int64_t *site_b);

#ifdef __cplusplus
}
#endif
#endif
