/*
 * smc.h -- C ABI of the GB300 swap Monte Carlo library (libsmc.so).
 *
 * Canonical, composition-conserving Metropolis swap Monte Carlo on a BCC
 * alloy lattice, scheduled over non-interacting link cells (SMC-X, Sec. II-A;
 * SMC-AI, Sec. III-A and Algorithm 1).  Energies come from pair interactions
 * over neighbour shells, from the qSRO model of local pair fractions, or from
 * a small BF16 MLP on per-shell species counts (Sec. IV-B).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice.  A box of nx x ny x nz BCC cells (each >= 2), N = 2 nx ny nz < 2^31
 *   sites.  Site (sub, x, y, z) sits at (x + sub/2, y + sub/2, z + sub/2) a.
 *   Occupancy is an int8 array of N species indices in [0, nspecies) in the
 *   canonical order s = ((sub*nz + z)*ny + y)*nx + x.  nspecies <= 8
 *   (MLP models: <= 5).
 * Shells.  1: 8 neighbours at sqrt(3)a/2, ordered lexicographically in
 *   (+-1/2)^3 with - before +; 2: 6 at a; 3: 12 at sqrt(2)a.
 * Link cells and mini-steps (Sec. II-A; Algorithm 1).  The link-cell
 *   edge along an axis of n cells is 4 if n >= 8 and n % 4 == 0, else n.
 *   A sweep is n_A = 2 Lx Ly Lz mini-steps; mini-step k visits the offset
 *   (sub, dx, dy, dz) with k = ((sub*Lz + dz)*Ly + dy)*Lx + dx, and every link
 *   cell tries to swap its site at that offset with a random first-shell
 *   neighbour.  One sweep = one trial per site (the paper's MC step, Sec. V-A).
 * Random numbers.  Philox4x32-10 with key (seed lo, seed hi) and counter
 *   (s >> 2, replica, sweep lo, sweep hi); site s uses output word s & 3:
 *   partner = shell-1 vector [word >> 29], r = word & (2^29 - 1).  Results do
 *   not depend on the launch configuration.  Sweep indices 2^64-2 and 2^64-1
 *   are reserved for the initial configuration.
 * Metropolis (Algorithm 1).  Integer models: accept iff dE <= 0 or
 *   r < floor(2^29 exp(-dE unit_ev / kT)) (table built on the host in FP64).
 *   Floating-point models: accept iff dE <= 0 or (r + 1/2) 2^-29 <
 *   exp(-dE / kT).  The BCC pair sweeps take dE in exact fixed point,
 *   dE = dE_fix 2^-sigma (coefficient differences D_m(q) - D_m(S-1) rounded
 *   once to multiples of 2^-sigma, sigma = floor(log2(2^30 / sum_m 8 (z_m - 1)
 *   max|V_m|)); within sum |c| 2^-(sigma+1) of the FP64 sum) and test
 *   2r + 1 < ceil(2^(dE_fix cx + 30)), cx = -log2(e) 2^-sigma / kT in FP32,
 *   2^x from ex2.approx; the other kernels evaluate exp(-dE / kT) in FP32.
 *   A swap of two equal species is an accepted no-op.  The BCC pair sweeps
 *   report a species byte outside [0, S) as SMC_ERR_ARG (smc_check) and use
 *   it modulo 8.
 * Energies.  Pair: E = sum_i 1/2 sum_m sum_{v in shell m} V_m(s_i, s_{i+v}).
 *   MLP: E = sum_i f(x_i), x_i = [onehot(s_i) | shell-1 counts | shell-2
 *   counts | shell-3 counts] (5 entries each), f = W3 silu(W2 silu(W1 x + b1)
 *   + b2) + b3 (MLPNet, Sec. IV-B).  Evaluated on the tensor cores with BF16
 *   weights and inputs (the integer features are exact in BF16), FP32
 *   accumulation, FP32 biases and output layer; the layer-1 activations are
 *   rounded to BF16 before the second product, and silu(z) is computed as
 *   h + h tanh(h), h = z/2, with the hardware tanh approximation.  A site's f
 *   is a fixed function of its features (the same bits wherever it is
 *   evaluated), so the MLP chains sample the Boltzmann distribution of that
 *   BF16 energy exactly; its departure from FP64 is what the tests report.
 *   MLPNet (SMC_MLPNET_BF16, the paper's shape): the same features,
 *   h1 = relu(W0 x + b0), h2 = relu(W1 h1 + b1), h3 = relu(W2 h2 + b2),
 *   f = W3 h3 + b3, 96 units per layer, with the same BF16 / FP32 split (the
 *   activations of the first two layers rounded to BF16); it runs everywhere
 *   the MLP does except smc_energy_grad.
 *   MLP sweeps and traces need every axis a multiple of 4 cells and >= 8,
 *   nx <= 1024, and occ 4-byte aligned.
 *
 * Memory and streams.  Pointers marked "device" are caller-owned device
 * memory (for example torch tensors); "host" pointers are read during the
 * call only.  All work is enqueued on `stream` and is complete when the
 * stream is synchronised.  The library owns a per-device workspace (link-cell
 * progress flags, partial sums, acceptance tables) that it grows with
 * cudaMalloc when needed and never frees before process exit; calls that use
 * it must not run concurrently on different streams of one device.
 *
 * Errors.  Argument errors return synchronously and leave every buffer
 * untouched.  Device-side failures (a progress wait that exceeded its time
 * limit) are latched in a device status word; smc_check(stream) synchronises
 * the stream and returns and clears it.  smc_last_error() gives the message of
 * the last failing call on the calling thread.  No call aborts the process.
 */
#ifndef SMC_H
#define SMC_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SMC_OK = 0,
    SMC_ERR_ARG = -1,          /* invalid argument */
    SMC_ERR_UNSUPPORTED = -2,  /* valid but not supported by this build */
    SMC_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    SMC_ERR_TIMEOUT = -4,      /* a device-side progress wait timed out */
    SMC_ERR_STATE = -5         /* inconsistent library state */
} smc_status;

typedef struct {
    int32_t nx, ny, nz;  /* cells per axis, each >= 2 */
    int32_t nspecies;    /* 1..8 */
} smc_lattice;

enum {
    SMC_PAIR_I32 = 0,          /* integer pair coefficients (exact path) */
    SMC_PAIR_F32 = 1,          /* FP32 pair coefficients, eV */
    SMC_MLP_BF16 = 2,          /* BF16 MLP site energies */
    SMC_PAIR_F32_MLP_BF16 = 3, /* sum of the two */
    SMC_QSRO_F32 = 4,          /* qSRO site energies (Sec. IV-B), FP32 parameters */
    SMC_MLPNET_BF16 = 5        /* MLPNet at the paper's shape (Sec. IV-B): 96-wide, ReLU, BF16 */
};

/* Energy model (all pointers host memory, read during the call).
 * Pair coefficients V_m(p, q) (Sec. IV-B, effective pair interactions) are
 * [nshells][S][S], symmetric in p, q.  MLP weights are BF16 bit patterns in
 * row-major [out][in] order: w1 [64][20], w2 [64][64], w3 [64].
 * qSRO (Sec. IV-B, Eq. quadratic_local_SRO): the local energy of site i is
 *   E_i = sum_{m, p'<=p} V_m^{pp'} pi_m^{pp'} + sum_{m,p} W_m^p (pi_m^{pp})^2 + C
 * with pi_m^{pp'} the fraction of the pairs (i, j), j in shell m of i, whose
 * species are {p, p'}; V_m^{pp'} in v_f32 ([nshells][S][S], symmetric),
 * W_m^p in qsro_w ([nshells][S]), C in qsro_c.  The constant lambda sum W^2
 * of the paper's equation is a training regulariser and is not part of E.
 * The paper's linear sum runs over p' < p; with same-element terms included
 * the model equals the paper's with V'^{pq} = V^{pq} - (V^{pp} + V^{qq})/2
 * plus sum_m sum_p N_p V_m^{pp}, a constant at fixed composition, so every
 * dE is the paper form's dE with V' (and V^{pp} = 0 gives that form as is). */
typedef struct {
    int32_t kind;            /* SMC_PAIR_I32 .. SMC_MLPNET_BF16 */
    int32_t nshells;         /* pair / qSRO shells 1..3 (ignored for SMC_MLP_BF16) */
    const int32_t *v_i32;    /* SMC_PAIR_I32: units of unit_ev, |V| <= 2^24 */
    const float *v_f32;      /* SMC_PAIR_F32*, SMC_QSRO_F32: eV */
    double unit_ev;          /* SMC_PAIR_I32: eV per integer unit (> 0) */
    const uint16_t *mlp_w1, *mlp_w2, *mlp_w3;
    const float *mlp_b1, *mlp_b2;
    float mlp_b3;
    const float *qsro_w;     /* SMC_QSRO_F32: W_m^p, [nshells][S], eV */
    float qsro_c;            /* SMC_QSRO_F32: C, eV per site */
    /* SMC_MLPNET_BF16: f = W3 h3 + b3, h3 = relu(W2 h2 + b2), h2 = relu(W1 h1
     * + b1), h1 = relu(W0 x + b0) on the MLP's 20 features; BF16 bit patterns
     * w0 [96][20], w1 [96][96], w2 [96][96], w3 [96], FP32 biases. */
    const uint16_t *net_w0, *net_w1, *net_w2, *net_w3;
    const float *net_b0, *net_b1, *net_b2;
    float net_b3;
} smc_model;

/* Composition-conserving random initial configuration (the starting state
 * of Algorithm 1).  Sites are ordered by the 64-bit key
 * (w(seed; s>>2, replica, 2^64-2)[s&3] << 32) | w(seed; s>>2, replica,
 * 2^64-1)[s&3] with ties broken by s; the first counts[0] sites in that order
 * get species 0, the next counts[1] species 1, and so on.
 *   counts  host [nspecies], non-negative, summing to N.
 *   occ     device [N] int8, written.
 * Errors: SMC_ERR_ARG for bad dimensions or counts. */
smc_status smc_init_lattice(const smc_lattice *lat, const int64_t *counts, uint64_t seed,
                            uint32_t replica, int8_t *occ, cudaStream_t stream);

/* nsweeps sweeps of Algorithm 1 on occ, sweeps sweep0 .. sweep0+nsweeps-1.
 *   occ     device [N] int8, updated in place.
 *   kT      host [nsweeps], temperature of each sweep in eV (> 0, may be +inf
 *           for floating-point models).
 *   e_acc   device double, nullable: += sum of dE of accepted trials (eV;
 *           integer units of unit_ev for SMC_PAIR_I32), summed in a fixed
 *           order (bit-reproducible).
 *   n_acc   device int64, nullable: += number of accepted trials.
 * MLP models keep a per-site energy cache E[i] = f(x_i) in the workspace
 * (4 N bytes), filled at the start of every call and updated over the
 * interaction zone of every accepted swap, so a trial evaluates only the 40
 * post-swap energies of its zone, and the per-site features (species and
 * per-shell species counts, 16 N bytes) the same way; they need every axis
 * a multiple of 4 cells and >= 8, nx <= 1024.  qSRO models keep each site's
 * own-species count per shell (N bytes for 1-2 shells, 2 N for 3), built at
 * the start of every call and updated by accepted swaps; a trial's dE comes
 * from the species of a, b and the sites within the model's shells of
 * either, and from those sites' counts, in FP32 (C left out, where it
 * cancels), within 1e-5 eV of FP64.  They need every axis a multiple of 4
 * cells and >= 8.
 * Pair models on lattices with every axis a multiple of 4 and >= 8 cells
 * whose rows fit the SMs' shared memory (128^3 and below) keep the lattice
 * there for the whole call (one cooperative launch per call, row versions
 * exchanged between CTAs through L2); larger lattices stream their rows from
 * device memory (rows of 128, 256 or 512 cells with a two-shell model of at
 * most 5 species and a 16-byte aligned occ: two groups of mini-steps per
 * staging of a column's rows).  All give the same trajectory bit for bit.
 * Errors: SMC_ERR_ARG (dimensions, model, kT), SMC_ERR_UNSUPPORTED (MLP or
 * qSRO models on lattices their kernels do not take), SMC_ERR_CUDA. */
smc_status smc_sweep(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                     uint32_t replica, uint64_t sweep0, int32_t nsweeps, const double *kT,
                     double *e_acc, int64_t *n_acc, cudaStream_t stream);

/* Allocation-free variant of smc_sweep for callers that cannot call
 * cudaMalloc: code running while a CUDA graph is being captured (where an
 * allocation is an error), or applications whose device memory is owned by
 * their own allocator and must not see a library allocate on its own.  The
 * paper has no counterpart; it is a deployment convenience.
 *
 * It runs the same kernels as smc_sweep for SMC_PAIR_F32 models: for the
 * same arguments and tuning it gives the same trajectory, and e_acc and
 * n_acc bit for bit.  Its scratch memory (progress flags and partial sums of
 * at most 16384 link-cell tiles) lives in a fixed 320 KB array inside the
 * library that every GPU which loads the library keeps until the process
 * exits.  It calls no cudaMalloc, cudaFree or allocating library routine,
 * and it does not touch the library workspace (smc_check does not see its
 * device-side failures: they go to `status`).
 *   status  device int32, required: set to 0 at the start of the call (also
 *           when nsweeps == 0) and to SMC_ERR_TIMEOUT if a device-side
 *           progress wait timed out, which leaves the trajectory incomplete.
 *   other arguments as for smc_sweep.
 * Every call looks up the array's device address (cudaGetSymbolAddress)
 * with the caller's device current; the first call on a device also loads
 * the library's kernels there, so make it before any stream capture.  Every
 * call shares the array and rewrites it (the flags and partial sums it needs
 * are cleared at the start of each launch), so calls that overlap on the GPU
 * (different streams, or a second host thread) race; serialise them on one
 * stream.
 * Errors: SMC_ERR_ARG as smc_sweep, and for a NULL status; SMC_ERR_UNSUPPORTED
 * for other model kinds or for lattices needing more than 16384 tiles;
 * SMC_ERR_CUDA. */
smc_status smc_sweep_noalloc(const smc_lattice *lat, const smc_model *model, int8_t *occ,
                             uint64_t seed, uint32_t replica, uint64_t sweep0, int32_t nsweeps,
                             const double *kT, double *e_acc, int64_t *n_acc, int32_t *status,
                             cudaStream_t stream);

/* Independent replicas of possibly different sizes (each its own lattice and
 * occupancy, shared model), advanced together in one persistent launch per
 * chunk of sweeps (pair models whose replicas all fit shared memory: one
 * launch per wave of replicas resident at once).  Replica r uses RNG replica
 * index replica0 + r, so it reproduces smc_sweep(..., replica0 + r, ...) bit
 * for bit.
 *   lats    host [R];  occ  host [R] array of device pointers.
 *   kT      host [R][nsweeps] (eV).
 *   e_acc, n_acc  device [R], nullable.
 * MLP and qSRO models: R must be 1 (SMC_ERR_UNSUPPORTED otherwise). */
smc_status smc_sweep_batched(int32_t R, const smc_lattice *lats, const smc_model *model,
                             int8_t *const *occ, uint64_t seed, uint32_t replica0,
                             uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc,
                             int64_t *n_acc, cudaStream_t stream);

/* Ordered pair counts n_m^{pq} = #{(i, v in shell m): s_i = p, s_{i+v} = q}
 * (the pair numbers of Eq. 2) and Warren-Cowley SRO
 * alpha_m^{pq} = 1 - n_m^{pq} / (N c_p z_m c_q) (NaN where c_p or c_q is 0).
 *   nshells  1..3.   occ  device [N].
 *   counts   device [nshells][S][S] int64, nullable.
 *   alpha    device [nshells][S][S] double, nullable. */
smc_status smc_sro(const smc_lattice *lat, int32_t nshells, const int8_t *occ, int64_t *counts,
                   double *alpha, cudaStream_t stream);

/* Total energy of occ.  MLP models: the site energies of the tensor-core
 * evaluation summed in FP64 in a fixed order (bit-reproducible); pair + MLP
 * models add the pair energy from the pair counts.  qSRO models: in FP64
 * from exact integer counts, sum V_m^{pq} n_m^{pq} / z_m + sum W_m^p Q_m^p /
 * z_m^2 + N C, with n the ordered pair counts and Q_m^p the sum over sites
 * of species p of their squared same-element count in shell m.
 *   e      device double (eV), nullable (required for MLP and qSRO models).
 *   e_int  device int64, nullable; integer models only: E in units of unit_ev
 *          (exact). */
smc_status smc_energy(const smc_lattice *lat, const smc_model *model, const int8_t *occ,
                      double *e, int64_t *e_int, cudaStream_t stream);

/* dE/dtheta of the total energy at configuration occ.
 * Layout: pair part [nshells][S(S+1)/2] with (p, q), p <= q, row-major over
 * p then q (one parameter per unordered pair: dE/dV_m^{pq} = n_m^{pq} for
 * p != q, n_m^{pp}/2 for p = q), then for MLP models the 5569 MLP parameters
 * W1, b1, W2, b2, W3, b3.  qSRO models: [V_m^{pq}, p <= q]
 * ((n_m^{pq} + n_m^{qp}) / z_m for p != q, n_m^{pp} / z_m for p = q), then
 * [W_m^p] (Q_m^p / z_m^2), then C (N).  MLPNet models: not offered
 * (smc_grad_size returns -1, smc_energy_grad SMC_ERR_UNSUPPORTED).
 *   grad   device float [smc_grad_size(lat, model)]. */
int64_t smc_grad_size(const smc_lattice *lat, const smc_model *model);
smc_status smc_energy_grad(const smc_lattice *lat, const smc_model *model, const int8_t *occ,
                           float *grad, cudaStream_t stream);

/* Lock-step trace of one mini-step: applies mini-step k of sweep `sweep`
 * (as smc_sweep would) and records, per trial in link-cell order
 * c = (cz*NLy + cy)*NLx + cx, the dE it computed (eV) and its decision.
 * MLP models recompute the pre-swap energies (no cache) with the sweep's
 * arithmetic, and qSRO models rebuild the own-species counts from occ and
 * run the sweep's kernel, so a sweep equals its 2 Lx Ly Lz traced
 * mini-steps bit for bit.
 *   dE   device float [N/n_A], nullable;  acc  device uint8 [N/n_A], nullable. */
smc_status smc_ministep_trace(const smc_lattice *lat, const smc_model *model, int8_t *occ,
                              uint64_t seed, uint32_t replica, uint64_t sweep, int32_t k,
                              double kT, float *dE, uint8_t *acc, cudaStream_t stream);

/* Mini-step k of sweep `sweep` on one x-slab of the box `lat` (Sec. III-B,
 * 1D slab decomposition; pair models).  The slab owns cells
 * x0 <= x < x0 + w of every row; win holds cells [x0 - g, x0 + w + g)
 * (x modulo nx) as [2][nz][ny][w + 2g] int8 (device, updated in place).
 * The slab's trials run exactly as in smc_sweep on the whole box -- the same
 * link cells, the random word of the global site id, the same dE and
 * decision -- so W slabs that run every mini-step and then exchange the
 * cells each changed within g of its edges (the ranges of the Python
 * module slab.py) reproduce smc_sweep bit for bit.
 *   x0, w    multiples of 4, w >= 4, x0 + w <= nx (nx a multiple of 4, >= 8).
 *   g        ghost cells per side, 2 <= g <= w (a pair trial reads 2 cells
 *            past its own along x).
 *   part     0: every link cell of the slab; 1: the first and last link cell
 *            of each x-row (the trials that change cells within 3 of the
 *            slab's edges, the cells the exchange sends); 2: the others
 *            (reads and writes inside the slab).  Parts 1 and 2 together
 *            equal part 0 in either order: a mini-step's trials touch
 *            disjoint cells.  Part 2 reads no ghost cell and writes none of
 *            the cells the exchange sends, so it may run while the frames of
 *            its own mini-step travel -- the cells part 1 changed going out,
 *            the neighbours' changes coming into the ghosts (the overlap of
 *            Sec. V-C).
 *   e_acc, n_acc  device, nullable: += accepted dE (eV) and count.
 * Errors: SMC_ERR_ARG for the ranges above; SMC_ERR_UNSUPPORTED for MLP,
 * MLPNet and qSRO models. */
smc_status smc_slab_ministep(const smc_lattice *lat, const smc_model *model, int8_t *win, int32_t x0,
                             int32_t w, int32_t g, uint64_t seed, uint32_t replica, uint64_t sweep,
                             int32_t k, double kT, double *e_acc, int64_t *n_acc, int32_t part,
                             cudaStream_t stream);

/* FCC lattice (the paper's lattice, Sec. IV-C), pair models (SMC_PAIR_I32,
 * SMC_PAIR_F32) and the qSRO model (SMC_QSRO_F32, Eq. quadratic_local_SRO
 * with the FCC shells, z_m = 12, 6, 24; the sweep keeps a cache of
 * own-species counts in the workspace, N bytes for 1-2 shells, 2 N for 3).  lat gives nx x ny x nz cubic cells of 4 sites at the
 * half-unit offsets (0,0,0), (1,1,0), (1,0,1), (0,1,1) (sublattices 0-3),
 * N = 4 nx ny nz, site s = ((sub*nz + z)*ny + y)*nx + x; every axis a
 * multiple of 4 and >= 8 cells (4x4x4 link cells, n_A = 256 mini-steps,
 * k = ((sub*4 + dz)*4 + dy)*4 + dx, Sec. V-C).  Shell m: the half-unit
 * vectors of squared length 2m with an even component sum (12, 6, 24), in
 * lexicographic order.  Random numbers: per trial site s,
 * w = Philox4x32-10(key seed, counter (s, replica, sweep lo, sweep hi)),
 * r = w0 & (2^29 - 1) for the Metropolis test, partner = floor(12 w1 / 2^32).
 * smc_fcc_init_lattice: the composition-conserving start state (the
 * smc_init_lattice order over the same N site ids).  The other calls have
 * the arguments and errors of their BCC counterparts; e_acc sums per link
 * cell, then over the link cells in a fixed order (bit-reproducible);
 * smc_fcc_ministep_trace runs the sweep
 * kernel on one mini-step and records its per-trial dE and decisions.
 * Errors: SMC_ERR_UNSUPPORTED for other model kinds, and for sweeps and
 * traces on a box whose axes are not multiples of 4 of at least 8 cells
 * (smc_fcc_energy takes any box of at least 1 cell per axis). */
smc_status smc_fcc_init_lattice(const smc_lattice *lat, const int64_t *counts, uint64_t seed, uint32_t replica,
                                int8_t *occ, cudaStream_t stream);
smc_status smc_fcc_sweep(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                         uint32_t replica, uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc,
                         int64_t *n_acc, cudaStream_t stream);
smc_status smc_fcc_ministep_trace(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                                  uint32_t replica, uint64_t sweep, int32_t k, double kT, float *dE, uint8_t *acc,
                                  cudaStream_t stream);
smc_status smc_fcc_energy(const smc_lattice *lat, const smc_model *model, const int8_t *occ, double *e,
                          int64_t *e_int, cudaStream_t stream);

/* Philox4x32-10 block function on the device, for tests: out[4i..4i+3] =
 * Philox(ctr[4i..4i+3], key[2i..2i+1]).  All pointers device memory. */
smc_status smc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                             cudaStream_t stream);

/* Synchronises `stream`, returns the latched device status and clears it. */
smc_status smc_check(cudaStream_t stream);

/* Message of the last failing call on this thread ("" if none). */
const char *smc_last_error(void);

/* Launch tuning (domain tile shape and CTA size) chosen by the caller's
 * autotuner; results never depend on it.  tile_y, tile_z: link-cell columns
 * per tile along y and z (0 = automatic); threads: CTA size, a multiple of 32
 * in [32, 512] (0 = automatic; the fast kernel uses at most 256); ctas_per_sm: resident CTAs per SM requested
 * (0 = automatic).  Applies to later sweeps on the calling thread. */
typedef struct {
    int32_t tile_y, tile_z, threads, ctas_per_sm;
} smc_tuning;
smc_status smc_set_tuning(const smc_tuning *t);

/* Test and tuning hooks.  SMC_DBG_TIMEOUT_MS sets the progress-wait limit
 * (default 2000 ms); SMC_DBG_SKIP_PUBLISH makes the tile (streaming sweeps)
 * or block (the resident pair sweep: its row versions and its progress) with
 * that index never publish, so that its neighbours time out (-1 = off).
 * SMC_DBG_FAST_TEAM (1, 2 or 4 warps per link-cell column),
 * SMC_DBG_FAST_BUFFERS (1 or 2 row buffers per column) and
 * SMC_DBG_FAST_STAGING (1: one bulk copy per row; 2: 16-byte cp.async) fix
 * those launch choices of the pair sweep on lattices with four-cell link
 * cells on every axis (0 = automatic); SMC_DBG_RESIDENT = 1 keeps the pair
 * sweep from holding a small lattice in shared memory for a whole call
 * (0 = automatic).  Results never depend on them. */
enum {
    SMC_DBG_TIMEOUT_MS = 1,
    SMC_DBG_SKIP_PUBLISH = 2,
    SMC_DBG_FAST_TEAM = 3,
    SMC_DBG_FAST_BUFFERS = 4,
    SMC_DBG_FAST_STAGING = 5,
    SMC_DBG_RESIDENT = 6
};
smc_status smc_debug_set(int32_t what, int64_t value);

#ifdef __cplusplus
}
#endif
#endif
