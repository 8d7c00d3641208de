// smc_api.cu -- C ABI entry points of libsmc.so: argument validation,
// per-device workspace, error reporting and dispatch to the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "smc_common.cuh"

namespace smc {

static thread_local char g_msg[512] = "";
static std::mutex g_lock;  // the workspace and parameter blocks are shared
static thread_local Tuning g_tuning;
static int64_t g_timeout_ns = 2000LL * 1000 * 1000;
static int64_t g_skip_tile = -1;
static int g_fast_team = 0, g_fast_nbuf = 0, g_fast_stage = 0, g_resident = 0;

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
}

smc_status cuda_fail(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return SMC_ERR_CUDA;
}

Tuning current_tuning() { return g_tuning; }
int64_t debug_timeout_ns() { return g_timeout_ns; }
int64_t debug_skip_tile() { return g_skip_tile; }
int debug_fast_team() { return g_fast_team; }
int debug_fast_nbuf() { return g_fast_nbuf; }
int debug_fast_stage() { return g_fast_stage; }
int debug_resident() { return g_resident; }

static Workspace g_ws[64];

Workspace *workspace(smc_status *st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        *st = cuda_fail(e == cudaSuccess ? cudaErrorInvalidDevice : e, "cudaGetDevice");
        return nullptr;
    }
    Workspace *ws = &g_ws[dev];
    if (ws->device < 0) {
        int sms = 0, optin = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaDeviceGetAttribute");
            return nullptr;
        }
        const size_t cap = 1 << 20;
        void *buf = nullptr;
        e = cudaMalloc(&buf, cap);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaMalloc(workspace)");
            return nullptr;
        }
        e = cudaMemset(buf, 0, 256);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaMemset(workspace)");
            return nullptr;
        }
        ws->buf = buf;
        ws->cap = cap;
        ws->status = (int *)buf;
        ws->num_sms = sms;
        ws->smem_optin = (size_t)optin;
        ws->device = dev;
    }
    *st = SMC_OK;
    return ws;
}

// Scratch starts 256 bytes into the buffer (after the status word).  Growing
// frees the old buffer only after the device has finished with it.
void *workspace_scratch(Workspace *ws, size_t bytes, smc_status *st)
{
    const size_t need = bytes + 256;
    if (need > ws->cap) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaDeviceSynchronize(workspace growth)");
            return nullptr;
        }
        int status = 0;
        e = cudaMemcpy(&status, ws->status, sizeof status, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaMemcpy(status)");
            return nullptr;
        }
        size_t cap = ws->cap;
        while (cap < need) cap *= 2;
        void *buf = nullptr;
        e = cudaMalloc(&buf, cap);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaMalloc(workspace)");
            return nullptr;
        }
        e = cudaMemset(buf, 0, 256);
        if (e == cudaSuccess) e = cudaMemcpy(buf, &status, sizeof status, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            *st = cuda_fail(e, "cudaMemset(workspace)");
            return nullptr;
        }
        cudaFree(ws->buf);
        ws->buf = buf;
        ws->cap = cap;
        ws->status = (int *)buf;
    }
    *st = SMC_OK;
    return (unsigned char *)ws->buf + 256;
}

bool lattice_valid(const smc_lattice *lat, bool mlp)
{
    if (!lat) {
        set_error("lattice is NULL");
        return false;
    }
    if (lat->nx < 2 || lat->ny < 2 || lat->nz < 2) {
        set_error("lattice dimensions must be >= 2 (got %d x %d x %d)", lat->nx, lat->ny, lat->nz);
        return false;
    }
    if (lat->nspecies < 1 || lat->nspecies > (mlp ? 5 : kMaxSpecies)) {
        set_error("nspecies must be in [1, %d] (got %d)", mlp ? 5 : kMaxSpecies, lat->nspecies);
        return false;
    }
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    if (N >= (1LL << 31)) {
        set_error("lattice too large: N = %lld sites (limit 2^31 - 1)", N);
        return false;
    }
    return true;
}

static bool is_mlp(const smc_model *m)
{
    return m->kind == SMC_MLP_BF16 || m->kind == SMC_PAIR_F32_MLP_BF16 || m->kind == SMC_MLPNET_BF16;
}
static bool is_qsro(const smc_model *m) { return m->kind == SMC_QSRO_F32; }
static bool has_pair(const smc_model *m)
{
    return m->kind == SMC_PAIR_I32 || m->kind == SMC_PAIR_F32 || m->kind == SMC_PAIR_F32_MLP_BF16;
}

bool model_valid(const smc_lattice *lat, const smc_model *m)
{
    if (!m) {
        set_error("model is NULL");
        return false;
    }
    if (m->kind < SMC_PAIR_I32 || m->kind > SMC_MLPNET_BF16) {
        set_error("unknown model kind %d", m->kind);
        return false;
    }
    const int S = lat->nspecies;
    if (has_pair(m)) {
        if (m->nshells < 1 || m->nshells > kMaxShells) {
            set_error("nshells must be in [1, 3] (got %d)", m->nshells);
            return false;
        }
        if (m->kind == SMC_PAIR_I32) {
            if (!m->v_i32 || !(m->unit_ev > 0.0) || !std::isfinite(m->unit_ev)) {
                set_error("integer model needs v_i32 and unit_ev > 0");
                return false;
            }
            for (int i = 0; i < m->nshells * S * S; ++i)
                if (m->v_i32[i] > (1 << 24) || m->v_i32[i] < -(1 << 24)) {
                    set_error("|V| must be <= 2^24 (entry %d = %d)", i, m->v_i32[i]);
                    return false;
                }
        } else if (!m->v_f32) {
            set_error("floating-point pair model needs v_f32");
            return false;
        }
        for (int mm = 0; mm < m->nshells; ++mm)
            for (int p = 0; p < S; ++p)
                for (int q = 0; q < p; ++q) {
                    const int a = (mm * S + p) * S + q, b = (mm * S + q) * S + p;
                    const bool sym = m->kind == SMC_PAIR_I32 ? m->v_i32[a] == m->v_i32[b] : m->v_f32[a] == m->v_f32[b];
                    if (!sym) {
                        set_error("pair coefficients must be symmetric (shell %d, %d-%d)", mm + 1, p, q);
                        return false;
                    }
                }
    }
    if (is_qsro(m)) {
        if (m->nshells < 1 || m->nshells > kMaxShells) {
            set_error("nshells must be in [1, 3] (got %d)", m->nshells);
            return false;
        }
        if (!m->v_f32 || !m->qsro_w) {
            set_error("qSRO model needs v_f32 and qsro_w");
            return false;
        }
        for (int mm = 0; mm < m->nshells; ++mm)
            for (int p = 0; p < S; ++p) {
                if (!std::isfinite(m->qsro_w[mm * S + p])) {
                    set_error("qSRO W must be finite (shell %d, species %d)", mm + 1, p);
                    return false;
                }
                for (int q = 0; q < S; ++q) {
                    const float a = m->v_f32[(mm * S + p) * S + q], b = m->v_f32[(mm * S + q) * S + p];
                    if (!std::isfinite(a) || a != b) {
                        set_error("qSRO V must be finite and symmetric (shell %d, %d-%d)", mm + 1, p, q);
                        return false;
                    }
                }
            }
        if (!std::isfinite(m->qsro_c)) {
            set_error("qSRO C must be finite");
            return false;
        }
    }
    if (m->kind == SMC_MLPNET_BF16) {
        if (!m->net_w0 || !m->net_w1 || !m->net_w2 || !m->net_w3 || !m->net_b0 || !m->net_b1 || !m->net_b2) {
            set_error("MLPNet model needs w0, w1, w2, w3, b0, b1, b2");
            return false;
        }
        if (S > 5) {
            set_error("MLP models support at most 5 species");
            return false;
        }
    } else if (is_mlp(m)) {
        if (!m->mlp_w1 || !m->mlp_w2 || !m->mlp_w3 || !m->mlp_b1 || !m->mlp_b2) {
            set_error("MLP model needs w1, w2, w3, b1, b2");
            return false;
        }
        if (S > 5) {
            set_error("MLP models support at most 5 species");
            return false;
        }
    }
    return true;
}

}  // namespace smc

using namespace smc;

#define API_LOCK std::lock_guard<std::mutex> _guard(g_lock)

extern "C" {

const char *smc_last_error(void) { return g_msg; }

smc_status smc_check(cudaStream_t stream)
{
    API_LOCK;
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int code = 0;
    e = cudaMemcpy(&code, ws->status, sizeof code, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
    if (code != 0) {
        const int zero = 0;
        e = cudaMemcpy(ws->status, &zero, sizeof zero, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status reset)");
        if (code == SMC_ERR_TIMEOUT) set_error("a device-side progress wait timed out");
        if (code == SMC_ERR_ARG)
            set_error("an occupancy value lies outside [0, nspecies) (the sweep took it modulo 8; the result is "
                      "undefined)");
        return (smc_status)code;
    }
    return SMC_OK;
}

smc_status smc_set_tuning(const smc_tuning *t)
{
    if (!t) {
        g_tuning = Tuning();
        return SMC_OK;
    }
    if (t->tile_y < 0 || t->tile_z < 0 || t->threads < 0 || t->ctas_per_sm < 0 ||
        (t->threads && (t->threads % 32 || t->threads > 1024))) {
        set_error("invalid tuning");
        return SMC_ERR_ARG;
    }
    g_tuning.tile_y = t->tile_y;
    g_tuning.tile_z = t->tile_z;
    g_tuning.threads = t->threads;
    g_tuning.ctas_per_sm = t->ctas_per_sm;
    return SMC_OK;
}

smc_status smc_debug_set(int32_t what, int64_t value)
{
    API_LOCK;
    if (what == SMC_DBG_TIMEOUT_MS) {
        if (value <= 0) {
            set_error("timeout must be positive");
            return SMC_ERR_ARG;
        }
        g_timeout_ns = value * 1000 * 1000;
        return SMC_OK;
    }
    if (what == SMC_DBG_SKIP_PUBLISH) {
        g_skip_tile = value;
        return SMC_OK;
    }
    if (what == SMC_DBG_FAST_TEAM) {
        if (value != 0 && value != 1 && value != 2 && value != 4) {
            set_error("team size must be 0, 1, 2 or 4");
            return SMC_ERR_ARG;
        }
        g_fast_team = (int)value;
        return SMC_OK;
    }
    if (what == SMC_DBG_FAST_BUFFERS) {
        if (value < 0 || value > 2) {
            set_error("buffer count must be 0, 1 or 2");
            return SMC_ERR_ARG;
        }
        g_fast_nbuf = (int)value;
        return SMC_OK;
    }
    if (what == SMC_DBG_FAST_STAGING) {
        if (value < 0 || value > 2) {
            set_error("staging must be 0, 1 or 2");
            return SMC_ERR_ARG;
        }
        g_fast_stage = (int)value;
        return SMC_OK;
    }
    if (what == SMC_DBG_RESIDENT) {
        if (value < 0 || value > 1) {
            set_error("resident must be 0 or 1");
            return SMC_ERR_ARG;
        }
        g_resident = (int)value;
        return SMC_OK;
    }
    set_error("unknown debug key %d", what);
    return SMC_ERR_ARG;
}

smc_status smc_init_lattice(const smc_lattice *lat, const int64_t *counts, uint64_t seed, uint32_t replica,
                            int8_t *occ, cudaStream_t stream)
{
    API_LOCK;
    if (!lattice_valid(lat, false)) return SMC_ERR_ARG;
    if (!counts || !occ) {
        set_error("counts and occ must be non-NULL");
        return SMC_ERR_ARG;
    }
    const long long N = 2LL * lat->nx * lat->ny * lat->nz;
    long long tot = 0;
    for (int p = 0; p < lat->nspecies; ++p) {
        if (counts[p] < 0) {
            set_error("negative count for species %d", p);
            return SMC_ERR_ARG;
        }
        tot += counts[p];
    }
    if (tot != N) {
        set_error("counts sum to %lld, lattice has %lld sites", tot, N);
        return SMC_ERR_ARG;
    }
    return launch_init(lat, counts, seed, replica, occ, stream);
}

static smc_status check_sweep_args(const smc_lattice *lat, const smc_model *model, int8_t *occ, int32_t nsweeps,
                                   const double *kT, int nkT, uint64_t sweep0)
{
    if (!lattice_valid(lat, model && is_mlp(model))) return SMC_ERR_ARG;
    if (!model_valid(lat, model)) return SMC_ERR_ARG;
    if (!occ) {
        set_error("occ is NULL");
        return SMC_ERR_ARG;
    }
    if (nsweeps < 0) {
        set_error("nsweeps must be >= 0");
        return SMC_ERR_ARG;
    }
    if (nsweeps > 0 && !kT) {
        set_error("kT is NULL");
        return SMC_ERR_ARG;
    }
    if (sweep0 + (uint64_t)nsweeps > 0xFFFFFFFFFFFFFFFEull || sweep0 + (uint64_t)nsweeps < sweep0) {
        set_error("sweep indices reach the reserved values 2^64-2, 2^64-1");
        return SMC_ERR_ARG;
    }
    for (int i = 0; i < nkT; ++i) {
        const double t = kT[i];
        if (!(t > 0.0) || (model->kind == SMC_PAIR_I32 && !std::isfinite(t))) {
            set_error("kT[%d] = %g is invalid (must be > 0; finite for integer models)", i, t);
            return SMC_ERR_ARG;
        }
        if (model->kind == SMC_PAIR_I32 && model->unit_ev / t < 29.0 * 0.6931471805599453 / (double)(1 << 24)) {
            set_error("kT[%d] too high for the integer acceptance table", i);
            return SMC_ERR_UNSUPPORTED;
        }
    }
    if ((long long)nsweeps * 2 * lc_edge(lat->ny) * lc_edge(lat->nz) >= (1LL << 31)) {
        set_error("too many sweeps in one call");
        return SMC_ERR_ARG;
    }
    return SMC_OK;
}

smc_status smc_sweep(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed, uint32_t replica,
                     uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc, int64_t *n_acc,
                     cudaStream_t stream)
{
    API_LOCK;
    smc_status st = check_sweep_args(lat, model, occ, nsweeps, kT, nsweeps, sweep0);
    if (st != SMC_OK) return st;
    if (nsweeps == 0) return SMC_OK;
    if (is_mlp(model))
        return launch_mlp_sweep(lat, model, occ, seed, replica, sweep0, nsweeps, kT, e_acc, n_acc, stream);
    if (is_qsro(model))
        return launch_qsro_ministeps(lat, model, occ, seed, replica, sweep0, nsweeps, kT, e_acc, n_acc, nullptr, nullptr,
                                     -1, stream);
    int8_t *occs[1] = {occ};
    return launch_pair_sweep(1, lat, model, occs, seed, replica, sweep0, nsweeps, kT, e_acc, n_acc, stream);
}

smc_status smc_sweep_noalloc(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                             uint32_t replica, uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc,
                             int64_t *n_acc, int32_t *status, cudaStream_t stream)
{
    API_LOCK;
    if (!lattice_valid(lat, false)) return SMC_ERR_ARG;
    if (!model_valid(lat, model)) return SMC_ERR_ARG;
    if (model->kind != SMC_PAIR_F32) {
        set_error("smc_sweep_noalloc supports SMC_PAIR_F32 models only");
        return SMC_ERR_UNSUPPORTED;
    }
    if (!occ || !status || nsweeps < 0 || (nsweeps > 0 && !kT)) {
        set_error("occ, status and kT must be non-NULL and nsweeps >= 0");
        return SMC_ERR_ARG;
    }
    if (sweep0 + (uint64_t)nsweeps > 0xFFFFFFFFFFFFFFFEull || sweep0 + (uint64_t)nsweeps < sweep0) {
        set_error("sweep indices reach the reserved values 2^64-2, 2^64-1");
        return SMC_ERR_ARG;
    }
    for (int i = 0; i < nsweeps; ++i)
        if (!(kT[i] > 0.0)) {
            set_error("kT[%d] = %g is invalid (must be > 0)", i, kT[i]);
            return SMC_ERR_ARG;
        }
    if ((long long)nsweeps * 2 * lc_edge(lat->ny) * lc_edge(lat->nz) >= (1LL << 31)) {
        set_error("too many sweeps in one call");
        return SMC_ERR_ARG;
    }
    if (nsweeps == 0) {
        const cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), stream);
        return e == cudaSuccess ? SMC_OK : cuda_fail(e, "cudaMemsetAsync(status)");
    }
    return launch_pair_sweep_noalloc(lat, model, occ, seed, replica, sweep0, nsweeps, kT, e_acc, n_acc, status,
                                     stream);
}

smc_status smc_sweep_batched(int32_t R, const smc_lattice *lats, const smc_model *model, int8_t *const *occ,
                             uint64_t seed, uint32_t replica0, uint64_t sweep0, int32_t nsweeps, const double *kT,
                             double *e_acc, int64_t *n_acc, cudaStream_t stream)
{
    API_LOCK;
    if (R < 1 || R > kMaxReplicas || !lats || !occ) {
        set_error("R must be in [1, %d] with lats and occ non-NULL", kMaxReplicas);
        return SMC_ERR_ARG;
    }
    for (int r = 0; r < R; ++r) {
        smc_status st = check_sweep_args(&lats[r], model, occ[r], nsweeps, kT + (size_t)r * nsweeps, nsweeps, sweep0);
        if (st != SMC_OK) return st;
    }
    if ((uint64_t)replica0 + (uint64_t)R > 0x100000000ull) {
        set_error("replica indices overflow 32 bits");
        return SMC_ERR_ARG;
    }
    if (nsweeps == 0) return SMC_OK;
    if (is_mlp(model) || is_qsro(model)) {
        if (R != 1) {
            set_error("batched MLP and qSRO sweeps take one replica per call");
            return SMC_ERR_UNSUPPORTED;
        }
        if (is_qsro(model))
            return launch_qsro_ministeps(lats, model, occ[0], seed, replica0, sweep0, nsweeps, kT, e_acc, n_acc, nullptr,
                                         nullptr, -1, stream);
        return launch_mlp_sweep(lats, model, occ[0], seed, replica0, sweep0, nsweeps, kT, e_acc, n_acc, stream);
    }
    return launch_pair_sweep(R, lats, model, occ, seed, replica0, sweep0, nsweeps, kT, e_acc, n_acc, stream);
}

smc_status smc_ministep_trace(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                              uint32_t replica, uint64_t sweep, int32_t k, double kT, float *dE, uint8_t *acc,
                              cudaStream_t stream)
{
    API_LOCK;
    smc_status st = check_sweep_args(lat, model, occ, 1, &kT, 1, sweep);
    if (st != SMC_OK) return st;
    const int nA = 2 * lc_edge(lat->nx) * lc_edge(lat->ny) * lc_edge(lat->nz);
    if (k < 0 || k >= nA) {
        set_error("mini-step %d out of range [0, %d)", k, nA);
        return SMC_ERR_ARG;
    }
    if (is_mlp(model)) return launch_mlp_trace(lat, model, occ, seed, replica, sweep, k, kT, dE, acc, stream);
    if (is_qsro(model))
        return launch_qsro_ministeps(lat, model, occ, seed, replica, sweep, 1, &kT, nullptr, nullptr, dE, acc, k,
                                     stream);
    return launch_ministep_trace(lat, model, occ, seed, replica, sweep, k, kT, dE, acc, stream);
}

smc_status smc_slab_ministep(const smc_lattice *lat, const smc_model *model, int8_t *win, int32_t x0, int32_t w,
                             int32_t g, uint64_t seed, uint32_t replica, uint64_t sweep, int32_t k, double kT,
                             double *e_acc, int64_t *n_acc, int32_t part, cudaStream_t stream)
{
    API_LOCK;
    smc_status st = check_sweep_args(lat, model, win, 1, &kT, 1, sweep);
    if (st != SMC_OK) return st;
    if (model->kind != SMC_PAIR_I32 && model->kind != SMC_PAIR_F32) {
        set_error("the slab mini-step takes pair models");
        return SMC_ERR_UNSUPPORTED;
    }
    if (lc_edge(lat->nx) != 4) {
        set_error("slabs need nx >= 8 and a multiple of 4 (got %d)", lat->nx);
        return SMC_ERR_ARG;
    }
    if (x0 < 0 || w < 4 || x0 % 4 != 0 || w % 4 != 0 || x0 + w > lat->nx) {
        set_error("slab [%d, %d) must be whole link cells inside [0, %d)", x0, x0 + w, lat->nx);
        return SMC_ERR_ARG;
    }
    if (g < 2 || g > w) {
        set_error("ghost cells g = %d must lie in [2, w = %d]", g, w);
        return SMC_ERR_ARG;
    }
    if (part < 0 || part > 2) {
        set_error("part must be 0 (all), 1 (edge link cells) or 2 (interior)");
        return SMC_ERR_ARG;
    }
    const int nA = 2 * 4 * lc_edge(lat->ny) * lc_edge(lat->nz);
    if (k < 0 || k >= nA) {
        set_error("mini-step %d out of range [0, %d)", k, nA);
        return SMC_ERR_ARG;
    }
    return launch_slab_ministep(lat, model, win, x0, w, g, seed, replica, sweep, k, kT, e_acc, n_acc, part, stream);
}

// ---- FCC lattice (Sec. IV-C), pair models ----

static bool fcc_lattice_valid(const smc_lattice *lat)
{
    if (!lat) {
        set_error("lattice is NULL");
        return false;
    }
    if (lat->nx < 1 || lat->ny < 1 || lat->nz < 1) {
        set_error("lattice dimensions must be >= 1 (got %d x %d x %d)", lat->nx, lat->ny, lat->nz);
        return false;
    }
    if (lat->nspecies < 1 || lat->nspecies > kMaxSpecies) {
        set_error("nspecies must be in [1, %d] (got %d)", kMaxSpecies, lat->nspecies);
        return false;
    }
    if (4LL * lat->nx * lat->ny * lat->nz >= (1LL << 31)) {
        set_error("lattice too large: N = %lld sites (limit 2^31 - 1)", 4LL * lat->nx * lat->ny * lat->nz);
        return false;
    }
    return true;
}

static smc_status fcc_check(const smc_lattice *lat, const smc_model *model, const void *occ, bool sweep)
{
    if (!fcc_lattice_valid(lat) || !model_valid(lat, model)) return SMC_ERR_ARG;
    if (model->kind != SMC_PAIR_I32 && model->kind != SMC_PAIR_F32 && model->kind != SMC_QSRO_F32) {
        set_error("the FCC lattice takes pair models (SMC_PAIR_I32, SMC_PAIR_F32) and qSRO models only");
        return SMC_ERR_UNSUPPORTED;
    }
    if (!occ) {
        set_error("occ is NULL");
        return SMC_ERR_ARG;
    }
    if (sweep && !fcc_shape_ok(lat)) {
        set_error("FCC sweeps need every axis a multiple of 4 and >= 8 cells (got %d x %d x %d)", lat->nx, lat->ny,
                  lat->nz);
        return SMC_ERR_UNSUPPORTED;
    }
    return SMC_OK;
}

smc_status smc_fcc_init_lattice(const smc_lattice *lat, const int64_t *counts, uint64_t seed, uint32_t replica,
                                int8_t *occ, cudaStream_t stream)
{
    if (!fcc_lattice_valid(lat)) return SMC_ERR_ARG;
    // the same start-state order over N = 4 nx ny nz ids: a BCC box of 2nx x ny x nz
    const smc_lattice twice = {2 * lat->nx, lat->ny, lat->nz, lat->nspecies};
    return smc_init_lattice(&twice, counts, seed, replica, occ, stream);
}

smc_status smc_fcc_sweep(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                         uint32_t replica, uint64_t sweep0, int32_t nsweeps, const double *kT, double *e_acc,
                         int64_t *n_acc, cudaStream_t stream)
{
    API_LOCK;
    smc_status st = fcc_check(lat, model, occ, true);
    if (st != SMC_OK) return st;
    if (nsweeps < 0 || nsweeps > (1 << 24)) {
        set_error("nsweeps must be in [0, 2^24]");
        return SMC_ERR_ARG;
    }
    if (nsweeps > 0 && !kT) {
        set_error("kT is NULL");
        return SMC_ERR_ARG;
    }
    if (sweep0 + (uint64_t)nsweeps > 0xFFFFFFFFFFFFFFFEull || sweep0 + (uint64_t)nsweeps < sweep0) {
        set_error("sweep indices reach the reserved values 2^64-2, 2^64-1");
        return SMC_ERR_ARG;
    }
    for (int i = 0; i < nsweeps; ++i) {
        const double t = kT[i];
        if (!(t > 0.0) || (model->kind == SMC_PAIR_I32 && !std::isfinite(t))) {
            set_error("kT[%d] = %g is invalid (must be > 0; finite for integer models)", i, t);
            return SMC_ERR_ARG;
        }
        if (model->kind == SMC_PAIR_I32 && model->unit_ev / t < 29.0 * 0.6931471805599453 / (double)(1 << 24)) {
            set_error("kT[%d] too high for the integer acceptance table", i);
            return SMC_ERR_UNSUPPORTED;
        }
    }
    if (nsweeps == 0) return SMC_OK;
    return launch_fcc_sweep(lat, model, occ, seed, replica, sweep0, nsweeps, kT, e_acc, n_acc, nullptr, nullptr, -1,
                            stream);
}

smc_status smc_fcc_ministep_trace(const smc_lattice *lat, const smc_model *model, int8_t *occ, uint64_t seed,
                                  uint32_t replica, uint64_t sweep, int32_t k, double kT, float *dE, uint8_t *acc,
                                  cudaStream_t stream)
{
    API_LOCK;
    smc_status st = fcc_check(lat, model, occ, true);
    if (st != SMC_OK) return st;
    if (k < 0 || k >= 256) {
        set_error("mini-step %d out of range [0, 256)", k);
        return SMC_ERR_ARG;
    }
    if (sweep > 0xFFFFFFFFFFFFFFFDull) {
        set_error("sweep index reaches the reserved values 2^64-2, 2^64-1");
        return SMC_ERR_ARG;
    }
    if (!(kT > 0.0) || (model->kind == SMC_PAIR_I32 && !std::isfinite(kT))) {
        set_error("kT = %g is invalid (must be > 0; finite for integer models)", kT);
        return SMC_ERR_ARG;
    }
    if (model->kind == SMC_PAIR_I32 && model->unit_ev / kT < 29.0 * 0.6931471805599453 / (double)(1 << 24)) {
        set_error("kT too high for the integer acceptance table");
        return SMC_ERR_UNSUPPORTED;
    }
    return launch_fcc_sweep(lat, model, occ, seed, replica, sweep, 1, &kT, nullptr, nullptr, dE, acc, k, stream);
}

smc_status smc_fcc_energy(const smc_lattice *lat, const smc_model *model, const int8_t *occ, double *e,
                          int64_t *e_int, cudaStream_t stream)
{
    API_LOCK;
    smc_status st = fcc_check(lat, model, occ, false);
    if (st != SMC_OK) return st;
    if (e_int && model->kind != SMC_PAIR_I32) {
        set_error("e_int is only defined for integer models");
        return SMC_ERR_ARG;
    }
    return launch_fcc_energy(lat, model, occ, e, e_int, stream);
}

smc_status smc_sro(const smc_lattice *lat, int32_t nshells, const int8_t *occ, int64_t *counts, double *alpha,
                   cudaStream_t stream)
{
    API_LOCK;
    if (!lattice_valid(lat, false)) return SMC_ERR_ARG;
    if (nshells < 1 || nshells > kMaxShells || !occ) {
        set_error("nshells must be in [1, 3] and occ non-NULL");
        return SMC_ERR_ARG;
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    unsigned long long *cnt = (unsigned long long *)counts;
    if (!cnt) {
        cnt = (unsigned long long *)workspace_scratch(ws, sizeof(unsigned long long) * kMaxShells * 64, &st);
        if (!cnt) return st;
    }
    st = launch_pair_counts(lat, nshells, occ, cnt, stream);
    if (st != SMC_OK || !alpha) return st;
    return launch_sro_finish(lat, nshells, cnt, alpha, stream);
}

smc_status smc_energy(const smc_lattice *lat, const smc_model *model, const int8_t *occ, double *e, int64_t *e_int,
                      cudaStream_t stream)
{
    API_LOCK;
    if (!lattice_valid(lat, model && is_mlp(model)) || !model_valid(lat, model)) return SMC_ERR_ARG;
    if (!occ) {
        set_error("occ is NULL");
        return SMC_ERR_ARG;
    }
    if (e_int && model->kind != SMC_PAIR_I32) {
        set_error("e_int is only defined for integer models");
        return SMC_ERR_ARG;
    }
    if (is_mlp(model) || is_qsro(model)) {
        if (!e) {
            set_error("e is NULL");
            return SMC_ERR_ARG;
        }
        if (is_qsro(model)) return launch_qsro_energy(lat, model, occ, e, stream);
        return launch_mlp_energy(lat, model, occ, e, stream);
    }
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    unsigned long long *cnt =
        (unsigned long long *)workspace_scratch(ws, sizeof(unsigned long long) * kMaxShells * 64, &st);
    if (!cnt) return st;
    st = launch_pair_counts(lat, model->nshells, occ, cnt, stream);
    if (st != SMC_OK) return st;
    return launch_energy_finish(lat, model, cnt, e, e_int, stream);
}

int64_t smc_grad_size(const smc_lattice *lat, const smc_model *model)
{
    if (!lat || !model || lat->nspecies < 1) return -1;
    const int S = lat->nspecies;
    int64_t n = 0;
    if (has_pair(model)) n += (int64_t)model->nshells * S * (S + 1) / 2;
    if (model->kind == SMC_MLPNET_BF16) return -1;
    if (is_mlp(model)) n += 64 * 20 + 64 + 64 * 64 + 64 + 64 + 1;
    if (is_qsro(model)) n += (int64_t)model->nshells * S * (S + 1) / 2 + (int64_t)model->nshells * S + 1;
    return n;
}

smc_status smc_energy_grad(const smc_lattice *lat, const smc_model *model, const int8_t *occ, float *grad,
                           cudaStream_t stream)
{
    API_LOCK;
    if (!lattice_valid(lat, model && is_mlp(model)) || !model_valid(lat, model)) return SMC_ERR_ARG;
    if (!occ || !grad) {
        set_error("occ and grad must be non-NULL");
        return SMC_ERR_ARG;
    }
    if (model->kind == SMC_MLPNET_BF16) {
        set_error("smc_energy_grad does not take MLPNet models");
        return SMC_ERR_UNSUPPORTED;
    }
    if (is_mlp(model)) return launch_mlp_grad(lat, model, occ, grad, stream);
    if (is_qsro(model)) return launch_qsro_grad(lat, model, occ, grad, stream);
    smc_status st;
    Workspace *ws = workspace(&st);
    if (!ws) return st;
    unsigned long long *cnt =
        (unsigned long long *)workspace_scratch(ws, sizeof(unsigned long long) * kMaxShells * 64, &st);
    if (!cnt) return st;
    st = launch_pair_counts(lat, model->nshells, occ, cnt, stream);
    if (st != SMC_OK) return st;
    return launch_pair_grad_finish(lat, model, cnt, grad, stream);
}

smc_status smc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n, cudaStream_t stream)
{
    API_LOCK;
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) {
        set_error("invalid philox arguments");
        return SMC_ERR_ARG;
    }
    return launch_philox(ctr, key, out, n, stream);
}

}  // extern "C"
