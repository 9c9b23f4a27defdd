// fs_api.cu - the C ABI of include/fstat.h: plan lifetime, workspace and
// the launch sequence of one batched F-statistic evaluation.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fs_internal.h"

namespace {

thread_local char g_err[512] = "";

fs_status fail(fs_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

fs_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) return fail(FS_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

fs_status fs::set_error(fs_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

struct fs_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    cudaStream_t stream;
};

struct fs_plan {
    fs::Grid grid;
    int mode;
    int device;
    cudaStream_t stream;
    int tdi;                          // FS_TDI_X or FS_TDI_AE
    int nch;                          // channels of the data (1 or 2)
    fs::Tables tab[fs::kMaxChannels]; // per channel: shared frequency tables, the channel's dw and W
    double* tab_base;
    int data_set;
    // workspace
    int B_cap, Np_cap;
    fs::Particle* parts;
    double* H;
    double* T;
    double* S;
    double* Fpart;
    double2* rot;
    float2* rot32;
    int ntiles;
    // mixed mode: FP32 (dw, W) tables [nch][n] and their common scale exponent
    float4* tab32;
    int* emax;
    // launch variant of the fused kernel: forced (>= 0) or looked up per
    // (N_p, edge kind) among the autotuned choices, else variant 0
    int variant_forced;
    // response of the FP64 path: the paper's form (resp_on = 0) or the series of Eq. (freDres)
    int resp_on;
    fs::Resp resp;
    // orbits of the FP64 path: 0 the rigid constellation, > 0 to second order in this eccentricity
    double orbit_e;
    // response of the FP64 path: 0 long-wavelength, > 0 the finite-arm TDI response with this arm (s)
    double arm_s;
    unsigned long long* census;   // [fs::kCensusModes] device counters of fs_plan_census
    int census_on;
    struct TuneRec {
        int Np, global, variant;
    };
    static constexpr int kTuneMax = 64;
    TuneRec tuned[kTuneMax];
    int n_tuned;
    int* span_list;      // [B][nspans] in-band particles per span (mixed path)
    int* span_cnt;       // span_sched_ints(nspans): counts, item prefixes, persistent-kernel counters
    // swarm evaluation scratch and the captured PSO iteration
    fs_params* pso_params;   // [B_cap]
    double* pso_F;           // [B_cap]
    // surrogate screening candidates
    int64_t cand_cap;
    double *cand_x, *cand_v;
    float *cand_in, *cand_score;
    unsigned char* cand_inside;

    // segment start bins of the current call (global mode; converted on the device from the
    // caller's edge frequencies at the start of every evaluation) and the sticky error flags
    int64_t* edges_dev;
    int* flags_dev;   // [0] sticky flags (fs_plan_check), [1] scratch of the grid check
    double2* cis;     // FS_FP64: exp(2 pi i j 2^-20) table of the anchored kernels (16 MB)
    // single-particle scratch for fs_add_signal
    fs_params* one_param;
    fs::Particle* one_part;
    double* one_a;
    // kernel timing
    struct ProfRec {
        int kind;
        cudaEvent_t a, b;
    };
    int profiling;
    std::vector<ProfRec>* prof;       // recorded, unread
    std::vector<cudaEvent_t>* spare;  // reusable events
};

namespace {

constexpr int kKinds = 4;

// Launch variants of the fused kernel.  FS_FP64: direct form with a tile of
// 2048, 1024 or 4096 bins per (particle, tile) item, anchored form (grid or
// persistent).  FS_MIXED: grid form with 2 or 3 resident CTAs per SM,
// persistent form with 2 or 3, grid form with the tables staged through
// shared memory by bulk copies.
int n_variants(int mode) { return 5; }

int fp64_tile(int variant) { return variant == 1 ? 1024 : variant == 2 ? 4096 : fs::kTile; }

// The grid as channel c of the plan's channel set sees it (orientation and projection scale).
fs::Grid channel_grid(const fs_plan* p, int c) {
    fs::Grid g = p->grid;
    const fs::Channel ch = fs::channel_of(p->tdi, c);
    if ((p->orbit_e > 0.0 || p->arm_s > 0.0) && p->mode == FS_FP64) {
        // the eccentric orbits' patterns (and the finite-arm response) are formed per channel
        // from the three arms
        g.orb.e = p->orbit_e;
        g.orb.L = p->arm_s;
        g.orb.chan = p->tdi == FS_TDI_X ? 0 : 1 + c;
        for (int k = 0; k < 3; k++) {
            const double b = 2.0 * fs::kPi * k / 3.0 + p->grid.orient;
            g.orb.cb[k] = cos(b);
            g.orb.sb[k] = sin(b);
            g.orb.c2b[k] = cos(2.0 * b);
            g.orb.s2b[k] = sin(2.0 * b);
        }
    }
    g.orient += ch.orient_shift;
    g.pscale = ch.pscale;
    return g;
}

// Untuned default: the anchored persistent form (FS_FP64), the persistent
// form with 3 CTAs per SM (FS_MIXED).
int default_variant(int mode) { return mode == FS_MIXED ? 3 : 4; }

int resolve_variant(const fs_plan* p, int Np, int global) {
    if (p->variant_forced >= 0) return p->variant_forced;
    for (int i = 0; i < p->n_tuned; i++)
        if (p->tuned[i].Np == Np && p->tuned[i].global == global) return p->tuned[i].variant;
    return default_variant(p->mode);
}

void record_tuned(fs_plan* p, int Np, int global, int variant) {
    for (int i = 0; i < p->n_tuned; i++)
        if (p->tuned[i].Np == Np && p->tuned[i].global == global) {
            p->tuned[i].variant = variant;
            return;
        }
    if (p->n_tuned < fs_plan::kTuneMax) p->tuned[p->n_tuned++] = {Np, global, variant};
}

cudaEvent_t take_event(fs_plan* p) {
    if (!p->spare->empty()) {
        cudaEvent_t e = p->spare->back();
        p->spare->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Bracket a launch sequence with events when profiling is on.
struct ProfScope {
    fs_plan* p;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(fs_plan* pl, int k) : p(pl), kind(k) {
        if (p->profiling) {
            a = take_event(p);
            if (a) cudaEventRecord(a, p->stream);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEvent_t b = take_event(p);
            if (b) {
                cudaEventRecord(b, p->stream);
                p->prof->push_back({kind, a, b});
            } else {
                p->spare->push_back(a);
            }
        }
    }
};

void free_workspace(fs_plan* p) {
    cudaFree(p->parts);
    cudaFree(p->H);
    cudaFree(p->T);
    cudaFree(p->S);
    cudaFree(p->Fpart);
    cudaFree(p->rot);
    cudaFree(p->rot32);
    cudaFree(p->span_list);
    cudaFree(p->span_cnt);
    cudaFree(p->pso_params);
    cudaFree(p->pso_F);
    p->pso_params = nullptr;
    p->pso_F = nullptr;
    p->span_list = p->span_cnt = nullptr;
    p->parts = nullptr;
    p->rot = nullptr;
    p->rot32 = nullptr;
    p->H = p->T = p->S = p->Fpart = nullptr;
    p->B_cap = p->Np_cap = 0;
}

// sums per partial slot the workspace is sized for: 7, or 8 with the response series
constexpr size_t kSlotMax = 8;

fs_status ensure_workspace(fs_plan* p, int B, int Np) {
    if (B <= p->B_cap && Np <= p->Np_cap) return FS_OK;
    int nb = B > p->B_cap ? B : p->B_cap;
    int nn = Np > p->Np_cap ? Np : p->Np_cap;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    free_workspace(p);
    size_t nt = (size_t)p->ntiles;
    const size_t nc = (size_t)p->nch;
    if ((e = cudaMalloc(&p->parts, sizeof(fs::Particle) * nb * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->H, sizeof(double) * kSlotMax * nt * nb * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->T, sizeof(double) * kSlotMax * nt * nb * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->S, sizeof(double) * kSlotMax * (size_t)nn * nb * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->Fpart, sizeof(double) * (size_t)nn * nb)) != cudaSuccess ||
        (e = cudaMalloc(&p->rot, sizeof(double2) * (size_t)nn * nb)) != cudaSuccess ||
        (e = cudaMalloc(&p->rot32, sizeof(float2) * (size_t)nn * nb)) != cudaSuccess ||
        (e = cudaMalloc(&p->span_list, sizeof(int) * (size_t)nb * (nt > 0 ? nt : 1))) != cudaSuccess ||
        (e = cudaMalloc(&p->span_cnt, sizeof(int) * fs::span_sched_ints(nt))) != cudaSuccess ||
        (e = cudaMemsetAsync(p->span_cnt, 0, sizeof(int) * fs::span_sched_ints(nt), p->stream)) != cudaSuccess ||
        (e = cudaMalloc(&p->pso_params, sizeof(fs_params) * (size_t)nb)) != cudaSuccess ||
        (e = cudaMalloc(&p->pso_F, sizeof(double) * (size_t)nb)) != cudaSuccess) {
        free_workspace(p);
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    p->B_cap = nb;
    p->Np_cap = nn;
    return FS_OK;
}

// Candidate buffers of the screened step (grown synchronously, never during capture).
fs_status ensure_candidates(fs_plan* p, int64_t nc) {
    if (nc <= p->cand_cap) return FS_OK;
    cudaError_t e;
    if ((e = cudaStreamSynchronize(p->stream)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    cudaFree(p->cand_x);
    cudaFree(p->cand_v);
    cudaFree(p->cand_in);
    cudaFree(p->cand_score);
    cudaFree(p->cand_inside);
    p->cand_x = p->cand_v = nullptr;
    p->cand_in = p->cand_score = nullptr;
    p->cand_inside = nullptr;
    p->cand_cap = 0;
    if ((e = cudaMalloc(&p->cand_x, sizeof(double) * 5 * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->cand_v, sizeof(double) * 5 * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->cand_in, sizeof(float) * 5 * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->cand_score, sizeof(float) * nc)) != cudaSuccess ||
        (e = cudaMalloc(&p->cand_inside, nc)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(candidates)");
    p->cand_cap = nc;
    return FS_OK;
}

}  // namespace

extern "C" {

const char* fs_last_error(void) { return g_err; }

fs_status fs_constants(double* out) {
    if (!out) return fail(FS_EINVAL, "fs_constants: out is NULL");
    out[0] = fs::kMsunS;
    out[1] = fs::kYearS;
    out[2] = fs::kAuS;
    out[3] = fs::kF0Ecc;
    return FS_OK;
}

fs_status fs_plan_create(fs_plan** out, int64_t n_bins, double f_min, double df, double T_obs, int mode,
                         void* stream) {
    return fs_plan_create_tdi(out, n_bins, f_min, df, T_obs, mode, FS_TDI_X, stream);
}

int fs_plan_channels(const fs_plan* p) { return p ? p->nch : -1; }

fs_status fs_plan_create_tdi(fs_plan** out, int64_t n_bins, double f_min, double df, double T_obs, int mode,
                             int tdi, void* stream) {
    g_err[0] = 0;
    if (!out) return fail(FS_EINVAL, "fs_plan_create: out is NULL");
    if (tdi != FS_TDI_X && tdi != FS_TDI_AE) return fail(FS_EINVAL, "fs_plan_create_tdi: unknown channel set %d", tdi);
    *out = nullptr;
    if (n_bins <= 0 || !(f_min > 0.0) || !(df > 0.0) || !(T_obs > 0.0) || !isfinite(f_min) || !isfinite(df) ||
        !isfinite(T_obs))
        return fail(FS_EINVAL, "fs_plan_create: need n_bins > 0 and finite f_min, df, T_obs > 0");
    if (mode != FS_FP64 && mode != FS_MIXED) return fail(FS_EINVAL, "fs_plan_create: unknown mode %d", mode);
    if (mode == FS_MIXED && n_bins >= ((int64_t)1 << 31))
        return fail(FS_EINVAL, "fs_plan_create: FS_MIXED needs n_bins < 2^31");
    if (n_bins > ((int64_t)1 << 40)) return fail(FS_EINVAL, "fs_plan_create: n_bins too large");
    fs_plan* p = new (std::nothrow) fs_plan;
    if (!p) return fail(FS_ENOMEM, "fs_plan_create: host allocation failed");
    memset(p, 0, sizeof(*p));
    p->grid.n = n_bins;
    p->grid.f_min = f_min;
    p->grid.df = df;
    p->grid.T_obs = T_obs;
    p->grid.alpha0 = 0.0;
    p->grid.orient = 0.0;
    p->grid.pscale = 1.0;
    p->tdi = tdi;
    p->nch = tdi == FS_TDI_AE ? 2 : 1;
    p->mode = mode;
    p->stream = (cudaStream_t)stream;
    p->ntiles = (int)((n_bins + fs::kTileMin - 1) / fs::kTileMin);
    p->variant_forced = -1;
    p->n_tuned = 0;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    // six frequency tables shared by the channels, then (dw re, dw im, W) per channel
    size_t bytes = sizeof(double) * (size_t)n_bins * (6 + 3 * (size_t)p->nch);
    if ((e = cudaMalloc(&p->tab_base, bytes)) != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaMalloc(tables)");
    }
    double* q = p->tab_base;
    for (int c = 0; c < p->nch; c++) {
        fs::Tables& t = p->tab[c];
        double** slots[fs::kNumTables] = {&t.fh, &t.fl, &t.u, &t.g0h, &t.g0l, &t.e19, &t.dwr, &t.dwi, &t.W};
        for (int i = 0; i < fs::kNumTables; i++) {
            const size_t slot = i < 6 ? (size_t)i : 6 + 3 * (size_t)c + (i - 6);
            *slots[i] = q + slot * n_bins;
        }
    }
    if ((e = cudaMalloc(&p->edges_dev, sizeof(int64_t) * (fs::kNpMax + 2))) != cudaSuccess ||
        (e = cudaMalloc(&p->flags_dev, 2 * sizeof(int))) != cudaSuccess ||
        (e = cudaMemsetAsync(p->flags_dev, 0, 2 * sizeof(int), p->stream)) != cudaSuccess ||
        (e = cudaMalloc(&p->one_param, sizeof(fs_params))) != cudaSuccess ||
        (e = cudaMalloc(&p->one_part, sizeof(fs::Particle))) != cudaSuccess ||
        (e = cudaMalloc(&p->one_a, sizeof(double) * 4)) != cudaSuccess) {
        fs_plan_destroy(p);
        return cuda_fail(e, "cudaMalloc(plan)");
    }
    if (mode == FS_FP64 &&
        ((e = cudaMalloc(&p->cis, sizeof(double2) << fs::kCisBits)) != cudaSuccess ||
         (e = fs::launch_cis_table(p->cis, p->stream)) != cudaSuccess)) {
        fs_plan_destroy(p);
        return cuda_fail(e, "exp table");
    }
    if (mode == FS_MIXED &&
        ((e = cudaMalloc(&p->tab32, sizeof(float4) * (size_t)n_bins * p->nch)) != cudaSuccess ||
         (e = cudaMalloc(&p->emax, sizeof(int))) != cudaSuccess)) {
        fs_plan_destroy(p);
        return cuda_fail(e, "cudaMalloc(mixed tables)");
    }
    p->prof = new std::vector<fs_plan::ProfRec>();
    p->spare = new std::vector<cudaEvent_t>();
    *out = p;
    return FS_OK;
}

fs_status fs_plan_destroy(fs_plan* p) {
    if (!p) return FS_OK;
    cudaStreamSynchronize(p->stream);
    free_workspace(p);
    cudaFree(p->census);
    cudaFree(p->tab_base);
    cudaFree(p->edges_dev);
    cudaFree(p->flags_dev);
    cudaFree(p->cis);
    cudaFree(p->one_param);
    cudaFree(p->one_part);
    cudaFree(p->one_a);
    cudaFree(p->tab32);
    cudaFree(p->emax);
    cudaFree(p->cand_x);
    cudaFree(p->cand_v);
    cudaFree(p->cand_in);
    cudaFree(p->cand_score);
    cudaFree(p->cand_inside);
    if (p->prof) {
        for (auto& r : *p->prof) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        delete p->prof;
    }
    if (p->spare) {
        for (auto e : *p->spare) cudaEventDestroy(e);
        delete p->spare;
    }
    delete p;
    return FS_OK;
}

fs_status fs_plan_set_data(fs_plan* p, const double* data_dev, const double* psd_dev, const double* f_grid_dev) {
    g_err[0] = 0;
    if (!p || !data_dev || !psd_dev) return fail(FS_EINVAL, "fs_plan_set_data: NULL argument");
    if (f_grid_dev) {
        // the kernels step the phase in the bin index, which needs the uniform grid
        // f_k = f_min + k df: check the caller's grid against it and wait for the answer
        // the check's own word (flags_dev[1]), so that the sticky word keeps what it holds
        int h = 0;
        cudaError_t e;
        if ((e = cudaMemsetAsync(p->flags_dev + 1, 0, sizeof(int), p->stream)) != cudaSuccess ||
            (e = fs::launch_grid_check(p->grid, f_grid_dev, p->flags_dev + 1, p->stream)) != cudaSuccess ||
            (e = cudaMemcpyAsync(&h, p->flags_dev + 1, sizeof(int), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess ||
            (e = cudaStreamSynchronize(p->stream)) != cudaSuccess)
            return cuda_fail(e, "fs_plan_set_data: grid check");
        if (h & fs::kFlagBadGrid)
            return fail(FS_EUNSUPPORTED,
                        "fs_plan_set_data: f_grid is not the uniform grid f_min + k df of the plan (to 4 ulp); "
                        "non-uniform grids are not supported");
    }
    ProfScope ps(p, 3);
    cudaError_t e;
    for (int c = 0; c < p->nch; c++)   // channel c's data and PSD follow channel c - 1's
        if ((e = fs::launch_precompute(p->grid, data_dev + (size_t)2 * p->grid.n * c, psd_dev + (size_t)p->grid.n * c,
                                       p->tab[c], p->stream)) != cudaSuccess)
            return cuda_fail(e, "precompute launch");
    if (p->mode == FS_MIXED &&
        (e = fs::launch_tables32(p->grid, p->tab, p->nch, p->emax, p->tab32, p->stream)) != cudaSuccess)
        return cuda_fail(e, "mixed tables launch");
    p->data_set = 1;
    return FS_OK;
}

fs_status fs_plan_reserve(fs_plan* p, int B_max, int Np_max) {
    g_err[0] = 0;
    if (!p || B_max < 0 || Np_max < 1 || Np_max > fs::kNpMax)
        return fail(FS_EINVAL, "fs_plan_reserve: need B_max >= 0 and 1 <= Np_max <= %d", fs::kNpMax);
    return ensure_workspace(p, B_max > 0 ? B_max : 1, Np_max);
}

fs_status fs_plan_check(fs_plan* p, int* flags_out) {
    g_err[0] = 0;
    if (flags_out) *flags_out = 0;
    if (!p) return fail(FS_EINVAL, "fs_plan_check: plan is NULL");
    int h = 0;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(&h, p->flags_dev, sizeof(int), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(p->flags_dev, 0, sizeof(int), p->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(p->stream)) != cudaSuccess)
        return cuda_fail(e, "fs_plan_check");
    if (flags_out) *flags_out = h;
    if (h & fs::kFlagTimeout)
        return fail(FS_ETIMEOUT, "fs_plan_check: a bounded device-side wait of an earlier call ran out (its F values "
                                 "are invalid)");
    if (h & fs::kFlagBadEdges)
        return fail(FS_EINVAL, "fs_plan_check: an earlier call was given partition edges that are not finite or "
                               "decrease (its F values are NaN)");
    return FS_OK;
}

namespace {
fs_status fstat_impl(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np,
                     double* F_dev, double* F_part_dev, double* amp_dev);
}

fs_status fs_fstat_batch(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np,
                         double* F_dev, double* F_part_dev) {
    g_err[0] = 0;
    return fstat_impl(p, params_dev, B, edges_dev, Np, F_dev, F_part_dev, nullptr);
}

fs_status fs_amplitudes(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np,
                        double* F_dev, double* a_dev, double* ext_dev) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_amplitudes: plan is NULL");
    if (!a_dev) return fail(FS_EINVAL, "fs_amplitudes: a is NULL");
    if (B <= 0) return B == 0 ? FS_OK : fail(FS_EINVAL, "fs_amplitudes: B = %d < 0", B);
    if (Np < 1 || Np > fs::kNpMax) return fail(FS_EINVAL, "fs_amplitudes: N_p = %d not in [1, %d]", Np, fs::kNpMax);
    fs_status st = ensure_workspace(p, B, Np);
    if (st != FS_OK) return st;
    if ((st = fstat_impl(p, params_dev, B, edges_dev, Np, F_dev ? F_dev : p->pso_F, nullptr, a_dev)) != FS_OK)
        return st;
    if (ext_dev) {
        cudaError_t e = fs::launch_extrinsic((int64_t)B * Np, a_dev, ext_dev, p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "extrinsic launch");
    }
    return FS_OK;
}

fs_status fs_plan_census(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np,
                         int64_t* counts) {
    g_err[0] = 0;
    if (!p || !counts) return fail(FS_EINVAL, "fs_plan_census: NULL plan or counts");
    for (int i = 0; i < fs::kCensusModes; i++) counts[i] = 0;
    if (B <= 0) return B == 0 ? FS_OK : fail(FS_EINVAL, "fs_plan_census: B = %d < 0", B);
    cudaError_t e;
    if (!p->census && (e = cudaMalloc(&p->census, fs::kCensusModes * sizeof(unsigned long long))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(census)");
    fs_status st = ensure_workspace(p, B, Np);
    if (st != FS_OK) return st;
    if ((e = cudaMemsetAsync(p->census, 0, fs::kCensusModes * sizeof(unsigned long long), p->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(census)");
    p->census_on = 1;
    st = fstat_impl(p, params_dev, B, edges_dev, Np, p->pso_F, nullptr, nullptr);
    p->census_on = 0;
    if (st != FS_OK) return st;
    unsigned long long h[fs::kCensusModes];
    if ((e = cudaMemcpyAsync(h, p->census, sizeof(h), cudaMemcpyDeviceToHost, p->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(p->stream)) != cudaSuccess)
        return cuda_fail(e, "census read-back");
    for (int i = 0; i < fs::kCensusModes; i++) counts[i] = (int64_t)h[i];
    return FS_OK;
}

namespace {
fs_status fstat_impl(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np,
                     double* F_dev, double* F_part_dev, double* amp_dev) {
    if (!p) return fail(FS_EINVAL, "fs_fstat_batch: plan is NULL");
    if (B < 0) return fail(FS_EINVAL, "fs_fstat_batch: B = %d < 0", B);
    if (Np < 1 || Np > fs::kNpMax) return fail(FS_EINVAL, "fs_fstat_batch: N_p = %d not in [1, %d]", Np, fs::kNpMax);
    if (B > 65535 * 8) return fail(FS_EINVAL, "fs_fstat_batch: B = %d exceeds %d", B, 65535 * 8);
    if (B == 0) return FS_OK;
    if (!params_dev || !F_dev) return fail(FS_EINVAL, "fs_fstat_batch: NULL params or F");
    if (!p->data_set) return fail(FS_EINVAL, "fs_fstat_batch: fs_plan_set_data was not called");
    const int global = edges_dev != nullptr;
    fs_status st = ensure_workspace(p, B, Np);
    if (st != FS_OK) return st;
    cudaError_t e;
    // segment starts from the caller's edge frequencies, on the stream (no host wait)
    if (global && (e = fs::launch_edges(p->grid, edges_dev, Np, p->edges_dev, p->flags_dev, p->stream)) != cudaSuccess)
        return cuda_fail(e, "edges launch");
    fs::Segs sg;
    sg.Np = Np;
    sg.global = global;
    sg.edges = p->edges_dev;
    fs::Partials pa;
    pa.census = p->census_on ? p->census : nullptr;
    pa.flags = p->flags_dev;
    pa.cis = p->cis;
    pa.H = p->H;
    pa.T = p->T;
    pa.S = p->S;
    pa.rot = p->rot;
    const bool mixed = p->mode == FS_MIXED;
    pa.rot32 = mixed ? p->rot32 : nullptr;
    const int variant = resolve_variant(p, Np, global);
    // the response series runs in the direct form only (the anchored form's expansions
    // are built for the paper's response): its variants 3 and 4 take the default tile
    const bool mb = !mixed && p->resp_on;
    const bool fin = !mixed && p->arm_s > 0.0;
    // the eccentric orbits and the finite-arm response run in the direct form too
    const bool direct_only = mb || fin || (!mixed && p->orbit_e > 0.0);
    const bool anchored = !mixed && !direct_only && variant >= 3;
    pa.nsum = (mb || fin) ? 8 : 7;
    pa.tile = mixed ? fs::mixed_span() : anchored ? fs::fp64a_span() : fp64_tile(direct_only && variant >= 3 ? 0 : variant);
    pa.ntiles = (int)((p->grid.n + pa.tile - 1) / pa.tile);
    double* Fpart = F_part_dev ? F_part_dev : p->Fpart;
    // channel c: its response (turned orientation, scaled projections), its particles and partial sums
    pa.nch = p->nch;
    pa.ch_HT = (int64_t)pa.nsum * p->ntiles * p->B_cap;
    pa.ch_S = (int64_t)pa.nsum * p->Np_cap * p->B_cap;
    {
        ProfScope ps(p, 0);
        for (int c = 0; c < p->nch; c++)
            if ((e = fs::launch_setup(channel_grid(p, c), params_dev, B, p->parts + (size_t)c * p->B_cap, global,
                                      p->stream)) != cudaSuccess)
                return cuda_fail(e, "setup launch");
        // one basis rotation per segment for every channel (channel 0's patterns at its centre): the
        // amplitudes are common to the channels, so their sums must share the basis
        if ((e = fs::launch_rotation(p->grid, p->parts, B, sg, p->rot, pa.rot32, p->stream)) != cudaSuccess)
            return cuda_fail(e, "rotation launch");
    }
    {
        ProfScope ps(p, 1);
        for (int c = 0; c < p->nch; c++) {
            const fs::Grid gc = channel_grid(p, c);
            const fs::Particle* pc = p->parts + (size_t)c * p->B_cap;
            fs::Partials pc_pa = pa;
            pc_pa.H = pa.H + c * pa.ch_HT;
            pc_pa.T = pa.T + c * pa.ch_HT;
            pc_pa.S = pa.S + c * pa.ch_S;
            if (mixed) {
                if ((e = fs::launch_mixed_main(gc, p->tab[c], p->tab32 + (size_t)c * p->grid.n, pc, B, sg, pc_pa,
                                               variant, p->span_list, p->span_cnt, p->stream)) != cudaSuccess)
                    return cuda_fail(e, "mixed main launch");
            } else if (anchored) {
                if ((e = fs::launch_fp64a_main(gc, p->tab[c], pc, B, sg, pc_pa, variant == 4, p->span_list,
                                               p->span_cnt, p->stream)) != cudaSuccess)
                    return cuda_fail(e, "fp64 anchored main launch");
            } else if ((e = fs::launch_fp64_main(gc, p->tab[c], pc, B, sg, pc_pa, p->stream,
                                                 mb ? &p->resp : nullptr)) != cudaSuccess) {
                return cuda_fail(e, "fp64 main launch");
            }
        }
    }
    {
        ProfScope ps(p, 2);
        if ((e = fs::launch_reduce(p->grid, p->parts, B, sg, pa, Fpart, F_dev, p->stream, amp_dev,
                                   mixed ? p->emax : nullptr)) != cudaSuccess)
            return cuda_fail(e, "reduce launch");
    }
    return FS_OK;
}
}  // namespace

fs_status fs_mixed_probe(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np, int b,
                         int64_t k0, int64_t nbins, float* out_dev) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_mixed_probe: plan is NULL");
    if (p->mode != FS_MIXED) return fail(FS_EINVAL, "fs_mixed_probe: the plan is not FS_MIXED");
    if (B < 1 || b < 0 || b >= B) return fail(FS_EINVAL, "fs_mixed_probe: need 0 <= b < B");
    if (Np < 1 || Np > fs::kNpMax) return fail(FS_EINVAL, "fs_mixed_probe: N_p = %d not in [1, %d]", Np, fs::kNpMax);
    if (k0 < 0 || nbins < 0 || k0 + nbins > p->grid.n)
        return fail(FS_EINVAL, "fs_mixed_probe: bins [k0, k0 + nbins) must lie in [0, n_bins)");
    if (!params_dev || (nbins > 0 && !out_dev)) return fail(FS_EINVAL, "fs_mixed_probe: NULL params or out");
    if (!p->data_set) return fail(FS_EINVAL, "fs_mixed_probe: fs_plan_set_data was not called");
    fs_status st = ensure_workspace(p, B, Np);
    if (st != FS_OK) return st;
    const int global = edges_dev != nullptr;
    cudaError_t e;
    if (global && (e = fs::launch_edges(p->grid, edges_dev, Np, p->edges_dev, p->flags_dev, p->stream)) != cudaSuccess)
        return cuda_fail(e, "edges launch");
    fs::Segs sg;
    sg.Np = Np;
    sg.global = global;
    sg.edges = p->edges_dev;
    fs::Partials pa;
    pa.H = p->H;
    pa.T = p->T;
    pa.S = p->S;
    pa.rot = p->rot;
    pa.rot32 = p->rot32;
    pa.tile = fs::mixed_span();
    pa.ntiles = (int)((p->grid.n + pa.tile - 1) / pa.tile);
    const fs::Grid g0 = channel_grid(p, 0);
    if ((e = fs::launch_setup(g0, params_dev, B, p->parts, global, p->stream)) != cudaSuccess ||
        (e = fs::launch_rotation(g0, p->parts, B, sg, p->rot, p->rot32, p->stream)) != cudaSuccess ||
        (e = fs::launch_mixed_probe(g0, p->tab[0], p->tab32, p->parts, sg, pa, b, k0, k0 + nbins, out_dev,
                                    p->stream)) != cudaSuccess)
        return cuda_fail(e, "probe launch");
    return FS_OK;
}

fs_status fs_particle_bands(fs_plan* p, const fs_params* params_dev, int B, int64_t* bands_dev) {
    g_err[0] = 0;
    if (!p || B < 0) return fail(FS_EINVAL, "fs_particle_bands: bad plan or B");
    if (B == 0) return FS_OK;
    if (!params_dev || !bands_dev) return fail(FS_EINVAL, "fs_particle_bands: NULL argument");
    fs_status st = ensure_workspace(p, B, p->Np_cap > 0 ? p->Np_cap : 1);
    if (st != FS_OK) return st;
    cudaError_t e;
    if ((e = fs::launch_setup(channel_grid(p, 0), params_dev, B, p->parts, 0, p->stream)) != cudaSuccess)
        return cuda_fail(e, "setup launch");
    if ((e = fs::launch_bands(p->parts, B, bands_dev, p->stream)) != cudaSuccess)
        return cuda_fail(e, "bands launch");
    return FS_OK;
}

// Dimensions of a swarm's search space: 5, or 6 with delta_mu free (0 reads as 5).
static int swarm_dims(const fs_swarm* w) { return w->dims == 6 ? 6 : 5; }

static fs_status check_swarm(const fs_swarm* w) {
    if (!w || w->R < 0 || w->n_part < 1 || !w->x || !w->v || !w->pbest_x || !w->pbest_f || !w->fit)
        return fail(FS_EINVAL, "swarm: need R >= 0, n_part >= 1 and non-NULL state arrays");
    if (w->dims != 0 && w->dims != 5 && w->dims != 6) return fail(FS_EINVAL, "swarm: dims must be 5 or 6");
    if ((int64_t)w->R * w->n_part > 65535 * 8) return fail(FS_EINVAL, "swarm: R * n_part too large");
    if (w->run0 < 0 || (int64_t)w->run0 + w->R > (1 << 20))
        return fail(FS_EINVAL, "swarm: need 0 <= run0 and run0 + R <= 2^20 (the Philox run field)");
    return FS_OK;
}

fs_status fs_pso_init(fs_plan* p, const fs_swarm* w, uint64_t seed) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_pso_init: plan is NULL");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    cudaError_t e = fs::launch_pso_init(w->R, w->n_part, swarm_dims(w), seed, w->x, w->v, w->pbest_x, w->pbest_f,
                                        w->fit, w->run0,
                                        p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pso init launch");
    if (w->iter && (e = cudaMemsetAsync(w->iter, 0, sizeof(unsigned int), p->stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(iter)");
    return FS_OK;
}

fs_status fs_pso_evaluate(fs_plan* p, const fs_swarm* w, const double* edges_dev, int Np) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_pso_evaluate: plan is NULL");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (!w->box) return fail(FS_EINVAL, "fs_pso_evaluate: box is NULL");
    const int n = w->R * w->n_part;
    if (n == 0) return FS_OK;
    if ((st = ensure_workspace(p, n, Np)) != FS_OK) return st;
    cudaError_t e = fs::launch_pso_map(w->R, w->n_part, swarm_dims(w), w->x, w->box, w->q, p->pso_params, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pso map launch");
    if ((st = fs_fstat_batch(p, p->pso_params, n, edges_dev, Np, p->pso_F, nullptr)) != FS_OK) return st;
    if ((e = fs::launch_pso_fitness(n, p->pso_F, Np, w->fit, p->stream)) != cudaSuccess)
        return cuda_fail(e, "pso fitness launch");
    return FS_OK;
}

fs_status fs_pso_autotune(fs_plan* p, const fs_swarm* w, const double* edges_dev, int Np, int reps,
                          int* variant_out, float* ms_out) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_pso_autotune: plan is NULL");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (!w->box) return fail(FS_EINVAL, "fs_pso_autotune: box is NULL");
    const int n = w->R * w->n_part;
    if (n == 0) return fail(FS_EINVAL, "fs_pso_autotune: empty swarm");
    if ((st = ensure_workspace(p, n, Np)) != FS_OK) return st;
    cudaError_t e = fs::launch_pso_map(w->R, w->n_part, swarm_dims(w), w->x, w->box, w->q, p->pso_params, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pso map launch");
    return fs_plan_autotune(p, p->pso_params, n, edges_dev, Np, reps, variant_out, ms_out);
}

fs_status fs_pso_step(fs_plan* p, const fs_swarm* w, uint64_t seed, int iteration, double w0, double w1, int n_iter,
                      double c1, double c2, double vmax, int* lbest_dev) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_pso_step: plan is NULL");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (n_iter < 1 || !(vmax > 0.0)) return fail(FS_EINVAL, "fs_pso_step: need n_iter >= 1 and vmax > 0");
    if (iteration < 0 && !w->iter) return fail(FS_EINVAL, "fs_pso_step: iteration < 0 needs swarm->iter");
    const bool dev_iter = iteration < 0;
    cudaError_t e = fs::launch_pso_step(w->R, w->n_part, swarm_dims(w), seed, dev_iter ? w->iter : nullptr,
                                        dev_iter ? 0u : (unsigned int)iteration, w0, w1, n_iter, c1, c2, vmax, w->x,
                                        w->v, w->pbest_x, w->pbest_f, w->fit, lbest_dev,
                                        dev_iter ? w->iter : nullptr, w->run0, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pso step launch");
    return FS_OK;
}

fs_status fs_pso_step_screened(fs_plan* p, const fs_swarm* w, fs_mlp* const* mlps, int n_mlp, int n_cand,
                               uint64_t seed, int iteration, double w0, double w1, int n_iter, double c1, double c2,
                               double vmax) {
    g_err[0] = 0;
    if (!p || !mlps || n_mlp < 1) return fail(FS_EINVAL, "fs_pso_step_screened: NULL plan or no network");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (swarm_dims(w) != 5)
        return fail(FS_EUNSUPPORTED, "fs_pso_step_screened: the surrogate networks take 5 inputs; the swarm has 6 "
                                     "dimensions");
    int ng = 0;
    for (int i = 0; i < n_mlp; i++) {
        if (!mlps[i]) return fail(FS_EINVAL, "fs_pso_step_screened: network %d is NULL", i);
        ng += fs_mlp_groups(mlps[i]);
    }
    if (w->R % ng != 0)
        return fail(FS_EINVAL, "fs_pso_step_screened: R = %d is not a multiple of the %d network groups", w->R, ng);
    if (n_cand < 1 || n_cand > 64) return fail(FS_EINVAL, "fs_pso_step_screened: n_cand must be in [1, 64]");
    if (n_iter < 1 || !(vmax > 0.0)) return fail(FS_EINVAL, "fs_pso_step_screened: need n_iter >= 1 and vmax > 0");
    if (iteration < 0 && !w->iter) return fail(FS_EINVAL, "fs_pso_step_screened: iteration < 0 needs swarm->iter");
    const int64_t nc = (int64_t)w->R * w->n_part * n_cand;
    if ((st = ensure_candidates(p, nc)) != FS_OK) return st;
    cudaError_t e;
    const bool dev_iter = iteration < 0;
    e = fs::launch_pso_screened(w->R, w->n_part, n_cand, seed, dev_iter ? w->iter : nullptr,
                                dev_iter ? 0u : (unsigned int)iteration, w0, w1, n_iter, c1, c2, vmax, w->x, w->v,
                                w->pbest_x, w->pbest_f, w->fit, p->cand_x, p->cand_v, p->cand_in, p->cand_inside,
                                p->cand_score, mlps, n_mlp, dev_iter ? w->iter : nullptr, w->run0, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "screened step");
    return FS_OK;
}

fs_status fs_pso_best(fs_plan* p, const fs_swarm* w, double* best_f, int* best_i) {
    g_err[0] = 0;
    if (!p || !best_f || !best_i) return fail(FS_EINVAL, "fs_pso_best: NULL argument");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    cudaError_t e = fs::launch_pso_best(w->R, w->n_part, w->pbest_f, best_f, best_i, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pso best launch");
    return FS_OK;
}

fs_status fs_pso_graph_build(fs_plan* p, const fs_swarm* w, const double* edges_dev, int Np, uint64_t seed,
                             double w0, double w1, int n_iter, double c1, double c2, double vmax, fs_graph** out) {
    g_err[0] = 0;
    if (!out) return fail(FS_EINVAL, "fs_pso_graph_build: out is NULL");
    *out = nullptr;
    if (!p) return fail(FS_EINVAL, "fs_pso_graph_build: plan is NULL");
    if (!p->stream) return fail(FS_EINVAL, "fs_pso_graph_build: the plan's stream is the legacy default stream");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (!w->iter) return fail(FS_EINVAL, "fs_pso_graph_build: swarm->iter is NULL");
    const int n = w->R * w->n_part;
    // everything that may allocate, copy or synchronise happens before capture
    if ((st = ensure_workspace(p, n > 0 ? n : 1, Np)) != FS_OK) return st;
    if ((st = fs_pso_evaluate(p, w, edges_dev, Np)) != FS_OK) return st;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const int prof = p->profiling;
    p->profiling = 0;
    if ((e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        p->profiling = prof;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    fs_status s1 = fs_pso_evaluate(p, w, edges_dev, Np);
    fs_status s2 = s1 == FS_OK ? fs_pso_step(p, w, seed, -1, w0, w1, n_iter, c1, c2, vmax, nullptr) : s1;
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(p->stream, &gr);
    p->profiling = prof;
    if (s2 != FS_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s2;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    fs_graph* gobj = new (std::nothrow) fs_graph;
    if (!gobj) {
        cudaGraphDestroy(gr);
        return fail(FS_ENOMEM, "fs_pso_graph_build: host allocation failed");
    }
    gobj->graph = gr;
    gobj->stream = p->stream;
    if ((e = cudaGraphInstantiate(&gobj->exec, gr, 0)) != cudaSuccess) {
        cudaGraphDestroy(gr);
        delete gobj;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = gobj;
    return FS_OK;
}

fs_status fs_pso_record(fs_plan* p, const fs_swarm* w, const fs_sample_ring* rings, int n_rings) {
    g_err[0] = 0;
    if (!p || !rings || n_rings < 1) return fail(FS_EINVAL, "fs_pso_record: NULL plan or no ring");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (w->R % n_rings != 0)
        return fail(FS_EINVAL, "fs_pso_record: R = %d is not a multiple of n_rings = %d", w->R, n_rings);
    const int per = (w->R / n_rings) * w->n_part;   // particles per ring (their runs are contiguous)
    for (int g = 0; g < n_rings; g++) {
        const fs_sample_ring& r = rings[g];
        if (!r.x || !r.f || !r.count || r.cap < 1)
            return fail(FS_EINVAL, "fs_pso_record: ring %d needs x, f, count and cap >= 1", g);
        if ((r.dims == 6 ? 6 : 5) != swarm_dims(w) || (r.dims != 0 && r.dims != 5 && r.dims != 6))
            return fail(FS_EINVAL, "fs_pso_record: ring %d holds %d floats per sample, the swarm has %d dimensions",
                        g, r.dims == 0 ? 5 : r.dims, swarm_dims(w));
    }
    // one launch per kRingBatch rings
    for (int g0 = 0; g0 < n_rings; g0 += fs::kRingBatch) {
        const int nr = n_rings - g0 < fs::kRingBatch ? n_rings - g0 : fs::kRingBatch;
        fs::RingBatch rb{};
        for (int j = 0; j < nr; j++) {
            rb.x[j] = rings[g0 + j].x;
            rb.f[j] = rings[g0 + j].f;
            rb.count[j] = rings[g0 + j].count;
            rb.cap[j] = rings[g0 + j].cap;
        }
        const int D = swarm_dims(w);
        cudaError_t e = fs::launch_pso_record(nr, per, D, w->x + (int64_t)g0 * per * D, w->fit + (int64_t)g0 * per, rb,
                                              p->stream);
        if (e != cudaSuccess) return cuda_fail(e, "pso record launch");
    }
    return FS_OK;
}

fs_status fs_mlp_stream(fs_mlp* m, cudaStream_t* s);

fs_status fs_pso_graph_build_ex(fs_plan* p, const fs_swarm* w, const double* edges_dev, int Np, uint64_t seed,
                                double w0, double w1, int n_iter, double c1, double c2, double vmax, int parts,
                                const fs_sample_ring* rings, int n_rings, fs_mlp* const* mlps, int n_mlp, int n_cand,
                                fs_graph** out) {
    g_err[0] = 0;
    if (!out) return fail(FS_EINVAL, "fs_pso_graph_build_ex: out is NULL");
    *out = nullptr;
    if (!p) return fail(FS_EINVAL, "fs_pso_graph_build_ex: plan is NULL");
    if (!p->stream) return fail(FS_EINVAL, "fs_pso_graph_build_ex: the plan's stream is the legacy default stream");
    if (parts <= 0 || parts > 15 || ((parts & 4) && (parts & 8)))
        return fail(FS_EINVAL, "fs_pso_graph_build_ex: parts must combine bits 1, 2 and one of 4, 8");
    fs_status st = check_swarm(w);
    if (st != FS_OK) return st;
    if (!w->iter) return fail(FS_EINVAL, "fs_pso_graph_build_ex: swarm->iter is NULL");
    if ((parts & 2) && (!rings || n_rings < 1)) return fail(FS_EINVAL, "fs_pso_graph_build_ex: bit 2 needs rings");
    if (parts & 8) {
        if (!mlps || n_mlp < 1) return fail(FS_EINVAL, "fs_pso_graph_build_ex: bit 8 needs networks");
        for (int i = 0; i < n_mlp; i++) {
            cudaStream_t ms = nullptr;
            if (!mlps[i]) return fail(FS_EINVAL, "fs_pso_graph_build_ex: network %d is NULL", i);
            if ((st = fs_mlp_stream(mlps[i], &ms)) != FS_OK) return st;
            if (ms != p->stream)
                return fail(FS_EINVAL, "fs_pso_graph_build_ex: the networks must use the plan's stream");
        }
    }
    const int n = w->R * w->n_part;
    if ((st = ensure_workspace(p, n > 0 ? n : 1, Np)) != FS_OK) return st;
    if (parts & 1) {
        if ((st = fs_pso_evaluate(p, w, edges_dev, Np)) != FS_OK) return st;
    }
    if (parts & 8) {
        if (n_cand < 1 || n_cand > 64) return fail(FS_EINVAL, "fs_pso_graph_build_ex: n_cand must be in [1, 64]");
        if ((st = ensure_candidates(p, (int64_t)n * n_cand)) != FS_OK) return st;   // outside the capture
    }
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const int prof = p->profiling;
    p->profiling = 0;
    if ((e = cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        p->profiling = prof;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    st = FS_OK;
    if (parts & 1) st = fs_pso_evaluate(p, w, edges_dev, Np);
    if (st == FS_OK && (parts & 2)) st = fs_pso_record(p, w, rings, n_rings);
    if (st == FS_OK && (parts & 4)) st = fs_pso_step(p, w, seed, -1, w0, w1, n_iter, c1, c2, vmax, nullptr);
    if (st == FS_OK && (parts & 8))
        st = fs_pso_step_screened(p, w, mlps, n_mlp, n_cand, seed, -1, w0, w1, n_iter, c1, c2, vmax);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(p->stream, &gr);
    p->profiling = prof;
    if (st != FS_OK) {
        if (gr) cudaGraphDestroy(gr);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    fs_graph* gobj = new (std::nothrow) fs_graph;
    if (!gobj) {
        cudaGraphDestroy(gr);
        return fail(FS_ENOMEM, "fs_pso_graph_build_ex: host allocation failed");
    }
    gobj->graph = gr;
    gobj->stream = p->stream;
    if ((e = cudaGraphInstantiate(&gobj->exec, gr, 0)) != cudaSuccess) {
        cudaGraphDestroy(gr);
        delete gobj;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = gobj;
    return FS_OK;
}

fs_status fs_mlp_train_graph_build(fs_mlp* const* mlps, int n, const fs_sample_ring* rings, int steps, float lr,
                                   fs_graph** out) {
    g_err[0] = 0;
    if (!out) return fail(FS_EINVAL, "fs_mlp_train_graph_build: out is NULL");
    *out = nullptr;
    if (!mlps || !rings || n < 1 || steps < 1 || !(lr > 0.f))
        return fail(FS_EINVAL, "fs_mlp_train_graph_build: need n >= 1 networks and rings, steps >= 1, lr > 0");
    cudaStream_t s = nullptr;
    for (int i = 0, k = 0; i < n; i++) {
        cudaStream_t si = nullptr;
        if (!mlps[i]) return fail(FS_EINVAL, "fs_mlp_train_graph_build: network %d is NULL", i);
        fs_status st = fs_mlp_stream(mlps[i], &si);
        if (st != FS_OK) return st;
        if (i == 0) s = si;
        if (si != s || !s) return fail(FS_EINVAL, "fs_mlp_train_graph_build: the networks must share one non-default stream");
        // a batch of G networks trains on G consecutive rings that are slices of one buffer
        const fs_sample_ring& r0 = rings[k];
        for (int j = 0; j < fs_mlp_groups(mlps[i]); j++, k++) {
            const fs_sample_ring& r = rings[k];
            if (!r.x || !r.f || r.cap < 1)
                return fail(FS_EINVAL, "fs_mlp_train_graph_build: ring %d needs x, f and cap >= 1", k);
            if (r.dims != 0 && r.dims != 5)
                return fail(FS_EINVAL, "fs_mlp_train_graph_build: ring %d holds %d floats per sample; the networks "
                                       "take 5 inputs", k, r.dims);
            if (r.cap != r0.cap || r.x != r0.x + (int64_t)j * r0.cap * 5 || r.f != r0.f + (int64_t)j * r0.cap)
                return fail(FS_EINVAL,
                            "fs_mlp_train_graph_build: the rings of network %d must be consecutive slices of one "
                            "buffer with one capacity", i);
        }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    fs_status st = FS_OK;
    for (int i = 0, k = 0; i < n && st == FS_OK; k += fs_mlp_groups(mlps[i]), i++)
        st = fs_mlp_train(mlps[i], rings[k].x, rings[k].f, rings[k].cap, steps, lr, nullptr);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(s, &gr);
    if (st != FS_OK) {
        if (gr) cudaGraphDestroy(gr);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    fs_graph* gobj = new (std::nothrow) fs_graph;
    if (!gobj) {
        cudaGraphDestroy(gr);
        return fail(FS_ENOMEM, "fs_mlp_train_graph_build: host allocation failed");
    }
    gobj->graph = gr;
    gobj->stream = s;
    if ((e = cudaGraphInstantiate(&gobj->exec, gr, 0)) != cudaSuccess) {
        cudaGraphDestroy(gr);
        delete gobj;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    *out = gobj;
    return FS_OK;
}

fs_status fs_graph_run(fs_graph* g, int n) {
    g_err[0] = 0;
    if (!g || n < 0) return fail(FS_EINVAL, "fs_graph_run: bad argument");
    for (int i = 0; i < n; i++) {
        cudaError_t e = cudaGraphLaunch(g->exec, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    }
    return FS_OK;
}

fs_status fs_graph_destroy(fs_graph* g) {
    if (!g) return FS_OK;
    cudaStreamSynchronize(g->stream);
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return FS_OK;
}

fs_status fs_plan_set_variant(fs_plan* p, int variant) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_plan_set_variant: plan is NULL");
    if (variant < -1 || variant >= n_variants(p->mode))
        return fail(FS_EINVAL, "fs_plan_set_variant: variant must be -1 or in [0, %d)", n_variants(p->mode));
    p->variant_forced = variant;
    return FS_OK;
}

fs_status fs_plan_set_variant_for(fs_plan* p, int Np, int global_edges, int variant) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_plan_set_variant_for: plan is NULL");
    if (Np < 1 || Np > fs::kNpMax) return fail(FS_EINVAL, "fs_plan_set_variant_for: N_p = %d out of range", Np);
    if (variant < 0 || variant >= n_variants(p->mode))
        return fail(FS_EINVAL, "fs_plan_set_variant_for: variant must be in [0, %d)", n_variants(p->mode));
    record_tuned(p, Np, global_edges ? 1 : 0, variant);
    return FS_OK;
}

fs_status fs_plan_get_variant(fs_plan* p, int Np, int global_edges, int* variant) {
    g_err[0] = 0;
    if (!p || !variant) return fail(FS_EINVAL, "fs_plan_get_variant: NULL argument");
    *variant = resolve_variant(p, Np, global_edges ? 1 : 0);
    return FS_OK;
}

fs_status fs_plan_autotune(fs_plan* p, const fs_params* params_dev, int B, const double* edges_dev, int Np,
                           int reps, int* variant_out, float* ms_out) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_plan_autotune: plan is NULL");
    if (reps < 1 || reps > 1000) return fail(FS_EINVAL, "fs_plan_autotune: reps = %d not in [1, 1000]", reps);
    if (B < 1) return fail(FS_EINVAL, "fs_plan_autotune: need B >= 1");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(p->stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone) return fail(FS_EINVAL, "fs_plan_autotune: the stream is being captured");
    fs_status st = ensure_workspace(p, B, Np);
    if (st != FS_OK) return st;
    double* F = p->pso_F;   // scratch output, distinct from every parameter buffer
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        return cuda_fail(e, "cudaEventCreate");
    }
    const int saved = p->variant_forced;
    const int global = edges_dev != nullptr;
    int best = 0;
    float best_ms = 0.f;
    st = FS_OK;
    for (int v = 0; v < n_variants(p->mode) && st == FS_OK; v++) {
        p->variant_forced = v;
        if ((st = fs_fstat_batch(p, params_dev, B, edges_dev, Np, F, nullptr)) != FS_OK) break;   // warm-up
        if ((e = cudaEventRecord(ev[0], p->stream)) != cudaSuccess) {
            st = cuda_fail(e, "cudaEventRecord");
            break;
        }
        for (int r = 0; r < reps && st == FS_OK; r++) st = fs_fstat_batch(p, params_dev, B, edges_dev, Np, F, nullptr);
        if (st != FS_OK) break;
        float ms = 0.f;
        if ((e = cudaEventRecord(ev[1], p->stream)) != cudaSuccess || (e = cudaEventSynchronize(ev[1])) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, ev[0], ev[1])) != cudaSuccess) {
            st = cuda_fail(e, "autotune timing");
            break;
        }
        ms /= (float)reps;
        if (ms_out) ms_out[v] = ms;
        if (v == 0 || ms < best_ms) {
            best = v;
            best_ms = ms;
        }
    }
    p->variant_forced = saved;
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st != FS_OK) return st;
    record_tuned(p, Np, global, best);
    if (variant_out) *variant_out = best;
    return FS_OK;
}

fs_status fs_plan_set_profiling(fs_plan* p, int enable) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_plan_set_profiling: plan is NULL");
    p->profiling = enable ? 1 : 0;
    return FS_OK;
}

fs_status fs_plan_read_profile(fs_plan* p, int kind, double* total_ms, int64_t* launches) {
    g_err[0] = 0;
    if (!p || kind < 0 || kind >= kKinds || !total_ms || !launches)
        return fail(FS_EINVAL, "fs_plan_read_profile: bad argument");
    cudaError_t e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    double tot = 0.0;
    int64_t n = 0;
    std::vector<fs_plan::ProfRec> keep;
    for (auto& r : *p->prof) {
        if (r.kind != kind) {
            keep.push_back(r);
            continue;
        }
        float ms = 0.0f;
        if ((e = cudaEventElapsedTime(&ms, r.a, r.b)) != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        tot += ms;
        n++;
        p->spare->push_back(r.a);
        p->spare->push_back(r.b);
    }
    *p->prof = keep;
    *total_ms = tot;
    *launches = n;
    return FS_OK;
}

fs_status fs_add_signal(fs_plan* p, const fs_params* params_host, const double* a_host, double* data_dev) {
    g_err[0] = 0;
    if (!p || !params_host || !a_host || !data_dev) return fail(FS_EINVAL, "fs_add_signal: NULL argument");
    if (!p->data_set) return fail(FS_EINVAL, "fs_add_signal: fs_plan_set_data was not called");
    cudaError_t e;
    if ((e = cudaMemcpyAsync(p->one_param, params_host, sizeof(fs_params), cudaMemcpyHostToDevice, p->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(p->one_a, a_host, sizeof(double) * 4, cudaMemcpyHostToDevice, p->stream)) !=
            cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync(signal parameters)");
    for (int c = 0; c < p->nch; c++) {   // the signal as each channel sees it, into that channel's data
        const fs::Grid gc = channel_grid(p, c);
        if ((e = fs::launch_setup(gc, p->one_param, 1, p->one_part, 0, p->stream)) != cudaSuccess)
            return cuda_fail(e, "setup launch");
        if ((e = fs::launch_add_signal(gc, p->tab[c], p->one_part, p->one_a, data_dev + (size_t)2 * p->grid.n * c,
                                       p->stream, p->resp_on ? &p->resp : nullptr)) != cudaSuccess)
            return cuda_fail(e, "add_signal launch");
    }
    e = cudaStreamSynchronize(p->stream);   // the host arguments are pageable: finish before returning
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return FS_OK;
}

fs_status fs_plan_set_response(fs_plan* p, int filter_order, int k_max) {
    g_err[0] = 0;
    if (filter_order < -1 || filter_order > 2)
        return fail(FS_EINVAL, "fs_plan_set_response: filter order %d not in [-1, 2]", filter_order);
    if (k_max < 0 || k_max > 1) return fail(FS_EINVAL, "fs_plan_set_response: k_max %d not in [0, 1]", k_max);
    if (!p) return fail(FS_EINVAL, "fs_plan_set_response: plan is NULL");
    if (filter_order >= 0 && p->mode != FS_FP64)
        return fail(FS_EUNSUPPORTED, "fs_plan_set_response: the response series needs an FS_FP64 plan");
    if (filter_order >= 0 && p->arm_s > 0.0)
        return fail(FS_EUNSUPPORTED, "fs_plan_set_response: the series is not offered with the finite-arm response");
    if (filter_order < 0) {
        p->resp_on = 0;
        return FS_OK;
    }
    // weights a_j solving sum_j a_j j^(2m) = (2m-1)!! (i/pi)^m, m = 0..N (closed forms)
    const double pi = fs::kPi, pi2 = fs::kPi * fs::kPi;
    fs::Resp r{};
    r.N = filter_order;
    r.K = k_max;
    if (filter_order == 0) {
        r.ar[0] = 1.0;
    } else if (filter_order == 1) {
        r.ar[0] = 1.0;
        r.ai[0] = -1.0 / pi;
        r.ai[1] = 1.0 / pi;
    } else {
        r.ar[0] = 1.0 - 3.0 / (4.0 * pi2);
        r.ai[0] = -5.0 / (4.0 * pi);
        r.ar[1] = 1.0 / pi2;
        r.ai[1] = 4.0 / (3.0 * pi);
        r.ar[2] = -1.0 / (4.0 * pi2);
        r.ai[2] = -1.0 / (12.0 * pi);
    }
    p->resp = r;
    p->resp_on = 1;
    return FS_OK;
}

fs_status fs_plan_set_orbit(fs_plan* p, double eccentricity) {
    g_err[0] = 0;
    if (!(eccentricity >= 0.0 && eccentricity <= 0.05))
        return fail(FS_EINVAL, "fs_plan_set_orbit: eccentricity %g not in [0, 0.05]", eccentricity);
    if (!p) return fail(FS_EINVAL, "fs_plan_set_orbit: plan is NULL");
    if (eccentricity > 0.0 && p->mode != FS_FP64)
        return fail(FS_EUNSUPPORTED, "fs_plan_set_orbit: the eccentric orbits need an FS_FP64 plan");
    p->orbit_e = eccentricity;
    return FS_OK;
}

fs_status fs_plan_set_arm(fs_plan* p, double arm_seconds) {
    g_err[0] = 0;
    if (!(arm_seconds >= 0.0 && arm_seconds <= 100.0))
        return fail(FS_EINVAL, "fs_plan_set_arm: arm length %g s not in [0, 100]", arm_seconds);
    if (!p) return fail(FS_EINVAL, "fs_plan_set_arm: plan is NULL");
    if (arm_seconds > 0.0 && p->mode != FS_FP64)
        return fail(FS_EUNSUPPORTED, "fs_plan_set_arm: the finite-arm response needs an FS_FP64 plan");
    if (arm_seconds > 0.0 && p->resp_on)
        return fail(FS_EUNSUPPORTED, "fs_plan_set_arm: the finite-arm response is not offered with the series");
    p->arm_s = arm_seconds;
    return FS_OK;
}

fs_status fs_plan_get_arm(const fs_plan* p, double* arm_seconds) {
    g_err[0] = 0;
    if (!p || !arm_seconds) return fail(FS_EINVAL, "fs_plan_get_arm: NULL argument");
    *arm_seconds = p->arm_s;
    return FS_OK;
}

fs_status fs_plan_selftest_timeout(fs_plan* p) {
    g_err[0] = 0;
    if (!p) return fail(FS_EINVAL, "fs_plan_selftest_timeout: plan is NULL");
    cudaError_t e = fs::launch_wait_probe(p->flags_dev, p->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wait probe launch");
    return FS_OK;
}

fs_status fs_plan_get_orbit(const fs_plan* p, double* eccentricity) {
    g_err[0] = 0;
    if (!p || !eccentricity) return fail(FS_EINVAL, "fs_plan_get_orbit: NULL argument");
    *eccentricity = p->orbit_e;
    return FS_OK;
}

fs_status fs_plan_get_response(const fs_plan* p, int* filter_order, int* k_max) {
    g_err[0] = 0;
    if (!p || !filter_order || !k_max) return fail(FS_EINVAL, "fs_plan_get_response: NULL argument");
    *filter_order = p->resp_on ? p->resp.N : -1;
    *k_max = p->resp_on ? p->resp.K : 0;
    return FS_OK;
}

}  // extern "C"
