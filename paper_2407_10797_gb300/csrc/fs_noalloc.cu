// fs_noalloc.cu - fs_fstat_batch_noalloc: the FP64 F-statistic with every
// intermediate buffer carved from one file-scope device array, for callers
// that cannot allocate device memory.
//
// Who needs this: code that runs where cudaMalloc is not available or not
// allowed -- inside a host callback or a library that must not touch the
// allocator, a process whose memory pool is owned by another runtime, or an
// embedded caller with a fixed memory budget.  Such callers own their inputs
// and outputs but cannot give the library a workspace, so the workspace lives
// in a static __device__ array that every GPU loading this library holds until
// the process exits.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "fs_internal.h"

namespace {

// Limits of one call and the fixed scratch capacity they need (checked below).
constexpr int64_t kMaxBins = 32768;
constexpr int kMaxB = 1024;
constexpr int kMaxNp = 64;
constexpr size_t kScratchBytes = 10u << 20;   // 10 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices];   // device address of g_scratch, per device ordinal

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte layout of the scratch for one call.
struct Layout {
    size_t tables, parts, H, T, S, Fpart, rot, edges, total;
};

constexpr Layout layout_for(int64_t n, int B, int Np) {
    Layout L{};
    size_t ntiles = (size_t)((n + fs::kTile - 1) / fs::kTile);
    size_t off = 0;
    L.tables = off;
    off += align256(sizeof(double) * fs::kNumTables * (size_t)n);
    L.parts = off;
    off += align256(sizeof(fs::Particle) * (size_t)B);
    L.H = off;
    off += align256(sizeof(double) * 7 * ntiles * (size_t)B);
    L.T = off;
    off += align256(sizeof(double) * 7 * ntiles * (size_t)B);
    L.S = off;
    off += align256(sizeof(double) * 7 * (size_t)Np * B);
    L.Fpart = off;
    off += align256(sizeof(double) * (size_t)Np * B);
    L.rot = off;
    off += align256(sizeof(double2) * (size_t)Np * B);
    L.edges = off;
    off += align256(sizeof(int64_t) * (size_t)(Np + 2));   // segment starts and the validity word
    L.total = off;
    return L;
}

static_assert(layout_for(kMaxBins, kMaxB, kMaxNp).total <= kScratchBytes,
              "the scratch array must hold a call at the stated limits");

// Device address of g_scratch on the current device (looked up once per device
// and kept for the life of the process, so a cudaDeviceReset after the first
// call on a device is not supported).
fs_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fs::set_error(FS_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fs::set_error(FS_EUNSUPPORTED, "device ordinal %d >= %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fs::set_error(FS_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return FS_OK;
}

}  // namespace

extern "C" fs_status fs_fstat_batch_noalloc(int64_t n_bins, double f_min, double df, double T_obs,
                                            const double* data_dev, const double* psd_dev,
                                            const fs_params* params_dev, int B, const double* edges_dev,
                                            int N_p, double* F_dev, double* F_part_dev, void* stream) {
    fs::set_error(FS_OK, "");
    if (n_bins <= 0 || !(f_min > 0.0) || !(df > 0.0) || !(T_obs > 0.0) || !isfinite(f_min) || !isfinite(df) ||
        !isfinite(T_obs))
        return fs::set_error(FS_EINVAL, "fs_fstat_batch_noalloc: need n_bins > 0 and finite f_min, df, T_obs > 0");
    if (n_bins > kMaxBins)
        return fs::set_error(FS_EINVAL, "fs_fstat_batch_noalloc: n_bins = %lld exceeds the limit %lld",
                             (long long)n_bins, (long long)kMaxBins);
    if (B < 0 || B > kMaxB)
        return fs::set_error(FS_EINVAL, "fs_fstat_batch_noalloc: B = %d not in [0, %d]", B, kMaxB);
    if (N_p < 1 || N_p > kMaxNp)
        return fs::set_error(FS_EINVAL, "fs_fstat_batch_noalloc: N_p = %d not in [1, %d]", N_p, kMaxNp);
    if (B == 0) return FS_OK;
    if (!data_dev || !psd_dev || !params_dev || !F_dev)
        return fs::set_error(FS_EINVAL, "fs_fstat_batch_noalloc: NULL data, psd, params or F");
    const int global = edges_dev != nullptr;
    void* base = nullptr;
    fs_status st = scratch_address(&base);
    if (st != FS_OK) return st;
    const Layout L = layout_for(n_bins, B, N_p);
    unsigned char* sp = (unsigned char*)base;
    cudaStream_t s = (cudaStream_t)stream;

    fs::Grid g;
    g.n = n_bins;
    g.f_min = f_min;
    g.df = df;
    g.T_obs = T_obs;
    g.alpha0 = 0.0;
    g.orient = 0.0;
    fs::Tables tb;
    double* tab = (double*)(sp + L.tables);
    double** slots[fs::kNumTables] = {&tb.fh, &tb.fl, &tb.u, &tb.g0h, &tb.g0l, &tb.e19, &tb.dwr, &tb.dwi, &tb.W};
    for (int i = 0; i < fs::kNumTables; i++) *slots[i] = tab + (size_t)i * n_bins;
    fs::Particle* parts = (fs::Particle*)(sp + L.parts);
    int64_t* starts = (int64_t*)(sp + L.edges);
    fs::Segs sg;
    sg.Np = N_p;
    sg.global = global;
    sg.edges = starts;
    fs::Partials pa;
    pa.H = (double*)(sp + L.H);
    pa.T = (double*)(sp + L.T);
    pa.S = (double*)(sp + L.S);
    pa.rot = (double2*)(sp + L.rot);
    pa.rot32 = nullptr;
    pa.ntiles = (int)((n_bins + fs::kTile - 1) / fs::kTile);
    pa.tile = fs::kTile;
    double* Fpart = F_part_dev ? F_part_dev : (double*)(sp + L.Fpart);

    // Every scratch byte a kernel reads is written earlier in this same call
    // (segment starts, tables, particles, rotations, the partial sums of the
    // tiles a segment spans), so nothing needs clearing between calls.  Edge
    // frequencies that are not finite or decrease give F = NaN (no flag word).
    cudaError_t e;
    if ((global && (e = fs::launch_edges(g, edges_dev, N_p, starts, nullptr, s)) != cudaSuccess) ||
        (e = fs::launch_precompute(g, data_dev, psd_dev, tb, s)) != cudaSuccess ||
        (e = fs::launch_setup(g, params_dev, B, parts, global, s)) != cudaSuccess ||
        (e = fs::launch_rotation(g, parts, B, sg, pa.rot, nullptr, s)) != cudaSuccess ||
        (e = fs::launch_fp64_main(g, tb, parts, B, sg, pa, s)) != cudaSuccess ||
        (e = fs::launch_reduce(g, parts, B, sg, pa, Fpart, F_dev, s)) != cudaSuccess)
        return fs::set_error(FS_ECUDA, "fs_fstat_batch_noalloc launch: %s", cudaGetErrorString(e));
    return FS_OK;
}
