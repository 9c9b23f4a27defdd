// fs_internal.h - plan layout and kernel launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fs_common.cuh"
#include "fstat.h"

namespace fs {

constexpr int kTile = 2048;          // bins per (particle, tile) work item of the FP64 kernel (default)
constexpr int kTileMin = 1024;       // smallest FP64 tile a launch variant uses (sizes the workspace)
constexpr int kWarpsPerCta = 8;      // particles per CTA of the FP64 kernel
constexpr int kNpMax = 4096;
constexpr int kCisBits = 20;         // entries 2^kCisBits of the anchored FP64 kernels' exp table

// Per-bin tables (structure of arrays, length n).
struct Tables {
    double* fh;    // f_k, double-double head
    double* fl;    // f_k, double-double tail
    double* u;     // f^-1/3
    double* g0h;   // f^-5/3 head
    double* g0l;   // f^-5/3 tail
    double* e19;   // (f0/f)^(19/9)
    double* dwr;   // Re 4 df d_k f^-7/6 / S_k
    double* dwi;   // Im of the same
    double* W;     // 4 df f^-7/3 / S_k
};
constexpr int kNumTables = 9;

struct Grid {
    int64_t n;
    double f_min, df, T_obs;
    double alpha0, orient;   // detector orbital phase and orientation at t = 0
    double pscale = 1.0;     // scale of the arm projections: the patterns, quadratic in them, carry pscale^2
    Orbit orb{};             // orbits to second order in eccentricity when orb.e > 0 (direct kernels only)
};

// TDI channels in the long-wavelength limit (Sec. II.A, Eq. eq2): with the
// vertex Michelsons X, Y, Z of the rigid constellation, A = (Z - X)/sqrt2 and
// E = (X - 2Y + Z)/sqrt6 are the X Michelson with the constellation turned in
// its plane by 75 and 30 degrees, times sqrt(3/2) (the three detector
// tensors are 120 degrees apart in the plane of traceless in-plane tensors,
// where a turn by r moves a tensor by 2r).
constexpr int kMaxChannels = 2;
struct Channel {
    double orient_shift;   // rad, added to the grid's orientation
    double pscale;         // arm-projection scale (patterns scale by its square)
};
__host__ __device__ constexpr Channel channel_of(int tdi, int c) {
    return tdi == 0 ? Channel{0.0, 1.0}
                    : (c == 0 ? Channel{1.3089969389957472, 1.1066819197003215}      // A: 75 deg, (3/2)^(1/4)
                              : Channel{0.5235987755982988, 1.1066819197003215});    // E: 30 deg
}

// Segment description for one batch.
struct Segs {
    int Np;
    int global;               // 1: edges[] apply to every particle
    const int64_t* edges;     // device (global mode only): Np+1 segment start bins, then a validity word
                              // at edges[Np+1] (0: the caller's edge frequencies were invalid)
};

// Bits of a plan's sticky device flag word (read and cleared by fs_plan_check).
constexpr int kFlagBadEdges = 1;   // partition edges not finite or decreasing
constexpr int kFlagBadGrid = 2;    // a caller's frequency grid is not f_min + k df
constexpr int kFlagTimeout = 4;    // a bounded device-side wait ran out (that call's F values are invalid)

struct Partials {
    double* H;    // [B][ntiles][7] first segment of each (particle, tile)
    double* T;    // [B][ntiles][7] last segment of each (particle, tile)
    double* S;    // [B][Np][7] segments complete inside one tile
    double2* rot; // [B][Np] (c, s): antenna basis G1 = c F+ + s Fx, G2 = c Fx - s F+ of each segment
    float2* rot32; // the same rotations in FP32 (mixed mode), or NULL
    int ntiles;   // number of tiles (slots of H and T per particle)
    int tile;     // bins per tile
    unsigned long long* census = nullptr;   // [6] in-band bins per anchor mode (anchored kernels), or NULL
    int* flags = nullptr;                   // the plan's sticky flag word (kFlag*), for device-detected errors
    // channels summed by the solve kernel: channel c's slots at H + c ch_HT, T + c ch_HT, S + c ch_S
    int nch = 1;
    int64_t ch_HT = 0, ch_S = 0;
    int nsum = 7;   // sums per slot: 7, or 8 for the response series (K12' of the complex responses)
    const double2* cis = nullptr;   // the plan's exp(2 pi i j 2^-kCisBits) table (anchored FP64 kernels)
};

// Record an error message for fs_last_error() and return st.
fs_status set_error(fs_status st, const char* fmt, ...);

// Segment starts from N_p + 1 edge frequencies (device), validity word at starts[Np+1].
cudaError_t launch_edges(const Grid& g, const double* edges_hz, int Np, int64_t* starts, int* flags,
                         cudaStream_t s);
cudaError_t launch_grid_check(const Grid& g, const double* f_grid, int* flags, cudaStream_t s);
cudaError_t launch_precompute(const Grid& g, const double* data, const double* psd, const Tables& t,
                              cudaStream_t s);
cudaError_t launch_setup(const Grid& g, const ::fs_params* params, int B, Particle* parts, int global,
                         cudaStream_t s);
cudaError_t launch_rotation(const Grid& g, const Particle* parts, int B, const Segs& sg, double2* rot,
                            float2* rot32, cudaStream_t s);
// resp != NULL: the response series (eight sums per slot, pa.nsum = 8)
cudaError_t launch_fp64_main(const Grid& g, const Tables& t, const Particle* parts, int B, const Segs& sg,
                             const Partials& pa, cudaStream_t s, const Resp* resp = nullptr);
cudaError_t launch_reduce(const Grid& g, const Particle* parts, int B, const Segs& sg, const Partials& pa,
                          double* Fpart, double* F, cudaStream_t s,
                          double* amp = nullptr, const int* amp_exp = nullptr);
// In-band particle lists per span of span_len bins: list [nspans][B] holds
// span s's in-band particles, the heavy ones (kHeavyBounds or more segment
// boundaries inside the span) first, each class in increasing particle
// order.  The int buffer `cnt` (span_sched_ints(nspans) entries) holds
//   [0, ns)            cnt[s]: in-band particles of span s
//   [ns, 2 ns + 1)     exclusive prefix over spans of the heavy counts (with offsets)
//   [2 ns + 1, +3)     persistent-kernel counters
//   [2 ns + 4, 3 ns + 4)  heavy count of span s
//   [3 ns + 4, 4 ns + 5)  exclusive prefix over spans of the other counts (with offsets)
// The persistent kernels take every heavy item before the others, so that
// the items with the most per-segment work do not start last.
constexpr int kHeavyBounds = 16;
constexpr int kCensusModes = 9;   // anchor modes counted by fs_plan_census
inline int span_sched_ints(int nspans) { return 4 * nspans + 8; }
cudaError_t launch_span_lists(const Particle* parts, int B, const Segs& sg, int nspans, int span_len, int* list,
                              int* cnt, bool offsets, cudaStream_t s);
// FS_FP64 anchored form (spans of fp64a_span() bins; partial slots per span).
int fp64a_span();
cudaError_t launch_fp64a_main(const Grid& g, const Tables& t, const Particle* parts, int B, const Segs& sg,
                              const Partials& pa, bool persistent, int* list, int* cnt, cudaStream_t s);
cudaError_t launch_extrinsic(int64_t n, const double* amp, double* ext, cudaStream_t s);
// Fill the 2^kCisBits-entry table of exp(2 pi i j 2^-kCisBits) (double2: cos, sin).
cudaError_t launch_cis_table(double2* tab, cudaStream_t s);
// One bounded mbarrier wait that runs out (nothing arrives): sets kFlagTimeout in *flags.
cudaError_t launch_wait_probe(int* flags, cudaStream_t s);
// FP32 tables of nch channels (t32 [nch][n]) with one common power-of-two scale (exponent in *emax)
cudaError_t launch_tables32(const Grid& g, const Tables* t, int nch, int* emax, float4* t32, cudaStream_t s);
// variant 0: grid, 2 CTAs/SM (up to 128 registers); 1: grid, 3 CTAs/SM (up to 80 registers);
// 2, 3: persistent with 2 or 3 CTAs/SM; 4: grid, tables staged through shared memory by bulk copies
cudaError_t launch_mixed_main(const Grid& g, const Tables& t, const float4* t32, const Particle* parts, int B,
                              const Segs& sg, const Partials& pa, int variant, int* list, int* cnt,
                              cudaStream_t s);
int mixed_span();   // bins per H/T slot of the mixed path
// Per-bin values of the mixed body for particle b over bins [k0, k1): out [k1 - k0][mixed_probe_fields()].
cudaError_t launch_mixed_probe(const Grid& g, const Tables& t, const float4* t32, const Particle* parts,
                               const Segs& sg, const Partials& pa, int b, int64_t k0, int64_t k1, float* out,
                               cudaStream_t s);
int mixed_probe_fields();
cudaError_t launch_pso_init(int R, int Np, int D, unsigned long long seed, double* x, double* v, double* pbx,
                            double* pbf, double* fit, int run0, cudaStream_t s);
cudaError_t launch_pso_map(int R, int Np, int D, const double* x, const double* box, double q, ::fs_params* out,
                           cudaStream_t s);
cudaError_t launch_pso_fitness(int n, const double* F, int Np, double* fit, cudaStream_t s);
cudaError_t launch_pso_step(int R, int Np, int D, unsigned long long seed, const unsigned int* iter_dev,
                            unsigned int iter_host, double w0, double w1, int n_iter, double c1, double c2, double vmax,
                            double* x, double* v, double* pbx, double* pbf, const double* fit, int* lbest,
                            unsigned int* iter_advance, int run0, cudaStream_t s);
cudaError_t launch_pso_best(int R, int Np, const double* pbf, double* best_f, int* best_i, cudaStream_t s);
cudaError_t launch_pso_screened(int R, int Np, int C, unsigned long long seed, const unsigned int* iter_dev,
                                unsigned int iter_host, double w0, double w1, int n_iter, double c1, double c2,
                                double vmax, double* x, double* v, double* pbx, double* pbf, const double* fit,
                                double* cx, double* cv, float* cin, unsigned char* inside, float* score,
                                ::fs_mlp* const* mlps, int n_mlp, unsigned int* iter_advance, int run0, cudaStream_t s);
// Up to kRingBatch sample rings, passed to the record kernels by value.
constexpr int kRingBatch = 32;
struct RingBatch {
    float* x[kRingBatch];
    float* f[kRingBatch];
    unsigned long long* count[kRingBatch];
    int cap[kRingBatch];
};
cudaError_t launch_pso_record(int nr, int per, int D, const double* x, const double* fit, const RingBatch& rb,
                              cudaStream_t s);
cudaError_t launch_bands(const Particle* parts, int B, int64_t* bands, cudaStream_t s);
cudaError_t launch_add_signal(const Grid& g, const Tables& t, const Particle* part, const double* a,
                              double* data, cudaStream_t s, const Resp* resp = nullptr);

}  // namespace fs
