/*
 * fstat.h - C ABI of the GB300 (sm_103a) semi-coherent F-statistic library.
 *
 * The library evaluates, for a batch of particles (intrinsic parameters
 * Theta_I), the semi-coherent F-statistic of the hierarchical SmBBH search of
 * Fu, Wang & Mohanty (arXiv:2407.10797):
 *
 *   F_sum(Theta_I) = sum_{l=1..N_seg} F_l,  F_l = 1/2 N_l^T M_l^{-1} N_l,
 *   N_l^i = <d, A^i>_l,  M_l^ij = <A^i, A^j>_l,
 *   <a, b>_l = 4 Re sum_{k in segment l} a_k conj(b_k) / S_k * df
 *
 * (Sec. II.A Eqs. inner_product, response, coherent_F_stat, aandMN-aandMN3;
 * Sec. II.B Eq. semi-cohF and the segment inner product).  The paper's
 * F-hat is F_sum / N_seg.  Templates follow Appendix A (restricted PN phase,
 * TaylorF2 through 2PN, leading e0^2 eccentricity correction at 10 mHz) with
 * the frequency-domain LISA response of Sec. IV (Eq. freDres, N = 0): the
 * antenna patterns and the Doppler phase are taken at the stationary-phase
 * time t(f) = (1/2pi) dPsi/df.
 *
 * Conventions
 *   - Units: G = c = 1 with times in seconds; masses in solar masses on input.
 *   - Frequency grid: f_k = f_min + k*df, k = 0..n_bins-1 (uniform; the
 *     paper's data are the DFT grid of a regularly sampled series, Sec. V.A).
 *   - Segment edges (Sec. II.B): N_p + 1 non-decreasing frequencies e_p (Hz) in
 *     device memory; bin k lies in segment p iff e_p <= f_k < e_{p+1}, the last
 *     segment closed at e_{N_p}; bins outside [e_0, e_{N_p}] take no part.  NULL
 *     instead means per-particle edges (see fs_fstat_batch).
 *   - All `*_dev` pointers are device pointers owned by the caller; `*_host`
 *     pointers are host memory owned by the caller.  The plan owns its own
 *     workspace (per-bin tables, per-particle coefficients, partial sums).
 *   - Every call is asynchronous and ordered on the plan's stream, unless its
 *     comment says otherwise.  A call reads caller memory when its work runs
 *     on the stream, and keeps no pointer afterwards; a captured graph reads
 *     the buffers it was built with every time it is launched.
 *   - Errors: every function returns fs_status; on failure fs_last_error()
 *     returns a message (thread-local, valid until the next call on the same
 *     thread).  Invalid sizes or arguments give FS_EINVAL and launch nothing.
 *   - Thread safety: one plan must not be used from two threads at once.
 */
#ifndef FSTAT_H
#define FSTAT_H

#include <stdint.h>

#if defined(__GNUC__)
#define FS_API __attribute__((visibility("default")))
#else
#define FS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FS_OK = 0,
    FS_EINVAL = -1,        /* invalid argument or size */
    FS_ECUDA = -2,         /* a CUDA runtime call failed */
    FS_ENOMEM = -3,        /* device allocation failed */
    FS_ETIMEOUT = -4,      /* a bounded device-side wait expired */
    FS_EUNSUPPORTED = -5   /* valid request the library does not implement */
} fs_status;

typedef enum {
    FS_FP64 = 0,   /* every step in FP64; the phase in double-double where it exceeds 2^23 cycles */
    FS_MIXED = 1   /* FP64 anchors + exact fixed-point phase steps, FP32 response and products */
} fs_precision;

/* TDI channels of the data (Sec. II.A, Eq. eq2: the log-likelihood, and with
 * it N and M of every segment, sums over the channels).  In the
 * long-wavelength response of Sec. IV (N = 0) the Michelson combinations X,
 * Y, Z with vertices at the three spacecraft give A = (Z - X)/sqrt2 and
 * E = (X - 2Y + Z)/sqrt6 (noise-orthogonal; T = (X + Y + Z)/sqrt3 vanishes
 * identically in this limit and is not offered). */
typedef enum {
    FS_TDI_X = 0,   /* one channel: X (the paper's choice) */
    FS_TDI_AE = 1   /* two channels: A, then E */
} fs_tdi;

/* Intrinsic parameters of one particle (Sec. II.A, Theta_I without delta_mu;
 * the mass ratio q = m1/m2 >= 1 fixes eta = q/(1+q)^2). */
typedef struct {
    double Mc;   /* chirp mass, solar masses (> 0) */
    double tc;   /* time of coalescence, s, measured from the start of the data */
    double lat;  /* ecliptic latitude beta, rad (theta = pi/2 - beta) */
    double lon;  /* ecliptic longitude lambda = phi, rad */
    double e0;   /* orbital eccentricity at GW frequency 10 mHz */
    double q;    /* mass ratio (1 = equal masses) */
} fs_params;

typedef struct fs_plan fs_plan;

/* Create a plan for one frequency grid and precision mode.
 *   n_bins > 0, f_min > 0, df > 0, T_obs > 0 (observation span: segment outer
 *   edges are the bins whose stationary-phase time lies in [0, T_obs],
 *   Sec. II.B); mode is an fs_precision; stream is a cudaStream_t (NULL = the
 *   legacy default stream).  Allocates the per-bin tables on the current
 *   device.  Synchronous.  *out is NULL on failure. */
FS_API fs_status fs_plan_create(fs_plan** out, int64_t n_bins, double f_min, double df, double T_obs,
                         int mode, void* stream);

/* fs_plan_create for data in the TDI channels `tdi` (an fs_tdi): every
 * per-bin input (data, PSD) then holds one array per channel, channel after
 * channel, and every F is the sum over the channels' inner products.
 * fs_plan_create is the case FS_TDI_X.  Synchronous. */
FS_API fs_status fs_plan_create_tdi(fs_plan** out, int64_t n_bins, double f_min, double df, double T_obs,
                                    int mode, int tdi, void* stream);

/* Number of channels of a plan (1 for FS_TDI_X, 2 for FS_TDI_AE), -1 for NULL. */
FS_API int fs_plan_channels(const fs_plan* plan);

/* Free a plan and its workspace (waits for the plan's stream).  NULL is a no-op. */
FS_API fs_status fs_plan_destroy(fs_plan* plan);

/* Load one data set (Sec. II.A, Eq. inner_product: the noise-weighted inner
 * product on the frequency grid).  data_dev: n_bins complex values as
 * interleaved FP64 (re, im) per channel; psd_dev: n_bins one-sided PSD
 * values S_k > 0 per channel (channels one after the other, in the order of
 * the plan's fs_tdi);
 * f_grid_dev: NULL for the plan's grid f_k = f_min + k df, or the n_bins
 * frequencies of the data (device, FP64), which must equal that grid to 4 units
 * in the last place: the kernels step the template phase in the bin index, so
 * a non-uniform grid returns FS_EUNSUPPORTED (and loads nothing).  Precomputes
 * the particle-independent per-bin tables (noise-weighted data 4 df d_k
 * f^-7/6 / S_k, weights 4 df f^-7/3 / S_k, frequency powers).  Asynchronous
 * with f_grid_dev = NULL; with a grid it waits for the plan's stream to read
 * the check's answer.  The caller's buffers may be reused once the plan's
 * stream has passed this call. */
FS_API fs_status fs_plan_set_data(fs_plan* plan, const double* data_dev, const double* psd_dev,
                                  const double* f_grid_dev);

/* Pre-size the plan's workspace for batches of up to B_max particles and
 * N_p_max segments, so that later fs_fstat_batch calls allocate nothing (and
 * can be captured in a CUDA graph).  Synchronous. */
FS_API fs_status fs_plan_reserve(fs_plan* plan, int B_max, int N_p_max);

/* Batched semi-coherent F-statistic (Sec. II.B, Eq. semi-cohF).
 *   params_dev : B particles (device array of fs_params).
 *   B          : 0 <= B; B = 0 launches nothing.
 *   partition_edges_dev : NULL for per-particle segments: the outer edges are
 *                the first and last bin whose t(f_k) lies in [0, T_obs] and the
 *                N_p segments are equal-width in frequency between them (bin k
 *                is in segment p iff e_p <= f_k < e_{p+1}, the last one closed).
 *                Otherwise N_p + 1 edge frequencies in device memory, the same
 *                for every particle (see Conventions).  They are read on the
 *                plan's stream when the call runs (also when it is replayed
 *                from a captured graph), so the caller keeps the buffer alive
 *                until then.  Edges that are not finite or decrease cannot be
 *                refused without waiting for the device: F is then NaN for
 *                every particle and fs_plan_check reports it.
 *   N_p        : 1 <= N_p <= 4096.
 *   F_dev      : B doubles, F_sum = sum_p F_p (the paper's F-hat times N_p).
 *   F_part_dev : B*N_p doubles (F_p, row-major by particle) or NULL.
 * A segment with fewer than 4 bins, or with M11 M22 - M12^2 <= 1e-12 M11 M22,
 * contributes F_p = 0.  A particle with a non-finite parameter, Mc <= 0 or
 * q <= 0 gets F = NaN (and NaN segments).  Grows the workspace (synchronously)
 * if B or N_p exceed the reservation. */
FS_API fs_status fs_fstat_batch(fs_plan* plan, const fs_params* params_dev, int B,
                                const double* partition_edges_dev, int N_p, double* F_dev, double* F_part_dev);

/* Errors the device found in earlier calls on this plan: waits for the plan's
 * stream, writes the flag bits seen since the last check to *flags_out (may be
 * NULL; bit 0: partition edges that were not finite or decreased; bit 2: a
 * bounded device-side wait ran out, so that call's F values are invalid) and
 * clears them.  Returns FS_ETIMEOUT when bit 2 was set, else FS_EINVAL when
 * bit 0 was set, FS_OK otherwise. */
FS_API fs_status fs_plan_check(fs_plan* plan, int* flags_out);

/* Self-test of the timeout path that fs_plan_check reports (bit 2): launches
 * on the plan's stream one device wait that runs out by design -- an
 * mbarrier that nothing arrives at, polled a bounded number of times, as the
 * staged FS_MIXED kernel polls its copies -- which sets the plan's timeout
 * bit and returns.  The next fs_plan_check returns FS_ETIMEOUT and clears the
 * bit; the plan and its context stay usable.  No counterpart in the paper:
 * it lets a caller (and the tests) see that a device-side wait that gives up
 * is reported on the host without faulting the GPU.  Asynchronous. */
FS_API fs_status fs_plan_selftest_timeout(fs_plan* plan);

/* Maximum-likelihood amplitudes and extrinsic parameters (Eq. aandMN3 and
 * App. B, Eqs. B2-B3), per particle and segment.
 *   Arguments as in fs_fstat_batch; F_dev may be NULL (plan scratch).
 *   a_dev   : B*N_p*4 doubles, a = M^-1 N of each segment in the basis
 *             A1 = F+ h0, A2 = Fx h0, A3 = -i F+ h0, A4 = -i Fx h0 with
 *             h0 = f^-7/6 exp(-i Psi): the data's best fit in the segment is
 *             sum_i a_i A^i.  The amplitude constant of Eq. A2 and the phase
 *             constants -phi_c - pi/4 are part of a.  A segment that
 *             contributes F_p = 0 (fewer than 4 bins or singular M) gets a = 0;
 *             a particle with F = NaN gets NaN.
 *   ext_dev : B*N_p*4 doubles (D_L, iota, psi, phi_c) from a by Eqs. B2-B3
 *             (arctan of a ratio read as atan2; D_L in the units of a, i.e.
 *             1/D_L = the overall amplitude of a), NaN where a = 0; or NULL.
 * With N_p = 1 these are the fully coherent estimates the search reports
 * after its last stage.  Asynchronous, stream-ordered. */
FS_API fs_status fs_amplitudes(fs_plan* plan, const fs_params* params_dev, int B, const double* edges_dev,
                               int N_p, double* F_dev, double* a_dev, double* ext_dev);

/* Add the signal h = sum_i a_i A^i of one particle to data_dev (n_bins
 * interleaved complex FP64 per channel, device, as for fs_plan_set_data; each
 * channel receives the signal through its own response) at the bins of the
 * particle's band [first, last bin with t(f_k) in [0, T_obs]]; the other bins
 * are untouched.
 * The basis is A1 = F+ h0, A2 = Fx h0, A3 = -i F+ h0, A4 = -i Fx h0 with
 * h0 = f^-7/6 exp(-i Psi(f)) (Appendix A with the Sec. IV response); a_host
 * holds the four amplitudes of Eq. (response).  Evaluated in FP64. */
FS_API fs_status fs_add_signal(fs_plan* plan, const fs_params* params_host, const double* a_host,
                        double* data_dev);

/* Precision accounting of the FS_MIXED mode (the segment inner product of
 * Sec. II.B evaluated with an FP32 body): per-bin values that the mixed kernel
 * feeds into its sums, for particle b of a batch over the bins
 * [k0, k0 + nbins), so that each stage can be compared with an FP64
 * evaluation.  The values come from the production per-bin code (the same
 * anchors, the same polynomial and fallback evaluation); nothing is summed.
 *   Arguments as in fs_fstat_batch (the batch fixes the segments and their
 *   rotated antenna bases); 0 <= b < B; 0 <= k0, k0 + nbins <= n_bins.
 *   out_dev : nbins records of 28 floats (device):
 *     [0] tile mode (0 no in-band anchor, 1 FP32 polynomial body, 2 bin-by-bin
 *         FP64), [1] the tile's anchor bin, [2] segment index,
 *     [3] fixed-point phase polynomial: orbital phase minus the anchor's
 *         Doppler phase (cycles, mod 1), [4] orbital-phase offset d(alpha)
 *         from the anchor (rad), [5] Doppler phase minus its anchor value
 *         (cycles), [6] the phase fed to sincos (cycles in [-1/2, 1/2]),
 *     [7] G1, [8] G2 (antenna patterns in the segment's rotated basis
 *         G1 = c F+ + s Fx, G2 = c Fx - s F+), [9] c, [10] s,
 *     [11] cos, [12] sin of 2 pi [6] (SFU), [13] Re dw, [14] Im dw, [15] W
 *         (the FP32 tables, scaled by powers of two), [16..22] the seven
 *         summed terms G1 zr, G1 zi, G2 zr, G2 zi, W G1^2, W G1 G2, W G2^2
 *         with z = dw e^{2 pi i ph}, [23] c - [9], [24] s - [10] (the FP64
 *         rotation's low parts), [25..27] unused.
 *   Fields a mode does not produce are NaN.  FS_EINVAL unless the plan is
 *   FS_MIXED.  With several channels the values are channel 0's.
 *   Asynchronous. */
FS_API fs_status fs_mixed_probe(fs_plan* plan, const fs_params* params_dev, int B, const double* edges_dev,
                                int N_p, int b, int64_t k0, int64_t nbins, float* out_dev);

/* Segment outer edges of each particle (Sec. II.B): bands_dev receives
 * 2*B int64 values (first, last) per particle, the first and last bin whose
 * stationary-phase time lies in [0, T_obs]; first > last means no such bin
 * (and a particle with invalid parameters reports (1, 0)).  Asynchronous. */
FS_API fs_status fs_particle_bands(fs_plan* plan, const fs_params* params_dev, int B, int64_t* bands_dev);

/* ---- Particle swarm optimisation on the device (Sec. III.A) ------------- */

/* State of R independent PSO runs of n_part particles each in the
 * normalised search space [0,1]^D of (M_c, t_c, sin(lat), lon, e0) (D = 5,
 * every particle with the mass ratio q) or of (M_c, t_c, sin(lat), lon, e0,
 * delta_mu) (D = 6: the dimensionless mass difference delta_mu = (m1 - m2)/M
 * of Sec. II.A's Theta_I is searched too, the paper's [0, 0.9] range of
 * Table I, and a particle has q = (1 + delta_mu)/(1 - delta_mu)).  All
 * pointers are device memory owned by the caller; the D-sized rows below are
 * D = dims values. */
typedef struct {
    int R;                 /* independent runs */
    int n_part;            /* particles per run */
    double* x;             /* [R][n_part][D] normalised positions */
    double* v;             /* [R][n_part][D] velocities */
    double* pbest_x;       /* [R][n_part][D] personal-best positions */
    double* pbest_f;       /* [R][n_part] personal-best fitness */
    double* fit;           /* [R][n_part] fitness of x (written by fs_pso_evaluate) */
    const double* box;     /* [R][D][2] search box of each run: (lo, hi) of M_c [Msun], t_c [s],
                              sin(lat), lon [rad], e0 (and delta_mu in [0, 1)); x maps linearly onto it */
    double q;              /* mass ratio of every particle (D = 5) */
    unsigned int* iter;    /* device iteration counter, used by fs_pso_step(iteration < 0) and the graph */
    int run0;              /* global index of run 0: the Philox counters use run0 + r, so a process that
                              holds runs [run0, run0 + R) of a larger search draws their numbers (0: default) */
    int dims;              /* D: 5 (or 0) or 6 */
} fs_swarm;

/* Initial state: x ~ U[0,1)^D, v ~ U[-x, 1-x) (Sec. III.A), pbest_x = x,
 * pbest_f = fit = -inf; random numbers from Philox4x32-10 with counter
 * (0xFFFFFFFF, particle, dim, run) and key = seed.  Asynchronous. */
FS_API fs_status fs_pso_init(fs_plan* plan, const fs_swarm* swarm, uint64_t seed);

/* Fitness of the current positions: fit = F_sum / N_p (the paper's F-hat,
 * Eq. semi-cohF) with the segments of fs_fstat_batch (edges_dev as its
 * partition_edges_dev);
 * a particle outside [0,1]^D is not evaluated and gets -inf ("let them fly").
 * R * n_part must not exceed the plan's reservation if the call is captured. */
FS_API fs_status fs_pso_evaluate(fs_plan* plan, const fs_swarm* swarm, const double* edges_dev, int N_p);

/* One PSO update (Eqs. pso_position_update, pso_velocity_update): personal
 * bests on a strictly greater fitness, ring local best {i-1, i, i+1} with ties
 * to the lowest index, v <- w v + c1 r1 (p - x) + c2 r2 (l - x) clamped to
 * [-vmax, vmax], x <- x + v.  w = w0 - (w0 - w1) k / (n_iter - 1) at iteration
 * k; r1, r2 from Philox4x32-10 with counter (k, particle, dim, run), key = seed.
 * iteration >= 0 gives k directly; iteration < 0 reads k from *swarm->iter and
 * increments it afterwards (on the device).  lbest_dev: optional [R][n_part]
 * local-best indices.  Asynchronous. */
FS_API fs_status fs_pso_step(fs_plan* plan, const fs_swarm* swarm, uint64_t seed, int iteration, double w0,
                             double w1, int n_iter, double c1, double c2, double vmax, int* lbest_dev);

/* Best personal best of every run: best_f_dev [R], best_idx_dev [R] (lowest
 * particle index among equals).  Asynchronous. */
FS_API fs_status fs_pso_best(fs_plan* plan, const fs_swarm* swarm, double* best_f_dev, int* best_idx_dev);

typedef struct fs_graph fs_graph;

/* Capture one full PSO iteration (fs_pso_evaluate + fs_pso_step with the
 * device iteration counter) as a CUDA graph on the plan's stream, which must
 * not be the legacy default stream.  The graph reads and writes the swarm's
 * buffers and the plan's workspace as they are at capture time: keep both
 * alive and do not grow the workspace (reserve B >= R * n_part first).  Runs
 * one untimed evaluation before capturing.  Synchronous.  *out is NULL on
 * failure. */
FS_API fs_status fs_pso_graph_build(fs_plan* plan, const fs_swarm* swarm, const double* edges_dev, int N_p,
                                    uint64_t seed, double w0, double w1, int n_iter, double c1, double c2,
                                    double vmax, fs_graph** out);

/* Launch a captured iteration n times on its plan's stream.  Asynchronous. */
FS_API fs_status fs_graph_run(fs_graph* graph, int n);

/* Free a captured graph (waits for its stream).  NULL is a no-op. */
FS_API fs_status fs_graph_destroy(fs_graph* graph);

/* ---- Surrogate MLP (not in the paper: ranks candidate PSO moves) ---------- */

/* A 5 -> width -> width -> width -> 1 network with ReLU hidden layers: bf16
 * weights and layer inputs, fp32 accumulation on the tensor cores, fp32
 * master weights trained with Adam on the (particle, F-hat) pairs a search
 * produces.  Inputs are normalised PSO positions in [0,1]^5. */
typedef struct fs_mlp fs_mlp;

/* Number of fp32 parameters: W1 [width][5], b1, W2 [width][width], b2, W3, b3,
 * W4 [width], b4, in that order (row-major), -1 for an invalid width. */
FS_API int64_t fs_mlp_num_params(int width);

/* Create with Kaiming-uniform weights from Philox4x32-10 (key = seed), zero
 * biases and Adam state.  width: a multiple of 8 in [8, 1024]; max_batch:
 * rows per internal pass (larger forward batches are chunked, training
 * batches must fit).  stream: cudaStream_t.  Synchronous. */
FS_API fs_status fs_mlp_create(fs_mlp** out, int width, int max_batch, uint64_t seed, void* stream);
FS_API fs_status fs_mlp_destroy(fs_mlp* mlp);

/* A batch of `groups` independent networks (1 <= groups <= 1024) of one
 * width, evaluated and trained together: every kernel of a pass, the GEMMs
 * included, covers all of them in one launch.  Network g is initialised
 * with key seed + g, so it starts as fs_mlp_create(seed + g) would; its
 * results equal those of that single network run alone (same summation
 * order).  max_batch counts rows per network.  Through the calls below a
 * batch reads and writes per-network blocks laid end to end: parameters
 * [groups][P], inputs X_dev [groups][N][5], targets and outputs
 * [groups][N], losses [groups] (per step); the networks share the Adam step
 * count.  fs_mlp_create is the case groups = 1. */
FS_API fs_status fs_mlp_create_group(fs_mlp** out, int groups, int width, int max_batch, uint64_t seed,
                                     void* stream);

/* Networks in the batch (1 for fs_mlp_create), -1 for NULL. */
FS_API int fs_mlp_groups(const fs_mlp* mlp);

/* Tensor-core path of the network's GEMMs: 1 = tcgen05 (5th-generation
 * tensor cores, accumulators in tensor memory) for the products whose
 * output width is a multiple of 64 or equals 16 -- the forward layers' with
 * operands copied by the tensor memory accelerator, the backward ones' by the
 * CTA's threads -- mma.sync for the others; 2 = tcgen05 for the forward
 * layers, mma.sync for the backward pass (the default at creation); 0 =
 * mma.sync throughout.  All accumulate bf16 products in fp32; results
 * differ only in summation order. */
FS_API fs_status fs_mlp_set_tensor_path(fs_mlp* mlp, int tcgen05);

/* FS_ETIMEOUT (and *timed_out = 1) if a tcgen05 GEMM of this network gave up
 * waiting for its MMAs (its outputs are then invalid); FS_OK otherwise.
 * Waits for the network's stream. */
FS_API fs_status fs_mlp_tensor_status(fs_mlp* mlp, int* timed_out);

/* Copy the fp32 master weights in or out (device buffers of
 * groups x fs_mlp_num_params floats).  Setting weights resets the Adam step count
 * and the target standardisation.  set is synchronous, get asynchronous. */
FS_API fs_status fs_mlp_set_params(fs_mlp* mlp, const float* theta_dev);
FS_API fs_status fs_mlp_get_params(fs_mlp* mlp, float* theta_dev);

/* Predictions y_dev [groups][N] for X_dev [groups][N][5] (fp32, device), in the units of
 * the targets of the last fs_mlp_train call (raw network output before any
 * training).  Asynchronous. */
FS_API fs_status fs_mlp_forward(fs_mlp* mlp, const float* X_dev, int N, float* y_dev);

/* Loss L = (1/2n) sum (y - t)^2 over the n finite targets t_dev [groups][N]
 * (NaN = ignored, no standardisation), per network, and its gradient with
 * respect to the fp32 master weights (grad_dev: groups x fs_mlp_num_params
 * floats, may be NULL; loss_dev: groups floats, may be NULL).
 * 1 <= N <= max_batch.  Asynchronous. */
FS_API fs_status fs_mlp_loss_grad(fs_mlp* mlp, const float* X_dev, const float* t_dev, int N, float* grad_dev,
                                  float* loss_dev);

/* `steps` full-batch Adam steps (lr, beta1 = 0.9, beta2 = 0.999, eps = 1e-8)
 * on (X_dev, t_dev) with the finite targets standardised by their mean and
 * standard deviation (per network); loss_dev: optional [steps][groups]
 * losses.  Asynchronous. */
FS_API fs_status fs_mlp_train(fs_mlp* mlp, const float* X_dev, const float* t_dev, int N, int steps, float lr,
                              float* loss_dev);

/* fs_pso_step with surrogate screening: after the personal-best update, n_cand
 * candidate moves are drawn per particle (candidate c uses the Philox counter
 * (k, particle, dim, run | c << 20), so candidate 0 is the fs_pso_step move),
 * a network predicts their fitness, and each particle takes the candidate
 * with the highest prediction (lowest index among equals; candidates outside
 * [0,1]^5 rank last; a swarm with D = 6 gets FS_EUNSUPPORTED, the networks
 * taking 5 inputs).  mlps: n_mlp >= 1 network batches holding ng networks
 * in all (in order); R must be a multiple of ng and the j-th network ranks
 * the candidates of runs [j R/ng, (j+1) R/ng) (one network per search box,
 * since positions are normalised to each run's box).  1 <= n_cand <= 64; candidates go through a network in chunks
 * of its max_batch.  The networks must run on the plan's stream.
 * Asynchronous; allocates its candidate buffers in the plan (synchronously)
 * when they are too small. */
FS_API fs_status fs_pso_step_screened(fs_plan* plan, const fs_swarm* swarm, fs_mlp* const* mlps, int n_mlp,
                                      int n_cand, uint64_t seed, int iteration, double w0, double w1, int n_iter,
                                      double c1, double c2, double vmax);

/* Ring buffer of (position, fitness) samples a search collects to train the
 * surrogate.  x: [cap][D] floats (D of the swarms that append), f: [cap] floats, count: one unsigned
 * 64-bit counter of samples appended so far (all device memory, owned by
 * the caller; set count to 0 to start).  Sample i of an append of n goes to
 * slot (count + i) mod cap, and count advances by n. */
typedef struct {
    float* x;
    float* f;
    int cap;
    unsigned long long* count;
    int dims;   /* floats per sample: 5 (or 0) or 6; must equal the appending swarm's D */
} fs_sample_ring;

/* Append the swarm's current positions (as floats) and fitness (NaN where
 * not finite) to the rings: R must be a multiple of n_rings and ring g takes
 * the particles of runs [g R/n_rings, (g+1) R/n_rings).  Asynchronous. */
FS_API fs_status fs_pso_record(fs_plan* plan, const fs_swarm* swarm, const fs_sample_ring* rings, int n_rings);

/* Capture a chosen part of a PSO iteration as a CUDA graph (as
 * fs_pso_graph_build does for the whole of it).  parts: bit 1 = evaluate
 * (fs_pso_evaluate), bit 2 = append to the rings (fs_pso_record), bit 4 =
 * fs_pso_step, bit 8 = fs_pso_step_screened with the networks and n_cand (4
 * and 8 exclusive); both steps use the device iteration counter.  The
 * networks' stream must be the plan's stream; their weights are read when
 * the graph runs, so training between launches takes effect.  The ring and
 * network arrays are read at capture time.  Synchronous; runs one untimed
 * evaluation first when bit 1 is set. */
FS_API fs_status fs_pso_graph_build_ex(fs_plan* plan, const fs_swarm* swarm, const double* edges_dev, int N_p,
                                       uint64_t seed, double w0, double w1, int n_iter, double c1, double c2,
                                       double vmax, int parts, const fs_sample_ring* rings, int n_rings,
                                       fs_mlp* const* mlps, int n_mlp, int n_cand, fs_graph** out);

/* Capture `steps` Adam steps of fs_mlp_train for each network on its ring's
 * whole contents (all cap slots; empty slots hold NaN targets, which the loss
 * ignores) as one CUDA graph, run with fs_graph_run.  rings holds one ring
 * per network (the sum of the batches' group counts); the rings of a batch
 * of G networks must be consecutive slices of one buffer (ring j of the
 * batch at x + j cap 5 and f + j cap, one cap).  The networks must share
 * one stream that is not the legacy default stream; the rings' buffers are
 * read when the graph runs.  The Adam step count lives on the device, so
 * replays continue the optimisation.  Synchronous. */
FS_API fs_status fs_mlp_train_graph_build(fs_mlp* const* mlps, int n, const fs_sample_ring* rings, int steps,
                                          float lr, fs_graph** out);

/* Response model of the FS_FP64 path (Sec. IV, Eq. freDres).
 *   filter_order = -1 (default): the paper's own choice, N = 0 with the
 *     higher-order d(t) terms neglected: T(f) = F(t_f) e^{2 pi i f d(t_f)}.
 *   filter_order = N in 0..2: the series of Eq. (freDres) itself,
 *     T(f) = sum_{k=0}^{k_max} (-i T_A1)^k / k!  F^N_{T_f}[d^k G/dtau^k](t_f),
 *     G(tau) = F(tau - d(tau)) / (1 + ddot(tau)) e^{2 pi i f d(tau)(1 - ddot(tau))},
 *     F^N_{T_f}[G](t) = 1/2 sum_{j=0}^{N} a_j (G(t + j T_f) + G(t - j T_f)),
 *     T_A1 = (7/6)/(2 pi f), T_f^2 = |d^2 Psi/df^2|/(4 pi), with the antenna
 *     pattern at the retarded time, the 1/(1 + ddot) factor and the ddot
 *     phase term.  The weights a_j (defined in a reference the paper cites)
 *     are taken as those that make the filter reproduce the even moments of
 *     the stationary-phase kernel e^{i pi fdot s^2} up to order 2N: a_0 = 1
 *     (N = 0); 1 - i/pi, i/pi (N = 1); 1 - 3/(4 pi^2) - 5i/(4 pi),
 *     1/pi^2 + 4i/(3 pi), -1/(4 pi^2) - i/(12 pi) (N = 2).
 *   k_max: 0 or 1 (the paper defines T_A1 only).
 * With the series the responses are complex, so each segment carries an
 * eighth sum (the imaginary part of the cross Gram term) and the 4x4 solve
 * of Eq. (aandMN3) takes the Hermitian 2x2 form.  It applies to every later
 * F-statistic, amplitude, swarm evaluation and fs_add_signal of the plan;
 * graphs built earlier keep the response they were captured with.  It runs
 * in the direct form of the fused kernel (launch variants 0-2; variants 3
 * and 4 take variant 0's tile), at several times the per-bin cost.
 * FS_EINVAL for arguments out of range, FS_EUNSUPPORTED for a series on an
 * FS_MIXED plan.  Host only, no device work. */
FS_API fs_status fs_plan_set_response(fs_plan* plan, int filter_order, int k_max);
FS_API fs_status fs_plan_get_response(const fs_plan* plan, int* filter_order, int* k_max);

/* Spacecraft orbits of the FS_FP64 path (Sec. IV: the paper's analytic orbit
 * is accurate to second order in eccentricity).
 *   eccentricity = 0 (default): the rigid equilateral constellation (the
 *     orbits to first order in e), whose patterns are trig polynomials of
 *     degree 4 in the orbital phase alpha.
 *   eccentricity = e in (0, 0.05]: each spacecraft on the Keplerian ellipse
 *     of semi-major axis 1 AU, eccentricity e and inclination sqrt(3) e,
 *     perihelia 120 degrees apart in mean anomaly, expanded to second order
 *     in e; arms normalised exactly, patterns of the long-wavelength
 *     Michelsons (and of A and E) from the three arm directions at each bin.
 *     The first order in e gives the rigid form; the second makes the arms
 *     breathe and tilt by O(e).  LISA's 2.5e9 m arms give
 *     e = L / (2 sqrt(3) AU) = 4.824e-3.
 * The Doppler delay stays that of the guiding centre.  The eccentric orbits
 * run in the direct form of the fused kernel (launch variants 0-2; 3 and 4
 * take variant 0's tile) and combine with fs_plan_set_response.  It applies
 * to every later F-statistic, amplitude, swarm evaluation and fs_add_signal
 * of the plan; graphs built earlier keep the orbits they were captured with.
 * FS_EINVAL for e outside [0, 0.05], FS_EUNSUPPORTED for e > 0 on an
 * FS_MIXED plan.  Host only, no device work. */
FS_API fs_status fs_plan_set_orbit(fs_plan* plan, double eccentricity);
FS_API fs_status fs_plan_get_orbit(const fs_plan* plan, double* eccentricity);

/* Arm transfer of the FS_FP64 path's response (Sec. IV: a TDI combination is
 * a sum of time-delayed single-arm responses).
 *   arm_seconds = 0 (default): the long-wavelength limit, patterns
 *     D : e_A of the Michelson detector tensors.
 *   arm_seconds = L > 0: the finite-arm response of the first-generation TDI
 *     Michelsons with nominal arm L (LISA: 2.5e9 m = 8.339 s), constellation
 *     frozen at t_f.  Link s -> r (n = (x_r - x_s)/L_sr, k the propagation
 *     direction): y = (n.e_A.n) (-i pi f L_sr) sinc(pi f L_sr (1 - k.n))
 *     e^{-i pi f (L_sr + k.(x_s + x_r))}; vertex v with arms to a and b:
 *     R_v = [e^{-2 pi i f L_va} y_va + y_av - e^{-2 pi i f L_vb} y_vb - y_bv]
 *     / (-4 pi i f L), which tends to the long-wavelength pattern as f L -> 0
 *     (the TDI factor 1 - e^{-4 pi i f L}, common to signal and noise, is
 *     divided out); X = R_0, A = (R_2 - R_0)/sqrt2, E = (R_0 - 2R_1 + R_2)/sqrt6.
 *     Positions x are the guiding centre (whose delay is the Doppler term of
 *     the template phase) plus L/(2 sqrt3) times the orbit offsets, rigid or
 *     to second order in eccentricity (fs_plan_set_orbit).  The responses are
 *     complex, so each segment carries eight sums, as for the series.
 * It applies to every later evaluation and fs_add_signal of the plan (graphs
 * built earlier keep what they were captured with); it runs in the direct
 * form of the fused kernel.  FS_EINVAL for L outside [0, 100] s;
 * FS_EUNSUPPORTED for L > 0 on an FS_MIXED plan or together with the response
 * series (fs_plan_set_response with a filter order >= 0).  Host only. */
FS_API fs_status fs_plan_set_arm(fs_plan* plan, double arm_seconds);
FS_API fs_status fs_plan_get_arm(const fs_plan* plan, double* arm_seconds);

/* Launch variants of the fused bin-loop kernel (the tile shape of the
 * ragged batch, Sec. IV's particle x frequency parallelism).
 *   FS_FP64 : direct form, the whole template evaluated at every bin:
 *             0 = 2048-bin tiles per (particle, tile) item, 1 = 1024, 2 = 4096;
 *             anchored form, each 1024-bin tile expanded about its centre
 *             bin (exact 64-bit fixed-point cubic phase plus FP64 higher
 *             terms and polynomials, truncation bounded per tile, bin-by-bin
 *             fallback): 3 = grid form, 4 = persistent form.  The direct
 *             variants differ by rounding only (relative 1e-15); the
 *             anchored ones by their truncation bounds as well (phase
 *             1e-11 cycle per bin: relative 1e-10 or less on F).
 *   FS_MIXED: 0 = one CTA per (span of 32768 bins, 8 in-band particles), 2
 *             CTAs per SM; 1 = the same with 3 CTAs per SM; 2 = persistent
 *             kernel (one grid of SMs x resident CTAs whose warps take
 *             (span, particle) items from a device-side counter), 2 CTAs per
 *             SM; 3 = persistent, 3 CTAs per SM; 4 = the CTA form of 0 with
 *             each 1024-bin tile of the FP32 tables copied once per CTA into
 *             shared memory by a bulk asynchronous copy and read by all 8
 *             warps (bounded waits: a wait that runs out is reported by
 *             fs_plan_check).  F is bit-identical across the five.
 * Which variant a call uses: the forced one if fs_plan_set_variant gave one
 * (>= 0), else the one recorded for (N_p, edge kind) by fs_plan_autotune,
 * fs_pso_autotune or fs_plan_set_variant_for, else the mode's default
 * (FS_FP64: 4, FS_MIXED: 3).
 *
 * fs_plan_set_variant: force `variant` for every call, or -1 to return to
 * the per-(N_p, edge kind) choice.  FS_EINVAL if out of range. */
FS_API fs_status fs_plan_set_variant(fs_plan* plan, int variant);

/* Record `variant` for calls with this N_p and edge kind (global_edges != 0:
 * edge frequencies given; 0: per-particle edges), as the autotuner would.  Lets a
 * resumed search reuse the choices of the run it continues. */
FS_API fs_status fs_plan_set_variant_for(fs_plan* plan, int N_p, int global_edges, int variant);

/* The variant a call with this N_p and edge kind would use now. */
FS_API fs_status fs_plan_get_variant(fs_plan* plan, int N_p, int global_edges, int* variant);

/* Census of the anchored kernels' evaluation modes for one batch: runs
 * fs_fstat_batch once (F to plan scratch) with the variant the call resolves
 * to, counting in-band particle*bins per tile mode, and returns them in
 * counts[9]: [2] bin-by-bin fallback; FS_MIXED: [1] FP32 polynomial body,
 * [3] its low-degree tier (antenna degree 3, Doppler to d(alpha)^3);
 * FS_FP64 anchored variants: the degree tiers (antenna polynomial degree,
 * phase-remainder degree) [5] (6, 6), [4] (7, 7), [3] (8, 9), [1] (10, 11),
 * [6] (6, 6) with the phase remainder (at most 6.7e-8 cycle) evaluated
 * in FP32, [7] the same with antenna degree 5 and [8] with degree 4; [0]
 * unused.  All zero for the direct FS_FP64 variants (0-2), which have no
 * anchors.  Synchronous; must not be called while the plan's stream is being
 * captured.  For roofline accounting (the operation count per bin differs
 * between modes and tiers). */
FS_API fs_status fs_plan_census(fs_plan* plan, const fs_params* params_dev, int B, const double* edges_dev,
                                int N_p, int64_t* counts);

/* Autotuner: time every variant on this batch (one untimed call, then `reps`
 * calls between CUDA events on the plan's stream, 1 <= reps <= 1000), record
 * the fastest for (N_p, edge kind) and return it in *variant_out (may be
 * NULL); ms_out (may be NULL) receives the mean ms per call of each variant
 * (5 entries in either mode).  Synchronous; FS_EINVAL while the
 * plan's stream is being captured.  Arguments as in fs_fstat_batch; the F
 * values computed go to plan scratch, not to the caller. */
FS_API fs_status fs_plan_autotune(fs_plan* plan, const fs_params* params_dev, int B, const double* edges_dev,
                                  int N_p, int reps, int* variant_out, float* ms_out);

/* fs_plan_autotune on the swarm's current positions (mapped to physical
 * parameters as fs_pso_evaluate does).  The swarm is not modified. */
FS_API fs_status fs_pso_autotune(fs_plan* plan, const fs_swarm* swarm, const double* edges_dev, int N_p,
                                 int reps, int* variant_out, float* ms_out);

/* Kernel timing on the plan's stream.  While enabled, every kernel the plan
 * launches is bracketed by CUDA events.  fs_plan_read_profile waits for the
 * plan's stream, returns the summed duration (ms) and launch count of one
 * kernel kind since the last read (0 = per-particle setup, 1 = fused
 * template/reduction kernel, 2 = segment solve and sum, 3 = per-bin
 * precompute) and resets that kind's counters. */
FS_API fs_status fs_plan_set_profiling(fs_plan* plan, int enable);
FS_API fs_status fs_plan_read_profile(fs_plan* plan, int kernel, double* total_ms, int64_t* launches);

/* fs_fstat_batch without any device allocation, for callers that cannot
 * call cudaMalloc (code inside an allocator-free library or host callback, a
 * process whose device memory is owned by another runtime, or a caller with a
 * fixed memory budget).  The paper has no counterpart: it is a deployment
 * variant of fs_fstat_batch in FS_FP64 mode, not part of the method.
 *   Inputs are the grid (n_bins, f_min, df, T_obs as for fs_plan_create), the
 *   data and PSD (as for fs_plan_set_data with f_grid_dev = NULL), params_dev
 *   / B / edges_dev / N_p (as for fs_fstat_batch: edge frequencies in device
 *   memory, converted to bins inside the call; invalid edges give F = NaN,
 *   there is no flag word to check); outputs F_dev and F_part_dev (may be
 *   NULL) as for fs_fstat_batch; stream is a cudaStream_t (NULL = legacy
 *   default stream).
 *   Limits: n_bins <= 32768, 0 <= B <= 1024, 1 <= N_p <= 64; larger requests
 *   return FS_EINVAL with a message naming the limit.
 * Workspace: a 10 MiB file-scope device array of the library, held by every
 * GPU that loads the library until the process exits.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process (a cudaDeviceReset
 * afterwards is not supported); make that first call before any stream
 * capture.  All calls
 * share the one array and each call overwrites what it needs, so calls that
 * may overlap on the GPU (different streams, or different host threads on the
 * same device) race and must be serialised by the caller.  Calls no
 * cudaMalloc, cudaFree or other allocating routine.  Asynchronous. */
FS_API fs_status fs_fstat_batch_noalloc(int64_t n_bins, double f_min, double df, double T_obs,
                                        const double* data_dev, const double* psd_dev, const fs_params* params_dev,
                                        int B, const double* edges_dev, int N_p, double* F_dev,
                                        double* F_part_dev, void* stream);

/* Constants compiled into the library: out[0] = solar mass in s, out[1] =
 * year in s, out[2] = AU/c in s, out[3] = eccentricity reference frequency (Hz). */
FS_API fs_status fs_constants(double* out_host);

/* Message of the last failed call on this thread ("" if none). */
FS_API const char* fs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FSTAT_H */
