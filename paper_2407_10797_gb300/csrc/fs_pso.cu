// fs_pso.cu - device-side particle swarm optimisation (Sec. III.A).
//
//   x_{i,j}[k+1] = x_{i,j}[k] + clamp(v_{i,j}[k+1], -v_max, v_max)      Eq. (pso_position_update)
//   v_{i,j}[k+1] = w[k] v + c1 r1 (p - x) + c2 r2 (l - x)                 Eq. (pso_velocity_update)
// with p the personal best (replaced only on a strictly greater fitness), l
// the best personal best on the ring {i-1, i, i+1} (ties to the lowest
// index), r1, r2 ~ U[0,1) from Philox4x32-10 with counter (iteration,
// particle, dim, run) and key = seed, "let them fly" boundaries (a particle
// outside the unit box gets fitness -inf and is not evaluated), and a
// linearly decaying inertia weight.  The update is written with explicit
// round-to-nearest multiplies and adds (no contraction), so it is bit-exact
// against a plain CPU implementation of the same order of operations.
//
// Not in the paper: a screened step (each particle draws several candidate
// moves with distinct Philox counters, the surrogate networks of its run's
// group rank them, and the best-ranked in-box candidate is taken), and the
// recording of (position, fitness) samples into the device rings the
// networks train on.
#include <cmath>

#include "fs_internal.h"

namespace fs {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__device__ __forceinline__ double u53(uint32_t lo, uint32_t hi) {
    const unsigned long long w = ((unsigned long long)hi << 32) | lo;
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

// x ~ U[0,1)^D, v ~ U[-x, 1-x): counter (0xFFFFFFFF, particle, dim, run).
__global__ void pso_init_kernel(int R, int Np, int D, unsigned long long seed, double* x, double* v, double* pbx,
                                double* pbf, double* fit, int run0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)R * Np * D;
    if (i >= n) return;
    const int j = (int)(i % D);
    const int p = (int)((i / D) % Np);
    const int r = (int)(i / ((int64_t)D * Np));
    uint32_t c[4] = {0xFFFFFFFFu, (uint32_t)p, (uint32_t)j, (uint32_t)(r + run0)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
    x[i] = u1;
    v[i] = __dsub_rn(u2, u1);
    pbx[i] = u1;
    if (j == 0) {
        pbf[i / D] = -INFINITY;
        fit[i / D] = -INFINITY;
    }
}

// Map normalised positions to physical parameters in each run's box; a
// particle outside [0, 1]^D gets NaN parameters (the F-statistic skips it).
// box: [R][D][2] = (lo, hi) of (Mc [Msun], tc [s], sin(lat), lon [rad], e0)
// and, with D = 6, of the dimensionless mass difference delta_mu = (m1 - m2)/M
// (Sec. II.A's Theta_I), whose mass ratio is q = (1 + delta_mu)/(1 - delta_mu);
// with D = 5 every particle takes the swarm's q.
__global__ void pso_map_kernel(int R, int Np, int D, const double* __restrict__ x, const double* __restrict__ box,
                               double q, ::fs_params* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * Np) return;
    const int r = i / Np;
    const double* xi = x + (int64_t)i * D;
    const double* bx = box + (int64_t)r * 2 * D;
    bool inside = true;
    double y[6];
    for (int j = 0; j < D; j++) {
        inside = inside && xi[j] >= 0.0 && xi[j] <= 1.0;
        y[j] = bx[2 * j] + xi[j] * (bx[2 * j + 1] - bx[2 * j]);
    }
    ::fs_params p;
    if (inside && D == 6 && !(y[5] >= 0.0 && y[5] < 1.0)) inside = false;   // delta_mu outside [0, 1)
    if (inside) {
        p.Mc = y[0];
        p.tc = y[1];
        p.lat = asin(fmin(1.0, fmax(-1.0, y[2])));
        p.lon = y[3];
        p.e0 = y[4];
        p.q = D == 6 ? (1.0 + y[5]) / (1.0 - y[5]) : q;
    } else {
        p.Mc = p.tc = p.lat = p.lon = p.e0 = p.q = __longlong_as_double(0x7ff8000000000000LL);
    }
    out[i] = p;
}

// fitness = F_sum / N_p (the paper's F-hat); -inf outside the box (NaN F).
__global__ void pso_fitness_kernel(int n, const double* __restrict__ F, int Np, double* fit) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double f = F[i];
    fit[i] = isnan(f) ? -INFINITY : f / (double)Np;
}

// One iteration, one thread per (run, particle): personal best, ring local
// best, then the D velocity/position updates.  Local bests read personal
// bests that neighbours update in the same launch, so the personal-best pass
// is a separate kernel.
__global__ void pso_pbest_kernel(int R, int Np, int D, const double* __restrict__ x, const double* __restrict__ fit,
                                 double* pbx, double* pbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * Np) return;
    const double f = fit[i];
    if (f > pbf[i]) {   // NaN compares false
        pbf[i] = f;
        for (int j = 0; j < D; j++) pbx[(int64_t)i * D + j] = x[(int64_t)i * D + j];
    }
}

__global__ void pso_move_kernel(int R, int Np, int D, unsigned long long seed, const unsigned int* iter_dev,
                                unsigned int iter_host, double w0, double w1, int n_iter, double c1, double c2,
                                double vmax, double* x, double* v, const double* __restrict__ pbx,
                                const double* __restrict__ pbf, int* lbest_out, int run0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * Np) return;
    const unsigned int it = iter_dev ? *iter_dev : iter_host;
    // linearly decaying inertia weight over n_iter iterations
    const double w = (n_iter > 1) ? __dsub_rn(w0, __dmul_rn(__dsub_rn(w0, w1), __ddiv_rn((double)it, (double)(n_iter - 1))))
                                  : w0;
    const int r = i / Np, p = i % Np;
    const int cand[3] = {(p + Np - 1) % Np, p, (p + 1) % Np};
    int best = -1;
    for (int c = 0; c < 3; c++) {
        const int jn = cand[c];
        if (best < 0) {
            best = jn;
            continue;
        }
        const double fj = pbf[r * Np + jn], fb = pbf[r * Np + best];
        if (fj > fb || (fj == fb && jn < best)) best = jn;
    }
    if (lbest_out) lbest_out[i] = best;
    const int64_t li = (int64_t)r * Np + best;
    for (int j = 0; j < D; j++) {
        uint32_t c[4] = {it, (uint32_t)p, (uint32_t)j, (uint32_t)(r + run0)};
        philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double r1 = u53(c[0], c[1]), r2 = u53(c[2], c[3]);
        const int64_t ij = (int64_t)i * D + j;
        const double xv = x[ij];
        double cog = __dmul_rn(c1, r1);
        cog = __dmul_rn(cog, __dsub_rn(pbx[ij], xv));
        double soc = __dmul_rn(c2, r2);
        soc = __dmul_rn(soc, __dsub_rn(pbx[li * D + j], xv));
        double nv = __dmul_rn(w, v[ij]);
        nv = __dadd_rn(nv, cog);
        nv = __dadd_rn(nv, soc);
        if (nv > vmax) nv = vmax;
        if (nv < -vmax) nv = -vmax;
        v[ij] = nv;
        x[ij] = __dadd_rn(xv, nv);
    }
}

__global__ void pso_advance_kernel(unsigned int* iter_dev) { *iter_dev += 1u; }

// Candidate moves for surrogate screening: n_cand velocity draws per particle,
// candidate c with Philox counter (k, particle, dim, run | c << 20), so
// candidate 0 is the plain move.  Writes x, v of every candidate (fp64) and
// the fp32 network input; `inside` flags candidates in the unit box.
__global__ void pso_candidates_kernel(int R, int Np, int D, int C, unsigned long long seed,
                                      const unsigned int* iter_dev, unsigned int iter_host, double w0, double w1,
                                      int n_iter, double c1, double c2, double vmax, const double* __restrict__ x,
                                      const double* __restrict__ v, const double* __restrict__ pbx,
                                      const double* __restrict__ pbf, double* cx, double* cv, float* cin,
                                      unsigned char* inside, int run0) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * Np * C) return;
    const int c = (int)(idx % C);
    const int i = (int)(idx / C);
    const unsigned int it = iter_dev ? *iter_dev : iter_host;
    const double w = (n_iter > 1) ? __dsub_rn(w0, __dmul_rn(__dsub_rn(w0, w1), __ddiv_rn((double)it, (double)(n_iter - 1))))
                                  : w0;
    const int r = i / Np, p = i % Np;
    const int cand[3] = {(p + Np - 1) % Np, p, (p + 1) % Np};
    int best = -1;
    for (int q = 0; q < 3; q++) {
        const int jn = cand[q];
        if (best < 0) {
            best = jn;
            continue;
        }
        const double fj = pbf[r * Np + jn], fb = pbf[r * Np + best];
        if (fj > fb || (fj == fb && jn < best)) best = jn;
    }
    const int64_t li = (int64_t)r * Np + best;
    bool in = true;
    for (int j = 0; j < D; j++) {
        uint32_t ctr[4] = {it, (uint32_t)p, (uint32_t)j, (uint32_t)(r + run0) | ((uint32_t)c << 20)};
        philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
        const double r1 = u53(ctr[0], ctr[1]), r2 = u53(ctr[2], ctr[3]);
        const int64_t ij = (int64_t)i * D + j;
        const double xv = x[ij];
        double cog = __dmul_rn(c1, r1);
        cog = __dmul_rn(cog, __dsub_rn(pbx[ij], xv));
        double soc = __dmul_rn(c2, r2);
        soc = __dmul_rn(soc, __dsub_rn(pbx[li * D + j], xv));
        double nv = __dmul_rn(w, v[ij]);
        nv = __dadd_rn(nv, cog);
        nv = __dadd_rn(nv, soc);
        if (nv > vmax) nv = vmax;
        if (nv < -vmax) nv = -vmax;
        const double nx = __dadd_rn(xv, nv);
        cv[idx * D + j] = nv;
        cx[idx * D + j] = nx;
        cin[idx * D + j] = (float)nx;
        in = in && nx >= 0.0 && nx <= 1.0;
    }
    inside[idx] = in ? 1 : 0;
}

// Keep the candidate with the highest predicted fitness (lowest index among
// equals; out-of-box candidates rank last, and if all are out of the box the
// plain move, candidate 0, is kept).
__global__ void pso_select_kernel(int R, int Np, int D, int C, const float* __restrict__ score,
                                  const unsigned char* __restrict__ inside, const double* __restrict__ cx,
                                  const double* __restrict__ cv, double* x, double* v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * Np) return;
    int best = 0;
    float bs = -INFINITY;
    bool any = false;
    for (int c = 0; c < C; c++) {
        const int64_t k = (int64_t)i * C + c;
        if (!inside[k]) continue;
        const float sc = isnan(score[k]) ? -INFINITY : score[k];
        if (!any || sc > bs) {
            bs = sc;
            best = c;
            any = true;
        }
    }
    const int64_t k = (int64_t)i * C + best;
    for (int j = 0; j < D; j++) {
        x[(int64_t)i * D + j] = cx[k * D + j];
        v[(int64_t)i * D + j] = cv[k * D + j];
    }
}

// Best personal best of every run (lowest index among equals).
__global__ void pso_best_kernel(int R, int Np, const double* __restrict__ pbf, double* best_f, int* best_i) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int bi = 0;
    double bf = pbf[(int64_t)r * Np];
    for (int p = 1; p < Np; p++) {
        const double f = pbf[(int64_t)r * Np + p];
        if (f > bf) {
            bf = f;
            bi = p;
        }
    }
    best_f[r] = bf;
    best_i[r] = bi;
}

cudaError_t launch_pso_init(int R, int Np, int D, unsigned long long seed, double* x, double* v, double* pbx,
                            double* pbf, double* fit, int run0, cudaStream_t s) {
    const int64_t n = (int64_t)R * Np * D;
    if (n == 0) return cudaSuccess;
    pso_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, Np, D, seed, x, v, pbx, pbf, fit, run0);
    return cudaGetLastError();
}

cudaError_t launch_pso_map(int R, int Np, int D, const double* x, const double* box, double q, ::fs_params* out,
                           cudaStream_t s) {
    const int n = R * Np;
    if (n == 0) return cudaSuccess;
    pso_map_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, Np, D, x, box, q, out);
    return cudaGetLastError();
}

cudaError_t launch_pso_fitness(int n, const double* F, int Np, double* fit, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    pso_fitness_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, F, Np, fit);
    return cudaGetLastError();
}

cudaError_t launch_pso_step(int R, int Np, int D, unsigned long long seed, const unsigned int* iter_dev,
                            unsigned int iter_host, double w0, double w1, int n_iter, double c1, double c2, double vmax,
                            double* x, double* v, double* pbx, double* pbf, const double* fit, int* lbest,
                            unsigned int* iter_advance, int run0, cudaStream_t s) {
    const int n = R * Np;
    if (n == 0) return cudaSuccess;
    pso_pbest_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, Np, D, x, fit, pbx, pbf);
    pso_move_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, Np, D, seed, iter_dev, iter_host, w0, w1, n_iter, c1, c2, vmax,
                                                    x, v, pbx, pbf, lbest, run0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !iter_advance) return e;
    pso_advance_kernel<<<1, 1, 0, s>>>(iter_advance);
    return cudaGetLastError();
}

// Surrogate training samples: positions as floats, non-finite fitness as
// NaN, into slot (count + i) mod cap of a ring; the counter advances after.
// Sample append for up to kRingBatch rings in one launch: particle k of ring g
// (the g-th block of `per` particles) goes to slot (count_g + k) mod cap_g.
__global__ void pso_record_kernel(int nr, int per, int D, const double* __restrict__ x,
                                  const double* __restrict__ fit, RingBatch rb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nr * per) return;
    const int g = (int)(i / per), k = (int)(i % per);
    const int64_t j = (int64_t)((*rb.count[g] + (unsigned long long)k) % (unsigned long long)rb.cap[g]);
    float* rx = rb.x[g];
    for (int d = 0; d < D; d++) rx[j * D + d] = (float)x[i * D + d];
    const double f = fit[i];
    rb.f[g][j] = isfinite(f) ? (float)f : __int_as_float(0x7fc00000);
}

__global__ void ring_advance_kernel(int nr, int per, RingBatch rb) {
    const int g = threadIdx.x;
    if (g < nr) *rb.count[g] += (unsigned long long)per;
}

cudaError_t launch_pso_record(int nr, int per, int D, const double* x, const double* fit, const RingBatch& rb,
                              cudaStream_t s) {
    if (nr <= 0 || per <= 0) return cudaSuccess;
    const int64_t n = (int64_t)nr * per;
    pso_record_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(nr, per, D, x, fit, rb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ring_advance_kernel<<<1, kRingBatch, 0, s>>>(nr, per, rb);
    return cudaGetLastError();
}

cudaError_t launch_pso_screened(int R, int Np, int C, unsigned long long seed, const unsigned int* iter_dev,
                                unsigned int iter_host, double w0, double w1, int n_iter, double c1, double c2,
                                double vmax, double* x, double* v, double* pbx, double* pbf, const double* fit,
                                double* cx, double* cv, float* cin, unsigned char* inside, float* score,
                                fs_mlp* const* mlps, int n_mlp, unsigned int* iter_advance, int run0, cudaStream_t s) {
    const int n = R * Np;
    if (n == 0) return cudaSuccess;
    pso_pbest_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, Np, 5, x, fit, pbx, pbf);
    const int64_t nc = (int64_t)n * C;
    pso_candidates_kernel<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(R, Np, 5, C, seed, iter_dev, iter_host, w0, w1,
                                                                       n_iter, c1, c2, vmax, x, v, pbx, pbf, cx, cv,
                                                                       cin, inside, run0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the networks' groups, in order, split the runs into equal contiguous blocks:
    // group j ranks the candidates of runs [j R / ng, (j + 1) R / ng)
    int ng = 0;
    for (int i = 0; i < n_mlp; i++) ng += fs_mlp_groups(mlps[i]);
    const int64_t per = nc / ng;
    for (int i = 0, j = 0; i < n_mlp; j += fs_mlp_groups(mlps[i]), i++)
        if (fs_mlp_forward(mlps[i], cin + j * per * 5, (int)per, score + j * per) != FS_OK)
            return cudaErrorLaunchFailure;
    pso_select_kernel<<<(n + 127) / 128, 128, 0, s>>>(R, Np, 5, C, score, inside, cx, cv, x, v);
    if ((e = cudaGetLastError()) != cudaSuccess || !iter_advance) return e;
    pso_advance_kernel<<<1, 1, 0, s>>>(iter_advance);
    return cudaGetLastError();
}

cudaError_t launch_pso_best(int R, int Np, const double* pbf, double* best_f, int* best_i, cudaStream_t s) {
    if (R == 0) return cudaSuccess;
    pso_best_kernel<<<(R + 63) / 64, 64, 0, s>>>(R, Np, pbf, best_f, best_i);
    return cudaGetLastError();
}

}  // namespace fs
