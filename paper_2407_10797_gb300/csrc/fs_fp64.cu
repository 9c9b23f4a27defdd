// fs_fp64.cu - per-dataset precompute, per-particle setup, the FP64 fused
// template + segmented-reduction kernel and the per-segment 4x4 solve.
//
//   precompute (once per data set)      Sec. II.A Eq. inner_product, App. A Eq. A1
//   setup (per particle)                App. A Eq. A3, Sec. II.B segment edges, Sec. IV t_f
//   fp64_main (per particle x bin)      Sec. II.A Eqs. response, aandMN, aandMN2; Sec. IV Eq. freDres
//   reduce (per particle x segment)     Sec. II.A Eq. coherent_F_stat, Sec. II.B Eq. semi-cohF
#include <cfloat>
#include <climits>

#include "fs_internal.h"
#include "fs_device.cuh"

namespace fs {

// ---------------------------------------------------------------------------
// A0: per-bin tables.  Templates are f^-7/6 e^{-i Psi}; the amplitude and the
// noise weighting do not depend on the particle, so they are folded into the
// data (dw) and into the weight W of the Gram matrix.
// ---------------------------------------------------------------------------
__global__ void precompute_kernel(Grid g, const double* __restrict__ data, const double* __restrict__ psd,
                                  Tables t) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    // f_k = f_min + k df as a double-double
    double p, e, s, s2;
    two_prod((double)k, g.df, p, e);
    two_sum(g.f_min, p, s, s2);
    double fh, fl;
    fast_two_sum(s, s2 + e, fh, fl);
    double u = rcbrt(fh);
    // f^-5/3 to double-double: y0 ~ u^5, then one Newton step on y^-3 = f^5
    double y0 = u * u;
    y0 = y0 * y0 * u;
    double y2h, y2l, y3h, y3l, f2h, f2l, f4h, f4l, f5h, f5l, ph, pl;
    dd_mul(y0, 0.0, y0, 0.0, y2h, y2l);
    dd_mul(y2h, y2l, y0, 0.0, y3h, y3l);
    dd_mul(fh, fl, fh, fl, f2h, f2l);
    dd_mul(f2h, f2l, f2h, f2l, f4h, f4l);
    dd_mul(f4h, f4l, fh, fl, f5h, f5l);
    dd_mul(y3h, y3l, f5h, f5l, ph, pl);
    double r = (1.0 - ph) - pl;
    double gh, gl;
    fast_two_sum(y0, y0 * r * (1.0 / 3.0), gh, gl);
    double S = psd[k];
    double w4 = 4.0 * g.df / S;
    double amp = pow(fh, -7.0 / 6.0);
    double u7 = u * u * u;
    u7 = u7 * u7 * u;
    t.fh[k] = fh;
    t.fl[k] = fl;
    t.u[k] = u;
    t.g0h[k] = gh;
    t.g0l[k] = gl;
    t.e19[k] = pow(kF0Ecc / fh, 19.0 / 9.0);
    t.dwr[k] = w4 * amp * data[2 * k];
    t.dwi[k] = w4 * amp * data[2 * k + 1];
    t.W[k] = w4 * u7;
}

cudaError_t launch_precompute(const Grid& g, const double* data, const double* psd, const Tables& t,
                              cudaStream_t s) {
    int threads = 256;
    int64_t blocks = (g.n + threads - 1) / threads;
    precompute_kernel<<<(unsigned)blocks, threads, 0, s>>>(g, data, psd, t);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A1: per-particle coefficients and band edges.
// ---------------------------------------------------------------------------
// First k in [lo, hi) with pred(k) true for a predicate that is false then
// true along k (hi if none), searched by a whole warp: each round probes 32
// points and keeps the interval between the last false and first true probe.
template <typename Pred>
__device__ int64_t warp_search_first(int64_t lo, int64_t hi, Pred pred) {
    const int lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const int64_t w = hi - lo;
        const int64_t q = lo + (w * (lane + 1)) / 33;   // strictly increasing in lane, inside [lo, hi)
        const unsigned m = __ballot_sync(0xffffffffu, pred(q));
        if (m == 0u) {
            lo = __shfl_sync(0xffffffffu, q, 31) + 1;
        } else {
            const int f = __ffs(m) - 1;
            const int64_t qf = __shfl_sync(0xffffffffu, q, f);
            const int64_t qp = __shfl_sync(0xffffffffu, q, f > 0 ? f - 1 : 0);
            if (f > 0) lo = qp + 1;
            hi = qf;
        }
    }
    const int64_t k = lo + lane;
    const unsigned m = __ballot_sync(0xffffffffu, k < hi && pred(k));
    return m ? lo + (__ffs(m) - 1) : hi;
}

// Continuous solution f of t(f) = target (the band edge's frequency, Sec. II's
// band [f(t = 0), f(t = T_obs)]): the Newtonian chirp t - t_c = T0 f^-8/3 gives
// the start, Newton steps with the slope of the same series refine it,
//   dt/df = -(1/f) [8/3 T0 f^-8/3 + 2 T2 f^-2 + 5/3 T3 f^-5/3 + 4/3 T4 f^-4/3
//                   + (8/3 + 19/9) TE f^-8/3 (f0/f)^(19/9)].
// +inf when the target is at or after coalescence at Newtonian order, NaN if
// the steps fail; the caller only uses it to place a window that it checks.
__device__ double edge_freq(const Particle& P, double target) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (!(P.T0 < 0.0)) return nan;
    const double x0 = (target - P.tc) / P.T0;
    if (!(x0 > 0.0)) return __longlong_as_double(0x7ff0000000000000LL);
    double f = pow(x0, -0.375);
    for (int it = 0; it < 8; it++) {
        const FreqPowers w = powers_of(f);
        const double u2 = w.u * w.u, u3 = u2 * w.u, u4 = u2 * u2, u6 = u3 * u3;
        const double g83 = w.g0h * u3;
        double s = P.T0 * g83;
        s = fma(P.T2, u6, s);
        s = fma(P.T3, w.g0h, s);
        s = fma(P.T4, u4, s);
        s = fma(P.TE * g83, w.e19, s);
        double sl = (8.0 / 3.0) * P.T0 * g83;
        sl = fma(2.0 * P.T2, u6, sl);
        sl = fma((5.0 / 3.0) * P.T3, w.g0h, sl);
        sl = fma((4.0 / 3.0) * P.T4, u4, sl);
        sl = fma((8.0 / 3.0 + 19.0 / 9.0) * P.TE * g83, w.e19, sl);
        const double step = (P.tc + s - target) * f / sl;   // (t - target) / (dt/df), dt/df = -sl / f
        const double fn = f + step;
        if (!(fn > 0.0)) return nan;
        f = fn;
        if (fabs(step) <= 1e-10 * f) break;
    }
    return f;
}

constexpr int kEdgeWin = 16;   // bins per edge window (half a warp)

// First bin of the window that should hold the boundary at frequency fe: 7
// bins below it, clamped into [0, n - kEdgeWin]; -1 if fe gives no position.
__device__ int64_t edge_window(const Grid& g, double fe) {
    const int64_t top = g.n > kEdgeWin ? g.n - kEdgeWin : 0;
    if (fe != fe) return -1;
    const double kf = (fe - g.f_min) / g.df;
    if (!(kf < (double)g.n)) return top;   // includes +inf: above the grid
    if (kf < 8.0) return 0;
    const int64_t k0 = (int64_t)floor(kf) - 7;
    return k0 < top ? k0 : top;
}

// First k in [0, n) with pred(k) true (n if none), for a predicate that is
// false then true along k, from the probes of the window [k0, k0 + kEdgeWin)
// (bit j of m: pred(k0 + j), false for k0 + j >= n): exact when the window
// shows the change (a false probe right before the first true one, or the
// window at an end of [0, n)); *ok = false otherwise.
__device__ int64_t first_in_window(int64_t n, int64_t k0, unsigned m, bool* ok) {
    if (k0 < 0) {
        *ok = false;
        return n;
    }
    if (m) {
        const int f = __ffs(m) - 1;
        *ok = f > 0 || k0 == 0;
        return k0 + f;
    }
    *ok = k0 + kEdgeWin - 1 >= n - 1;   // no true probe and the window reaches the last bin
    return n;
}

// One warp per particle: lane 0 derives the coefficients, nine lanes sample the
// antenna patterns for their harmonics, and the warp searches the band edges.
__global__ void setup_kernel(Grid g, const ::fs_params* __restrict__ params, int B, Particle* parts, int global) {
    __shared__ Particle sp[4];
    __shared__ double fs9[4][2][9], cs9[4][9], sn9[4][9];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int b = blockIdx.x * 4 + wl;
    if (b >= B) return;   // warp-uniform
    Particle& P = sp[wl];
    const ::fs_params in = params[b];
    const bool ok = isfinite(in.Mc) && isfinite(in.tc) && isfinite(in.lat) && isfinite(in.lon) &&
                    isfinite(in.e0) && isfinite(in.q) && in.Mc > 0.0 && in.q > 0.0;
    if (!ok) {
        if (lane == 0) {
            Particle Q;
            memset(&Q, 0, sizeof(Q));
            Q.valid = 0;
            Q.klo = 1;
            Q.khi = 0;
            parts[b] = Q;
        }
        return;
    }
    if (lane == 0) {
        memset(&P, 0, sizeof(P));
        P.valid = 1;
        const double eta = in.q / ((1.0 + in.q) * (1.0 + in.q));
        // Mc in seconds (exact product as a double-double), x = pi Mc
        double mh, ml;
        two_prod(in.Mc, kMsunS, mh, ml);
        double xh, xl;
        dd_mul(kPi, kPiLo, mh, ml, xh, xl);
        // y = x^-5/3 (double-double): Newton step on y^-3 = x^5
        const double y0 = pow(xh, -5.0 / 3.0);
        double y2h, y2l, y3h, y3l, x2h, x2l, x4h, x4l, x5h, x5l, ph, pl;
        dd_mul(y0, 0.0, y0, 0.0, y2h, y2l);
        dd_mul(y2h, y2l, y0, 0.0, y3h, y3l);
        dd_mul(xh, xl, xh, xl, x2h, x2l);
        dd_mul(x2h, x2l, x2h, x2l, x4h, x4l);
        dd_mul(x4h, x4l, xh, xl, x5h, x5l);
        dd_mul(y3h, y3l, x5h, x5l, ph, pl);
        const double r = (1.0 - ph) - pl;
        double yh, yl;
        fast_two_sum(y0, y0 * r * (1.0 / 3.0), yh, yl);
        // P0 = (3/256) y / pi   (Psi_PN/(2 pi) with (3/128)(pi Mc f)^-5/3 at leading order)
        double ah, al;
        dd_mul(3.0 / 256.0, 0.0, yh, yl, ah, al);
        dd_mul(ah, al, kInvPi, kInvPiLo, P.P0h, P.P0l);
        // PN coefficients alpha_k (non-spinning TaylorF2 to 2PN)
        const double a2 = 3715.0 / 756.0 + 55.0 * eta / 9.0;
        const double a3 = -16.0 * kPi;
        const double a4 = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta * eta / 72.0;
        const double M = mh * pow(eta, -0.6);
        const double v1 = cbrt(kPi * M);   // (pi M)^(1/3)
        const double P0 = P.P0h;
        P.P2 = P0 * a2 * v1 * v1;
        P.P3 = P0 * a3 * v1 * v1 * v1;
        P.P4 = P0 * a4 * v1 * v1 * v1 * v1;
        P.E0 = -(2355.0 / 1462.0) * in.e0 * in.e0 * P0;
        // t(f) = dPhi/df: T_k = P_k (k - 5)/3, eccentric part -(34/9) E0 f^-8/3 (f0/f)^(19/9)
        P.T0 = -(5.0 / 3.0) * P0;
        P.T2 = -P.P2;
        P.T3 = -(2.0 / 3.0) * P.P3;
        P.T4 = -(1.0 / 3.0) * P.P4;
        P.TE = -(34.0 / 9.0) * P.E0;
        P.tc = in.tc;
        // Doppler: d(t) = R sin(theta) cos(alpha - phi), theta = pi/2 - beta
        double sb, cb, sl, cl;
        sincos(in.lat, &sb, &cb);
        sincos(in.lon, &sl, &cl);
        P.AD = kAuS * cb;
        P.clon = cl;
        P.slon = sl;
        // antenna: arm unit vectors u_nm = (dr_m - dr_n)/L of the rigid constellation,
        // u = [k(dc C2 + ds S2 - 3 dc), k(dc S2 - ds C2 - 3 ds), -(dc C1 + ds S1)/2],
        // k = 1/(4 sqrt 3), dc = cos b_m - cos b_n, ds = sin b_m - sin b_n, b_n = 2 pi n/3 + orient.
        double cbn[3], sbn[3];
        for (int n = 0; n < 3; n++) sincos(2.0 * kPi * n / 3.0 + g.orient, &sbn[n], &cbn[n]);
        const double kap = 1.0 / (4.0 * sqrt(3.0));
        const double pv[3] = {sb * cl, sb * sl, -cb};   // theta-hat
        const double qv[3] = {-sl, cl, 0.0};            // phi-hat
        for (int j = 0; j < 3; j++) {
            P.pq[j] = pv[j];
            P.pq[3 + j] = qv[j];
        }
        for (int arm = 0; arm < 2; arm++) {
            const int m = arm + 1;
            const double dc = cbn[m] - cbn[0], ds = sbn[m] - sbn[0];
            for (int j = 0; j < 2; j++) {
                const double* w = j == 0 ? pv : qv;
                double* c = P.pr[arm * 2 + j];
                c[0] = g.pscale * (-3.0 * kap * (dc * w[0] + ds * w[1]));
                c[1] = g.pscale * (-0.5 * dc * w[2]);
                c[2] = g.pscale * (-0.5 * ds * w[2]);
                c[3] = g.pscale * (kap * (dc * w[0] - ds * w[1]));
                c[4] = g.pscale * (kap * (ds * w[0] + dc * w[1]));
            }
        }
    }
    __syncwarp();
    // F+ and Fx are degree-4 trig polynomials in alpha: their harmonics by a
    // 9-point discrete Fourier transform (exact for degree <= 4); lane j < 9
    // samples alpha_j = 2 pi j / 9.
    if (lane < 9) {
        double sj, cj;
        sincospi(2.0 * lane / 9.0, &sj, &cj);
        cs9[wl][lane] = cj;
        sn9[wl][lane] = sj;
        antenna_of(P, cj, sj, fs9[wl][0][lane], fs9[wl][1][lane]);
    }
    __syncwarp();
    if (lane < 10) {   // lane = 2 h + f: harmonic h of pattern f (h = 0..4)
        const int h = lane >> 1, f = lane & 1;
        double ah = 0.0, bh = 0.0;
        for (int j = 0; j < 9; j++) {
            const int a = (h * j) % 9;   // cos/sin(2 pi h j / 9) = table entry (h j mod 9)
            ah += fs9[wl][f][j] * cs9[wl][a];
            bh += fs9[wl][f][j] * sn9[wl][a];
        }
        if (h == 0) {
            P.harm[f][0] = ah / 9.0;
        } else {
            P.harm[f][2 * h - 1] = 2.0 * ah / 9.0;
            P.harm[f][2 * h] = 2.0 * bh / 9.0;
        }
    }
    __syncwarp();
    // band: first bin with t >= 0 and last bin with t <= T_obs. Lanes 0 and 1
    // solve t(f) = 0 and t(f) = T_obs for the edges' frequencies; one round of
    // the predicates over a 16-bin window around each edge (lanes 0-15 and
    // 16-31) settles the bins exactly, and a window that does not show the
    // change falls back to the search over all bins (same predicate, same
    // result).
    int64_t klo = 0, khi = g.n - 1;
    if (!global) {
        auto before = [&](int64_t k) { return time_of(P, powers_of(bin_freq(g, k))) >= 0.0; };
        auto after = [&](int64_t k) { return time_of(P, powers_of(bin_freq(g, k))) > g.T_obs; };
        double fe = 0.0;
        if (lane < 2) fe = edge_freq(P, lane == 0 ? 0.0 : g.T_obs);
        const int64_t w_lo = edge_window(g, __shfl_sync(0xffffffffu, fe, 0));
        const int64_t w_hi = edge_window(g, __shfl_sync(0xffffffffu, fe, 1));
        const int half = lane / kEdgeWin;
        const int64_t k = (half ? w_hi : w_lo) + (lane % kEdgeWin);
        const bool probe = (half ? w_hi : w_lo) >= 0 && k < g.n && (half ? after(k) : before(k));
        const unsigned m = __ballot_sync(0xffffffffu, probe);
        bool ok;
        klo = first_in_window(g.n, w_lo, m & 0xffffu, &ok);
        if (!ok) klo = warp_search_first(0, g.n, before);
        khi = first_in_window(g.n, w_hi, m >> 16, &ok);
        if (!ok) khi = warp_search_first(0, g.n, after);
        khi -= 1;
    }
    __syncwarp();
    if (lane == 0) {
        P.klo = klo;
        P.khi = khi;
        parts[b] = P;
    }
}

cudaError_t launch_setup(const Grid& g, const ::fs_params* params, int B, Particle* parts, int global,
                         cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    setup_kernel<<<(B + 3) / 4, 128, 0, s>>>(g, params, B, parts, global);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-segment antenna basis.  F_p is invariant under any invertible change of
// the amplitude basis (Eq. coherent_F_stat), so each segment uses
//   G1 = c F+ + s Fx,  G2 = c Fx - s F+,  (c, s) = F(t_mid)/|F(t_mid)|
// taken at the segment's central bin.  On a short segment F+ and Fx are nearly
// proportional and the Gram matrix of (F+, Fx) is close to singular; in the
// rotated basis G2 is small but computed directly, and the Gram matrix of
// (G1, G2) is well conditioned, so FP64 sums keep F_p accurate.
// ---------------------------------------------------------------------------
__global__ void rotation_kernel(Grid g, const Particle* __restrict__ parts, int B, Segs sg, double2* rot,
                                float2* rot32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * sg.Np) return;
    const int b = (int)(i / sg.Np);
    const int p = (int)(i % sg.Np);
    const Particle& P = parts[b];
    double2 r = make_double2(1.0, 0.0);
    if (P.valid) {
        const SegView sv = seg_view(sg, P);
        if (sv.lo <= sv.hi) {
            int64_t s0 = sv.start(p), s1 = sv.start(p + 1);
            if (s1 > s0) {
                int64_t mid = s0 + (s1 - 1 - s0) / 2;
                double f = bin_freq(g, mid);
                double t = time_of(P, powers_of(f));
                double sn, cs;
                sincos(fma(kTwoPi / kYearS, t, g.alpha0), &sn, &cs);
                double Fp, Fx;
                antenna_of(P, cs, sn, Fp, Fx);
                double nrm = sqrt(Fp * Fp + Fx * Fx);
                if (nrm > 1e-300) r = make_double2(Fp / nrm, Fx / nrm);
            }
        }
    }
    rot[i] = r;
    if (rot32) rot32[i] = make_float2((float)r.x, (float)r.y);
}

cudaError_t launch_rotation(const Grid& g, const Particle* parts, int B, const Segs& sg, double2* rot,
                            float2* rot32, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    int64_t n = (int64_t)B * sg.Np;
    rotation_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, parts, B, sg, rot, rot32);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A2-A4 (FP64): one warp per (particle, tile); lanes stride over the bins.
// Each bin: phase, t(f), response, z = dw e^{+2 pi i Phi}; accumulate, in the
// segment's rotated antenna basis (G1, G2),
//   X1 = sum G1 z, X2 = sum G2 z, K11 = sum W G1^2, K12 = sum W G1 G2, K22 = sum W G2^2
// per segment.  The first segment touched in the tile goes to H, the last to
// T, segments that start and end inside the tile go straight to S.
// NS = 8: the response series of Eq. (freDres) (eval_bin_mb), whose T+ and Tx
// are complex; the rotated responses G1 = c T+ + s Tx, G2 = c Tx - s T+ give
//   X1 = sum z conj(G1), X2 = sum z conj(G2), K11 = sum W |G1|^2,
//   K12 = sum W Re(G1 conj G2), K22 = sum W |G2|^2 and K12' = sum W Im(G1 conj G2).
// ---------------------------------------------------------------------------
// RESP: 0 the paper's form (real patterns, seven sums), 1 the response series,
// 2 the paper's form with the finite-arm TDI response (complex, eight sums).
// ECC: antenna patterns of the orbits to second order in eccentricity (g.orb).
template <int RESP, bool ECC>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 1)
fp64_main_kernel(Grid g, Tables tb, const Particle* __restrict__ parts, int B, Segs sg, Partials pa, Resp resp) {
    constexpr int NS = RESP == 0 ? 7 : 8;
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.y * kWarpsPerCta + (threadIdx.x >> 5);
    const int tile = blockIdx.x;
    if (b >= B) return;
    const Particle P = parts[b];
    if (!P.valid) return;
    const SegView sv = seg_view(sg, P);
    int64_t lo = (int64_t)tile * pa.tile, hi = lo + pa.tile;
    if (lo < sv.lo) lo = sv.lo;
    if (hi > sv.hi + 1) hi = sv.hi + 1;
    if (lo >= hi) return;
    const int64_t slot = (int64_t)b * pa.ntiles + tile;

    double acc[NS];
#pragma unroll
    for (int c = 0; c < NS; c++) acc[c] = 0.0;
    int cur = sv.seg(lo);
    int nflush = 0;

    for (int64_t base = lo; base < hi; base += 32) {
        const int64_t k = base + lane;
        const bool valid = k < hi;
        int pk = INT_MAX;
        double t7[NS];
#pragma unroll
        for (int c = 0; c < NS; c++) t7[c] = 0.0;
        if (valid) {
            pk = sv.seg(k);
            FreqPowers w;
            w.u = tb.u[k];
            w.g0h = tb.g0h[k];
            w.e19 = tb.e19[k];
            const double2 rc = pa.rot[(int64_t)b * sg.Np + pk];
            double dr = tb.dwr[k], di = tb.dwi[k], W = tb.W[k];
            if constexpr (RESP == 0) {
                BinEval ev = eval_bin_fp64_t<ECC>(P, tb.fh[k], tb.fl[k], w, tb.g0l[k], g.alpha0, g.orb);
                double sn, cs;
                sincospi(2.0 * ev.frac, &sn, &cs);
                const double G1 = fma(rc.x, ev.Fp, rc.y * ev.Fx);
                const double G2 = fma(rc.x, ev.Fx, -rc.y * ev.Fp);
                double zr = fma(dr, cs, -di * sn);
                double zi = fma(dr, sn, di * cs);
                t7[0] = G1 * zr;
                t7[1] = G1 * zi;
                t7[2] = G2 * zr;
                t7[3] = G2 * zi;
                double wg = W * G1;
                t7[4] = wg * G1;
                t7[5] = wg * G2;
                t7[6] = W * G2 * G2;
            } else {
                const BinEvalMB ev = RESP == 1
                                         ? eval_bin_mb<ECC>(P, tb.fh[k], tb.fl[k], w, tb.g0l[k], g.alpha0, resp, g.orb)
                                         : eval_bin_fin(P, tb.fh[k], tb.fl[k], w, tb.g0l[k], g.alpha0, g.orb);
                double sn, cs;
                sincospi(2.0 * ev.frac, &sn, &cs);
                const double G1r = fma(rc.x, ev.Tpr, rc.y * ev.Txr), G1i = fma(rc.x, ev.Tpi, rc.y * ev.Txi);
                const double G2r = fma(rc.x, ev.Txr, -rc.y * ev.Tpr), G2i = fma(rc.x, ev.Txi, -rc.y * ev.Tpi);
                double zr = fma(dr, cs, -di * sn);
                double zi = fma(dr, sn, di * cs);
                // z conj(G) = (zr G_r + zi G_i) + i (zi G_r - zr G_i)
                t7[0] = fma(zr, G1r, zi * G1i);
                t7[1] = fma(zi, G1r, -zr * G1i);
                t7[2] = fma(zr, G2r, zi * G2i);
                t7[3] = fma(zi, G2r, -zr * G2i);
                t7[4] = W * fma(G1r, G1r, G1i * G1i);
                t7[5] = W * fma(G1r, G2r, G1i * G2i);
                t7[6] = W * fma(G2r, G2r, G2i * G2i);
                t7[7] = W * fma(G1i, G2r, -G1r * G2i);
            }
        }
        while (true) {
            if (valid && pk == cur) {
#pragma unroll
                for (int c = 0; c < NS; c++) acc[c] += t7[c];
            }
            unsigned more = __ballot_sync(0xffffffffu, valid && pk > cur);
            if (!more) break;
            // segment `cur` ends inside this tile: flush it
            double* dst = (nflush == 0) ? pa.H + slot * NS : pa.S + ((int64_t)b * sg.Np + cur) * NS;
#pragma unroll
            for (int c = 0; c < NS; c++) {
                double v = warp_sum(acc[c]);
                if (lane == 0) dst[c] = v;
                acc[c] = 0.0;
            }
            nflush++;
            int cand = (valid && pk > cur) ? pk : INT_MAX;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
            cur = cand;
        }
    }
    double* dst = (nflush == 0) ? pa.H + slot * NS : pa.T + slot * NS;
#pragma unroll
    for (int c = 0; c < NS; c++) {
        double v = warp_sum(acc[c]);
        if (lane == 0) dst[c] = v;
    }
}

cudaError_t launch_fp64_main(const Grid& g, const Tables& t, const Particle* parts, int B, const Segs& sg,
                             const Partials& pa, cudaStream_t s, const Resp* resp) {
    if (B <= 0) return cudaSuccess;
    dim3 grid((unsigned)pa.ntiles, (unsigned)((B + kWarpsPerCta - 1) / kWarpsPerCta));
    const bool ecc = g.orb.e > 0.0, fin = g.orb.L > 0.0;
    if (fin) {
        if (pa.nsum != 8 || resp) return cudaErrorInvalidValue;
        fp64_main_kernel<2, false><<<grid, kWarpsPerCta * 32, 0, s>>>(g, t, parts, B, sg, pa, Resp{});
    } else if (resp) {
        if (pa.nsum != 8) return cudaErrorInvalidValue;
        if (ecc)
            fp64_main_kernel<1, true><<<grid, kWarpsPerCta * 32, 0, s>>>(g, t, parts, B, sg, pa, *resp);
        else
            fp64_main_kernel<1, false><<<grid, kWarpsPerCta * 32, 0, s>>>(g, t, parts, B, sg, pa, *resp);
    } else if (ecc) {
        fp64_main_kernel<0, true><<<grid, kWarpsPerCta * 32, 0, s>>>(g, t, parts, B, sg, pa, Resp{});
    } else {
        fp64_main_kernel<0, false><<<grid, kWarpsPerCta * 32, 0, s>>>(g, t, parts, B, sg, pa, Resp{});
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A5: per-(particle, segment) sums over the tiles the segment spans, then
//   F_p = [K22 |X1|^2 - 2 K12 Re(X1 conj X2) + K11 |X2|^2] / (2 (K11 K22 - K12^2))
// which is 1/2 N^T M^-1 N for M = diag(K, K), K = [[K11, K12], [K12, K22]],
// N = (Re X1, Re X2, -Im X1, -Im X2) in the basis G1 h0, G2 h0, -i G1 h0, -i G2 h0.
// The degenerate-segment rule is stated in the (F+, Fx) basis:
// det <= 1e-12 P R with P = sum W F+^2, R = sum W Fx^2 recovered from K.
// ---------------------------------------------------------------------------
// G lanes per (particle, segment): G = 1 when a segment meets only a few
// tiles (large N_p), up to a warp when it meets hundreds.  G depends only on
// (n_bins, N_p, tile), so a plan's results stay bitwise reproducible.
// NS = 8 (the response series): K = [[K11, K12 - i K12'], [K12 + i K12', K22]] is
// the Hermitian Gram matrix of the complex responses (the 4x4 M is its real
// form) and F_p = X^H K^-1 X / 2:
//   F_p = [K22 |X1|^2 + K11 |X2|^2 - 2 K12 Re(conj X1 X2) - 2 K12' Im(conj X1 X2)]
//         / (2 (K11 K22 - K12^2 - K12'^2)),
// with the same degenerate-segment rule on K11 K22 - K12^2.
template <int G, int NS>
__global__ void reduce_kernel(Grid g, const Particle* __restrict__ parts, int B, Segs sg, Partials pa,
                              double* Fpart, double* amp, const int* amp_exp) {
    const int lane = threadIdx.x & (G - 1);
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (wid >= (int64_t)B * sg.Np) return;   // uniform within a group
    const int b = (int)(wid / sg.Np);
    const int p = (int)(wid % sg.Np);
    const Particle& P = parts[b];
    if (!P.valid || (sg.global && sg.edges[sg.Np + 1] == 0)) {   // invalid particle or invalid edge frequencies
        if (lane == 0) {
            Fpart[wid] = __longlong_as_double(0x7ff8000000000000LL);
            if (amp)
                for (int i = 0; i < 4; i++) amp[wid * 4 + i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        return;
    }
    const SegView sv = seg_view(sg, P);
    double acc[NS];
#pragma unroll
    for (int c = 0; c < NS; c++) acc[c] = 0.0;
    int64_t s0 = 0, s1 = 0;
    if (sv.lo <= sv.hi) {
        s0 = sv.start(p);
        s1 = sv.start(p + 1);
    }
    const int64_t nb = s1 > s0 ? s1 - s0 : 0;
    if (nb > 0) {
        const int64_t t0 = s0 / pa.tile, t1 = (s1 - 1) / pa.tile;
        for (int64_t t = t0 + lane; t <= t1; t += G) {
            int64_t tlo = t * pa.tile, thi = tlo + pa.tile - 1;
            if (tlo < sv.lo) tlo = sv.lo;
            if (thi > sv.hi) thi = sv.hi;
            const int pf = sv.seg(tlo), pl = sv.seg(thi);
            const double* src;
            int64_t stride;
            if (p == pf) {
                src = pa.H + ((int64_t)b * pa.ntiles + t) * NS;
                stride = pa.ch_HT;
            } else if (p == pl) {
                src = pa.T + ((int64_t)b * pa.ntiles + t) * NS;
                stride = pa.ch_HT;
            } else {
                src = pa.S + ((int64_t)b * sg.Np + p) * NS;
                stride = pa.ch_S;
            }
            for (int ch = 0; ch < pa.nch; ch++)   // the channels' sums add (Sec. II.A, Eq. eq2)
#pragma unroll
                for (int c = 0; c < NS; c++) acc[c] += src[ch * stride + c];
        }
    }
    if (G > 1) {
        // groups are aligned G-lane blocks of a warp whose members all reach this point
        const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (threadIdx.x & 31 & ~(G - 1)));
#pragma unroll
        for (int c = 0; c < NS; c++)
            for (int o = G / 2; o > 0; o >>= 1) acc[c] += __shfl_xor_sync(mask, acc[c], o);
    }
    if (lane == 0) {
        double X1r = acc[0], X1i = acc[1], X2r = acc[2], X2i = acc[3];
        double K11 = acc[4], K12 = acc[5], K22 = acc[6];
        const double K12p = NS == 8 ? acc[NS - 1] : 0.0;
        double det = K11 * K22 - K12 * K12;
        const double2 rc = pa.rot[wid];
        const double cc = rc.x * rc.x, ss = rc.y * rc.y, cs2 = 2.0 * rc.x * rc.y;
        double Pp = cc * K11 - cs2 * K12 + ss * K22;   // sum W F+^2
        double Rr = ss * K11 + cs2 * K12 + cc * K22;   // sum W Fx^2
        double F = 0.0;
        const bool solvable = nb >= 4 && det > 1e-12 * Pp * Rr;
        const double detH = NS == 8 ? det - K12p * K12p : det;
        if (solvable) {
            double num = K22 * (X1r * X1r + X1i * X1i) - 2.0 * K12 * (X1r * X2r + X1i * X2i) +
                         K11 * (X2r * X2r + X2i * X2i);
            if (NS == 8) num -= 2.0 * K12p * (X1r * X2i - X1i * X2r);
            F = 0.5 * num / detH;
        }
        Fpart[wid] = F;
        if (amp) {
            // Eq. aandMN3, a = M^-1 N with M = diag(K, K) and N = (Re X1, Re X2, -Im X1, -Im X2)
            // in the rotated basis (G1 h0, G2 h0, -i G1 h0, -i G2 h0), then back to the
            // (F+ h0, Fx h0, -i F+ h0, -i Fx h0) basis: G1 = c F+ + s Fx, G2 = c Fx - s F+.
            double a4v[4] = {0.0, 0.0, 0.0, 0.0};
            if (solvable) {
                // c = K^-1 X with c1 = b1 - i b3, c2 = b2 - i b4 (K12' = 0 unless NS = 8)
                const double id = 1.0 / detH;
                const double b1 = (K22 * X1r - K12 * X2r - K12p * X2i) * id;
                const double b2 = (K11 * X2r - K12 * X1r + K12p * X1i) * id;
                const double b3 = -(K22 * X1i - K12 * X2i + K12p * X2r) * id;
                const double b4 = -(K11 * X2i - K12 * X1i - K12p * X1r) * id;
                a4v[0] = rc.x * b1 - rc.y * b2;
                a4v[1] = rc.y * b1 + rc.x * b2;
                a4v[2] = rc.x * b3 - rc.y * b4;
                a4v[3] = rc.y * b3 + rc.x * b4;
                if (amp_exp) {
                    // sums from tables scaled by (2^-e/2, 2^-e) for (dw, W): a scales by 2^(e/2)
                    int ex = *amp_exp;
                    ex += ex & 1;
                    const double sc = ldexp(1.0, -ex / 2);
                    for (int i = 0; i < 4; i++) a4v[i] *= sc;
                }
            }
            for (int i = 0; i < 4; i++) amp[wid * 4 + i] = a4v[i];
        }
    }
}

// App. B, Eqs. B2-B3: (D_L, iota, psi, phi_c) from the amplitudes a of one
// segment, the printed arctan of a ratio read as atan2(numerator, denominator).
// A+^2 - Ax^2 is evaluated as 4 r1 r2 (the same quantity, without cancellation).
// All-zero amplitudes (a degenerate segment) give NaN.
__global__ void extrinsic_kernel(int64_t n, const double* __restrict__ amp, double* ext) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a1 = amp[i * 4], a2 = amp[i * 4 + 1], a3 = amp[i * 4 + 2], a4 = amp[i * 4 + 3];
    const double r1 = sqrt((a1 + a4) * (a1 + a4) + (a2 - a3) * (a2 - a3));
    const double r2 = sqrt((a1 - a4) * (a1 - a4) + (a2 + a3) * (a2 + a3));
    const double Ap = r1 + r2, Ax = r1 - r2;
    const double root = 2.0 * sqrt(r1 * r2);
    const double A = Ap + root;
    double out[4];
    if (!(A > 0.0)) {
        for (int j = 0; j < 4; j++) out[j] = __longlong_as_double(0x7ff8000000000000LL);
    } else {
        out[0] = 2.0 / A;                                            // D_L
        out[1] = acos(fmin(1.0, fmax(-1.0, -Ax / A)));                 // iota
        const double num = Ap * a4 - Ax * a1;
        const double psi = 0.5 * atan2(num, -(Ax * a2 + Ap * a3));
        out[2] = psi;
        const double s2 = sin(2.0 * psi);
        const double c = s2 > 0.0 ? 1.0 : (s2 < 0.0 ? -1.0 : 0.0);
        out[3] = atan2(c * num, -c * (Ax * a3 + Ap * a2));           // phi_c
    }
    for (int j = 0; j < 4; j++) ext[i * 4 + j] = out[j];
}

__global__ void sum_segments_kernel(const Particle* __restrict__ parts, int B, int Np, const double* Fpart,
                                    double* F) {
    const int lane = threadIdx.x & 31;
    const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= B) return;
    double s = 0.0;
    for (int p = lane; p < Np; p += 32) s += Fpart[b * Np + p];
    s = warp_sum(s);
    if (lane == 0) F[b] = parts[b].valid ? s : __longlong_as_double(0x7ff8000000000000LL);
}

cudaError_t launch_reduce(const Grid& g, const Particle* parts, int B, const Segs& sg, const Partials& pa,
                          double* Fpart, double* F, cudaStream_t s, double* amp, const int* amp_exp) {
    if (B <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t segs = (int64_t)B * sg.Np;
    // about two tiles per lane for a segment spanning the whole grid
    const int64_t tiles = (g.n + (int64_t)sg.Np * pa.tile - 1) / ((int64_t)sg.Np * pa.tile);
    int G = 1;
    while (G < 32 && 2 * G < tiles) G *= 2;
    const int64_t blocks = (segs * G + threads - 1) / threads;
#define FS_REDUCE(G_)                                                                                   \
    do {                                                                                                \
        if (pa.nsum == 8)                                                                               \
            reduce_kernel<G_, 8><<<(unsigned)blocks, threads, 0, s>>>(g, parts, B, sg, pa, Fpart, amp, amp_exp); \
        else                                                                                            \
            reduce_kernel<G_, 7><<<(unsigned)blocks, threads, 0, s>>>(g, parts, B, sg, pa, Fpart, amp, amp_exp); \
    } while (0)
    switch (G) {
        case 1: FS_REDUCE(1); break;
        case 2: FS_REDUCE(2); break;
        case 4: FS_REDUCE(4); break;
        case 8: FS_REDUCE(8); break;
        case 16: FS_REDUCE(16); break;
        default: FS_REDUCE(32); break;
    }
#undef FS_REDUCE
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int64_t blocks2 = ((int64_t)B * 32 + threads - 1) / threads;
    sum_segments_kernel<<<(unsigned)blocks2, threads, 0, s>>>(parts, B, sg.Np, Fpart, F);
    return cudaGetLastError();
}

cudaError_t launch_extrinsic(int64_t n, const double* amp, double* ext, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    extrinsic_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n, amp, ext);
    return cudaGetLastError();
}

__global__ void bands_kernel(const Particle* __restrict__ parts, int B, int64_t* bands) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    bands[2 * b] = parts[b].klo;
    bands[2 * b + 1] = parts[b].khi;
}

cudaError_t launch_bands(const Particle* parts, int B, int64_t* bands, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    bands_kernel<<<(B + 127) / 128, 128, 0, s>>>(parts, B, bands);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Signal synthesis: data += sum_i a_i A^i over the particle's band (FP64).
// ---------------------------------------------------------------------------
// With the response series (MB): h = (a1 - i a3) T+ h0 + (a2 - i a4) Tx h0.
// RESP as for fp64_main_kernel.
template <int RESP, bool ECC>
__global__ void add_signal_kernel(Grid g, Tables tb, const Particle* __restrict__ part, const double* a,
                                  double* data, Resp resp) {
    const Particle P = *part;
    if (!P.valid) return;
    int64_t k = P.klo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k > P.khi) return;
    FreqPowers w;
    w.u = tb.u[k];
    w.g0h = tb.g0h[k];
    w.e19 = tb.e19[k];
    double amp = pow(tb.fh[k], -7.0 / 6.0);
    double sn, cs;
    if constexpr (RESP != 0) {
        const BinEvalMB ev = RESP == 1 ? eval_bin_mb<ECC>(P, tb.fh[k], tb.fl[k], w, tb.g0l[k], g.alpha0, resp, g.orb)
                                       : eval_bin_fin(P, tb.fh[k], tb.fl[k], w, tb.g0l[k], g.alpha0, g.orb);
        sincospi(2.0 * ev.frac, &sn, &cs);
        // coefficient of h0: (a1 - i a3)(Tpr + i Tpi) + (a2 - i a4)(Txr + i Txi) = cr + i ci
        const double cr = a[0] * ev.Tpr + a[2] * ev.Tpi + a[1] * ev.Txr + a[3] * ev.Txi;
        const double ci = a[0] * ev.Tpi - a[2] * ev.Tpr + a[1] * ev.Txi - a[3] * ev.Txr;
        // (cr + i ci) (cos - i sin) * amp
        data[2 * k] += amp * (cr * cs + ci * sn);
        data[2 * k + 1] += amp * (ci * cs - cr * sn);
    } else {
        BinEval ev = eval_bin_fp64_t<ECC>(P, tb.fh[k], tb.fl[k], w, tb.g0l[k], g.alpha0, g.orb);
        sincospi(2.0 * ev.frac, &sn, &cs);
        double c = a[0] * ev.Fp + a[1] * ev.Fx;   // coefficient of h0
        double s = a[2] * ev.Fp + a[3] * ev.Fx;   // coefficient of -i h0
        // (c - i s) (cos - i sin) * amp
        data[2 * k] += amp * (c * cs - s * sn);
        data[2 * k + 1] += amp * (-c * sn - s * cs);
    }
}

cudaError_t launch_add_signal(const Grid& g, const Tables& t, const Particle* part, const double* a,
                              double* data, cudaStream_t s, const Resp* resp) {
    int threads = 256;
    int64_t blocks = (g.n + threads - 1) / threads;
    const bool ecc = g.orb.e > 0.0;
    if (g.orb.L > 0.0)
        add_signal_kernel<2, false><<<(unsigned)blocks, threads, 0, s>>>(g, t, part, a, data, Resp{});
    else if (resp && ecc)
        add_signal_kernel<1, true><<<(unsigned)blocks, threads, 0, s>>>(g, t, part, a, data, *resp);
    else if (resp)
        add_signal_kernel<1, false><<<(unsigned)blocks, threads, 0, s>>>(g, t, part, a, data, *resp);
    else if (ecc)
        add_signal_kernel<0, true><<<(unsigned)blocks, threads, 0, s>>>(g, t, part, a, data, Resp{});
    else
        add_signal_kernel<0, false><<<(unsigned)blocks, threads, 0, s>>>(g, t, part, a, data, Resp{});
    return cudaGetLastError();
}

}  // namespace fs
