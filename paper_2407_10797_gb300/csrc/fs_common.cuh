// fs_common.cuh - device-side model of the semi-coherent F-statistic path.
//
// Template (Appendix A of arXiv:2407.10797, Eqs. A1-A3) in cycles,
//   Phi(f) = f t_c + Phi_PN(f) + Phi_e(f) - f d(t_f),
//   Phi_PN = sum_{k=0,2,3,4} P_k f^{(k-5)/3},   P_k = (3/(256 pi)) (pi Mc)^{-5/3} alpha_k (pi M)^{k/3},
//   Phi_e  = E0 f^{-5/3} (f0/f)^{19/9},          E0  = -(2355/1462) e0^2 P_0,
// stationary-phase time (Sec. IV) t_f = dPhi_orb/df = t_c + sum_k T_k f^{(k-8)/3} + TE f^{-8/3} (f0/f)^{19/9},
// Doppler delay d(t) = R sin(theta) cos(alpha(t) - phi), alpha = 2 pi t / yr + alpha0,
// antenna patterns of the long-wavelength Michelson X of a rigid equilateral
// constellation as trig polynomials in alpha (degree 2 per arm projection).
//
// The constant phase -phi_c - pi/4 of Eq. (A3) and phi_p are carried by the
// amplitudes a_i of Eq. (response), whose basis is A1 = F+ h0, A2 = Fx h0,
// A3 = -i F+ h0, A4 = -i Fx h0 with h0 = f^{-7/6} exp(-2 pi i Phi).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fs {

// ---- constants (the library's own copy) ----------------------------------
constexpr double kMsunS = 4.925490947e-6;     // G Msun / c^3, s
constexpr double kYearS = 31557600.0;         // Julian year, s
constexpr double kAuS = 499.004784;           // AU / c, s
constexpr double kF0Ecc = 0.01;               // Hz, reference frequency of e0
constexpr double kPi = 3.141592653589793;
constexpr double kPiLo = 1.2246467991473532e-16;      // pi - kPi
constexpr double kInvPi = 0.3183098861837907;
constexpr double kInvPiLo = -1.9678676675182486e-17;  // 1/pi - kInvPi
constexpr double kTwoPi = 6.283185307179586;

// ---- error-free transformations and double-double arithmetic -------------
__host__ __device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    p = a * b;
    e = fma(a, b, -p);
}
__host__ __device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__host__ __device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
    s = a + b;
    e = b - (s - a);
}
// (ah + al) * (bh + bl) to ~2^-104 relative
__host__ __device__ __forceinline__ void dd_mul(double ah, double al, double bh, double bl, double& rh,
                                                double& rl) {
    double p, e;
    two_prod(ah, bh, p, e);
    e = fma(ah, bl, e);
    e = fma(al, bh, e);
    fast_two_sum(p, e, rh, rl);
}

// ---- per-particle coefficients --------------------------------------------
struct Particle {
    double P0h, P0l;          // leading phase coefficient (double-double), cycles * Hz^(5/3)
    double P2, P3, P4;        // phase: f^-1, f^-2/3, f^-1/3
    double E0;                // eccentric phase: f^-5/3 (f0/f)^(19/9)
    double T0, T2, T3, T4, TE;  // time: f^-8/3, f^-2, f^-5/3, f^-4/3, f^-8/3 (f0/f)^(19/9)
    double tc;
    double AD;                // R sin(theta) = AU cos(beta), s
    double clon, slon;
    double pr[4][5];          // a.p, a.q, b.p, b.q: c0 + c1 cos a + s1 sin a + c2 cos 2a + s2 sin 2a
    double harm[2][9];        // F+ and Fx as A0 + sum_{h=1..4} (A_h cos h a + B_h sin h a): A0, A1, B1, ..., A4, B4
    int64_t klo, khi;         // band: first/last bin with t(f_k) in [0, T_obs] (klo > khi: empty)
    int valid;                // 0: non-finite or unphysical parameters
    int pad;
};

// Powers of the bin frequency that the phase and t(f) need.
struct FreqPowers {
    double u;     // f^-1/3
    double g0h;   // f^-5/3 (head)
    double e19;   // (f0/f)^(19/9)
};

// Stationary-phase time t(f) (FP64).
__device__ __forceinline__ double time_of(const Particle& P, const FreqPowers& w) {
    double u2 = w.u * w.u;
    double u3 = u2 * w.u;
    double u4 = u2 * u2;
    double u6 = u3 * u3;
    double g83 = w.g0h * u3;  // f^-8/3
    double s = P.T0 * g83;
    s = fma(P.T2, u6, s);
    s = fma(P.T3, w.g0h, s);
    s = fma(P.T4, u4, s);
    s = fma(P.TE * g83, w.e19, s);
    return P.tc + s;
}

// Antenna patterns from cos/sin of the orbital phase alpha.
__device__ __forceinline__ void antenna_of(const Particle& P, double c1, double s1, double& Fp, double& Fx) {
    double c2 = fma(c1, c1, -s1 * s1);
    double s2 = 2.0 * s1 * c1;
    double pj[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        double v = P.pr[i][0];
        v = fma(P.pr[i][1], c1, v);
        v = fma(P.pr[i][2], s1, v);
        v = fma(P.pr[i][3], c2, v);
        v = fma(P.pr[i][4], s2, v);
        pj[i] = v;
    }
    // F+ = (a.p^2 - a.q^2 - b.p^2 + b.q^2)/2, Fx = a.p a.q - b.p b.q
    Fp = 0.5 * ((pj[0] * pj[0] - pj[1] * pj[1]) - (pj[2] * pj[2] - pj[3] * pj[3]));
    Fx = pj[0] * pj[1] - pj[2] * pj[3];
}

// Fractional part of the total phase in cycles (in [-1/2, 1/2]) at a bin with
// double-double frequency (fh, fl), plus the response there.
struct BinEval {
    double frac;   // Phi mod 1
    double Fp, Fx;
};

__device__ __forceinline__ BinEval eval_bin_fp64(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                 double g0l, double alpha0) {
    BinEval r;
    // leading PN term P0 * f^-5/3 in double-double, reduced mod 1 exactly
    double p, e;
    two_prod(P.P0h, w.g0h, p, e);
    e = fma(P.P0h, g0l, e);
    e = fma(P.P0l, w.g0h, e);
    double acc = (p - rint(p)) + e;
    // f t_c = (fh + fl) t_c, reduced mod 1
    double q, eq;
    two_prod(fh, P.tc, q, eq);
    eq = fma(fl, P.tc, eq);
    acc += (q - rint(q)) + eq;
    // remaining PN terms and the eccentric correction
    double u2 = w.u * w.u;
    double u3 = u2 * w.u;
    double rest = P.P2 * u3;
    rest = fma(P.P3, u2, rest);
    rest = fma(P.P4, w.u, rest);
    rest = fma(P.E0 * w.g0h, w.e19, rest);
    // response along t(f)
    double t = time_of(P, w);
    double alpha = fma(kTwoPi / kYearS, t, alpha0);
    double s1, c1;
    sincos(alpha, &s1, &c1);
    double cd = fma(c1, P.clon, s1 * P.slon);   // cos(alpha - phi)
    rest = fma(-fh * P.AD, cd, rest);            // - f d(t_f)
    acc += rest - rint(rest);
    r.frac = acc - rint(acc);
    antenna_of(P, c1, s1, r.Fp, r.Fx);
    return r;
}

// Segment index of bin k for a particle with per-particle segments.
__device__ __forceinline__ int seg_of_bin(int64_t k, int64_t klo, int64_t khi, int Np) {
    int64_t w = khi - klo;
    if (w <= 0) return 0;
    int64_t p = ((int64_t)Np * (k - klo)) / w;
    return p >= Np ? Np - 1 : (int)p;
}

}  // namespace fs
