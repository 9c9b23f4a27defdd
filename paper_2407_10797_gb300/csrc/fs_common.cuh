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
    double pq[6];             // polarisation basis of the source: p = theta-hat (0..2), q = phi-hat (3..5)
};

// Spacecraft orbits to second order in eccentricity (Sec. IV): e > 0 selects
// them (direct kernels only), e = 0 the rigid constellation of antenna_of.
struct Orbit {
    double e;                          // eccentricity
    int chan;                          // TDI channel the patterns are formed for: 0 X, 1 A, 2 E
    double cb[3], sb[3], c2b[3], s2b[3];   // cos, sin of beta_k and 2 beta_k, beta_k = 2 pi k/3 + orientation
    double L;                          // > 0: finite-arm TDI response with this nominal arm (s); 0: long wavelength
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

// Antenna patterns of the channel O.chan for the orbits of Orbit (and, with
// DERIV, their derivatives with respect to alpha) from cos/sin of alpha.
// Spacecraft k sits at the guiding centre plus e R times
//   (cos(2a - b)/2 - 3/2 cos b + e (-5/8 cos(a - 2b) + 3/8 cos(3a - 2b)),
//    sin(2a - b)/2 - 3/2 sin b + e (5/8 sin(a - 2b) + 3/8 sin(3a - 2b)),
//    -sqrt3 cos(a - b) - e sqrt3/2 cos(2a - 2b)),   b = beta_k
// (the terms common to the three spacecraft, which cancel in the arms,
// left out).  Arms n1 = r1 - r0, n2 = r2 - r1, n3 = r0 - r2, normalised;
// A_i = ((n_i.p)^2 - (n_i.q)^2)/2, B_i = (n_i.p)(n_i.q); the vertex
// Michelsons are X = (1, 3), Y = (2, 1), Z = (3, 2) (first arm minus second)
// and A = (Z - X)/sqrt2, E = (X - 2Y + Z)/sqrt6.
template <bool DERIV>
__device__ __forceinline__ void antenna_ecc(const Orbit& O, const Particle& P, double c1, double s1, double& Fp,
                                            double& Fx, double& dFp, double& dFx) {
    const double c2 = fma(c1, c1, -s1 * s1), s2 = 2.0 * s1 * c1;
    const double c3 = fma(c2, c1, -s2 * s1), s3 = fma(s2, c1, c2 * s1);
    const double e = O.e, r3 = 1.7320508075688772;
    double r[3][3], dr[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double cb = O.cb[k], sb = O.sb[k], c2b = O.c2b[k], s2b = O.s2b[k];
        const double c2ab = fma(c2, cb, s2 * sb), s2ab = fma(s2, cb, -c2 * sb);      // 2a - b
        const double cab = fma(c1, cb, s1 * sb), sab = fma(s1, cb, -c1 * sb);        // a - b
        const double ca2b = fma(c1, c2b, s1 * s2b), sa2b = fma(s1, c2b, -c1 * s2b);  // a - 2b
        const double c32 = fma(c3, c2b, s3 * s2b), s32 = fma(s3, c2b, -c3 * s2b);    // 3a - 2b
        const double c22 = fma(c2, c2b, s2 * s2b), s22 = fma(s2, c2b, -c2 * s2b);    // 2a - 2b
        r[k][0] = fma(0.5, c2ab, -1.5 * cb) + e * fma(-0.625, ca2b, 0.375 * c32);
        r[k][1] = fma(0.5, s2ab, -1.5 * sb) + e * fma(0.625, sa2b, 0.375 * s32);
        r[k][2] = -r3 * fma(0.5 * e, c22, cab);
        if (DERIV) {
            dr[k][0] = -s2ab + e * fma(0.625, sa2b, -1.125 * s32);
            dr[k][1] = c2ab + e * fma(0.625, ca2b, 1.125 * c32);
            dr[k][2] = r3 * fma(e, s22, sab);
        }
    }
    const double* p = P.pq;
    const double* q = P.pq + 3;
    double A[3], Bq[3], dA[3], dB[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int k0 = i, k1 = i == 2 ? 0 : i + 1;   // n_{i+1} = r_{k1} - r_{k0}
        double n[3], dn[3], nn = 0.0, nd = 0.0;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            n[j] = r[k1][j] - r[k0][j];
            nn = fma(n[j], n[j], nn);
            if (DERIV) {
                dn[j] = dr[k1][j] - dr[k0][j];
                nd = fma(n[j], dn[j], nd);
            }
        }
        const double inv = 1.0 / sqrt(nn);
        const double Pp = (n[0] * p[0] + n[1] * p[1] + n[2] * p[2]) * inv;
        const double Qq = (n[0] * q[0] + n[1] * q[1] + n[2] * q[2]) * inv;
        A[i] = 0.5 * (Pp * Pp - Qq * Qq);
        Bq[i] = Pp * Qq;
        if (DERIV) {
            // d(n/|n|) = (dn - (n/|n|) ((n/|n|).dn)) / |n|
            const double u = nd * inv * inv;
            const double dP = ((dn[0] * p[0] + dn[1] * p[1] + dn[2] * p[2]) * inv - Pp * u);
            const double dQ = ((dn[0] * q[0] + dn[1] * q[1] + dn[2] * q[2]) * inv - Qq * u);
            dA[i] = Pp * dP - Qq * dQ;
            dB[i] = dP * Qq + Pp * dQ;
        }
    }
    if (O.chan == 0) {
        Fp = A[0] - A[2];
        Fx = Bq[0] - Bq[2];
        if (DERIV) {
            dFp = dA[0] - dA[2];
            dFx = dB[0] - dB[2];
        }
    } else if (O.chan == 1) {
        const double k = 0.7071067811865476;   // 1/sqrt2
        Fp = k * (2.0 * A[2] - A[0] - A[1]);
        Fx = k * (2.0 * Bq[2] - Bq[0] - Bq[1]);
        if (DERIV) {
            dFp = k * (2.0 * dA[2] - dA[0] - dA[1]);
            dFx = k * (2.0 * dB[2] - dB[0] - dB[1]);
        }
    } else {
        const double k = 1.224744871391589;    // sqrt(3/2)
        Fp = k * (A[0] - A[1]);
        Fx = k * (Bq[0] - Bq[1]);
        if (DERIV) {
            dFp = k * (dA[0] - dA[1]);
            dFx = k * (dB[0] - dB[1]);
        }
    }
}

// Finite-arm response of the first-generation TDI Michelsons (Sec. IV: a TDI
// combination is a sum of time-delayed single-arm responses), constellation
// frozen at orbital phase alpha (cos/sin c1, s1), frequency f, for + and x.
// Spacecraft k at the guiding centre plus L/(2 sqrt3) times the orbit offsets
// (first order, plus e times the second order including its terms common to
// the three spacecraft, which shift the phase reference).  For the arm
// (i, j), u = (x_j - x_i)/L_ij, the link i -> j (n = u) and j -> i (n = -u):
//   y = (n.e_A.n) (-i pi f L_ij) sinc(pi f L_ij (1 - k.n)) exp(-i pi f (L_ij + k.(x_i + x_j))),
// k = -(source direction) = -(p x q).  Vertex v, arms to a = v+1, b = v+2:
//   R_v = [exp(-2 pi i f L_va) y_va + y_av - exp(-2 pi i f L_vb) y_vb - y_bv] / (-4 pi i f L);
// channels X = R_0, A = (R_2 - R_0)/sqrt2, E = (R_0 - 2 R_1 + R_2)/sqrt6.
__device__ __forceinline__ double sinc_d(double x) {
    const double x2 = x * x;
    return fabs(x) < 1e-4 ? fma(x2, fma(x2, 1.0 / 120.0, -1.0 / 6.0), 1.0) : sin(x) / x;
}

__device__ __forceinline__ void tdi_response(const Orbit& O, const Particle& P, double c1, double s1, double f,
                                             double T[4]) {
    const double c2 = fma(c1, c1, -s1 * s1), s2 = 2.0 * s1 * c1;
    const double c3 = fma(c2, c1, -s2 * s1), s3 = fma(s2, c1, c2 * s1);
    const double e = O.e, r3 = 1.7320508075688772, sc = O.L / (2.0 * r3);
    double x[3][3];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const double cb = O.cb[k], sb = O.sb[k], c2b = O.c2b[k], s2b = O.s2b[k];
        const double c2ab = fma(c2, cb, s2 * sb), s2ab = fma(s2, cb, -c2 * sb);
        const double cab = fma(c1, cb, s1 * sb);
        const double ca2b = fma(c1, c2b, s1 * s2b), sa2b = fma(s1, c2b, -c1 * s2b);
        const double c32 = fma(c3, c2b, s3 * s2b), s32 = fma(s3, c2b, -c3 * s2b);
        const double c22 = fma(c2, c2b, s2 * s2b);
        x[k][0] = sc * (fma(0.5, c2ab, -1.5 * cb) + e * (fma(-0.625, ca2b, 0.375 * c32) - 1.25 * c1));
        x[k][1] = sc * (fma(0.5, s2ab, -1.5 * sb) + e * (fma(0.625, sa2b, 0.375 * s32) - 1.25 * s1));
        x[k][2] = sc * (-r3 * cab + e * (0.5 * r3) * (3.0 - c22));
    }
    const double* p = P.pq;
    const double* q = P.pq + 3;
    const double kv[3] = {-(p[1] * q[2] - p[2] * q[1]), -(p[2] * q[0] - p[0] * q[2]), -(p[0] * q[1] - p[1] * q[0])};
    // per arm i = (i, i+1): projections, forward and backward link factors (without n.e.n), delay
    double qp[3], qx[3], yfr[3], yfi[3], ybr[3], ybi[3], dr[3], di[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int j = i == 2 ? 0 : i + 1;
        double u[3], L2 = 0.0;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            u[c] = x[j][c] - x[i][c];
            L2 = fma(u[c], u[c], L2);
        }
        const double Lij = sqrt(L2), inv = 1.0 / Lij;
        const double up = (u[0] * p[0] + u[1] * p[1] + u[2] * p[2]) * inv;
        const double uq = (u[0] * q[0] + u[1] * q[1] + u[2] * q[2]) * inv;
        const double ku = (u[0] * kv[0] + u[1] * kv[1] + u[2] * kv[2]) * inv;
        const double ks = kv[0] * (x[i][0] + x[j][0]) + kv[1] * (x[i][1] + x[j][1]) + kv[2] * (x[i][2] + x[j][2]);
        qp[i] = fma(up, up, -uq * uq);
        qx[i] = 2.0 * up * uq;
        const double pfl = kPi * f * Lij;
        double sp, cp;
        sincos(kPi * f * (Lij + ks), &sp, &cp);
        // (-i pfl) sinc * (cp - i sp) = pfl sinc (-sp - i cp)
        const double af = pfl * sinc_d(pfl * (1.0 - ku)), ab = pfl * sinc_d(pfl * (1.0 + ku));
        yfr[i] = -af * sp;
        yfi[i] = -af * cp;
        ybr[i] = -ab * sp;
        ybi[i] = -ab * cp;
        double sd, cd;
        sincos(2.0 * kPi * f * Lij, &sd, &cd);
        dr[i] = cd;
        di[i] = -sd;
    }
    // R_v per polarisation, divided by -4 pi i f L: 1/(-i c) = i/c
    double Rr[3][2], Ri[3][2];
    const double cn = 4.0 * kPi * f * O.L;
#pragma unroll
    for (int v = 0; v < 3; v++) {
        const int a = v == 2 ? 0 : v + 1, b = v == 0 ? 2 : v - 1;
        // links v -> a: arm v forward; a -> v: arm v backward; v -> b: arm b backward; b -> v: arm b forward
        const double mra = fma(dr[v], yfr[v], -di[v] * yfi[v]) + ybr[v];
        const double mia = fma(dr[v], yfi[v], di[v] * yfr[v]) + ybi[v];
        const double mrb = fma(dr[b], ybr[b], -di[b] * ybi[b]) + yfr[b];
        const double mib = fma(dr[b], ybi[b], di[b] * ybr[b]) + yfi[b];
#pragma unroll
        for (int A = 0; A < 2; A++) {
            const double wa = A == 0 ? qp[v] : qx[v], wb = A == 0 ? qp[b] : qx[b];
            const double Mr = wa * mra - wb * mrb, Mi = wa * mia - wb * mib;
            // (Mr + i Mi) * i / cn
            Rr[v][A] = -Mi / cn;
            Ri[v][A] = Mr / cn;
        }
    }
#pragma unroll
    for (int A = 0; A < 2; A++) {
        double tr, ti;
        if (O.chan == 0) {
            tr = Rr[0][A];
            ti = Ri[0][A];
        } else if (O.chan == 1) {
            tr = (Rr[2][A] - Rr[0][A]) * 0.7071067811865476;
            ti = (Ri[2][A] - Ri[0][A]) * 0.7071067811865476;
        } else {
            tr = (Rr[0][A] - 2.0 * Rr[1][A] + Rr[2][A]) * 0.4082482904638631;
            ti = (Ri[0][A] - 2.0 * Ri[1][A] + Ri[2][A]) * 0.4082482904638631;
        }
        T[2 * A] = tr;
        T[2 * A + 1] = ti;
    }
}

// Fractional part of the total phase in cycles (in [-1/2, 1/2]) at a bin with
// double-double frequency (fh, fl), plus the response there (antenna patterns
// of the rigid constellation, or with ECC those of the orbits of O).
struct BinEval {
    double frac;   // Phi mod 1
    double Fp, Fx;
};

template <bool ECC>
__device__ __forceinline__ BinEval eval_bin_fp64_t(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                   double g0l, double alpha0, const Orbit& O);

__device__ __forceinline__ BinEval eval_bin_fp64(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                 double g0l, double alpha0) {
    return eval_bin_fp64_t<false>(P, fh, fl, w, g0l, alpha0, Orbit{});
}

// The template phase mod 1 (orbital phase minus f d(t_f)) and cos/sin of the
// orbital phase alpha(t_f) at a bin.
__device__ __forceinline__ double phase_and_alpha(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                  double g0l, double alpha0, double& c1, double& s1) {
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
    sincos(alpha, &s1, &c1);
    double cd = fma(c1, P.clon, s1 * P.slon);   // cos(alpha - phi)
    rest = fma(-fh * P.AD, cd, rest);            // - f d(t_f)
    acc += rest - rint(rest);
    return acc - rint(acc);
}

template <bool ECC>
__device__ __forceinline__ BinEval eval_bin_fp64_t(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                   double g0l, double alpha0, const Orbit& O) {
    BinEval r;
    double c1, s1;
    r.frac = phase_and_alpha(P, fh, fl, w, g0l, alpha0, c1, s1);
    if (ECC) {
        double dp, dx;
        antenna_ecc<false>(O, P, c1, s1, r.Fp, r.Fx, dp, dx);
    } else {
        antenna_of(P, c1, s1, r.Fp, r.Fx);
    }
    return r;
}

// ---- the response series of Sec. IV, Eq. (freDres) -------------------------
//   T(f) = sum_{k=0}^{K} (-i T_A1)^k / k!  F^N_{T_f}[d^k G / dtau^k](t_f),
//   G(tau) = F(tau - d(tau)) / (1 + ddot(tau)) exp(2 pi i f d(tau) (1 - ddot(tau))),
//   F^N_{T_f}[G](t) = 1/2 sum_{j=0}^{N} a_j (G(t + j T_f) + G(t - j T_f)),
//   T_A1 = (7/6) / (2 pi f),  T_f^2 = |d^2 Psi/df^2| / (4 pi) = |dt_f/df| / 2.
// The weights a_j make the filter reproduce the even moments (2m-1)!! (i T_f^2/pi)^m
// (m <= N) of the stationary-phase kernel exp(i pi fdot s^2) around t_f; they are
// filled in by the host (fs_plan_set_response).  The phase factor of G at t_f,
// exp(2 pi i f D0) with D0 = d(t_f)(1 - ddot(t_f)), is carried by the template phase.
struct Resp {
    int N;               // filter order, 0..2
    int K;               // highest k, 0 or 1
    double ar[3], ai[3]; // a_0..a_N
};

// dt_f/df: the derivative of each power-law term of time_of.
__device__ __forceinline__ double dtime_df(const Particle& P, const FreqPowers& w, double f) {
    double u2 = w.u * w.u;
    double u3 = u2 * w.u;
    double u4 = u2 * u2;
    double u6 = u3 * u3;
    double g83 = w.g0h * u3;   // f^-8/3
    double s = (-8.0 / 3.0) * P.T0 * g83;
    s = fma(-2.0 * P.T2, u6, s);
    s = fma((-5.0 / 3.0) * P.T3, w.g0h, s);
    s = fma((-4.0 / 3.0) * P.T4, u4, s);
    s = fma((-43.0 / 9.0) * P.TE * g83, w.e19, s);
    return s / f;
}

// Antenna patterns (as antenna_of) and their derivatives with respect to alpha.
__device__ __forceinline__ void antenna_deriv(const Particle& P, double c1, double s1, double& Fp, double& Fx,
                                              double& dFp, double& dFx) {
    double c2 = fma(c1, c1, -s1 * s1);
    double s2 = 2.0 * s1 * c1;
    double pj[4], qj[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        double v = P.pr[i][0];
        v = fma(P.pr[i][1], c1, v);
        v = fma(P.pr[i][2], s1, v);
        v = fma(P.pr[i][3], c2, v);
        v = fma(P.pr[i][4], s2, v);
        pj[i] = v;
        double dv = -P.pr[i][1] * s1;
        dv = fma(P.pr[i][2], c1, dv);
        dv = fma(-2.0 * P.pr[i][3], s2, dv);
        dv = fma(2.0 * P.pr[i][4], c2, dv);
        qj[i] = dv;
    }
    Fp = 0.5 * ((pj[0] * pj[0] - pj[1] * pj[1]) - (pj[2] * pj[2] - pj[3] * pj[3]));
    Fx = pj[0] * pj[1] - pj[2] * pj[3];
    dFp = (pj[0] * qj[0] - pj[1] * qj[1]) - (pj[2] * qj[2] - pj[3] * qj[3]);
    dFx = (qj[0] * pj[1] + pj[0] * qj[1]) - (qj[2] * pj[3] + pj[2] * qj[3]);
}

// Phase (mod 1, with the phase factor of G at t_f) and the complex responses
// T+ and Tx of one bin under the series above.
struct BinEvalMB {
    double frac;
    double Tpr, Tpi, Txr, Txi;
};

// The paper's form of the response (N = 0, no higher d(t) terms) with the
// finite-arm TDI response of tdi_response in place of the long-wavelength
// pattern: the same phase as eval_bin_fp64, complex T+ and Tx.
__device__ __forceinline__ BinEvalMB eval_bin_fin(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                  double g0l, double alpha0, const Orbit& O) {
    BinEvalMB r;
    double c1, s1;
    r.frac = phase_and_alpha(P, fh, fl, w, g0l, alpha0, c1, s1);
    double T[4];
    tdi_response(O, P, c1, s1, fh, T);
    r.Tpr = T[0];
    r.Tpi = T[1];
    r.Txr = T[2];
    r.Txi = T[3];
    return r;
}

template <bool ECC>
__device__ __forceinline__ BinEvalMB eval_bin_mb(const Particle& P, double fh, double fl, const FreqPowers& w,
                                                 double g0l, double alpha0, const Resp& R, const Orbit& O) {
    BinEvalMB r;
    // orbital phase as in eval_bin_fp64
    double p, e;
    two_prod(P.P0h, w.g0h, p, e);
    e = fma(P.P0h, g0l, e);
    e = fma(P.P0l, w.g0h, e);
    double acc = (p - rint(p)) + e;
    double q, eq;
    two_prod(fh, P.tc, q, eq);
    eq = fma(fl, P.tc, eq);
    acc += (q - rint(q)) + eq;
    double u2 = w.u * w.u;
    double u3 = u2 * w.u;
    double rest = P.P2 * u3;
    rest = fma(P.P3, u2, rest);
    rest = fma(P.P4, w.u, rest);
    rest = fma(P.E0 * w.g0h, w.e19, rest);
    const double Om = kTwoPi / kYearS;
    const double t = time_of(P, w);
    double s1, c1;
    sincos(fma(Om, t, alpha0), &s1, &c1);
    const double cd = fma(c1, P.clon, s1 * P.slon);    // cos(alpha - phi)
    const double sd = fma(s1, P.clon, -c1 * P.slon);   // sin(alpha - phi)
    const double d0 = P.AD * cd, dd0 = -P.AD * Om * sd;
    rest = fma(-fh * P.AD, cd, rest);   // - f d(t_f)
    rest = fma(fh * d0, dd0, rest);     // + f d(t_f) ddot(t_f)
    acc += rest - rint(rest);
    r.frac = acc - rint(acc);
    const double D0 = d0 * (1.0 - dd0);
    // the stencil t_f + j T_f: alpha advances by j Om T_f
    const double Tf = sqrt(0.5 * fabs(dtime_df(P, w, fh)));
    double sdl, cdl;
    sincos(Om * Tf, &sdl, &cdl);
    const double c2dl = fma(-2.0 * sdl, sdl, 1.0), s2dl = 2.0 * sdl * cdl;
    const double TA1 = 7.0 / (12.0 * kPi * fh);
    double gr[2] = {0.0, 0.0}, gi[2] = {0.0, 0.0}, hr[2] = {0.0, 0.0}, hi[2] = {0.0, 0.0};
    for (int j = -R.N; j <= R.N; j++) {
        const int aj = j < 0 ? -j : j;
        const double cj = aj == 0 ? 1.0 : aj == 1 ? cdl : c2dl;
        const double sj = (aj == 0 ? 0.0 : aj == 1 ? sdl : s2dl) * (j < 0 ? -1.0 : 1.0);
        const double ca = fma(c1, cj, -s1 * sj), sa = fma(s1, cj, c1 * sj);
        const double cdj = fma(ca, P.clon, sa * P.slon), sdj = fma(sa, P.clon, -ca * P.slon);
        const double dj = P.AD * cdj, ddj = -P.AD * Om * sdj, d2j = -P.AD * Om * Om * cdj;
        // retarded orbital phase alpha - Om d (|Om d| < 1e-4 rad: series to x^5 exact in FP64)
        const double x = Om * dj, x2 = x * x;
        const double cx = fma(-0.5 * x2, fma(-x2, 1.0 / 12.0, 1.0), 1.0), sx = x * fma(-x2, 1.0 / 6.0, 1.0);
        const double cr = fma(ca, cx, sa * sx), sr = fma(sa, cx, -ca * sx);
        double F[2], dF[2];
        if (ECC)
            antenna_ecc<true>(O, P, cr, sr, F[0], F[1], dF[0], dF[1]);
        else
            antenna_deriv(P, cr, sr, F[0], F[1], dF[0], dF[1]);
        const double inv = 1.0 / (1.0 + ddj);
        double cph = 1.0, sph = 0.0;
        if (j != 0) sincos(kTwoPi * fh * (dj * (1.0 - ddj) - D0), &sph, &cph);
        const double h = j == 0 ? 1.0 : 0.5;   // (weights selected without a dynamic index: no local memory)
        const double wr = h * (aj == 0 ? R.ar[0] : aj == 1 ? R.ar[1] : R.ar[2]);
        const double wi = h * (aj == 0 ? R.ai[0] : aj == 1 ? R.ai[1] : R.ai[2]);
        const double Cr = cph * inv, Ci = sph * inv;
        const double wCr = fma(wr, Cr, -wi * Ci), wCi = fma(wr, Ci, wi * Cr);
        const double kr = -d2j * inv, ki = kTwoPi * fh * fma(ddj, 1.0 - ddj, -dj * d2j);
#pragma unroll
        for (int c = 0; c < 2; c++) {
            gr[c] = fma(wCr, F[c], gr[c]);
            gi[c] = fma(wCi, F[c], gi[c]);
            if (R.K >= 1) {
                // G' = C (Om dF/dalpha (1 - ddot) + F kappa), kappa = -d''/(1 + d') + 2 pi i f (d'(1 - d') - d d'')
                const double ur = fma(Om * dF[c], 1.0 - ddj, F[c] * kr), ui = F[c] * ki;
                hr[c] += fma(wCr, ur, -wCi * ui);
                hi[c] += fma(wCr, ui, wCi * ur);
            }
        }
    }
    // T = sum w G - i T_A1 sum w G'
    r.Tpr = fma(TA1, hi[0], gr[0]);
    r.Tpi = fma(-TA1, hr[0], gi[0]);
    r.Txr = fma(TA1, hi[1], gr[1]);
    r.Txi = fma(-TA1, hr[1], gi[1]);
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
