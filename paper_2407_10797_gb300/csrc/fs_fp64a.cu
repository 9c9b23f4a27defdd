// fs_fp64a.cu - FS_FP64 mode, anchored form of the fused bin loop (Sec. II.B
// segment sums of the Sec. IV template, Eqs. A1-A3).
//
// The direct FP64 kernel evaluates the whole template at every bin (powers
// of f, t(f), sin/cos of the orbital phase, the trig polynomials of the
// antenna patterns and sin/cos of the phase).  Here every (particle, 1024-bin
// tile) gets one FP64 anchor at its central in-band bin j_a, and each bin of
// the tile j_a + d is evaluated from expansions about it:
//   - orbital phase: Taylor coefficients in d to degree 12 from the
//     closed-form derivatives of its power-law terms;
//   - orbital-phase offset d(alpha) = Om (t(f) - t_a) as a quintic in d;
//   - Doppler phase and antenna patterns composed with d(alpha) into
//     polynomials in d (Horner's scheme on polynomials, truncated at degree
//     12), the antenna ones rotated into the segment's basis per piece;
//   - total phase: its cubic part in 64-bit fixed point (cycles mod 1, units
//     of 2^-64), stepped per lane by exact integer forward differences; the
//     degree 4..4+NR part a remainder added in units of 2^-48 cycle (FP64, or
//     FP32 in the lowest tier when it is at most 6.7e-8 cycle: error below
//     2.5e-14 cycle);
//   - exp(2 pi i Phi): a 2^20-entry table value in global memory (top 20
//     bits of the phase, rounded; 16 MB per plan, served by L2) times
//     1 - theta^2/2 + i theta for the remaining angle |theta| <= pi 2^-20
//     (dropped terms below 5e-18), folded into four FMAs.
// A tile takes the lowest degree tier (NG, NR) = (4, 2), (5, 2), (6, 2), (7, 3), (8, 5) or
// (10, 7) whose dropped terms, summed over the tile at the anchor, stay below
// 1e-13 cycle (phase) and 1e-15 (antenna); a tile whose d(alpha) quintic or
// degree-12 series does not converge is evaluated bin by bin exactly as the
// direct kernel does.  All other arithmetic is FP64 or exact integer; results agree
// with the direct form to rounding level (1e-10 on the F-statistic at full
// size, 1e-9 against the oracle).
//
// Work decomposition (spans of 32 tiles, in-band particle lists per span,
// grid or persistent form) is that of the mixed-precision kernel.
#include <cfloat>
#include <climits>

#include "fs_internal.h"
#include "fs_device.cuh"

namespace fs {

namespace {

constexpr int kTileA = 1024;                     // bins per anchor
constexpr int kTilesA = 32;                      // tiles per span (one anchor per lane)
constexpr int kSpanA = kTileA * kTilesA;         // 32768 bins
constexpr int kWarpsA = 4;                       // warps (particles) per CTA


constexpr int kDeg = 12;                         // Taylor degree in the bin offset d computed at an anchor
constexpr double kRem32Max = 6.7e-8;             // largest phase remainder (cycles) evaluated in FP32

struct AnchorD {
    unsigned long long c[4];   // cubic of the total phase (orbital minus Doppler), cycles mod 1, units 2^-64
    double R[kDeg - 3];        // its degree 4..12 coefficients (2^-48 cycle per bin^k), FP64
    double FU[2][kDeg + 1];    // F+ and Fx along the tile as polynomials in d (degree 0..12)
    int ja, lo, hi;            // anchor bin and in-band range [lo, hi) of the tile, relative to the span start
    int mode;                  // 0: no in-band bin, 2: bin by bin, 1/3/4/5/6: expansion tiers (see expansion_tile)
};

__device__ __noinline__ void make_anchor_d(const Grid& g, const Tables& tb, const Particle& P, int64_t span_lo,
                                           int64_t lo, int64_t hi, AnchorD& A) {
    A.lo = (int)(lo - span_lo);
    A.hi = (int)(hi - span_lo);
    if (lo >= hi) {
        A.mode = 0;
        return;
    }
    const int64_t ja = lo + (hi - lo - 1) / 2;
    const double hmax = (double)max(ja - lo, hi - 1 - ja);
    A.ja = (int)(ja - span_lo);
    const double fh = tb.fh[ja], fl = tb.fl[ja], u = tb.u[ja], g0h = tb.g0h[ja], g0l = tb.g0l[ja],
                 e19 = tb.e19[ja];
    // orbital phase mod 1 at the anchor (double-double leading term, exact f t_c)
    double p, e;
    two_prod(P.P0h, g0h, p, e);
    e = fma(P.P0h, g0l, e);
    e = fma(P.P0l, g0h, e);
    double acc = (p - rint(p)) + e;
    double q, eq;
    two_prod(fh, P.tc, q, eq);
    eq = fma(fl, P.tc, eq);
    acc += (q - rint(q)) + eq;
    const double u2 = u * u, u3 = u2 * u;
    const double Tm[5] = {P.P0h * g0h, P.P2 * u3, P.P3 * u2, P.P4 * u, P.E0 * g0h * e19};
    double rest = Tm[1] + Tm[2] + Tm[3] + Tm[4];
    acc += rest - rint(rest);
    // S_n = sum_m [p_m]_n T_m (falling factorials of the exponents p_m of the
    // terms T_m = c_m f^p_m): d^n Phi_orb / df^n = S_n / f^n for n >= 2 and
    // t(f) = t_c + S_1 / f.
    const double pm[5] = {-5.0 / 3.0, -1.0, -2.0 / 3.0, -1.0 / 3.0, -34.0 / 9.0};
    double fac[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
    double S[kDeg + 1];
    S[0] = 0.0;
    for (int n = 1; n <= kDeg; n++) {
        double sn = 0.0;
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fac[m] *= pm[m] - (double)(n - 1);
            sn = fma(fac[m], Tm[m], sn);
        }
        S[n] = sn;
    }
    const double inv = 1.0 / fh;
    const double r = g.df * inv;                    // df / f
    const double ta = P.tc + S[1] * inv;            // t(f_a)
    const double Om = kTwoPi / kYearS;
    double sa, ca;
    sincos(fma(Om, ta, g.alpha0), &sa, &ca);
    const double cda = fma(ca, P.clon, sa * P.slon);   // cos(alpha_a - phi)
    const double sda = fma(sa, P.clon, -ca * P.slon);  // sin(alpha_a - phi)
    // orbital Taylor coefficients in d: O_k = S_k r^k / k! (k >= 2), O_1 = t_a df
    double O[kDeg + 1];
    {
        double rk = r, kf = 1.0;
        O[0] = 0.0;
        O[1] = ta * g.df;
        for (int k = 2; k <= kDeg; k++) {
            rk *= r;
            kf *= (double)k;
            O[k] = S[k] * rk / kf;
        }
    }
    // orbital-phase offset d(alpha) = Om (t(f_a + d df) - t_a) = sum_{j=1..5} S_{j+1} r^j d^j Om / (f_a j!)
    double U[6];
    {
        const double Omf = Om * inv;
        double rj = 1.0, jf = 1.0;
        U[0] = 0.0;
        for (int j = 1; j <= 5; j++) {
            rj *= r;
            jf *= (double)j;
            U[j] = Omf * S[j + 1] * rj / jf;
        }
    }
    // Doppler phase AD (f_a + d df) cos(x_a + d(alpha)) as a polynomial in d:
    // cos(x_a + u) = sum_n cos^(n)(x_a) u^n / n!, cos^(n) cycling through (c, -s, -c, s)
    double Dk[kDeg + 1];
    {
        double cn[11];
        const double cyc[4] = {cda, -sda, -cda, sda};
        double nf = 1.0;
        for (int n = 0; n <= 10; n++) {
            if (n > 0) nf *= (double)n;
            cn[n] = cyc[n & 3] / nf;
        }
        double CU[kDeg + 1];
        poly_compose<kDeg, 5, double>(cn, 10, U, CU);
        const double ADfa = P.AD * fh, ADdf = P.AD * g.df;
        Dk[0] = ADfa * CU[0];
        for (int k = 1; k <= kDeg; k++) Dk[k] = fma(ADfa, CU[k], ADdf * CU[k - 1]);
    }
    // total phase: the cubic in fixed point (exact steps), degree 4..12 in FP64
    A.c[0] = to_fixed(acc - Dk[0]);
    A.c[1] = to_fixed(O[1] - Dk[1]);
    A.c[2] = to_fixed_small(O[2] - Dk[2]);
    A.c[3] = to_fixed_small(O[3] - Dk[3]);
    for (int k = 4; k <= kDeg; k++) A.R[k - 4] = O[k] - Dk[k];   // scaled by 2^48 once the tails are known
    // antenna along the tile: F(alpha_a + u) = sum_n F^(n)(alpha_a) u^n / n!, composed with u = d(alpha)
    {
        double ch[5], sh[5];
        ch[1] = ca;
        sh[1] = sa;
#pragma unroll
        for (int h = 2; h <= 4; h++) {
            ch[h] = ch[h - 1] * ca - sh[h - 1] * sa;
            sh[h] = sh[h - 1] * ca + ch[h - 1] * sa;
        }
#pragma unroll
        for (int f = 0; f < 2; f++) {
            const double* H = P.harm[f];
            double uu[5], vv[5];
            double Fd[11];
            Fd[0] = H[0];
#pragma unroll
            for (int h = 1; h <= 4; h++) {
                uu[h] = H[2 * h - 1] * ch[h] + H[2 * h] * sh[h];    // A cos + B sin
                vv[h] = H[2 * h] * ch[h] - H[2 * h - 1] * sh[h];    // derivative / h
                Fd[0] += uu[h];
            }
            double nf = 1.0;
            for (int n = 1; n <= 10; n++) {
                nf *= (double)n;
                double sum = 0.0;
#pragma unroll
                for (int h = 1; h <= 4; h++) {
                    double hn = 1.0;
                    for (int j = 0; j < n; j++) hn *= (double)h;
                    const int rr = n & 3;
                    const double t = (rr == 0) ? uu[h] : (rr == 1) ? vv[h] : (rr == 2) ? -uu[h] : -vv[h];
                    sum = fma(hn, t, sum);
                }
                Fd[n] = sum / nf;
            }
            poly_compose<kDeg, 5, double>(Fd, 10, U, A.FU[f]);
        }
    }
    // validity: the quintic d(alpha) (remainder from S_7, 20% margin) and the degree-12
    // truncations (the last two terms over |d| <= hmax) must be negligible; then the
    // tier is the lowest whose dropped terms, summed over |d| <= hmax, stay below
    // 1e-13 cycle (phase) and 1e-15 (antenna: on a short segment G2 varies by as little
    // as ~1e-4 of the pattern's scale, so its error budget is relative to that)
    const double x = hmax * r;
    double x6 = x * x * x;
    x6 *= x6;
    const double rem_alpha = 1.2 * Om * inv * fabs(S[7]) * x6 * (1.0 / 720.0);
    double hk[kDeg + 1];
    hk[0] = 1.0;
    for (int k = 1; k <= kDeg; k++) hk[k] = hk[k - 1] * hmax;
    double tG[kDeg + 2], tR[kDeg + 2];   // tails: sum over k >= n of |coef_k| hmax^k
    tG[kDeg + 1] = 0.0;
    tR[kDeg + 1] = 0.0;
    for (int k = kDeg; k >= 0; k--) {
        tG[k] = tG[k + 1] + (fabs(A.FU[0][k]) + fabs(A.FU[1][k])) * hk[k];
        tR[k] = tR[k + 1] + (k >= 4 ? fabs(A.R[k - 4]) * hk[k] : 0.0);
    }
    const bool finite = isfinite(rem_alpha) && isfinite(tG[0]) && isfinite(tR[4]);
    const bool converged = finite && rem_alpha <= 1e-13 && tG[kDeg - 1] <= 1e-17 && tR[kDeg - 1] <= 1e-16 &&
                           fabs(U[1]) * hmax <= 0.1;
    // tiers (antenna degree NG, phase remainder degree 4 + NR): 5:(6,2) 4:(7,3) 3:(8,5) 1:(10,7)
    auto ok = [&](int NG, int NR) { return tG[NG + 1] <= 1e-15 && tR[5 + NR] <= 1e-13; };
    A.mode = !converged ? 2 : ok(6, 2) ? 5 : ok(7, 3) ? 4 : ok(8, 5) ? 3 : ok(10, 7) ? 1 : 2;
    // tier (6, 2) with the remainder evaluated in FP32 (mode 6): when the remainder is at most
    // kRem32Max cycle over the tile, the FP32 evaluation's error (within 6 roundings of 2^-24 of
    // sum_k |R_k| hmax^k) stays below 2.5e-14 cycle
    if (A.mode == 5 && tR[4] <= kRem32Max) A.mode = 6;
    // the same with antenna degree 5 (mode 7) when the antenna terms beyond degree 5 meet the budget
    if (A.mode == 6 && tG[6] <= 1e-15) A.mode = 7;
    if (A.mode == 7 && tG[5] <= 1e-15) A.mode = 8;   // and antenna degree 4
    // the remainder is added to the fixed-point phase in units of 2^-48 cycle
    for (int k = 0; k <= kDeg - 4; k++) A.R[k] *= 0x1p48;
}

// Per-segment antenna polynomials in d: G1 = c F+ + s Fx, G2 = c Fx - s F+.
template <int NG>
__device__ __forceinline__ void segment_coeffs_d(const AnchorD& A, double2 rc, double g1[NG + 1], double g2[NG + 1]) {
#pragma unroll
    for (int n = 0; n <= NG; n++) {
        g1[n] = fma(rc.x, A.FU[0][n], rc.y * A.FU[1][n]);
        g2[n] = fma(rc.x, A.FU[1][n], -rc.y * A.FU[0][n]);
    }
}

template <int N>
__device__ __forceinline__ double horner(const double* c, double x) {
    double v = c[N];
#pragma unroll
    for (int i = N - 1; i >= 0; i--) v = fma(v, x, c[i]);
    return v;
}

// exp(2 pi i Phi) from the phase in 64-bit fixed point (cycles mod 1 in
// units of 2^-64): the nearest multiple of 2^-20 cycle indexes the table
// (kCisBits bits), the remaining 44 bits give the angle |theta| <= pi 2^-20,
// and exp(i theta) = 1 - theta^2/2 + i theta to below 5e-18 (the theta^3/6 of
// the sine is the largest dropped term):
//   cos = t.x + theta (t.x (-theta/2) - t.y),  sin = t.y + theta (t.y (-theta/2) + t.x).
__device__ __forceinline__ void cis_fixed(unsigned long long Ft, const double2* __restrict__ tab, double& cs,
                                          double& sn) {
    const unsigned idx = (unsigned)((Ft + (1ull << (63 - kCisBits))) >> (64 - kCisBits));
    const double th = (double)(long long)(Ft << kCisBits) * (kTwoPi * 0x1p-84);
    const double hth = -0.5 * th;
    const double2 t = __ldg(&tab[idx & ((1u << kCisBits) - 1u)]);
    cs = fma(th, fma(t.x, hth, -t.y), t.x);
    sn = fma(th, fma(t.y, hth, t.x), t.y);
}

// One bin of an expansion tile inside a single segment: the phase is the
// fixed-point cubic Fv plus the FP64 remainder d^4 (R_4 + R_5 d + ... ), NR + 1
// terms in units of 2^-48 cycle, added as an integer; the antenna pair is two
// degree-NG polynomials in d.
template <int NG, int NR, bool R32>
__device__ __forceinline__ void bin_d(unsigned long long Fv, double d, float dfl, double dr, double di, double W,
                                      const double Rc[NR + 1], const float Rcf[NR + 1], const double g1[NG + 1],
                                      const double g2[NG + 1], const double2* __restrict__ tab, double acc[7]) {
    long long corr;   // the remainder in units of 2^-48 cycle (Rc, Rcf scaled by 2^48)
    if (R32) {
        // |remainder| <= kRem32Max cycle: FP32 (|corr| < 2^31), error below 2.5e-14 cycle
        const float dd = dfl * dfl;
        float v = Rcf[NR];
#pragma unroll
        for (int i = NR - 1; i >= 0; i--) v = fmaf(v, dfl, Rcf[i]);
        corr = (long long)__float2int_rn((dd * dd) * v);
    } else {
        const double dd = d * d;
        corr = __double2ll_rn((dd * dd) * horner<NR>(Rc, d));
    }
    double cs, sn;
    cis_fixed(Fv + ((unsigned long long)corr << 16), tab, cs, sn);
    const double G1 = horner<NG>(g1, d);
    const double G2 = horner<NG>(g2, d);
    const double zr = fma(dr, cs, -di * sn);
    const double zi = fma(dr, sn, di * cs);
    acc[0] = fma(G1, zr, acc[0]);
    acc[1] = fma(G1, zi, acc[1]);
    acc[2] = fma(G2, zr, acc[2]);
    acc[3] = fma(G2, zi, acc[3]);
    const double wg = W * G1;
    acc[4] = fma(wg, G1, acc[4]);
    acc[5] = fma(wg, G2, acc[5]);
    acc[6] = fma(W * G2, G2, acc[6]);
}

// The warp's sums of acc[0..6] into dst[0..6], and acc cleared: a
// reduce-scatter butterfly over eight slots (the eighth zero).  At the XOR
// distances 16, 8 and 4 each lane keeps half of its slots -- the upper half
// if its lane bit is set -- and adds the partner's copies, so that lane l then
// holds slot 4 b4 + 2 b3 + b2 (b_j bit j of l); distances 2 and 1 sum the
// four lanes that hold the same slot, and the first of them writes it.
// 9 FP64 additions per lane instead of the 35 of seven warp trees.
__device__ __forceinline__ void flush_d(double acc[7], double* dst, int lane) {
    double v4[4];
    const bool h16 = (lane & 16) != 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const double lo = acc[i], hi = i + 4 < 7 ? acc[i + 4] : 0.0;
        const double give = h16 ? lo : hi;
        v4[i] = (h16 ? hi : lo) + __shfl_xor_sync(0xffffffffu, give, 16);
    }
    double v2[2];
    const bool h8 = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const double give = h8 ? v4[i] : v4[i + 2];
        v2[i] = (h8 ? v4[i + 2] : v4[i]) + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    const bool h4 = (lane & 4) != 0;
    double v1 = (h4 ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? v2[0] : v2[1], 4);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 2);
    v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
    const int slot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && slot < 7) dst[slot] = v1;
#pragma unroll
    for (int c = 0; c < 7; c++) acc[c] = 0.0;
}

// An expansion tile walked as single-segment pieces [pa_lo, pa_hi): flushes the
// running segment when a piece starts a new one.
template <int NG, int NR, bool R32 = false>
__device__ __forceinline__ void expansion_tile(const AnchorD& A, const SegView& sv, int64_t span_lo, int lo, int hi,
                                               const double2* __restrict__ rot, const double* __restrict__ dwr,
                                               const double* __restrict__ dwi, const double* __restrict__ Wt,
                                               const double2* __restrict__ tab, const Partials& pa, int64_t slot,
                                               int b, int Np, int lane, int& cur, int& nflush, int& trk,
                                               int64_t& trk_nxt, double acc[7]) {
    double g1[NG + 1], g2[NG + 1], Rc[NR + 1];
    float Rcf[NR + 1];
#pragma unroll
    for (int i = 0; i <= NR; i++) {
        Rc[i] = A.R[i];
        Rcf[i] = (float)A.R[i];
    }
    int pa_lo = lo;
    while (pa_lo < hi) {
        // segment of the piece's first bin (sv.seg of it), tracked forward across the item's
        // pieces: a segment boundary costs one sv.start
        const int64_t kabs = span_lo + pa_lo;
        if (trk < 0) {
            trk = sv.seg(kabs);
            trk_nxt = sv.start(trk + 1);
        }
        while (kabs >= trk_nxt) {
            trk++;
            trk_nxt = sv.start(trk + 1);
        }
        const int sp = trk;   // warp-uniform
        if (sp != cur) {
            flush_d(acc, (nflush == 0) ? pa.H + slot * 7 : pa.S + ((int64_t)b * Np + cur) * 7, lane);
            nflush++;
            cur = sp;
        }
        const int64_t nb = trk_nxt - span_lo;
        const int pa_hi = nb < hi ? (int)nb : hi;
        segment_coeffs_d<NG>(A, rot[sp], g1, g2);
        const int k0 = pa_lo + lane;
        const long long d0 = (long long)(k0 - A.ja);
        const unsigned long long y0 = poly_fx(A.c, d0), y1 = poly_fx(A.c, d0 + 32),
                                 y2 = poly_fx(A.c, d0 + 64), y3 = poly_fx(A.c, d0 + 96);
        unsigned long long F = y0, D1 = y1 - y0, D2 = y2 - 2ull * y1 + y0,
                           D3 = y3 - 3ull * y2 + 3ull * y1 - y0;
        double d = (double)(k0 - A.ja);
        float dfl = (float)(k0 - A.ja);   // the same offset in FP32 (exact: |d| < 2^24)
        int k = k0;
        // two bins per lane per iteration (k and k + 32): two independent chains
        for (; k + 32 < pa_hi; k += 64, d += 64.0, dfl += 64.f) {
            const unsigned long long Fa = F, Fb = F + D1;
            F = Fb + D1 + D2;
            D1 += 2ull * D2 + D3;
            D2 += 2ull * D3;
            bin_d<NG, NR, R32>(Fa, d, dfl, dwr[k], dwi[k], Wt[k], Rc, Rcf, g1, g2, tab, acc);
            bin_d<NG, NR, R32>(Fb, d + 32.0, dfl + 32.f, dwr[k + 32], dwi[k + 32], Wt[k + 32], Rc, Rcf, g1, g2, tab,
                               acc);
        }
        if (k < pa_hi) bin_d<NG, NR, R32>(F, d, dfl, dwr[k], dwi[k], Wt[k], Rc, Rcf, g1, g2, tab, acc);
        pa_lo = pa_hi;
    }
}

// One work item: particle b over span `span`, by one warp (see mixed_item).
__device__ __forceinline__ void fp64a_item(const Grid& g, const Tables& tb, const Particle* __restrict__ parts,
                                           const Segs& sg, const Partials& pa, const double2* __restrict__ tab,
                                           int span, int b, AnchorD* anc, int lane) {
    const int64_t span_lo = (int64_t)span * kSpanA;
    const Particle& P = parts[b];
    const SegView sv = seg_view(sg, P);
    {
        int64_t lo = span_lo + (int64_t)lane * kTileA, hi = lo + kTileA;
        if (lo < sv.lo) lo = sv.lo;
        if (hi > sv.hi + 1) hi = sv.hi + 1;
        make_anchor_d(g, tb, P, span_lo, lo, hi, anc[lane]);
        if (pa.census && lo < hi) atomicAdd(&pa.census[anc[lane].mode], (unsigned long long)(hi - lo));
    }
    __syncwarp();

    const int64_t slot = (int64_t)b * pa.ntiles + span;
    const double2* rot = pa.rot + (int64_t)b * sg.Np;
    const double* dwr = tb.dwr + span_lo;
    const double* dwi = tb.dwi + span_lo;
    const double* Wt = tb.W + span_lo;

    double acc[7];
#pragma unroll
    for (int c = 0; c < 7; c++) acc[c] = 0.0;
    int cur = -1;        // warp-uniform current segment
    int nflush = 0;
    int pk = -1;         // this lane's segment (bin-by-bin tiles)
    int nxt = -1;        // first bin (span-relative) of the segment after pk
    int trk = -1;        // warp-uniform segment of the latest piece start (expansion tiles) and
    int64_t trk_nxt = 0; // the first bin (absolute) of the segment after it

    for (int ti = 0; ti < kTilesA; ti++) {
        const AnchorD& A = anc[ti];
        if (A.mode == 0) continue;
        const int lo = A.lo, hi = A.hi;
        if (cur < 0) cur = sv.seg(span_lo + lo);
        if (A.mode != 2) {
            if (A.mode == 8)
                expansion_tile<4, 2, true>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane,
                                           cur, nflush, trk, trk_nxt, acc);
            else if (A.mode == 7)
                expansion_tile<5, 2, true>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane,
                                           cur, nflush, trk, trk_nxt, acc);
            else if (A.mode == 6)
                expansion_tile<6, 2, true>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane,
                                           cur, nflush, trk, trk_nxt, acc);
            else if (A.mode == 5)
                expansion_tile<6, 2>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane, cur,
                                     nflush, trk, trk_nxt, acc);
            else if (A.mode == 4)
                expansion_tile<7, 3>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane, cur,
                                     nflush, trk, trk_nxt, acc);
            else if (A.mode == 3)
                expansion_tile<8, 5>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane, cur,
                                     nflush, trk, trk_nxt, acc);
            else
                expansion_tile<10, 7>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane, cur,
                                      nflush, trk, trk_nxt, acc);
            pk = -1;
            nxt = -1;
        } else {
            // bin-by-bin FP64 tile (expansion bounds not met): the direct evaluation
            for (int base = lo; base < hi; base += 32) {
                const int k = base + lane;
                const bool valid = k < hi;
                double t7[7];
#pragma unroll
                for (int c = 0; c < 7; c++) t7[c] = 0.0;
                if (valid) {
                    if (k >= nxt) {
                        pk = sv.seg(span_lo + k);
                        nxt = (int)(sv.start(pk + 1) - span_lo);
                    }
                    const int64_t kk = span_lo + k;
                    FreqPowers fw;
                    fw.u = tb.u[kk];
                    fw.g0h = tb.g0h[kk];
                    fw.e19 = tb.e19[kk];
                    const BinEval ev = eval_bin_fp64(P, tb.fh[kk], tb.fl[kk], fw, tb.g0l[kk], g.alpha0);
                    double sn, cs;
                    sincospi(2.0 * ev.frac, &sn, &cs);
                    const double2 rc = rot[pk];
                    const double G1 = fma(rc.x, ev.Fp, rc.y * ev.Fx);
                    const double G2 = fma(rc.x, ev.Fx, -rc.y * ev.Fp);
                    const double dr = dwr[k], di = dwi[k], W = Wt[k];
                    const double zr = fma(dr, cs, -di * sn);
                    const double zi = fma(dr, sn, di * cs);
                    t7[0] = G1 * zr;
                    t7[1] = G1 * zi;
                    t7[2] = G2 * zr;
                    t7[3] = G2 * zi;
                    const double wg = W * G1;
                    t7[4] = wg * G1;
                    t7[5] = wg * G2;
                    t7[6] = W * G2 * G2;
                }
                while (true) {
                    if (valid && pk == cur) {
#pragma unroll
                        for (int c = 0; c < 7; c++) acc[c] += t7[c];
                    }
                    const unsigned more = __ballot_sync(0xffffffffu, valid && pk > cur);
                    if (!more) break;
                    flush_d(acc, (nflush == 0) ? pa.H + slot * 7 : pa.S + ((int64_t)b * sg.Np + cur) * 7, lane);
                    nflush++;
                    int cand = (valid && pk > cur) ? pk : INT_MAX;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
                    cur = cand;
                }
            }
        }
    }
    if (cur < 0) return;   // no in-band bin in this span (warp-uniform)
    flush_d(acc, (nflush == 0) ? pa.H + slot * 7 : pa.T + slot * 7, lane);
}

// The plan's exp(2 pi i j 2^-kCisBits) table (filled once per plan).
__global__ void cis_table_kernel(double2* tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (1 << kCisBits)) return;
    double s, c;
    sincospi((double)i * 0x1p-19, &s, &c);   // 2 i / 2^20
    tab[i] = make_double2(c, s);
}

// Grid form: CTA (span, group of 4 in-band particles of the span).
__global__ void __launch_bounds__(kWarpsA * 32, 3)
fp64a_main_kernel(Grid g, Tables tb, const Particle* __restrict__ parts, int B, Segs sg, Partials pa,
                  const int* __restrict__ list, const int* __restrict__ cnt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AnchorD* anc = reinterpret_cast<AnchorD*>(smem_raw);
    const double2* __restrict__ tab = pa.cis;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int span = blockIdx.x;
    const int j = blockIdx.y * kWarpsA + w;
    if (j >= cnt[span]) return;   // warp-uniform
    fp64a_item(g, tb, parts, sg, pa, tab, span, list[(int64_t)span * B + j], anc + w * 32, lane);
}

// Persistent form: warps take (span, particle) items from a device counter.
__global__ void __launch_bounds__(kWarpsA * 32, 3)
fp64a_persistent_kernel(Grid g, Tables tb, const Particle* __restrict__ parts, int B, Segs sg, Partials pa,
                        const int* __restrict__ list, const int* __restrict__ sched, int nspans, int* ctl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AnchorD* anc = reinterpret_cast<AnchorD*>(smem_raw) + (threadIdx.x >> 5) * 32;
    const double2* __restrict__ tab = pa.cis;
    const int lane = threadIdx.x & 31;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&ctl[1], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        int span, b;
        if (!sched_item(sched, nspans, B, list, item, span, b)) break;   // heavy items first
        __syncwarp();
        fp64a_item(g, tb, parts, sg, pa, tab, span, b, anc, lane);
    }
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t smem, int slot) {
    static bool done[64][2];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (done[dev][slot]) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done[dev][slot] = true;
    return e;
}

}  // namespace

int fp64a_span() { return kSpanA; }

cudaError_t launch_fp64a_main(const Grid& g, const Tables& t, const Particle* parts, int B, const Segs& sg,
                              const Partials& pa, bool persistent, int* list, int* cnt, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    if (!pa.cis) return cudaErrorInvalidValue;   // the plan's exp table is required
    const int nspans = pa.ntiles;
    const size_t smem = sizeof(AnchorD) * kWarpsA * 32;
    cudaError_t e = launch_span_lists(parts, B, sg, nspans, kSpanA, list, cnt, persistent, s);
    if (e != cudaSuccess) return e;
    if (persistent) {
        if ((e = allow_smem(fp64a_persistent_kernel, smem, 1)) != cudaSuccess) return e;
        const int grid = persistent_grid(fp64a_persistent_kernel, kWarpsA * 32, smem, 2);
        if (grid <= 0) return cudaErrorInvalidConfiguration;
        fp64a_persistent_kernel<<<grid, kWarpsA * 32, smem, s>>>(g, t, parts, B, sg, pa, list, cnt, nspans,
                                                                 cnt + 2 * nspans + 1);
        return cudaGetLastError();
    }
    if ((e = allow_smem(fp64a_main_kernel, smem, 0)) != cudaSuccess) return e;
    dim3 grid((unsigned)nspans, (unsigned)((B + kWarpsA - 1) / kWarpsA));
    fp64a_main_kernel<<<grid, kWarpsA * 32, smem, s>>>(g, t, parts, B, sg, pa, list, cnt);
    return cudaGetLastError();
}

cudaError_t launch_cis_table(double2* tab, cudaStream_t s) {
    cis_table_kernel<<<(1 << kCisBits) / 256, 256, 0, s>>>(tab);
    return cudaGetLastError();
}

}  // namespace fs
