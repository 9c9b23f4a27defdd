// fs_fp64a.cu - FS_FP64 mode, anchored form of the fused bin loop (Sec. II.B
// segment sums of the Sec. IV template, Eqs. A1-A3).
//
// The direct FP64 kernel evaluates the whole template at every bin (powers
// of f, t(f), sin/cos of the orbital phase, the trig polynomials of the
// antenna patterns and sin/cos of the phase).  Here every (particle, 1024-bin
// tile) gets one FP64 anchor at its centre bin j_a, and each bin of the tile
// j_a + d is evaluated from an expansion about it:
//   - orbital phase: an exact cubic in d in 64-bit fixed point (cycles mod 1,
//     units of 2^-64), stepped by integer forward differences, plus the FP64
//     quartic and quintic terms;
//   - orbital-phase offset d(alpha) = Om (t(f) - t_a) as a quartic in d;
//   - Doppler phase and antenna patterns as FP64 polynomials in d(alpha)
//     (degrees 7 and 8), the antenna ones folded with the segment's rotation;
//   - exp(2 pi i Phi) as a 256-entry table value times a degree-6/7 Taylor
//     series of the remaining angle (|angle| <= pi/256).
// The truncation remainders are bounded at the anchor (phase <= 1e-11 cycle,
// d(alpha) remainder <= 1e-11 rad, |d(alpha)| <= 0.06); a tile that fails a
// bound is evaluated bin by bin exactly as the direct kernel does.  All
// arithmetic is FP64 or exact integer; results agree with the direct form to
// rounding level (relative 1e-12 or better on the F-statistic).
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
constexpr int kTabA = 256;                       // exp(2 pi i j / 256) table

struct AnchorD {
    unsigned long long c[4];   // cubic of the orbital-minus-Doppler phase, cycles mod 1 in units of 2^-64
    double c4, c5;             // quartic and quintic phase terms, cycles per bin^4, bin^5
    double w[4];               // d(alpha) = sum_j w_j d^j, j = 1..4, rad
    double e[7];               // Doppler: AD f_a cos^(n)(x_a)/n!, n = 1..7 (cycles)
    double q[6];               // Doppler: AD df cos^(n)(x_a)/n!, n = 0..5 (cycles per bin)
    double Fpa, Fxa;           // F+ and Fx at alpha_a
    double Fd[8][2];           // F+^(n)(alpha_a)/n!, Fx^(n)(alpha_a)/n!, n = 1..8
    int ja, lo, hi;            // anchor bin and in-band range [lo, hi) of the tile, relative to the span start
    int mode;                  // 0: no in-band bin, 2: bin by bin, 1/3/4: expansion (wide/mid/narrow degrees)
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
    // terms T_m = c_m f^p_m), so that d^n Phi_orb / df^n = S_n / f^n for n >= 2
    // and t(f) = t_c + S_1 / f.
    const double pm[5] = {-5.0 / 3.0, -1.0, -2.0 / 3.0, -1.0 / 3.0, -34.0 / 9.0};
    double fac[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
    double S[7];
#pragma unroll
    for (int n = 1; n <= 6; n++) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < 5; m++) {
            fac[m] *= pm[m] - (double)(n - 1);
            s = fma(fac[m], Tm[m], s);
        }
        S[n] = s;
    }
    const double inv = 1.0 / fh;
    const double r = g.df * inv;                    // df / f
    const double ta = P.tc + S[1] * inv;            // t(f_a)
    // Taylor coefficients in d of Phi_orb: S_n r^n / n!
    const double r2 = r * r, r3 = r2 * r, r4 = r2 * r2, r5 = r4 * r;
    const double Om = kTwoPi / kYearS;
    double sa, ca;
    sincos(fma(Om, ta, g.alpha0), &sa, &ca);
    const double cda = fma(ca, P.clon, sa * P.slon);   // cos(alpha_a - phi)
    const double sda = fma(sa, P.clon, -ca * P.slon);  // sin(alpha_a - phi)
    acc -= fh * P.AD * cda;
    A.c[0] = to_fixed(acc);
    A.c[1] = to_fixed(ta * g.df);
    A.c[2] = to_fixed_small(0.5 * S[2] * r2);
    A.c[3] = to_fixed_small(S[3] * r3 * (1.0 / 6.0));
    A.c4 = S[4] * r4 * (1.0 / 24.0);
    A.c5 = S[5] * r5 * (1.0 / 120.0);
    // d(alpha) = Om (t(f_a + d df) - t_a) = Om sum_j S_{j+1} r^j d^j / (f_a j!)
    const double Omf = Om * inv;
    A.w[0] = Omf * S[2] * r;
    A.w[1] = Omf * S[3] * r2 * 0.5;
    A.w[2] = Omf * S[4] * r3 * (1.0 / 6.0);
    A.w[3] = Omf * S[5] * r4 * (1.0 / 24.0);
    // Doppler phase minus its anchor value, x = alpha - phi = x_a + d(alpha):
    //   AD [f_a (cos x - cos x_a) + d df cos x],  cos^(n)(x_a) cycles through (c, -s, -c, s)
    {
        const double cn[8] = {cda, -sda, -cda, sda, cda, -sda, -cda, sda};
        double fact = 1.0;
        const double ADfa = P.AD * fh, ADdf = P.AD * g.df;
#pragma unroll
        for (int n = 0; n <= 7; n++) {
            if (n > 0) fact *= (double)n;
            if (n >= 1) A.e[n - 1] = ADfa * cn[n] / fact;
            if (n <= 5) A.q[n] = ADdf * cn[n] / fact;
        }
    }
    // antenna: F(alpha_a + da) = sum_n F^(n)(alpha_a) da^n / n! from the harmonics
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
            double F0 = H[0];
            double uu[5], vv[5];
#pragma unroll
            for (int h = 1; h <= 4; h++) {
                uu[h] = H[2 * h - 1] * ch[h] + H[2 * h] * sh[h];    // A cos + B sin
                vv[h] = H[2 * h] * ch[h] - H[2 * h - 1] * sh[h];    // derivative / h
                F0 += uu[h];
            }
            if (f == 0) A.Fpa = F0;
            else A.Fxa = F0;
            double fact = 1.0;
#pragma unroll
            for (int n = 1; n <= 8; n++) {
                fact *= (double)n;
                double sum = 0.0;
#pragma unroll
                for (int h = 1; h <= 4; h++) {
                    double hn = 1.0;
#pragma unroll
                    for (int j = 0; j < n; j++) hn *= (double)h;
                    const int rr = n & 3;
                    const double t = (rr == 0) ? uu[h] : (rr == 1) ? vv[h] : (rr == 2) ? -uu[h] : -vv[h];
                    sum = fma(hn, t, sum);
                }
                A.Fd[n - 1][f] = sum / fact;
            }
        }
    }
    // truncation remainders over |d| <= hmax (20% margin).  The polynomial
    // degrees in d(alpha) go by tier: narrow (antenna 5, Doppler 4 and 3),
    // mid (6, 5, 4), wide (8, 7, 5); each tier's remainders (antenna:
    // (4 da)^(n+1)/(n+1)! times the pattern scale, Doppler: its scale times
    // da^(n+1)/(n+1)!) must stay below 1e-12 (1e-11 for the wide antenna).
    const double x = hmax * r;                      // H / f_a
    const double x5 = x * x * x * x * x;
    const double rem_phase = 1.2 * fabs(S[6]) * x5 * x * (1.0 / 720.0);   // cycles
    const double rem_alpha = 1.2 * Omf * fabs(S[6]) * x5 * (1.0 / 120.0);  // rad
    const double da =
        1.2 * hmax * (fabs(A.w[0]) + hmax * (fabs(A.w[1]) + hmax * (fabs(A.w[2]) + hmax * fabs(A.w[3]))));
    const double sE = fabs(P.AD * fh), sQ = fabs(P.AD * g.df) * hmax;
    double sG = 0.0;
#pragma unroll
    for (int i = 0; i < 9; i++) sG += fabs(P.harm[0][i]) + fabs(P.harm[1][i]);
    const double g4 = 4.0 * da;
    // x^(n+1)/(n+1)! for the degrees used
    const double da4 = da * da * da * da, da5 = da4 * da, da6 = da5 * da, da8 = da6 * da * da;
    const double g6 = g4 * g4 * g4 * g4 * g4 * g4, g7 = g6 * g4, g9 = g7 * g4 * g4;
    const bool narrow = sG * g6 / 720.0 <= 1e-12 && sE * da5 / 120.0 <= 1e-12 && sQ * da4 / 24.0 <= 1e-12;
    const bool mid = sG * g7 / 5040.0 <= 1e-12 && sE * da6 / 720.0 <= 1e-12 && sQ * da5 / 120.0 <= 1e-12;
    const bool wide = da <= 0.06 && sG * g9 / 362880.0 <= 1e-11 && sE * da8 / 40320.0 <= 1e-12 &&
                      sQ * da6 / 720.0 <= 1e-12;
    const bool finite = isfinite(rem_phase) && isfinite(da) && isfinite(A.c4) && isfinite(A.c5);
    const bool phase_ok = finite && rem_phase <= 1e-11 && rem_alpha <= 1e-11;
    A.mode = !phase_ok ? 2 : narrow ? 4 : mid ? 3 : wide ? 1 : 2;
}

// Per-segment antenna polynomials: G1 = c F+ + s Fx, G2 = c Fx - s F+ in powers of d(alpha).
__device__ __forceinline__ void segment_coeffs_d(const AnchorD& A, double2 rc, double g1[9], double g2[9]) {
    g1[0] = fma(rc.x, A.Fpa, rc.y * A.Fxa);
    g2[0] = fma(rc.x, A.Fxa, -rc.y * A.Fpa);
#pragma unroll
    for (int n = 1; n <= 8; n++) {
        g1[n] = fma(rc.x, A.Fd[n - 1][0], rc.y * A.Fd[n - 1][1]);
        g2[n] = fma(rc.x, A.Fd[n - 1][1], -rc.y * A.Fd[n - 1][0]);
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
// units of 2^-64): the nearest multiple of 1/256 cycle indexes the table, the
// remaining 56 bits give the angle |theta| <= pi/256, whose cos and sin come
// from their Taylor series (cos to degree 6, sin to degree 7; truncation
// below 1e-19).
__device__ __forceinline__ void cis_fixed(unsigned long long Ft, const double2* __restrict__ tab, double& cs,
                                          double& sn) {
    const int idx = (int)((Ft + (1ull << 55)) >> 56);
    const double th = (double)(long long)(Ft << 8) * (kTwoPi * 0x1p-72);
    const double t2 = th * th;
    const double cr = fma(fma(fma(-1.0 / 720.0, t2, 1.0 / 24.0), t2, -0.5), t2, 1.0);
    const double sr = th * fma(fma(fma(-1.0 / 5040.0, t2, 1.0 / 120.0), t2, -1.0 / 6.0), t2, 1.0);
    const double2 t = tab[idx & (kTabA - 1)];
    cs = fma(t.x, cr, -t.y * sr);
    sn = fma(t.y, cr, t.x * sr);
}

// One bin of an expansion tile inside a single segment; NG, NE, NQ are the
// degrees of the antenna, Doppler (f_a term, without its zero constant) and
// Doppler (d df term) polynomials in d(alpha).
template <int NG, int NE, int NQ>
__device__ __forceinline__ void bin_d(unsigned long long Fv, double d, double dr, double di, double W,
                                      const double w[4], double c4, double c5, const double e[7], const double q[6],
                                      const double g1[9], const double g2[9], const double2* __restrict__ tab,
                                      double acc[7]) {
    const double dd = d * d;
    const double ext = dd * dd * fma(c5, d, c4);
    const double da = d * fma(fma(fma(w[3], d, w[2]), d, w[1]), d, w[0]);
    const double dop = fma(da, horner<NE - 1>(e, da), d * horner<NQ>(q, da));
    // quartic/quintic phase minus the Doppler offset, to 2^-48 cycle, added in fixed point
    const long long corr = __double2ll_rn((ext - dop) * 0x1p48);
    double cs, sn;
    cis_fixed(Fv + ((unsigned long long)corr << 16), tab, cs, sn);
    const double G1 = horner<NG>(g1, da);
    const double G2 = horner<NG>(g2, da);
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

__device__ __forceinline__ void flush_d(double acc[7], double* dst, int lane) {
#pragma unroll
    for (int c = 0; c < 7; c++) {
        const double v = warp_sum(acc[c]);
        if (lane == 0) dst[c] = v;
        acc[c] = 0.0;
    }
}

// An expansion tile walked as single-segment pieces [pa_lo, pa_hi): flushes the
// running segment when a piece starts a new one.
template <int NG, int NE, int NQ>
__device__ __forceinline__ void expansion_tile(const AnchorD& A, const SegView& sv, int64_t span_lo, int lo, int hi,
                                               const double2* __restrict__ rot, const double* __restrict__ dwr,
                                               const double* __restrict__ dwi, const double* __restrict__ Wt,
                                               const double2* __restrict__ tab, const Partials& pa, int64_t slot,
                                               int b, int Np, int lane, int& cur, int& nflush, double acc[7]) {
    double g1[9], g2[9];
    double w[4], e[7], q[6];
#pragma unroll
    for (int i = 0; i < 4; i++) w[i] = A.w[i];
#pragma unroll
    for (int i = 0; i < 7; i++) e[i] = A.e[i];
#pragma unroll
    for (int i = 0; i < 6; i++) q[i] = A.q[i];
    const double c4 = A.c4, c5 = A.c5;
    int pa_lo = lo;
    while (pa_lo < hi) {
        const int sp = sv.seg(span_lo + pa_lo);   // warp-uniform
        if (sp != cur) {
            flush_d(acc, (nflush == 0) ? pa.H + slot * 7 : pa.S + ((int64_t)b * Np + cur) * 7, lane);
            nflush++;
            cur = sp;
        }
        const int64_t nb = sv.start(sp + 1) - span_lo;
        const int pa_hi = nb < hi ? (int)nb : hi;
        segment_coeffs_d(A, rot[sp], g1, g2);
        const int k0 = pa_lo + lane;
        const long long d0 = (long long)(k0 - A.ja);
        const unsigned long long y0 = poly_fx(A.c, d0), y1 = poly_fx(A.c, d0 + 32),
                                 y2 = poly_fx(A.c, d0 + 64), y3 = poly_fx(A.c, d0 + 96);
        unsigned long long F = y0, D1 = y1 - y0, D2 = y2 - 2ull * y1 + y0,
                           D3 = y3 - 3ull * y2 + 3ull * y1 - y0;
        double d = (double)(k0 - A.ja);
        int k = k0;
        // two bins per lane per iteration (k and k + 32): two independent chains
        for (; k + 32 < pa_hi; k += 64, d += 64.0) {
            const unsigned long long Fa = F, Fb = F + D1;
            F = Fb + D1 + D2;
            D1 += 2ull * D2 + D3;
            D2 += 2ull * D3;
            bin_d<NG, NE, NQ>(Fa, d, dwr[k], dwi[k], Wt[k], w, c4, c5, e, q, g1, g2, tab, acc);
            bin_d<NG, NE, NQ>(Fb, d + 32.0, dwr[k + 32], dwi[k + 32], Wt[k + 32], w, c4, c5, e, q, g1, g2, tab,
                              acc);
        }
        if (k < pa_hi) bin_d<NG, NE, NQ>(F, d, dwr[k], dwi[k], Wt[k], w, c4, c5, e, q, g1, g2, tab, acc);
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

    for (int ti = 0; ti < kTilesA; ti++) {
        const AnchorD& A = anc[ti];
        if (A.mode == 0) continue;
        const int lo = A.lo, hi = A.hi;
        if (cur < 0) cur = sv.seg(span_lo + lo);
        if (A.mode != 2) {
            if (A.mode == 4)
                expansion_tile<5, 4, 3>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane,
                                        cur, nflush, acc);
            else if (A.mode == 3)
                expansion_tile<6, 5, 4>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane,
                                        cur, nflush, acc);
            else
                expansion_tile<8, 7, 5>(A, sv, span_lo, lo, hi, rot, dwr, dwi, Wt, tab, pa, slot, b, sg.Np, lane,
                                        cur, nflush, acc);
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

__device__ __forceinline__ void fill_table(double2* tab) {
    for (int i = threadIdx.x; i < kTabA; i += blockDim.x) {
        double s, c;
        sincospi((double)i * (2.0 / kTabA), &s, &c);
        tab[i] = make_double2(c, s);
    }
    __syncthreads();
}

// Grid form: CTA (span, group of 4 in-band particles of the span).
__global__ void __launch_bounds__(kWarpsA * 32, 3)
fp64a_main_kernel(Grid g, Tables tb, const Particle* __restrict__ parts, int B, Segs sg, Partials pa,
                  const int* __restrict__ list, const int* __restrict__ cnt) {
    __shared__ double2 tab[kTabA];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AnchorD* anc = reinterpret_cast<AnchorD*>(smem_raw);
    fill_table(tab);
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
                        const int* __restrict__ list, const int* __restrict__ off, int nspans, int* ctl) {
    __shared__ double2 tab[kTabA];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AnchorD* anc = reinterpret_cast<AnchorD*>(smem_raw) + (threadIdx.x >> 5) * 32;
    fill_table(tab);
    const int lane = threadIdx.x & 31;
    const int total = off[nspans];
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&ctl[1], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= total) break;
        int lo = 0, hi = nspans;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= item) lo = mid;
            else hi = mid;
        }
        const int b = list[(int64_t)lo * B + (item - off[lo])];
        __syncwarp();
        fp64a_item(g, tb, parts, sg, pa, tab, lo, b, anc, lane);
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
    const int nspans = pa.ntiles;
    const size_t smem = sizeof(AnchorD) * kWarpsA * 32;
    cudaError_t e = launch_span_lists(parts, B, sg, nspans, kSpanA, list, cnt, persistent, s);
    if (e != cudaSuccess) return e;
    if (persistent) {
        if ((e = allow_smem(fp64a_persistent_kernel, smem, 1)) != cudaSuccess) return e;
        const int grid = persistent_grid(fp64a_persistent_kernel, kWarpsA * 32, smem, 2);
        if (grid <= 0) return cudaErrorInvalidConfiguration;
        fp64a_persistent_kernel<<<grid, kWarpsA * 32, smem, s>>>(g, t, parts, B, sg, pa, list, cnt + nspans, nspans,
                                                                 cnt + 2 * nspans + 1);
        return cudaGetLastError();
    }
    if ((e = allow_smem(fp64a_main_kernel, smem, 0)) != cudaSuccess) return e;
    dim3 grid((unsigned)nspans, (unsigned)((B + kWarpsA - 1) / kWarpsA));
    fp64a_main_kernel<<<grid, kWarpsA * 32, smem, s>>>(g, t, parts, B, sg, pa, list, cnt);
    return cudaGetLastError();
}

}  // namespace fs
