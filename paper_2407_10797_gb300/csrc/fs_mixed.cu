// fs_mixed.cu - the FS_MIXED path: FP64 anchors, exact fixed-point phase
// steps, FP32 response and products, FP64 partial sums.
//
// Per (particle, tile of 1024 bins) an anchor at the tile's central in-band bin
// k_a is evaluated in FP64 (double-double where the phase needs it):
//   Phi(k) = Phi_orb(f_k) - f_k d(t_{f_k})                  (App. A Eq. A3, Sec. IV)
//   Phi_orb(f_a + dk df) ~ c0 + c1 dk + c2 dk^2 + c3 dk^3    (Taylor, cycles)
//   t(f_a + dk df)       ~ t_a + t' df dk + t'' df^2 dk^2 / 2
// The phase polynomial is kept in 64-bit fixed point (units of 2^-64 cycle):
// integer arithmetic is exact modulo one cycle, so each lane walks its bins
// (step 32) by forward differences with no phase drift.  The Doppler phase and
// the antenna patterns are evaluated per bin as polynomials in the offset
// d(alpha) from the anchor's orbital phase alpha_a (FP32; the antenna
// patterns' constant terms in FP64), the phase goes through the SFU sincos,
// and the seven segment sums accumulate with compensation: each lane sums a
// tile's bins in FP32 (at most 16 terms per f32x2 half per single-segment
// piece), folds the tile's sum into a per-lane (sum, error) pair by an exact
// TwoSum, the pairs are combined across the warp by TwoSum as well (a
// reduce-scatter over the seven sums), and the result goes to FP64 partials that the solve kernel adds in FP64.  A tile whose quartic phase
// remainder exceeds 1e-6 cycle, whose t(f) remainder moves alpha by more than
// 1e-6 rad, or whose |d(alpha)| exceeds 0.06 rad is evaluated bin by bin in
// FP64 instead, so the mode stays correct on any grid.
#include <cfloat>
#include <climits>

#include "fs_internal.h"
#include "fs_device.cuh"

namespace fs {

constexpr int kTileMix = 1024;                        // bins per anchor: 32 lanes x 32 steps
constexpr int kTilesPerSpan = 32;                     // anchors per warp span (one per lane in phase A)
constexpr int kSpanMix = kTileMix * kTilesPerSpan;    // 32768 bins: H/T granularity of this path
constexpr int kWarpsMix = 8;                          // particles per CTA
// Polynomial degrees of the FP32 body: antenna pair in d(alpha), Doppler
// E (times d(alpha)) and Q (times dk) -- the full tier (mode 1) and the
// low-degree tier (mode 3) that tiles with a small d(alpha) range take
constexpr int kNGFull = 6, kNEFull = 4, kNQFull = 3;
constexpr int kNGLow = 3, kNELow = 2, kNQLow = 2;

struct Anchor {
    unsigned long long c[4];   // c0..c3 of the orbital-minus-Doppler phase polynomial, cycles mod 1, units 2^-64
    double Fpa, Fxa;           // F+ and Fx at alpha_a (FP64)
    float w1, w2;              // d(alpha) = w1 dk + w2 dk^2, rad
    float e[5];                // Doppler: AU cos(beta) f_a cos^(n)(alpha_a - phi)/n!, n = 1..5 (cycles)
    float q[4];                // Doppler: AU cos(beta) df cos^(n)(alpha_a - phi)/n!, n = 0..3 (cycles per bin)
    float Fd[6][2];            // F+^(n)(alpha_a)/n!, Fx^(n)(alpha_a)/n!, n = 1..6
    int ja, lo, hi;            // anchor bin and in-band range [lo, hi) of the tile, relative to the span start
    int mode;                  // 0: no in-band bin, 1: polynomial, 3: low-degree polynomial, 2: bin-by-bin FP64
};

// Bin-by-bin FP64 evaluation for tiles where the anchor expansion is not
// valid; returns the phase mod 1 and the rotated antenna pair (G1, G2).
// fallback_terms below turns them into the seven terms.
__device__ __noinline__ void eval_bin_fallback(const Particle& P, const Tables& tb, int64_t k, double alpha0,
                                               double2 cs, float* ph, float* G1, float* G2) {
    FreqPowers fw;
    fw.u = tb.u[k];
    fw.g0h = tb.g0h[k];
    fw.e19 = tb.e19[k];
    const BinEval ev = eval_bin_fp64(P, tb.fh[k], tb.fl[k], fw, tb.g0l[k], alpha0);
    *ph = (float)ev.frac;
    *G1 = (float)fma(cs.x, ev.Fp, cs.y * ev.Fx);
    *G2 = (float)fma(cs.x, ev.Fx, -cs.y * ev.Fp);
}

// The seven terms of one bin-by-bin FP64 bin (phase and antenna from
// eval_bin_fallback, FP32 sincos and products).
__device__ __forceinline__ void fallback_terms(float ph, float G1, float G2, float4 tw, float t7[7], float* cs_out,
                                               float* sn_out) {
    float sn, cs;
    __sincosf(6.283185307179586f * ph, &sn, &cs);
    const float zr = fmaf(tw.x, cs, -tw.y * sn);
    const float zi = fmaf(tw.x, sn, tw.y * cs);
    t7[0] = G1 * zr;
    t7[1] = G1 * zi;
    t7[2] = G2 * zr;
    t7[3] = G2 * zi;
    const float wg = tw.z * G1;
    t7[4] = wg * G1;
    t7[5] = wg * G2;
    t7[6] = tw.z * G2 * G2;
    *cs_out = cs;
    *sn_out = sn;
}

__device__ __noinline__ void make_anchor(const Grid& g, const Tables& tb, const Particle& P, int64_t span_lo, int64_t lo,
                            int64_t hi, Anchor& A) {
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
    // orbital phase mod 1 (double-double leading term, exact f t_c)
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
    const double T0 = P.P0h * g0h, T2 = P.P2 * u3, T3 = P.P3 * u2, T4 = P.P4 * u, Te = P.E0 * g0h * e19;
    double rest = T2 + T3 + T4 + Te;
    acc += rest - rint(rest);
    // derivatives of sum_m T_m (f/f_a)^{p_m}: d^n/df^n = sum_m p_m (p_m - 1) ... T_m / f^n
    // (S1, S2 in FP64: t_a to 1e-15 relative and c2 to 1e-10; S3, S4 only
    // enter c3, the alpha offset and the validity bound, where FP32 suffices)
    const double p0 = -5.0 / 3.0, p2 = -1.0, p3 = -2.0 / 3.0, p4 = -1.0 / 3.0, pe = -34.0 / 9.0;
    const double S1 = p0 * T0 + p2 * T2 + p3 * T3 + p4 * T4 + pe * Te;
    const double S2 = (p0 * (p0 - 1.0)) * T0 + (p2 * (p2 - 1.0)) * T2 + (p3 * (p3 - 1.0)) * T3 +
                      (p4 * (p4 - 1.0)) * T4 + (pe * (pe - 1.0)) * Te;
    const float T0f = (float)T0, T2f = (float)T2, T3f = (float)T3, T4f = (float)T4, Tef = (float)Te;
    constexpr float q30 = (float)(p0 * (p0 - 1.0) * (p0 - 2.0)), q32 = (float)(p2 * (p2 - 1.0) * (p2 - 2.0)),
                    q33 = (float)(p3 * (p3 - 1.0) * (p3 - 2.0)), q34 = (float)(p4 * (p4 - 1.0) * (p4 - 2.0)),
                    q3e = (float)(pe * (pe - 1.0) * (pe - 2.0));
    const float S3 = q30 * T0f + q32 * T2f + q33 * T3f + q34 * T4f + q3e * Tef;
    const float S4 = q30 * (float)(p0 - 3.0) * T0f + q32 * (float)(p2 - 3.0) * T2f + q33 * (float)(p3 - 3.0) * T3f +
                     q34 * (float)(p4 - 3.0) * T4f + q3e * (float)(pe - 3.0) * Tef;
    const double inv = 1.0 / fh;
    const double ta = P.tc + S1 * inv;           // t(f_a) = dPhi_orb/df
    const double d2 = S2 * inv * inv;            // dt/df
    const float invf = (float)inv;
    const float d3 = S3 * invf * invf * invf;    // d2t/df2
    const float d4 = S4 * invf * invf * invf * invf;
    // orbit and Doppler at the anchor
    const double Om = kTwoPi / kYearS;
    double sa, ca;
    sincos(fma(Om, ta, g.alpha0), &sa, &ca);
    const double cda = fma(ca, P.clon, sa * P.slon);   // cos(alpha_a - phi)
    const double sda = fma(sa, P.clon, -ca * P.slon);  // sin(alpha_a - phi)
    acc -= fh * P.AD * cda;
    const double df = g.df;
    const float dff = (float)df;
    A.c[0] = to_fixed(acc);
    A.c[1] = to_fixed(ta * df);
    A.c[2] = to_fixed_small(0.5 * d2 * df * df);
    A.c[3] = to_fixed_small((double)(d3 * dff * dff * dff) * (1.0 / 6.0));
    const float Omf = (float)Om;
    A.w1 = (float)(Om * d2 * df);
    A.w2 = 0.5f * Omf * d3 * dff * dff;
    // Doppler phase minus its anchor value, with x = alpha - phi = x_a + da:
    //   AD [f_a (cos x - cos x_a) + dk df cos x],  cos^(n)(x_a) cycles through (c, -s, -c, s)
    {
        const float cf = (float)cda, sf = (float)sda;
        const float cn[6] = {cf, -sf, -cf, sf, cf, -sf};
        const float inv_fact[6] = {1.f, 1.f, 0.5f, 1.f / 6.f, 1.f / 24.f, 1.f / 120.f};
        const float ADfa = (float)(P.AD * fh), ADdf = (float)(P.AD * df);
#pragma unroll
        for (int n = 1; n <= 5; n++) A.e[n - 1] = ADfa * cn[n] * inv_fact[n];
#pragma unroll
        for (int n = 0; n <= 3; n++) A.q[n] = ADdf * cn[n] * inv_fact[n];
    }
    // antenna: F(alpha_a + da) = sum_n F^(n)(alpha_a) da^n / n!, from the harmonics;
    // F(alpha_a) in FP64, the derivative terms (multiplied by da^n <= 0.06^n) in FP32
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
            float uu[5], vv[5];
#pragma unroll
            for (int h = 1; h <= 4; h++) {
                const double u_h = H[2 * h - 1] * ch[h] + H[2 * h] * sh[h];    // A cos + B sin
                F0 += u_h;
                uu[h] = (float)u_h;
                vv[h] = (float)(H[2 * h] * ch[h] - H[2 * h - 1] * sh[h]);   // derivative / h
            }
            if (f == 0) A.Fpa = F0; else A.Fxa = F0;
            // d^n/da^n of (u cos + v sin)-pairs: h^n (u, v, -u, -v)[n mod 4]
            const float inv_fact[7] = {1.f, 1.f, 0.5f, 1.f / 6.f, 1.f / 24.f, 1.f / 120.f, 1.f / 720.f};
#pragma unroll
            for (int n = 1; n <= 6; n++) {
                float sum = 0.f;
#pragma unroll
                for (int h = 1; h <= 4; h++) {
                    float hn = 1.f;
#pragma unroll
                    for (int j = 0; j < n; j++) hn *= (float)h;
                    const int r = n & 3;
                    const float t = (r == 0) ? uu[h] : (r == 1) ? vv[h] : (r == 2) ? -uu[h] : -vv[h];
                    sum = fmaf(hn, t, sum);
                }
                A.Fd[n - 1][f] = sum * inv_fact[n];
            }
        }
    }
    // validity of the truncated expansions over |dk| <= hmax
    const float hm = (float)hmax;
    const float H = hm * dff;
    const float rem_phase = 1.2f * fabsf(d4) * H * H * H * H * (1.f / 24.f);    // cycles
    const float rem_alpha = 1.2f * Omf * fabsf(d4) * H * H * H * (1.f / 6.f);    // rad
    const float da_max = fabsf(A.w1) * hm + fabsf(A.w2) * hm * hm;
    const bool finite = isfinite(rem_phase) && isfinite(da_max);
    A.mode = (finite && rem_phase <= 1e-6f && rem_alpha <= 1e-6f && da_max <= 0.06f) ? 1 : 2;
    if (A.mode == 1) {
        // low-degree tier (antenna degree kNGLow, Doppler terms to d(alpha)^(kNELow + 1) and
        // dk d(alpha)^kNQLow): the dropped terms, bounded over |d(alpha)| <= da_max, stay below
        // 2^-26 of the antenna pair's magnitude and below 1e-8 cycle of Doppler phase -- under the
        // FP32 rounding of the values they would have changed
        float tG = 0.f, sF = fabsf((float)A.Fpa) + fabsf((float)A.Fxa), p = 1.f;
        for (int n = 1; n <= 6; n++) {
            p *= da_max;
            const float t = (fabsf(A.Fd[n - 1][0]) + fabsf(A.Fd[n - 1][1])) * p;
            sF += t;
            if (n > kNGLow) tG += t;
        }
        float tD = 0.f;
        p = 1.f;
        for (int n = 1; n <= 5; n++) {
            p *= da_max;
            if (n > kNELow + 1) tD += fabsf(A.e[n - 1]) * p;
        }
        p = 1.f;
        for (int n = 0; n <= 3; n++) {
            if (n > kNQLow) tD += hm * fabsf(A.q[n]) * p;
            p *= da_max;
        }
        if (tG <= 0x1p-26f * sF && tD <= 1e-8f) A.mode = 3;
    }
}

// Coefficients of G1 = c F+ + s Fx and G2 = c Fx - s F+ in powers of d(alpha)
// for one (tile, segment): the constant terms in FP64 (G2 nearly cancels on a
// short segment), the others in FP32.
__device__ __forceinline__ void segment_coeffs(const Anchor& A, double2 r64, float2 r32, float g1[7], float g2[7]) {
    g1[0] = (float)fma(r64.x, A.Fpa, r64.y * A.Fxa);
    g2[0] = (float)fma(r64.x, A.Fxa, -r64.y * A.Fpa);
#pragma unroll
    for (int n = 1; n <= 6; n++) {
        g1[n] = fmaf(r32.x, A.Fd[n - 1][0], r32.y * A.Fd[n - 1][1]);
        g2[n] = fmaf(r32.x, A.Fd[n - 1][1], -r32.y * A.Fd[n - 1][0]);
    }
}

// Knuth's TwoSum in FP32: s + e = a + b exactly (round-to-nearest, no
// overflow).  The explicit _rn intrinsics keep the compiler from reassociating.
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated accumulation of x into the pair (s, c): s takes the rounded sum,
// c collects the exact rounding errors.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    float t, e;
    two_sum_f(s, x, t, e);
    s = t;
    c = __fadd_rn(c, e);
}

// One compensated TwoSum step of the flush below: the pair kept by this lane
// plus the partner's copy of the same slot.
__device__ __forceinline__ void comp_merge(float ks, float kc, float rs, float rc, float& s, float& c) {
    float t, e;
    two_sum_f(ks, rs, t, e);
    s = t;
    c = __fadd_rn(__fadd_rn(kc, rc), e);
}

// The warp's sums of the seven compensated pairs (s[i], c[i]) into dst[0..6]:
// a reduce-scatter butterfly over eight slots (the eighth zero).  At the XOR
// distances 16, 8 and 4 each lane keeps half of its slots -- the upper half
// if its lane bit is set -- and adds the partner's copies of them, so that
// after three steps lane l holds slot 4 b4 + 2 b3 + b2 (b_j bit j of l) of
// its group of eight; distances 2 and 1 then sum the four lanes that hold
// the same slot, and the first of them writes it.  Every addition is a
// TwoSum with the rounding errors carried in c.  9 merges instead of the 35
// of seven separate warp trees.
__device__ __forceinline__ void warp_flush7_comp(const float s[7], const float c[7], double* dst, int lane) {
    float S4[4], C4[4];
    const bool h16 = (lane & 16) != 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const float lo_s = s[i], lo_c = c[i];
        const float hi_s = i + 4 < 7 ? s[i + 4] : 0.f, hi_c = i + 4 < 7 ? c[i + 4] : 0.f;
        const float ks = h16 ? hi_s : lo_s, kc = h16 ? hi_c : lo_c;
        const float gs = h16 ? lo_s : hi_s, gc = h16 ? lo_c : hi_c;
        const float rs = __shfl_xor_sync(0xffffffffu, gs, 16), rc = __shfl_xor_sync(0xffffffffu, gc, 16);
        comp_merge(ks, kc, rs, rc, S4[i], C4[i]);
    }
    float S2[2], C2[2];
    const bool h8 = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const float ks = h8 ? S4[i + 2] : S4[i], kc = h8 ? C4[i + 2] : C4[i];
        const float gs = h8 ? S4[i] : S4[i + 2], gc = h8 ? C4[i] : C4[i + 2];
        const float rs = __shfl_xor_sync(0xffffffffu, gs, 8), rc = __shfl_xor_sync(0xffffffffu, gc, 8);
        comp_merge(ks, kc, rs, rc, S2[i], C2[i]);
    }
    float S1, C1;
    {
        const bool h4 = (lane & 4) != 0;
        const float ks = h4 ? S2[1] : S2[0], kc = h4 ? C2[1] : C2[0];
        const float gs = h4 ? S2[0] : S2[1], gc = h4 ? C2[0] : C2[1];
        const float rs = __shfl_xor_sync(0xffffffffu, gs, 4), rc = __shfl_xor_sync(0xffffffffu, gc, 4);
        comp_merge(ks, kc, rs, rc, S1, C1);
    }
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) {
        const float rs = __shfl_xor_sync(0xffffffffu, S1, o), rc = __shfl_xor_sync(0xffffffffu, C1, o);
        comp_merge(S1, C1, rs, rc, S1, C1);
    }
    const int slot = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
    if ((lane & 3) == 0 && slot < 7) dst[slot] = (double)S1 + (double)C1;
}

// Per-bin values of the FS_MIXED body that the probe entry point reports (one
// record of kProbeFields floats per bin; the probe reuses the production code,
// so the values are those the sums receive).
enum ProbeField {
    PR_MODE = 0,     // tile mode: 0 no anchor / out of band, 1 polynomial, 2 bin-by-bin FP64
    PR_KA,           // anchor bin of the tile (absolute)
    PR_SEG,          // segment index
    PR_ORB,          // fixed-point phase polynomial (orbital phase minus the anchor's Doppler phase), cycles
    PR_DALPHA,       // orbital-phase offset d(alpha) from the anchor, rad
    PR_DOP,          // Doppler phase minus its anchor value, cycles
    PR_PH,           // phase fed to the SFU sincos, cycles in [-1/2, 1/2]
    PR_G1, PR_G2,    // antenna pair in the segment's rotated basis
    PR_ROTC, PR_ROTS,  // the segment's rotation (c, s)
    PR_COS, PR_SIN,  // SFU cos / sin of 2 pi ph
    PR_TX, PR_TY, PR_TW,   // FP32 tables: dw (re, im), W (scaled by powers of two)
    PR_T0,           // the seven terms G1 zr, G1 zi, G2 zr, G2 zi, W G1^2, W G1 G2, W G2^2 (PR_T0 .. PR_T0 + 6)
    PR_ROTC_LO = PR_T0 + 7,   // c - (float)c and s - (float)s: the FP64 rotation as two floats each
    PR_ROTS_LO,
    kProbeFields = 28
};

// One bin of a polynomial tile inside a single segment: phase from the
// fixed-point value Fv, antenna and Doppler from the orbital-phase offset,
// seven sums into acc.
// Horner's scheme on the first N + 1 coefficients.
template <int N>
__device__ __forceinline__ float horner_f(const float* c, float x) {
    float v = c[N];
#pragma unroll
    for (int n = N - 1; n >= 0; n--) v = fmaf(v, x, c[n]);
    return v;
}

template <bool PROBE, int NG, int NE, int NQ>
__device__ __forceinline__ void mixed_bin(unsigned long long Fv, float d, float4 tw, float w1, float w2,
                                          const float g1[7], const float g2[7], const float e[5], const float q[4],
                                          float acc[7], float* pr = nullptr) {
    const float da = fmaf(w2, d, w1) * d;
    const float G1 = horner_f<NG>(g1, da);
    const float G2 = horner_f<NG>(g2, da);
    const float dop = fmaf(da, horner_f<NE>(e, da), d * horner_f<NQ>(q, da));
    float ph = fmaf((float)(int)(Fv >> 32), 2.3283064365386963e-10f, -dop);
    ph -= rintf(ph);
    float sn, cs;
    __sincosf(6.283185307179586f * ph, &sn, &cs);
    const float zr = fmaf(tw.x, cs, -tw.y * sn);
    const float zi = fmaf(tw.x, sn, tw.y * cs);
    if (PROBE) {
        pr[PR_ORB] = (float)(int)(Fv >> 32) * 2.3283064365386963e-10f;
        pr[PR_DALPHA] = da;
        pr[PR_DOP] = dop;
        pr[PR_PH] = ph;
        pr[PR_G1] = G1;
        pr[PR_G2] = G2;
        pr[PR_COS] = cs;
        pr[PR_SIN] = sn;
        pr[PR_TX] = tw.x;
        pr[PR_TY] = tw.y;
        pr[PR_TW] = tw.z;
        const float wg = tw.z * G1;
        pr[PR_T0 + 0] = G1 * zr;
        pr[PR_T0 + 1] = G1 * zi;
        pr[PR_T0 + 2] = G2 * zr;
        pr[PR_T0 + 3] = G2 * zi;
        pr[PR_T0 + 4] = wg * G1;
        pr[PR_T0 + 5] = wg * G2;
        pr[PR_T0 + 6] = tw.z * G2 * G2;
        return;
    }
    acc[0] = fmaf(G1, zr, acc[0]);
    acc[1] = fmaf(G1, zi, acc[1]);
    acc[2] = fmaf(G2, zr, acc[2]);
    acc[3] = fmaf(G2, zi, acc[3]);
    const float wg = tw.z * G1;
    acc[4] = fmaf(wg, G1, acc[4]);
    acc[5] = fmaf(wg, G2, acc[5]);
    acc[6] = fmaf(tw.z * G2, G2, acc[6]);
}

// Two FP32 lanes in one 64-bit register: the packed f32x2 arithmetic of
// sm_100-class GPUs does the same operation on both halves in one
// instruction, each half rounded as its scalar counterpart.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void up2(f32x2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Coefficients of one single-segment piece, each duplicated into both halves;
// the Doppler ones negated so that one fused chain gives minus the offset.
template <int NG, int NE, int NQ>
struct PairCoeffs {
    f32x2 w1, w2;
    f32x2 ne[NE + 1], nq[NQ + 1];
    f32x2 g1[NG + 1], g2[NG + 1];
};

// Bins k (low half) and k + 32 (high half) of a polynomial piece: the same
// operations as mixed_bin on both, sums into the packed accumulators.
template <int NG, int NE, int NQ>
__device__ __forceinline__ void mixed_pair(unsigned long long Fa, unsigned long long Fb, float d, float4 ta,
                                           float4 tb, const PairCoeffs<NG, NE, NQ>& C, f32x2 acc[7]) {
    const f32x2 D = pk2(d, d + 32.f);
    const f32x2 DA = mul2(fma2(C.w2, D, C.w1), D);
    f32x2 G1 = C.g1[NG], G2 = C.g2[NG];
#pragma unroll
    for (int n = NG - 1; n >= 0; n--) {
        G1 = fma2(G1, DA, C.g1[n]);
        G2 = fma2(G2, DA, C.g2[n]);
    }
    f32x2 E = C.ne[NE];
#pragma unroll
    for (int n = NE - 1; n >= 0; n--) E = fma2(E, DA, C.ne[n]);
    f32x2 Q = C.nq[NQ];
#pragma unroll
    for (int n = NQ - 1; n >= 0; n--) Q = fma2(Q, DA, C.nq[n]);
    const f32x2 ndop = fma2(DA, E, mul2(D, Q));
    const f32x2 ph = fma2(pk2((float)(int)(Fa >> 32), (float)(int)(Fb >> 32)), pk2(2.3283064365386963e-10f,
                          2.3283064365386963e-10f), ndop);
    float pa, pb;
    up2(ph, pa, pb);
    pa -= rintf(pa);
    pb -= rintf(pb);
    float sa, ca, sb, cb;
    __sincosf(6.283185307179586f * pa, &sa, &ca);
    __sincosf(6.283185307179586f * pb, &sb, &cb);
    const f32x2 CS = pk2(ca, cb), SN = pk2(sa, sb);
    // table entry (dw_re, dw_im, W, -dw_im)
    const f32x2 X = pk2(ta.x, tb.x), Y = pk2(ta.y, tb.y), Wt = pk2(ta.z, tb.z), YN = pk2(ta.w, tb.w);
    const f32x2 zr = fma2(X, CS, mul2(YN, SN));
    const f32x2 zi = fma2(X, SN, mul2(Y, CS));
    acc[0] = fma2(G1, zr, acc[0]);
    acc[1] = fma2(G1, zi, acc[1]);
    acc[2] = fma2(G2, zr, acc[2]);
    acc[3] = fma2(G2, zi, acc[3]);
    const f32x2 wg = mul2(Wt, G1);
    acc[4] = fma2(wg, G1, acc[4]);
    acc[5] = fma2(wg, G2, acc[5]);
    acc[6] = fma2(mul2(Wt, G2), G2, acc[6]);
}

// Whether particle b's band meets bins [lo, hi], and whether the span holds
// kHeavyBounds or more of its segment boundaries.
__device__ __forceinline__ void span_member(const Particle* __restrict__ parts, int B, const Segs& sg, int b,
                                            int64_t lo, int64_t hi, bool& in, bool& heavy) {
    in = heavy = false;
    if (b >= B || !parts[b].valid) return;
    const SegView sv = seg_view(sg, parts[b]);
    in = sv.lo <= sv.hi && sv.lo <= hi && sv.hi >= lo;
    if (in) heavy = sv.seg(sv.hi < hi ? sv.hi : hi) - sv.seg(sv.lo > lo ? sv.lo : lo) >= kHeavyBounds;
}

// In-band particles of every span: one warp per span.  list[span * B + j] is
// the j-th particle whose band meets the span -- the heavy ones (kHeavyBounds
// or more segment boundaries in the span) first, each class in increasing
// particle order -- cnt[span] their number and nh[span] the heavy ones', so
// no warp of the fused kernel idles on a particle that has no bin in the
// span.  With `off` given, the last CTA to finish (counted on ctl[0]) also
// writes the exclusive prefixes over spans of the heavy counts (off) and of
// the others (off_l), each with its total at [nspans], and resets the
// persistent kernel's item counter ctl[1] and ctl[0] itself to zero.
__global__ void span_lists_kernel(const Particle* __restrict__ parts, int B, Segs sg, int nspans, int span_len,
                                  int* list, int* cnt, int* off, int* ctl, int* nh, int* off_l) {
    const int lane = threadIdx.x & 31;
    const int span = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (span < nspans) {   // warp-uniform
        const int64_t lo = (int64_t)span * span_len, hi = lo + span_len - 1;
        const unsigned below = (1u << lane) - 1u;
        int nheavy = 0;
        for (int b0 = 0; b0 < B; b0 += 32) {
            bool in, heavy;
            span_member(parts, B, sg, b0 + lane, lo, hi, in, heavy);
            nheavy += __popc(__ballot_sync(0xffffffffu, in && heavy));
        }
        int wh = 0, wl = nheavy;
        for (int b0 = 0; b0 < B; b0 += 32) {
            const int b = b0 + lane;
            bool in, heavy;
            span_member(parts, B, sg, b, lo, hi, in, heavy);
            const unsigned mh = __ballot_sync(0xffffffffu, in && heavy), ml = __ballot_sync(0xffffffffu, in && !heavy);
            if (in) list[(int64_t)span * B + (heavy ? wh + __popc(mh & below) : wl + __popc(ml & below))] = b;
            wh += __popc(mh);
            wl += __popc(ml);
        }
        if (lane == 0) {
            cnt[span] = wl;
            nh[span] = nheavy;
        }
    }
    if (off == nullptr) return;   // uniform over the grid
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctl[0], 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    int run_h = 0, run_l = 0;
    for (int s0 = 0; s0 < nspans; s0 += 32) {
        const int s = s0 + lane;
        const int vh = s < nspans ? __ldcg(&nh[s]) : 0;
        const int vl = s < nspans ? __ldcg(&cnt[s]) - vh : 0;
        int xh = vh, xl = vl;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int yh = __shfl_up_sync(0xffffffffu, xh, o), yl = __shfl_up_sync(0xffffffffu, xl, o);
            if (lane >= o) {
                xh += yh;
                xl += yl;
            }
        }
        if (s < nspans) {
            off[s] = run_h + xh - vh;
            off_l[s] = run_l + xl - vl;
        }
        run_h += __shfl_sync(0xffffffffu, xh, 31);
        run_l += __shfl_sync(0xffffffffu, xl, 31);
    }
    if (lane == 0) {
        off[nspans] = run_h;
        off_l[nspans] = run_l;
        ctl[1] = 0;
        ctl[0] = 0;
    }
}

cudaError_t launch_span_lists(const Particle* parts, int B, const Segs& sg, int nspans, int span_len, int* list,
                              int* cnt, bool offsets, cudaStream_t s) {
    int* off = cnt + nspans;
    int* ctl = cnt + 2 * nspans + 1;
    int* nh = cnt + 2 * nspans + 4;
    int* off_l = cnt + 3 * nspans + 4;
    span_lists_kernel<<<(unsigned)((nspans * 32 + 255) / 256), 256, 0, s>>>(
        parts, B, sg, nspans, span_len, list, cnt, offsets ? off : nullptr, ctl, nh, off_l);
    return cudaGetLastError();
}

// Phase A of a work item (particle b over span `span`, one warp): one anchor
// per lane (tile `lane` of the span) into the warp's 32 anchor slots.
__device__ __forceinline__ void mixed_anchors(const Grid& g, const Tables& tb, const Particle& P, const SegView& sv,
                                              const Partials& pa, int64_t span_lo, Anchor* anc, int lane) {
    int64_t lo = span_lo + (int64_t)lane * kTileMix, hi = lo + kTileMix;
    if (lo < sv.lo) lo = sv.lo;
    if (hi > sv.hi + 1) hi = sv.hi + 1;
    make_anchor(g, tb, P, span_lo, lo, hi, anc[lane]);
    if (pa.census && lo < hi) atomicAdd(&pa.census[anc[lane].mode], (unsigned long long)(hi - lo));
    __syncwarp();
}

// Table source of phase B: every warp reads the span's FP32 tables from
// global memory (served by L2 when several particles share a span).
struct GlobalTables {
    const float4* tw_span;
    __device__ int first() const { return 0; }
    __device__ int last() const { return kTilesPerSpan - 1; }
    __device__ const float4* begin(int) const { return tw_span; }   // indexed by span-relative bin
    __device__ void end(int, int) const {}
};

// The bins [pa_lo, pa_hi) of one single-segment piece of a polynomial tile
// with antenna degree NG and Doppler degrees NE, NQ: each lane walks bins
// pa_lo + lane + 32 j, two per iteration (k and k + 32, the f32x2 halves),
// the fixed-point phase by forward differences; sums into acc.
template <int NG, int NE, int NQ>
__device__ __forceinline__ void piece_bins(const Anchor& A, int pa_lo, int pa_hi, int lane, const float4* tw_span,
                                           const float g1[7], const float g2[7], const float e[5], const float q[4],
                                           float acc[7]) {
    const float w1 = A.w1, w2 = A.w2;
    const int k0 = pa_lo + lane;
    const long long d0 = (long long)(k0 - A.ja);
    const unsigned long long y0 = poly_fx(A.c, d0), y1 = poly_fx(A.c, d0 + 32),
                             y2 = poly_fx(A.c, d0 + 64), y3 = poly_fx(A.c, d0 + 96);
    unsigned long long F = y0, D1 = y1 - y0, D2 = y2 - 2ull * y1 + y0,
                       D3 = y3 - 3ull * y2 + 3ull * y1 - y0;
    float d = (float)(k0 - A.ja);
    int k = k0;
    if (k + 32 < pa_hi) {
        // two bins per lane per iteration (k and k + 32), packed into f32x2 halves
        PairCoeffs<NG, NE, NQ> C;
        C.w1 = pk2(w1, w1);
        C.w2 = pk2(w2, w2);
#pragma unroll
        for (int n = 0; n <= NE; n++) C.ne[n] = pk2(-e[n], -e[n]);
#pragma unroll
        for (int n = 0; n <= NQ; n++) C.nq[n] = pk2(-q[n], -q[n]);
#pragma unroll
        for (int n = 0; n <= NG; n++) {
            C.g1[n] = pk2(g1[n], g1[n]);
            C.g2[n] = pk2(g2[n], g2[n]);
        }
        f32x2 acc2[7];
#pragma unroll
        for (int c = 0; c < 7; c++) acc2[c] = 0ull;   // (+0.0f, +0.0f)
        for (; k + 32 < pa_hi; k += 64, d += 64.f) {
            const float4 twa = tw_span[k];
            const float4 twb = tw_span[k + 32];
            const unsigned long long Fa = F, Fb = F + D1;
            F = Fb + D1 + D2;
            D1 += 2ull * D2 + D3;
            D2 += 2ull * D3;
            mixed_pair(Fa, Fb, d, twa, twb, C, acc2);
        }
#pragma unroll
        for (int c = 0; c < 7; c++) {
            float lo2, hi2;
            up2(acc2[c], lo2, hi2);
            acc[c] += lo2 + hi2;
        }
    }
    if (k < pa_hi) mixed_bin<false, NG, NE, NQ>(F, d, tw_span[k], w1, w2, g1, g2, e, q, acc);
}

// Phase B: the warp walks tiles first()..last() of the span with the table
// source Src (begin(ti) gives the tile's table entries, indexed by
// span-relative bin, or NULL to stop; end(ti) releases them).  Partial sums
// go to the slots of (b, span) and to the per-segment slots of the segments
// that start and end inside the span.
template <class Src>
__device__ __forceinline__ void mixed_walk(const Grid& g, const Tables& tb, const Particle& P, const SegView& sv,
                                           const Segs& sg, const Partials& pa, int span, int b, const Anchor* anc,
                                           int lane, Src& src) {
    const int64_t span_lo = (int64_t)span * kSpanMix;
    const int64_t slot = (int64_t)b * pa.ntiles + span;
    const double2* rot64 = pa.rot + (int64_t)b * sg.Np;
    const float2* rot32 = pa.rot32 + (int64_t)b * sg.Np;

    // acc: this tile's FP32 sums; (accS, accC): the compensated per-lane sums
    // of the tiles since the last flush
    float accS[7], accC[7], acc[7];
#pragma unroll
    for (int c = 0; c < 7; c++) accS[c] = accC[c] = 0.f;
    int cur = -1;        // warp-uniform current segment
    int nflush = 0;
    int pk = -1;         // this lane's segment
    int nxt = -1;        // first bin (span-relative) of the segment after pk
    int trk = -1;        // warp-uniform segment of the latest piece start (polynomial tiles) and
    int64_t trk_nxt = 0; // the first bin (absolute) of the segment after it
    float g1[7], g2[7];

    for (int ti = src.first(); ti <= src.last(); ti++) {
        const float4* tw_span = src.begin(ti);
        if (!tw_span) break;   // the staged source gave up waiting (flag set)
        const Anchor& A = anc[ti];
        if (A.mode == 0) {
            src.end(ti, lane);
            continue;
        }
        const int lo = A.lo, hi = A.hi;
        if (cur < 0) cur = sv.seg(span_lo + lo);
#pragma unroll
        for (int c = 0; c < 7; c++) acc[c] = 0.f;
        if (A.mode == 1 || A.mode == 3) {
            // polynomial tile, walked as single-segment pieces [pa_lo, pa_hi)
            const float e[5] = {A.e[0], A.e[1], A.e[2], A.e[3], A.e[4]};
            const float q[4] = {A.q[0], A.q[1], A.q[2], A.q[3]};
            int pa_lo = lo;
            while (pa_lo < hi) {
                // segment of the piece's first bin (sv.seg of it), tracked forward: piece starts only
                // increase within a work item, so a segment boundary costs one sv.start
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
                    // segment `cur` ended before this piece: flush it
                    double* dst = (nflush == 0) ? pa.H + slot * 7 : pa.S + ((int64_t)b * sg.Np + cur) * 7;
#pragma unroll
                    for (int c = 0; c < 7; c++) comp_add(accS[c], accC[c], acc[c]);
                    warp_flush7_comp(accS, accC, dst, lane);
#pragma unroll
                    for (int c = 0; c < 7; c++) accS[c] = accC[c] = acc[c] = 0.f;
                    nflush++;
                    cur = sp;
                }
                const int64_t nb = trk_nxt - span_lo;
                const int pa_hi = nb < hi ? (int)nb : hi;
                segment_coeffs(A, rot64[sp], rot32[sp], g1, g2);
                if (A.mode == 1)
                    piece_bins<kNGFull, kNEFull, kNQFull>(A, pa_lo, pa_hi, lane, tw_span, g1, g2, e, q, acc);
                else
                    piece_bins<kNGLow, kNELow, kNQLow>(A, pa_lo, pa_hi, lane, tw_span, g1, g2, e, q, acc);
                pa_lo = pa_hi;
            }
            // lanes' segment trackers are stale after this tile; the fallback path re-derives them
            pk = -1;
            nxt = -1;
        } else {
            // bin-by-bin FP64 tile (anchor expansion not valid)
            for (int base = lo; base < hi; base += 32) {
                const int k = base + lane;
                const bool valid = k < hi;
                float t7[7];
#pragma unroll
                for (int c = 0; c < 7; c++) t7[c] = 0.f;
                if (valid) {
                    const float4 tw = tw_span[k];
                    if (k >= nxt) {
                        pk = sv.seg(span_lo + k);
                        nxt = (int)(sv.start(pk + 1) - span_lo);
                    }
                    float ph, G1, G2, cs, sn;
                    eval_bin_fallback(P, tb, span_lo + k, g.alpha0, rot64[pk], &ph, &G1, &G2);
                    fallback_terms(ph, G1, G2, tw, t7, &cs, &sn);
                }
                while (true) {
                    if (valid && pk == cur) {
#pragma unroll
                        for (int c = 0; c < 7; c++) acc[c] += t7[c];
                    }
                    const unsigned more = __ballot_sync(0xffffffffu, valid && pk > cur);
                    if (!more) break;
                    double* dst = (nflush == 0) ? pa.H + slot * 7 : pa.S + ((int64_t)b * sg.Np + cur) * 7;
#pragma unroll
                    for (int c = 0; c < 7; c++) comp_add(accS[c], accC[c], acc[c]);
                    warp_flush7_comp(accS, accC, dst, lane);
#pragma unroll
                    for (int c = 0; c < 7; c++) accS[c] = accC[c] = acc[c] = 0.f;
                    nflush++;
                    int cand = (valid && pk > cur) ? pk : INT_MAX;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, o));
                    cur = cand;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 7; c++) comp_add(accS[c], accC[c], acc[c]);
        src.end(ti, lane);
    }
    if (cur < 0) return;   // no in-band bin in this span (warp-uniform)
    warp_flush7_comp(accS, accC, (nflush == 0) ? pa.H + slot * 7 : pa.T + slot * 7, lane);
}

// One work item, both phases, tables from global memory.
__device__ __forceinline__ void mixed_item(const Grid& g, const Tables& tb, const float4* __restrict__ t32,
                                           const Particle* __restrict__ parts, const Segs& sg, const Partials& pa,
                                           int span, int b, Anchor* anc, int lane) {
    const int64_t span_lo = (int64_t)span * kSpanMix;
    const Particle& P = parts[b];
    const SegView sv = seg_view(sg, P);
    mixed_anchors(g, tb, P, sv, pa, span_lo, anc, lane);
    GlobalTables src{t32 + span_lo};
    mixed_walk(g, tb, P, sv, sg, pa, span, b, anc, lane, src);
}

// Grid form: CTA (span, group of 8 in-band particles of the span), one warp per particle.
template <int MINB>
__global__ void __launch_bounds__(kWarpsMix * 32, MINB)
mixed_main_kernel(Grid g, Tables tb, const float4* __restrict__ t32, const Particle* __restrict__ parts, int B,
                  Segs sg, Partials pa, const int* __restrict__ list, const int* __restrict__ cnt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Anchor* anc = reinterpret_cast<Anchor*>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int span = blockIdx.x;
    const int j = blockIdx.y * kWarpsMix + w;
    if (j >= cnt[span]) return;   // warp-uniform
    mixed_item(g, tb, t32, parts, sg, pa, span, list[(int64_t)span * B + j], anc + w * 32, lane);
}

// Persistent form: a grid of (SMs x resident CTAs) whose warps take work
// items (span, in-band particle) from a shared counter -- every heavy item
// (many segment boundaries in the span) first, then the others, each class
// in span-major order -- until the list is exhausted.  No warp waits on
// another: a warp that finds the counter past the end returns.
template <int MINB>
__global__ void __launch_bounds__(kWarpsMix * 32, MINB)
mixed_persistent_kernel(Grid g, Tables tb, const float4* __restrict__ t32, const Particle* __restrict__ parts,
                        int B, Segs sg, Partials pa, const int* __restrict__ list, const int* __restrict__ sched,
                        int nspans, int* ctl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Anchor* anc = reinterpret_cast<Anchor*>(smem_raw) + (threadIdx.x >> 5) * 32;
    const int lane = threadIdx.x & 31;
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&ctl[1], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        int span, b;
        if (!sched_item(sched, nspans, B, list, item, span, b)) break;
        __syncwarp();   // every lane is done with the previous item's anchors
        mixed_item(g, tb, t32, parts, sg, pa, span, b, anc, lane);
    }
}

// ---------------------------------------------------------------------------
// Staged form: the CTA's 8 warps take 8 in-band particles of one span and
// walk its tiles together.  Each 1024-bin tile of FP32 tables (16 KB) is
// copied once per CTA from global memory into a ring of kStageBufs
// shared-memory buffers by a bulk asynchronous copy (cp.async.bulk, the TMA
// engine) and read by all 8 warps, instead of by each warp from L2.  Per
// buffer a "full" mbarrier (one arrival plus the copy's transaction bytes)
// tells the warps that a tile has landed, an "empty" mbarrier (one arrival
// per warp) tells the copying thread (thread 0, which also computes) that
// every warp is done with it.  Every wait is bounded: a wait that runs out
// sets kFlagTimeout in the plan's flag word and a CTA-wide abort flag, the
// warps stop, and thread 0 waits (bounded) for its copies still in flight
// before the CTA exits.  The per-bin arithmetic and the order of every sum
// are those of the other forms, so F is bit-identical to them.
// ---------------------------------------------------------------------------
constexpr int kStageBufs = 4;
constexpr long long kMaxPolls = 1LL << 24;
constexpr size_t kStageSmem = (size_t)kStageBufs * kTileMix * sizeof(float4) + sizeof(Anchor) * kWarpsMix * 32 +
                              2 * kStageBufs * sizeof(unsigned long long) + 4 * sizeof(int);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase with the given parity to complete (at most `polls` polls).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, uint32_t parity, long long polls = kMaxPolls) {
    const uint32_t a = smem_u32(bar);
    for (long long i = 0; i < polls; i++) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// One bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Self-test of the timeout path: one thread initialises an mbarrier that
// nothing arrives at and waits for its phase with a short bound (4096 polls);
// the wait runs out and the kernel sets kFlagTimeout in the plan's flag word
// and returns, as the staged kernel does when a copy never lands.
__global__ void wait_probe_kernel(int* flags) {
    __shared__ unsigned long long bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0u, 4096)) atomicOr(flags, kFlagTimeout);
}

struct StagedTables {
    float4* buf;                   // [kStageBufs][kTileMix] shared
    unsigned long long* full;      // [kStageBufs]
    unsigned long long* empty;     // [kStageBufs]
    volatile int* abort_flag;      // shared: a wait of this CTA ran out
    int* flags;                    // the plan's sticky flag word
    const float4* g_span;          // the span's FP32 tables in global memory
    int64_t bins_left;             // bins of the grid from the span's start
    int t0, t1;                    // tiles of the CTA's walk
    int issued;                    // thread 0: last tile whose copy was issued
    int waited;                    // thread 0: last tile whose copy it saw land

    __device__ int first() const { return t0; }
    __device__ int last() const { return t1; }
    __device__ int slot(int ti) const { return (ti - t0) % kStageBufs; }
    __device__ uint32_t parity(int ti) const { return (uint32_t)((ti - t0) / kStageBufs) & 1u; }
    __device__ void fail() {
        *abort_flag = 1;
        atomicOr(flags, kFlagTimeout);
    }
    // thread 0: copy tile j into its slot
    __device__ void issue(int j) {
        int64_t nb = bins_left - (int64_t)j * kTileMix;
        if (nb > kTileMix) nb = kTileMix;
        const uint32_t bytes = (uint32_t)nb * (uint32_t)sizeof(float4);
        const int s = slot(j);
        mbar_arrive_tx(&full[s], bytes);
        bulk_copy(buf + (size_t)s * kTileMix, g_span + (int64_t)j * kTileMix, bytes, &full[s]);
        issued = j;
    }
    __device__ const float4* begin(int ti) {
        if (*abort_flag) return nullptr;
        if (!mbar_wait(&full[slot(ti)], parity(ti))) {
            fail();
            return nullptr;
        }
        if (threadIdx.x == 0) waited = ti;
        return buf + (size_t)slot(ti) * kTileMix - (int64_t)ti * kTileMix;
    }
    __device__ void end(int ti, int lane) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[slot(ti)]);
        if (threadIdx.x == 0 && ti + kStageBufs <= t1 && !*abort_flag) {
            // every warp is done with tile ti: its buffer takes tile ti + kStageBufs
            if (mbar_wait(&empty[slot(ti)], parity(ti))) issue(ti + kStageBufs);
            else fail();
        }
    }
    // thread 0, before the CTA exits: wait (bounded) for copies it issued and has not seen land
    __device__ void drain() {
        for (int j = waited + 1; j <= issued; j++)
            if (!mbar_wait(&full[slot(j)], parity(j))) atomicOr(flags, kFlagTimeout);
    }
};

template <int MINB>
__global__ void __launch_bounds__(kWarpsMix * 32, MINB)
mixed_staged_kernel(Grid g, Tables tb, const float4* __restrict__ t32, const Particle* __restrict__ parts, int B,
                    Segs sg, Partials pa, const int* __restrict__ list, const int* __restrict__ cnt) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float4* buf = reinterpret_cast<float4*>(smem_raw);
    Anchor* anc_all = reinterpret_cast<Anchor*>(smem_raw + (size_t)kStageBufs * kTileMix * sizeof(float4));
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(anc_all + kWarpsMix * 32);
    int* sh = reinterpret_cast<int*>(bars + 2 * kStageBufs);   // [0] first tile, [1] last tile, [2] abort
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int span = blockIdx.x;
    const int n_here = cnt[span];
    if ((int)blockIdx.y * kWarpsMix >= n_here) return;   // CTA-uniform: no particle for this CTA
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStageBufs; s++) {
            mbar_init(&bars[s], 1);                     // full: the copying thread's arrival + bytes
            mbar_init(&bars[kStageBufs + s], kWarpsMix);  // empty: one arrival per warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh[0] = INT_MAX;
        sh[1] = -1;
        sh[2] = 0;
    }
    __syncthreads();
    const int64_t span_lo = (int64_t)span * kSpanMix;
    const int j = blockIdx.y * kWarpsMix + w;
    Anchor* anc = anc_all + w * 32;
    int b = -1;
    SegView sv{};
    if (j < n_here) {   // warp-uniform
        b = list[(int64_t)span * B + j];
        sv = seg_view(sg, parts[b]);
        mixed_anchors(g, tb, parts[b], sv, pa, span_lo, anc, lane);
        const unsigned m = __ballot_sync(0xffffffffu, anc[lane].mode != 0);
        if (lane == 0 && m) {
            atomicMin(&sh[0], __ffs(m) - 1);
            atomicMax(&sh[1], 31 - __clz(m));
        }
    }
    __syncthreads();
    StagedTables src;
    src.buf = buf;
    src.full = bars;
    src.empty = bars + kStageBufs;
    src.abort_flag = sh + 2;
    src.flags = pa.flags;
    src.g_span = t32 + span_lo;
    src.bins_left = g.n - span_lo;
    src.t0 = sh[0];
    src.t1 = sh[1];
    src.issued = src.t0 - 1;
    src.waited = src.t0 - 1;
    if (src.t0 > src.t1) return;   // CTA-uniform: no in-band tile
    if (threadIdx.x == 0)
        for (int t = src.t0; t <= src.t1 && t < src.t0 + kStageBufs; t++) src.issue(t);
    if (b >= 0) {
        mixed_walk(g, tb, parts[b], sv, sg, pa, span, b, anc, lane, src);
    } else {
        // a warp without a particle still takes part in every tile's hand-over
        for (int ti = src.t0; ti <= src.t1; ti++) {
            if (!src.begin(ti)) break;
            src.end(ti, lane);
        }
    }
    if (threadIdx.x == 0) src.drain();
}

cudaError_t launch_mixed_main(const Grid& g, const Tables& t, const float4* t32, const Particle* parts, int B,
                              const Segs& sg, const Partials& pa, int variant, int* list, int* cnt,
                              cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const int nspans = pa.ntiles;
    const bool persistent = variant == 2 || variant == 3;
    int* off = cnt + nspans;            // [nspans + 1]
    int* ctl = cnt + 2 * nspans + 1;    // [3]: CTAs done, next item, spare
    const size_t smem = sizeof(Anchor) * kWarpsMix * 32;
    cudaError_t e = launch_span_lists(parts, B, sg, nspans, kSpanMix, list, cnt, persistent, s);
    if (e != cudaSuccess) return e;
    if (persistent) {
        const bool three = variant == 3;
        const int grid = three ? persistent_grid(mixed_persistent_kernel<3>, kWarpsMix * 32, smem, 1)
                               : persistent_grid(mixed_persistent_kernel<2>, kWarpsMix * 32, smem, 0);
        if (grid <= 0) return cudaErrorInvalidConfiguration;
        if (three)
            mixed_persistent_kernel<3><<<grid, kWarpsMix * 32, smem, s>>>(g, t, t32, parts, B, sg, pa, list, cnt,
                                                                          nspans, ctl);
        else
            mixed_persistent_kernel<2><<<grid, kWarpsMix * 32, smem, s>>>(g, t, t32, parts, B, sg, pa, list, cnt,
                                                                          nspans, ctl);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)nspans, (unsigned)((B + kWarpsMix - 1) / kWarpsMix));
    if (variant == 4) {
        static int attr_set[64];
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!attr_set[dev]) {
            if ((e = cudaFuncSetAttribute(mixed_staged_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kStageSmem)) != cudaSuccess)
                return e;
            attr_set[dev] = 1;
        }
        mixed_staged_kernel<2><<<grid, kWarpsMix * 32, kStageSmem, s>>>(g, t, t32, parts, B, sg, pa, list, cnt);
        return cudaGetLastError();
    }
    if (variant == 1)
        mixed_main_kernel<3><<<grid, kWarpsMix * 32, smem, s>>>(g, t, t32, parts, B, sg, pa, list, cnt);
    else
        mixed_main_kernel<2><<<grid, kWarpsMix * 32, smem, s>>>(g, t, t32, parts, B, sg, pa, list, cnt);
    return cudaGetLastError();
}

int mixed_span() { return kSpanMix; }

// ---------------------------------------------------------------------------
// Probe: per-bin values of the FS_MIXED body for one particle over the bins
// [k0, k1), one warp per span of 32768 bins.  Phase A is the production
// anchor computation (same tiles, same band clipping); phase B evaluates each
// requested bin with the production per-bin code (mixed_bin with the probe
// record, or the bin-by-bin FP64 fallback), the fixed-point phase taken from
// the anchor polynomial directly (integer arithmetic: the same value the
// forward differences reach).  Nothing is accumulated.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32, 1)
mixed_probe_kernel(Grid g, Tables tb, const float4* __restrict__ t32, const Particle* __restrict__ parts, Segs sg,
                   Partials pa, int b, int64_t k0, int64_t k1, float* __restrict__ out) {
    __shared__ Anchor anc[kTilesPerSpan];
    const int lane = threadIdx.x;
    const int64_t span = k0 / kSpanMix + blockIdx.x;
    const int64_t span_lo = span * kSpanMix;
    const Particle& P = parts[b];
    const SegView sv = seg_view(sg, P);
    const bool live = P.valid && sv.lo <= sv.hi;
    {
        int64_t lo = span_lo + (int64_t)lane * kTileMix, hi = lo + kTileMix;
        if (lo < sv.lo) lo = sv.lo;
        if (hi > sv.hi + 1) hi = sv.hi + 1;
        if (!live) hi = lo;
        make_anchor(g, tb, P, span_lo, lo, hi, anc[lane]);
    }
    __syncwarp();
    const double2* rot64 = pa.rot + (int64_t)b * sg.Np;
    const float2* rot32 = pa.rot32 + (int64_t)b * sg.Np;
    int64_t a = span_lo > k0 ? span_lo : k0;
    int64_t e = span_lo + kSpanMix < k1 ? span_lo + kSpanMix : k1;
    const float qnan = __int_as_float(0x7fc00000);
    for (int64_t k = a + lane; k < e; k += 32) {
        float* pr = out + (k - k0) * kProbeFields;
#pragma unroll 1
        for (int f = 0; f < kProbeFields; f++) pr[f] = qnan;
        const Anchor& A = anc[(k - span_lo) / kTileMix];
        const int rel = (int)(k - span_lo);
        if (A.mode == 0 || rel < A.lo || rel >= A.hi) {
            pr[PR_MODE] = 0.f;
            continue;
        }
        const int sp = sv.seg(k);
        pr[PR_MODE] = (float)A.mode;
        pr[PR_KA] = (float)(span_lo + A.ja);
        pr[PR_SEG] = (float)sp;
        pr[PR_ROTC] = (float)rot64[sp].x;
        pr[PR_ROTS] = (float)rot64[sp].y;
        pr[PR_ROTC_LO] = (float)(rot64[sp].x - (double)(float)rot64[sp].x);
        pr[PR_ROTS_LO] = (float)(rot64[sp].y - (double)(float)rot64[sp].y);
        const float4 tw = t32[k];
        if (A.mode == 1 || A.mode == 3) {
            float g1[7], g2[7], acc[7];
            segment_coeffs(A, rot64[sp], rot32[sp], g1, g2);
            const float e5[5] = {A.e[0], A.e[1], A.e[2], A.e[3], A.e[4]};
            const float q4[4] = {A.q[0], A.q[1], A.q[2], A.q[3]};
            const long long d = (long long)(rel - A.ja);
            if (A.mode == 1)
                mixed_bin<true, kNGFull, kNEFull, kNQFull>(poly_fx(A.c, d), (float)d, tw, A.w1, A.w2, g1, g2, e5, q4,
                                                           acc, pr);
            else
                mixed_bin<true, kNGLow, kNELow, kNQLow>(poly_fx(A.c, d), (float)d, tw, A.w1, A.w2, g1, g2, e5, q4,
                                                        acc, pr);
        } else {
            float ph, G1, G2, cs, sn, t7[7];
            eval_bin_fallback(P, tb, k, g.alpha0, rot64[sp], &ph, &G1, &G2);
            fallback_terms(ph, G1, G2, tw, t7, &cs, &sn);
            pr[PR_PH] = ph;
            pr[PR_G1] = G1;
            pr[PR_G2] = G2;
            pr[PR_COS] = cs;
            pr[PR_SIN] = sn;
            pr[PR_TX] = tw.x;
            pr[PR_TY] = tw.y;
            pr[PR_TW] = tw.z;
            for (int c = 0; c < 7; c++) pr[PR_T0 + c] = t7[c];
        }
    }
}

cudaError_t launch_mixed_probe(const Grid& g, const Tables& t, const float4* t32, const Particle* parts,
                               const Segs& sg, const Partials& pa, int b, int64_t k0, int64_t k1, float* out,
                               cudaStream_t s) {
    if (k1 <= k0) return cudaSuccess;
    const int64_t nspans = (k1 - 1) / kSpanMix - k0 / kSpanMix + 1;
    mixed_probe_kernel<<<(unsigned)nspans, 32, 0, s>>>(g, t, t32, parts, sg, pa, b, k0, k1, out);
    return cudaGetLastError();
}

int mixed_probe_fields() { return kProbeFields; }

// ---------------------------------------------------------------------------
// FP32 tables of the mixed path: (dw_re, dw_im, W) scaled by powers of two so
// that max W ~ 1 (F is invariant under (d, S) -> (c d, c^2 S), and a power of
// two changes no mantissa).  With several channels the scale is common to
// all of them: F is invariant under one scale for every channel, not under
// one per channel.
// ---------------------------------------------------------------------------
__global__ void w_exponent_kernel(Grid g, Tables t, int* emax) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int e = INT_MIN;
    if (k < g.n) {
        const double W = t.W[k];
        if (W > 0.0 && isfinite(W)) e = ilogb(W);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0 && e != INT_MIN) atomicMax(emax, e);
}

__global__ void tables32_kernel(Grid g, Tables t, const int* emax, float4* t32) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n) return;
    int e = *emax;
    e += e & 1;                       // even, so that the data scale is an exact power of two too
    const double sW = ldexp(1.0, -e), sd = ldexp(1.0, -e / 2);
    const float di = (float)(t.dwi[k] * sd);
    t32[k] = make_float4((float)(t.dwr[k] * sd), di, (float)(t.W[k] * sW), -di);
}

cudaError_t launch_tables32(const Grid& g, const Tables* t, int nch, int* emax, float4* t32, cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = (g.n + threads - 1) / threads;
    cudaError_t e = cudaMemsetAsync(emax, 0x80, sizeof(int), s);   // INT_MIN-ish start (0x80808080)
    if (e != cudaSuccess) return e;
    for (int c = 0; c < nch; c++) {
        w_exponent_kernel<<<(unsigned)blocks, threads, 0, s>>>(g, t[c], emax);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int c = 0; c < nch; c++) {
        tables32_kernel<<<(unsigned)blocks, threads, 0, s>>>(g, t[c], emax, t32 + (size_t)c * g.n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace fs

namespace fs {
cudaError_t launch_wait_probe(int* flags, cudaStream_t s) {
    wait_probe_kernel<<<1, 32, 0, s>>>(flags);
    return cudaGetLastError();
}
}  // namespace fs
