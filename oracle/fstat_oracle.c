/*
 * Plain, slow CPU oracle for the semi-coherent F-statistic of the hierarchical
 * SmBBH search (Fu, Wang, Mohanty, arXiv:2407.10797).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant generator with
 * the CUDA library: every formula below is written out again from the paper.
 *
 * Precision: FP64 throughout, except the template phase, which is evaluated in
 * long double (the phase reaches 1e8 rad, where one FP64 ulp is 1e-8 rad).
 * Compile with -ffp-contract=off so that the same source gives the same bits
 * on x86-64 and aarch64.
 *
 * What each part follows:
 *   inner product            Sec. II.A, Eq. (inner_product)
 *   amplitude basis A^i      Sec. II.A, Eq. (response)
 *   F = 1/2 N^T M^-1 N       Sec. II.A, Eqs. (coherent_F_stat), (aandMN)-(aandMN3)
 *   segments, F-hat          Sec. II.B, Eq. (semi-cohF) and the segment inner product
 *   segment outer edges      Sec. II.B, last paragraph before Fig. 1
 *   waveform h(f), Psi(f)    Appendix A, Eqs. (A1)-(A3)
 *   response x(f) = T(f)h(f) Sec. IV, Eq. (freDres) with N = 0 and no higher d(t) terms
 *                            (the paper's form), or the series of Eq. (freDres) itself: the
 *                            filter F^N_{T_f} of order N <= 2 and the terms k <= 1, with the
 *                            retarded time and the ddot(t) factors of its kernel G (or_mb_response)
 *   t(f)                     Sec. IV, stationary-phase time t_f = (1/2pi) dPhi/df
 *   PSO update               Sec. III.A, Eqs. (pso_position_update), (pso_velocity_update)
 *   extrinsic parameters     Appendix B, Eqs. (B1)-(B3)
 *   several TDI channels     Sec. II.A, Eq. (eq2): the log-likelihood sums over the
 *                            combinations I, so N and M of a segment are sums over channels
 *   finite-arm TDI response  Sec. IV (a TDI combination is a sum of time-delayed single-arm
 *                            responses): first-generation Michelsons built from the retarded
 *                            link responses of the constellation frozen at t_f (or_tdi_response)
 *
 * Readings of points the paper leaves open:
 *   - PN coefficients alpha_k: non-spinning TaylorF2 through 2PN (k <= 4).
 *   - phi_e: leading-order e0^2 correction with e0 defined at f0 = 10 mHz.
 *   - phi_p is carried by the F+/Fx basis (psi = 0); phi_D = 2 pi f R sin(theta)
 *     cos(alpha(t_f) - phi); t(f) uses the orbital phase only.
 *   - spacecraft orbits: Keplerian ellipses (semi-major axis 1 AU, eccentricity e,
 *     inclination sqrt(3) e, perihelia 120 degrees apart) expanded to first order in
 *     e -- the rigid equilateral constellation -- or, on request (model.ecc = e),
 *     to second order in e (Sec. IV); the rigid form and the long-wavelength
 *     Michelson X are the defaults.
 *   - constants -phi_c - pi/4 of Psi are carried by the amplitudes a_i.
 *   - segment outer edges at the first/last bin whose t(f_k) lies in [0, T];
 *     interior edges equal-width in frequency; a bin belongs to segment p iff
 *     e_p <= f_k < e_{p+1} (last segment closed).
 *   - a segment with fewer than 4 bins, or with M11 M22 - M12^2 <= 1e-12 M11 M22,
 *     contributes F_p = 0.
 *   - the Gram sums and the 4x4 solve are carried in long double (see
 *     or_segment_sums_ld: short segments make M nearly singular).
 *   - the library returns the SUM over segments; F-hat = sum / N_seg.
 *   - TDI channels in the long-wavelength limit: X is the Michelson with its
 *     vertex at spacecraft 0, Y and Z those with vertices at spacecraft 1 and
 *     2 (arms to the next two spacecraft in cyclic order); A = (Z - X)/sqrt2,
 *     E = (X - 2Y + Z)/sqrt6 and T = (X + Y + Z)/sqrt3 as combinations of their
 *     detector tensors.  T vanishes identically in this limit.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- constants (this file's own copy) ---------------------------------- */
#define OR_MSUN_S 4.925490947e-6
#define OR_YEAR_S 31557600.0
#define OR_AU_S 499.004784
#define OR_PI 3.14159265358979323846
#define OR_PI_L 3.141592653589793238462643383279502884L
#define OR_F0_ECC 0.01 /* Hz: e0 is the eccentricity at this GW frequency */

typedef struct {
    double Mc;  /* chirp mass, solar masses */
    double tc;  /* coalescence time, s */
    double lat; /* ecliptic latitude beta, rad (theta = pi/2 - beta) */
    double lon; /* ecliptic longitude lambda = phi, rad */
    double e0;  /* eccentricity at f0 = 10 mHz */
    double q;   /* mass ratio m1/m2 >= 1 */
} or_params;

typedef struct {
    double f_min, df, T_obs;
    int64_t n;
    int response; /* 0: LISA response; 1: F+ = 1, Fx = 0, no Doppler (test mode) */
    int pn_order; /* highest k kept in sum_k alpha_k x^(k/2), 0..4 */
    double alpha0; /* orbital phase of the guiding centre at t = 0, rad */
    double orient; /* orientation of the constellation at t = 0, rad */
    int channel;   /* TDI channel: 0 X, 1 A, 2 E, 3 T */
    int mb_order;  /* -1: the paper's response T = F(t_f) e^{2 pi i f d(t_f)}; 0..2: Eq. (freDres)
                      with the filter F^N_{T_f} of this order N (see or_mb_response) */
    int mb_kmax;   /* highest k of the sum in Eq. (freDres), 0 or 1 (only T_A1 is defined) */
    double ecc;    /* 0: rigid constellation (first-order orbits); > 0: the spacecraft orbits to
                      second order in this eccentricity (or_sc_offset) */
    double arm_s;  /* 0: long-wavelength response; > 0: the finite-arm TDI response
                      (or_tdi_response) with nominal arm length arm_s light seconds */
    int no_doppler; /* 1: drop the Doppler delay of the guiding centre (test knob) */
} or_model;

/* ---- masses and PN coefficients (Appendix A) --------------------------- */
static double or_eta(double q) { return q / ((1.0 + q) * (1.0 + q)); }

/* Non-spinning TaylorF2 coefficients alpha_k(eta), k = 0..4. */
static void or_alpha(double eta, int order, double a[5]) {
    a[0] = 1.0;
    a[1] = 0.0;
    a[2] = 3715.0 / 756.0 + 55.0 * eta / 9.0;
    a[3] = -16.0 * OR_PI;
    a[4] = 15293365.0 / 508032.0 + 27145.0 * eta / 504.0 + 3085.0 * eta * eta / 72.0;
    for (int k = order + 1; k < 5; k++) a[k] = 0.0;
}

/* Stationary-phase time t(f) = t_c + (1/2pi) d/df [Psi_PN(f) + phi_e(f)]. */
static double or_time(const or_params* P, const or_model* m, double f) {
    double eta = or_eta(P->q);
    double Mc = P->Mc * OR_MSUN_S;
    double M = Mc * pow(eta, -0.6);
    double a[5];
    or_alpha(eta, m->pn_order, a);
    double v = cbrt(OR_PI * M * f);
    double lead = (3.0 / 128.0) * pow(OR_PI * Mc * f, -5.0 / 3.0);
    /* d/df of lead * sum_k a_k v^k, with lead ~ f^-5/3 and v^k ~ f^(k/3) */
    double s = 0.0, vk = 1.0;
    for (int k = 0; k <= 4; k++) {
        s += a[k] * ((double)(k - 5) / 3.0) * vk;
        vk *= v;
    }
    double dpsi = lead * s / f;
    double phie = -(2355.0 / 1462.0) * P->e0 * P->e0 * lead * pow(OR_F0_ECC / f, 19.0 / 9.0);
    double dphie = -(34.0 / 9.0) * phie / f;
    return P->tc + (dpsi + dphie) / (2.0 * OR_PI);
}

/* Orbital part of the phase in cycles, Psi_orb(f)/(2 pi) with
 * Psi_orb = 2 pi f t_c + Psi_PN(f) + phi_e(f), in long double. */
static long double or_phase_orb_cycles(const or_params* P, const or_model* m, long double f) {
    long double eta = (long double)or_eta(P->q);
    long double Mc = (long double)P->Mc * (long double)OR_MSUN_S;
    long double M = Mc * powl(eta, -0.6L);
    long double a[5];
    a[0] = 1.0L;
    a[1] = 0.0L;
    a[2] = 3715.0L / 756.0L + 55.0L * eta / 9.0L;
    a[3] = -16.0L * OR_PI_L;
    a[4] = 15293365.0L / 508032.0L + 27145.0L * eta / 504.0L + 3085.0L * eta * eta / 72.0L;
    for (int k = m->pn_order + 1; k < 5; k++) a[k] = 0.0L;
    long double v = cbrtl(OR_PI_L * M * f);
    long double lead = (3.0L / 128.0L) * powl(OR_PI_L * Mc * f, -5.0L / 3.0L);
    long double s = 0.0L, vk = 1.0L;
    for (int k = 0; k <= 4; k++) {
        s += a[k] * vk;
        vk *= v;
    }
    long double e0 = (long double)P->e0;
    long double phie = -(2355.0L / 1462.0L) * e0 * e0 * lead * powl((long double)OR_F0_ECC / f, 19.0L / 9.0L);
    return f * (long double)P->tc + (lead * s + phie) / (2.0L * OR_PI_L);
}

/* ---- detector (Sec. IV): rigid constellation, vector geometry ----------- */
static double or_orbit_phase(const or_model* m, double t) {
    return 2.0 * OR_PI * t / OR_YEAR_S + m->alpha0;
}

/* Position of spacecraft n (0,1,2) relative to the guiding centre
 * R (cos alpha, sin alpha, 0), in units of e*R: the Keplerian ellipse of
 * semi-major axis R and eccentricity e whose mean anomaly is alpha - beta_n
 * (beta_n = 2 pi n/3 + orient), its plane tilted by sqrt(3) e about the axis
 * normal to the apsidal line and turned by beta_n about the ecliptic pole,
 * expanded in e (eccentric anomaly to second order by Kepler's equation):
 *   order 1: (cos(2a - b) - 3 cos b) / 2, (sin(2a - b) - 3 sin b) / 2, -sqrt3 cos(a - b)
 *   order 2 (times e): -5/4 cos a - 5/8 cos(a - 2b) + 3/8 cos(3a - 2b),
 *                      -5/4 sin a + 5/8 sin(a - 2b) + 3/8 sin(3a - 2b),
 *                      sqrt3/2 (3 - cos(2a - 2b)).
 * With model.ecc = 0 only the first order is kept (the rigid constellation).
 * Only differences of positions are used (arm directions). */
static void or_sc_offset(const or_model* m, int n, double alpha, double r[3]) {
    double beta = 2.0 * OR_PI * n / 3.0 + m->orient;
    r[0] = 0.5 * (cos(2.0 * alpha - beta) - 3.0 * cos(beta));
    r[1] = 0.5 * (sin(2.0 * alpha - beta) - 3.0 * sin(beta));
    r[2] = -sqrt(3.0) * cos(alpha - beta);
    if (m->ecc != 0.0) {
        const double e = m->ecc;
        r[0] += e * (-1.25 * cos(alpha) - 0.625 * cos(alpha - 2.0 * beta) + 0.375 * cos(3.0 * alpha - 2.0 * beta));
        r[1] += e * (-1.25 * sin(alpha) + 0.625 * sin(alpha - 2.0 * beta) + 0.375 * sin(3.0 * alpha - 2.0 * beta));
        r[2] += e * (0.5 * sqrt(3.0) * (3.0 - cos(2.0 * alpha - 2.0 * beta)));
    }
}

/* Public: spacecraft offset above (units of e R). */
void or_sc_offset_at(const or_model* m, int n, double alpha, double* r) { or_sc_offset(m, n, alpha, r); }

/* Detector tensor D = (a a - b b)/2 of the long-wavelength Michelson with
 * vertex at spacecraft v (a, b: unit vectors along its arms to spacecraft
 * v+1 and v+2, cyclic) at orbital phase alpha. */
static void or_vertex_detector(const or_model* m, int v, double alpha, double D[3][3]) {
    double r0[3], r1[3], r2[3], a[3], b[3];
    or_sc_offset(m, v, alpha, r0);
    or_sc_offset(m, (v + 1) % 3, alpha, r1);
    or_sc_offset(m, (v + 2) % 3, alpha, r2);
    double na = 0.0, nb = 0.0;
    for (int i = 0; i < 3; i++) {
        a[i] = r1[i] - r0[i];
        b[i] = r2[i] - r0[i];
        na += a[i] * a[i];
        nb += b[i] * b[i];
    }
    na = sqrt(na);
    nb = sqrt(nb);
    for (int i = 0; i < 3; i++) {
        a[i] /= na;
        b[i] /= nb;
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) D[i][j] = 0.5 * (a[i] * a[j] - b[i] * b[j]);
}

/* Detector tensor of the model's TDI channel at time t: X itself, or the
 * combinations A, E, T of the three vertex Michelsons X, Y, Z. */
static void or_detector(const or_model* m, double t, double D[3][3]) {
    double alpha = or_orbit_phase(m, t);
    if (m->channel == 0) {
        or_vertex_detector(m, 0, alpha, D);
        return;
    }
    double X[3][3], Y[3][3], Z[3][3];
    or_vertex_detector(m, 0, alpha, X);
    or_vertex_detector(m, 1, alpha, Y);
    or_vertex_detector(m, 2, alpha, Z);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            if (m->channel == 1) D[i][j] = (Z[i][j] - X[i][j]) / sqrt(2.0);
            else if (m->channel == 2) D[i][j] = (X[i][j] - 2.0 * Y[i][j] + Z[i][j]) / sqrt(6.0);
            else D[i][j] = (X[i][j] + Y[i][j] + Z[i][j]) / sqrt(3.0);
        }
}

/* F+ and Fx of the long-wavelength Michelson with vertex at spacecraft 0:
 * F_A = D : e_A, e+ = p p - q q, ex = p q + q p. */
static void or_antenna(const or_params* P, const or_model* m, double t, double* Fp, double* Fx) {
    if (m->response == 1) {
        *Fp = 1.0;
        *Fx = 0.0;
        return;
    }
    double D[3][3];
    or_detector(m, t, D);
    double sb = sin(P->lat), cb = cos(P->lat), sl = sin(P->lon), cl = cos(P->lon);
    /* theta = pi/2 - beta: p = theta-hat, q = phi-hat of the source direction */
    double p[3] = {sb * cl, sb * sl, -cb};
    double qv[3] = {-sl, cl, 0.0};
    double fp = 0.0, fx = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double ep = p[i] * p[j] - qv[i] * qv[j];
            double ex = p[i] * qv[j] + qv[i] * p[j];
            fp += D[i][j] * ep;
            fx += D[i][j] * ex;
        }
    *Fp = fp;
    *Fx = fx;
}

/* Finite-arm response of the first-generation TDI Michelsons (Sec. IV: a TDI
 * combination is a sum of time-delayed single-arm responses), for the
 * constellation frozen at time t, at frequency f, for the polarisations + and x.
 * Spacecraft i sits at the guiding centre plus dx_i = L/(2 sqrt3) rho_i
 * (rho of or_sc_offset: its arms are 2 sqrt3 long at first order, so L is the
 * nominal arm length in seconds).  Link s -> r (emitted at s, received at r),
 * n = (x_r - x_s)/L_sr, k = -(source direction):
 *   y_sr = (n.e_A.n) [exp(-2 pi i f (L_sr + k.dx_s)) - exp(-2 pi i f k.dx_r)] / (2 (1 - k.n))
 * per unit h_A(f) (the guiding centre's own delay is the Doppler factor that
 * the template phase carries).  Michelson with vertex v and arms to a = v+1,
 * b = v+2 (cyclic), normalised by -4 pi i f L:
 *   R_v = [exp(-2 pi i f L_va) y_va + y_av - exp(-2 pi i f L_vb) y_vb - y_bv] / (-4 pi i f L),
 * which tends to D_v : e_A (the long-wavelength pattern) as f L -> 0; the
 * common TDI factor 1 - exp(-4 pi i f L) of signal and noise is divided out.
 * Channels: X = R_0, A = (R_2 - R_0)/sqrt2, E = (R_0 - 2 R_1 + R_2)/sqrt6. */
static void or_tdi_response(const or_params* P, const or_model* m, double f, double t, double complex T[2]) {
    const double L = m->arm_s;
    const double alpha = or_orbit_phase(m, t);
    double x[3][3];
    for (int i = 0; i < 3; i++) {
        or_sc_offset(m, i, alpha, x[i]);
        for (int j = 0; j < 3; j++) x[i][j] *= L / (2.0 * sqrt(3.0));
    }
    double sb = sin(P->lat), cb = cos(P->lat), sl = sin(P->lon), cl = cos(P->lon);
    double p[3] = {sb * cl, sb * sl, -cb};
    double q[3] = {-sl, cl, 0.0};
    double k[3] = {-cb * cl, -cb * sl, -sb};
    /* y[s][r][A] for every ordered pair s != r, and the link lengths */
    double complex y[3][3][2];
    double Lsr[3][3];
    for (int s_ = 0; s_ < 3; s_++)
        for (int r = 0; r < 3; r++) {
            if (r == s_) continue;
            double n[3], len = 0.0;
            for (int j = 0; j < 3; j++) {
                n[j] = x[r][j] - x[s_][j];
                len += n[j] * n[j];
            }
            len = sqrt(len);
            for (int j = 0; j < 3; j++) n[j] /= len;
            Lsr[s_][r] = len;
            double np = 0.0, nq = 0.0, kn = 0.0, kxs = 0.0, kxr = 0.0;
            for (int j = 0; j < 3; j++) {
                np += n[j] * p[j];
                nq += n[j] * q[j];
                kn += k[j] * n[j];
                kxs += k[j] * x[s_][j];
                kxr += k[j] * x[r][j];
            }
            double complex ph = cexp(-2.0 * I * OR_PI * f * (len + kxs)) - cexp(-2.0 * I * OR_PI * f * kxr);
            double complex w = ph / (2.0 * (1.0 - kn));
            y[s_][r][0] = (np * np - nq * nq) * w;
            y[s_][r][1] = 2.0 * np * nq * w;
        }
    double complex R[3][2];
    const double complex norm = -4.0 * I * OR_PI * f * L;
    for (int v = 0; v < 3; v++) {
        int a = (v + 1) % 3, b = (v + 2) % 3;
        for (int A = 0; A < 2; A++)
            R[v][A] = (cexp(-2.0 * I * OR_PI * f * Lsr[v][a]) * y[v][a][A] + y[a][v][A] -
                       cexp(-2.0 * I * OR_PI * f * Lsr[v][b]) * y[v][b][A] - y[b][v][A]) / norm;
    }
    for (int A = 0; A < 2; A++) {
        if (m->channel == 0) T[A] = R[0][A];
        else if (m->channel == 1) T[A] = (R[2][A] - R[0][A]) / sqrt(2.0);
        else if (m->channel == 2) T[A] = (R[0][A] - 2.0 * R[1][A] + R[2][A]) / sqrt(6.0);
        else T[A] = (R[0][A] + R[1][A] + R[2][A]) / sqrt(3.0);
    }
}

/* The response's pattern at time t and frequency f: the long-wavelength
 * (F+, Fx) of or_antenna, or with model.arm_s > 0 the finite-arm TDI
 * response of or_tdi_response (complex). */
static void or_pattern(const or_params* P, const or_model* m, double f, double t, double complex F[2]) {
    if (m->arm_s > 0.0 && m->response != 1) {
        or_tdi_response(P, m, f, t, F);
        return;
    }
    double Fp, Fx;
    or_antenna(P, m, t, &Fp, &Fx);
    F[0] = Fp;
    F[1] = Fx;
}

/* Doppler delay d(t) = n . r_gc(t) = R sin(theta) cos(alpha(t) - phi). */
static double or_doppler_delay(const or_params* P, const or_model* m, double t) {
    if (m->response == 1 || m->no_doppler) return 0.0;
    double alpha = or_orbit_phase(m, t);
    return OR_AU_S * cos(P->lat) * cos(alpha - P->lon);
}

/* ---- the series of Eq. (freDres) (Sec. IV) ----------------------------- */

/* First and second time derivatives of the Doppler delay above (closed forms
 * of d/dt R cos(beta) cos(2 pi t / yr + alpha0 - lambda)). */
static void or_doppler_rates(const or_params* P, const or_model* m, double t, double* dd, double* d2) {
    if (m->response == 1 || m->no_doppler) {
        *dd = 0.0;
        *d2 = 0.0;
        return;
    }
    double Om = 2.0 * OR_PI / OR_YEAR_S;
    double x = or_orbit_phase(m, t) - P->lon;
    double R = OR_AU_S * cos(P->lat);
    *dd = -R * Om * sin(x);
    *d2 = -R * Om * Om * cos(x);
}

/* T_f of Sec. IV: T_f^2 = |d^2 Psi/df^2| / (4 pi) for the waveform phase
 * Psi = 2 pi Phi_orb, whose first derivative is 2 pi t_f; so T_f^2 =
 * |dt_f/df| / 2, dt_f/df by the five-point central difference of t(f) with
 * step 1e-4 f (truncation ~ (1e-4)^4 relative). */
static double or_tf_width(const or_params* P, const or_model* m, double f) {
    double h = 1e-4 * f;
    double d = (-or_time(P, m, f + 2.0 * h) + 8.0 * or_time(P, m, f + h) - 8.0 * or_time(P, m, f - h) +
                or_time(P, m, f - 2.0 * h)) / (12.0 * h);
    return sqrt(0.5 * fabs(d));
}

/* Weights a_j (j = 0..N) of the filter
 *   F^N_{T_f}[G](t) = 1/2 sum_j a_j (G(t + j T_f) + G(t - j T_f)).
 * The paper takes them from its ref. marsat2018fourier (App. 2), which is not
 * at hand.  Reading: the filter stands for the average of G over the
 * stationary-phase kernel exp(i pi fdot s^2) of the chirp around t_f
 * (fdot = 1/(2 T_f^2)), whose even moments are <s^2m> = (2m-1)!! (i T_f^2/pi)^m;
 * the weights make the filter reproduce them for m = 0..N, i.e. exact for G
 * polynomial of degree <= 2N+1: sum_j a_j j^(2m) = (2m-1)!! (i/pi)^m (with
 * 0^0 = 1).  Solved by Gaussian elimination (the system is a Vandermonde
 * system in j^2, well conditioned for N <= 2). */
void or_mb_weights(int N, double* a_re, double* a_im) {
    double complex A[3][4];
    for (int m = 0; m <= N; m++) {
        double complex rhs = 1.0;
        for (int i = 1; i <= m; i++) rhs *= (2.0 * i - 1.0) * (I / OR_PI);
        for (int j = 0; j <= N; j++) {
            double pw = 1.0;
            for (int i = 0; i < m; i++) pw *= (double)(j * j);
            A[m][j] = pw;
        }
        A[m][N + 1] = rhs;
    }
    for (int c = 0; c <= N; c++) {
        int piv = c;
        for (int r = c + 1; r <= N; r++)
            if (cabs(A[r][c]) > cabs(A[piv][c])) piv = r;
        for (int j = 0; j <= N + 1; j++) {
            double complex t = A[c][j];
            A[c][j] = A[piv][j];
            A[piv][j] = t;
        }
        for (int r = 0; r <= N; r++) {
            if (r == c) continue;
            double complex fct = A[r][c] / A[c][c];
            for (int j = c; j <= N + 1; j++) A[r][j] -= fct * A[c][j];
        }
    }
    for (int j = 0; j <= N; j++) {
        double complex v = A[j][N + 1] / A[j][j];
        a_re[j] = creal(v);
        a_im[j] = cimag(v);
    }
}

/* The kernel of Eq. (freDres) for (F+, Fx), times exp(-2 pi i f D0):
 *   G(tau) = F(tau - d(tau)) / (1 + ddot(tau)) exp(2 pi i f d(tau) (1 - ddot(tau)))
 * D0 = d(t_f) (1 - ddot(t_f)) is the phase factor at t_f, which the template
 * phase carries instead. */
static void or_mb_G(const or_params* P, const or_model* m, double f, double tau, double D0, double complex G[2]) {
    double d = or_doppler_delay(P, m, tau), dd, d2;
    or_doppler_rates(P, m, tau, &dd, &d2);
    double complex F[2];
    or_pattern(P, m, f, tau - d, F);
    double ph = 2.0 * OR_PI * f * (d * (1.0 - dd) - D0);
    double complex c = (cos(ph) + I * sin(ph)) / (1.0 + dd);
    G[0] = F[0] * c;
    G[1] = F[1] * c;
}

/* Eq. (freDres) at frequency f with t_f = t, divided by exp(2 pi i f D0):
 *   T = sum_{k=0}^{kmax} (-i T_A1)^k / k!  F^N_{T_f}[d^k G / dtau^k](t_f),
 *   T_A1 = (7/6) / (2 pi f)  (the k = 1 coefficient the paper prints; k <= 1).
 * dG/dtau by the five-point central difference with step 20 s (G turns at
 * most 2 pi f |ddot| ~ 3e-5 rad/s at 50 mHz: truncation ~ 1e-13 relative). */
static void or_mb_response(const or_params* P, const or_model* m, double f, double t, double D0,
                           double complex T[2]) {
    const int N = m->mb_order;
    double a_re[3], a_im[3];
    or_mb_weights(N, a_re, a_im);
    const double Tf = or_tf_width(P, m, f);
    const double TA1 = (7.0 / 6.0) / (2.0 * OR_PI * f);
    const double h = 20.0;
    T[0] = 0.0;
    T[1] = 0.0;
    for (int j = -N; j <= N; j++) {
        const int aj = j < 0 ? -j : j;
        const double complex w = (j == 0 ? 1.0 : 0.5) * (a_re[aj] + I * a_im[aj]);
        const double tau = t + (double)j * Tf;
        double complex G[2];
        or_mb_G(P, m, f, tau, D0, G);
        T[0] += w * G[0];
        T[1] += w * G[1];
        if (m->mb_kmax >= 1) {
            double complex Gp2[2], Gp1[2], Gm1[2], Gm2[2];
            or_mb_G(P, m, f, tau + 2.0 * h, D0, Gp2);
            or_mb_G(P, m, f, tau + h, D0, Gp1);
            or_mb_G(P, m, f, tau - h, D0, Gm1);
            or_mb_G(P, m, f, tau - 2.0 * h, D0, Gm2);
            for (int c = 0; c < 2; c++) {
                double complex dG = (-Gp2[c] + 8.0 * Gp1[c] - 8.0 * Gm1[c] + Gm2[c]) / (12.0 * h);
                T[c] += w * (-I * TA1) * dG;
            }
        }
    }
}

static int or_params_finite(const or_params* P) {
    return isfinite(P->Mc) && isfinite(P->tc) && isfinite(P->lat) && isfinite(P->lon) &&
           isfinite(P->e0) && isfinite(P->q) && P->Mc > 0.0 && P->q > 0.0;
}

/* ---- public helpers ----------------------------------------------------- */
double or_time_of_freq(const or_params* P, const or_model* m, double f) { return or_time(P, m, f); }

/* Total template phase in cycles at bin frequency f (long double), and its
 * fractional part.  Phi = Psi_orb/2pi - f d(t_f). */
double or_phase_frac(const or_params* P, const or_model* m, double f_min, double df, int64_t k) {
    long double f = (long double)f_min + (long double)k * (long double)df;
    long double ph = or_phase_orb_cycles(P, m, f);
    double t = or_time(P, m, (double)f);
    ph -= f * (long double)or_doppler_delay(P, m, t);
    long double fr = ph - roundl(ph);
    return (double)fr;
}

/* The response of Eq. (freDres) at frequency f (t_f from the model):
 * out = (Re T+, Im T+, Re Tx, Im Tx, D0, T_f), T divided by exp(2 pi i f D0). */
void or_mb_response_at(const or_params* P, const or_model* m, double f, double* out) {
    double t = or_time(P, m, f);
    double d = or_doppler_delay(P, m, t), dd, d2;
    or_doppler_rates(P, m, t, &dd, &d2);
    double complex T[2];
    or_mb_response(P, m, f, t, d * (1.0 - dd), T);
    out[0] = creal(T[0]);
    out[1] = cimag(T[0]);
    out[2] = creal(T[1]);
    out[3] = cimag(T[1]);
    out[4] = d * (1.0 - dd);
    out[5] = or_tf_width(P, m, f);
}

/* Public: the finite-arm TDI response (Re T+, Im T+, Re Tx, Im Tx) at frequency f and time t. */
void or_tdi_response_at(const or_params* P, const or_model* m, double f, double t, double* out) {
    double complex T[2];
    or_tdi_response(P, m, f, t, T);
    out[0] = creal(T[0]);
    out[1] = cimag(T[0]);
    out[2] = creal(T[1]);
    out[3] = cimag(T[1]);
}

void or_doppler_rates_at(const or_params* P, const or_model* m, double t, double* dd, double* d2) {
    or_doppler_rates(P, m, t, dd, d2);
}

long double or_phase_orb_cycles_ld(const or_params* P, const or_model* m, long double f) {
    return or_phase_orb_cycles(P, m, f);
}

double or_phase_orb_cycles_d(const or_params* P, const or_model* m, double f) {
    return (double)or_phase_orb_cycles(P, m, (long double)f);
}

void or_antenna_at(const or_params* P, const or_model* m, double t, double* Fp, double* Fx) {
    or_antenna(P, m, t, Fp, Fx);
}

double or_doppler_at(const or_params* P, const or_model* m, double t) { return or_doppler_delay(P, m, t); }

void or_detector_tensor_at(const or_model* m, double t, double* D9) {
    double D[3][3];
    or_detector(m, t, D);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) D9[3 * i + j] = D[i][j];
}

/* Basis waveforms A^i at bins k0..k1-1 (Eq. response with the Sec. IV
 * response): h0 = f^-7/6 e^{-2 pi i Phi}, A1 = F+ h0, A2 = Fx h0,
 * A3 = -i F+ h0, A4 = -i Fx h0.  out: [4][k1-k0] re and im. */
void or_basis(const or_params* P, const or_model* m, int64_t k0, int64_t k1, double* re, double* im) {
    int64_t n = k1 - k0;
    for (int64_t j = 0; j < n; j++) {
        int64_t k = k0 + j;
        double f = m->f_min + (double)k * m->df;
        double t = or_time(P, m, f);
        if (m->mb_order >= 0) {
            /* Eq. (freDres): A1 = T+ h0, A2 = Tx h0, A3 = -i T+ h0, A4 = -i Tx h0 with the
             * complex responses T of or_mb_response and h0 = f^-7/6 e^{-2 pi i Phi},
             * Phi = Phi_orb - f D0 (the phase factor of G at t_f) */
            double d = or_doppler_delay(P, m, t), dd, d2;
            or_doppler_rates(P, m, t, &dd, &d2);
            const double D0 = d * (1.0 - dd);
            long double fl = (long double)m->f_min + (long double)k * (long double)m->df;
            long double ph = or_phase_orb_cycles(P, m, fl) - fl * (long double)D0;
            double fr = (double)(ph - roundl(ph));
            double complex T[2];
            or_mb_response(P, m, f, t, D0, T);
            double amp = pow(f, -7.0 / 6.0);
            double complex h0 = amp * (cos(2.0 * OR_PI * fr) - I * sin(2.0 * OR_PI * fr));
            for (int c = 0; c < 2; c++) {
                double complex A = T[c] * h0, Am = -I * A;
                re[c * n + j] = creal(A);
                im[c * n + j] = cimag(A);
                re[(c + 2) * n + j] = creal(Am);
                im[(c + 2) * n + j] = cimag(Am);
            }
            continue;
        }
        if (m->arm_s > 0.0 && m->response != 1) {
            /* the paper's form with the finite-arm TDI response: A1 = T+ h0, A3 = -i T+ h0, ... */
            double complex T[2];
            or_tdi_response(P, m, f, t, T);
            double fr = or_phase_frac(P, m, m->f_min, m->df, k);
            double amp = pow(f, -7.0 / 6.0);
            double complex h0 = amp * (cos(2.0 * OR_PI * fr) - I * sin(2.0 * OR_PI * fr));
            for (int c = 0; c < 2; c++) {
                double complex A = T[c] * h0, Am = -I * A;
                re[c * n + j] = creal(A);
                im[c * n + j] = cimag(A);
                re[(c + 2) * n + j] = creal(Am);
                im[(c + 2) * n + j] = cimag(Am);
            }
            continue;
        }
        double Fp, Fx;
        or_antenna(P, m, t, &Fp, &Fx);
        double fr = or_phase_frac(P, m, m->f_min, m->df, k);
        double c = cos(2.0 * OR_PI * fr), s = sin(2.0 * OR_PI * fr);
        double amp = pow(f, -7.0 / 6.0);
        double h_re = amp * c, h_im = -amp * s;   /* h0 */
        re[0 * n + j] = Fp * h_re;
        im[0 * n + j] = Fp * h_im;
        re[1 * n + j] = Fx * h_re;
        im[1 * n + j] = Fx * h_im;
        /* -i (x + i y) = y - i x */
        re[2 * n + j] = Fp * h_im;
        im[2 * n + j] = -Fp * h_re;
        re[3 * n + j] = Fx * h_im;
        im[3 * n + j] = -Fx * h_re;
    }
}

/* Segment outer edges (Sec. II.B): first and last bin whose stationary-phase
 * time lies in [0, T_obs].  t(f) increases with f on the search range.
 * Returns 0 and sets *klo > *khi when no bin qualifies. */
int or_band(const or_params* P, const or_model* m, int64_t* klo, int64_t* khi) {
    int64_t n = m->n;
    /* smallest k with t(f_k) >= 0 */
    int64_t lo = 0, hi = n; /* answer in [lo, hi]; hi = n means none */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        double t = or_time(P, m, m->f_min + (double)mid * m->df);
        if (t >= 0.0) hi = mid; else lo = mid + 1;
    }
    int64_t a = lo;
    /* largest k with t(f_k) <= T: one less than the smallest k with t > T */
    lo = 0;
    hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        double t = or_time(P, m, m->f_min + (double)mid * m->df);
        if (t > m->T_obs) hi = mid; else lo = mid + 1;
    }
    int64_t b = lo - 1;
    *klo = a;
    *khi = b;
    return 0;
}

/* Start bin of every segment: starts[p] for p = 0..Np, segment p is
 * [starts[p], starts[p+1]).  Global edges (if given) are used as they are.
 * Per-particle edges: e_p = f_lo + p (f_hi - f_lo)/Np with f_lo = f_{klo},
 * f_hi = f_{khi}; bin k is in p iff e_p <= f_k < e_{p+1}, last segment closed.
 * In bin units e_p sits at klo + p (khi - klo)/Np, so the first bin of
 * segment p is klo + ceil(p (khi - klo) / Np). */
static void or_segment_starts(const or_params* P, const or_model* m, const int64_t* edges, int Np,
                              int64_t* starts) {
    if (edges) {
        for (int p = 0; p <= Np; p++) starts[p] = edges[p];
        return;
    }
    int64_t klo, khi;
    or_band(P, m, &klo, &khi);
    if (klo > khi) {
        for (int p = 0; p <= Np; p++) starts[p] = 0;
        return;
    }
    int64_t w = khi - klo;
    for (int p = 0; p < Np; p++) {
        int64_t num = (int64_t)p * w;
        starts[p] = klo + (num + Np - 1) / Np;
    }
    starts[Np] = khi + 1;
    if (w == 0)
        for (int p = 1; p < Np; p++) starts[p] = khi + 1;
}

/* Segment start bins from N_p + 1 global edge frequencies (Sec. II.B: bin k
 * lies in segment p iff e_p <= f_k < e_{p+1}, the last segment closed at
 * e_{N_p}), by the definition: starts[p] counts the bins with f_k < e_p for
 * p < N_p and starts[N_p] those with f_k <= e_{N_p}, every bin tested.  Since
 * f_k grows with k, segment p is then the bins [starts[p], starts[p+1]).
 * Returns -1 (and writes nothing) if an edge is not finite or the edges
 * decrease. */
int or_edge_starts(const or_model* m, const double* e, int Np, int64_t* starts) {
    for (int p = 0; p <= Np; p++) {
        if (!isfinite(e[p])) return -1;
        if (p > 0 && !(e[p - 1] <= e[p])) return -1;
    }
    for (int p = 0; p <= Np; p++) starts[p] = 0;
    for (int64_t k = 0; k < m->n; k++) {
        const double f = m->f_min + (double)k * m->df;
        for (int p = 0; p < Np; p++)
            if (f < e[p]) starts[p]++;
        if (f <= e[Np]) starts[Np]++;
    }
    return 0;
}

/* Per-segment N^i = <d, A^i> and M^ij = <A^i, A^j> (Eqs. aandMN, aandMN2)
 * with the segment inner product <a,b>_l = 4 df Re sum_k a_k conj(b_k)/S_k.
 * Products and sums are formed in long double: on short segments F+ and Fx
 * are nearly proportional and M is close to singular (M11 M22 - M12^2 down
 * to ~1e-10 M11 M22), so the Gram sums need more than FP64 precision for
 * F_p to be reliable to 1e-9. */
static void or_segment_sums_ld(const or_params* P, const or_model* m, const double* d_re, const double* d_im,
                               const double* psd, const int64_t* edges, int Np, long double* Nout,
                               long double* Mout, int64_t* nbins) {
    int64_t* starts = (int64_t*)malloc(sizeof(int64_t) * (Np + 1));
    or_segment_starts(P, m, edges, Np, starts);
    for (int p = 0; p < Np; p++) {
        int64_t k0 = starts[p], k1 = starts[p + 1];
        if (k1 < k0) k1 = k0;
        int64_t n = k1 - k0;
        nbins[p] = n;
        long double N[4] = {0, 0, 0, 0}, M[16];
        for (int i = 0; i < 16; i++) M[i] = 0.0L;
        if (n > 0) {
            double* re = (double*)malloc(sizeof(double) * 4 * n);
            double* im = (double*)malloc(sizeof(double) * 4 * n);
            or_basis(P, m, k0, k1, re, im);
            for (int64_t j = 0; j < n; j++) {
                int64_t k = k0 + j;
                long double w = 4.0L * (long double)m->df / (long double)psd[k];
                long double dr = d_re[k], di = d_im[k];
                for (int i = 0; i < 4; i++) {
                    long double ar = re[i * n + j], ai = im[i * n + j];
                    /* Re(d conj(A)) = d_re A_re + d_im A_im */
                    N[i] += w * (dr * ar + di * ai);
                    for (int l = 0; l < 4; l++)
                        M[i * 4 + l] += w * (ar * (long double)re[l * n + j] + ai * (long double)im[l * n + j]);
                }
            }
            free(re);
            free(im);
        }
        for (int i = 0; i < 4; i++) Nout[4 * p + i] = N[i];
        for (int i = 0; i < 16; i++) Mout[16 * p + i] = M[i];
    }
    free(starts);
}

void or_segment_sums(const or_params* P, const or_model* m, const double* d_re, const double* d_im,
                     const double* psd, const int64_t* edges, int Np, double* Nout /*[Np][4]*/,
                     double* Mout /*[Np][16]*/, int64_t* nbins /*[Np]*/) {
    long double* N = (long double*)malloc(sizeof(long double) * 4 * Np);
    long double* M = (long double*)malloc(sizeof(long double) * 16 * Np);
    or_segment_sums_ld(P, m, d_re, d_im, psd, edges, Np, N, M, nbins);
    for (int i = 0; i < 4 * Np; i++) Nout[i] = (double)N[i];
    for (int i = 0; i < 16 * Np; i++) Mout[i] = (double)M[i];
    free(N);
    free(M);
}

/* F_p = 1/2 N^T M^-1 N by Cholesky factorisation of the 4x4 M (long double);
 * the degenerate-segment rule returns 0. */
static long double or_segment_F_ld(const long double* N, const long double* M, int64_t nbins) {
    if (nbins < 4) return 0.0L;
    long double m11 = M[0], m12 = M[1], m22 = M[5];
    if (m11 * m22 - m12 * m12 <= 1e-12L * m11 * m22) return 0.0L;
    long double L[4][4];
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) L[i][j] = 0.0L;
    for (int i = 0; i < 4; i++) {
        for (int j = 0; j <= i; j++) {
            long double s = M[i * 4 + j];
            for (int k = 0; k < j; k++) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0.0L)) return 0.0L;
                L[i][i] = sqrtl(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    /* solve L y = N; then N^T M^-1 N = y . y */
    long double y[4];
    for (int i = 0; i < 4; i++) {
        long double s = N[i];
        for (int k = 0; k < i; k++) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    return 0.5L * (y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3]);
}

double or_segment_F(const double* N, const double* M, int64_t nbins) {
    long double Nl[4], Ml[16];
    for (int i = 0; i < 4; i++) Nl[i] = N[i];
    for (int i = 0; i < 16; i++) Ml[i] = M[i];
    return (double)or_segment_F_ld(Nl, Ml, nbins);
}

/* Batched semi-coherent F: F[b] = sum_p F_p (the paper's F-hat is F[b]/Np),
 * Fpart[b*Np + p] = F_p (may be NULL).  edges: Np+1 global segment start
 * bins, or NULL for per-particle segments.  nthreads <= 0: all cores. */
int or_fstat_batch(const or_params* params, int B, const or_model* m, const double* d_re,
                   const double* d_im, const double* psd, const int64_t* edges, int Np, double* F,
                   double* Fpart, int nthreads) {
    if (B < 0 || Np < 1 || !m || m->n < 1) return -1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; b++) {
        const or_params* P = params + b;
        long double* Nb = (long double*)malloc(sizeof(long double) * 4 * Np);
        long double* Mb = (long double*)malloc(sizeof(long double) * 16 * Np);
        int64_t* nb = (int64_t*)malloc(sizeof(int64_t) * Np);
        long double tot = 0.0L;
        if (!or_params_finite(P)) {
            tot = NAN;
            if (Fpart)
                for (int p = 0; p < Np; p++) Fpart[(int64_t)b * Np + p] = NAN;
        } else {
            or_segment_sums_ld(P, m, d_re, d_im, psd, edges, Np, Nb, Mb, nb);
            for (int p = 0; p < Np; p++) {
                long double Fp = or_segment_F_ld(Nb + 4 * p, Mb + 16 * p, nb[p]);
                if (Fpart) Fpart[(int64_t)b * Np + p] = (double)Fp;
                tot += Fp;
            }
        }
        F[b] = (double)tot;
        free(Nb);
        free(Mb);
        free(nb);
    }
    return 0;
}

/* The same for data in several TDI channels (Sec. II.A, Eq. eq2): models[c]
 * fixes channel c's response (its `channel` field; grid and orbit shared),
 * d_re, d_im, psd hold nch arrays of n values one after the other, and N, M
 * of each segment are summed over the channels before the 4x4 solve. */
int or_fstat_batch_multi(const or_params* params, int B, const or_model* models, int nch, const double* d_re,
                         const double* d_im, const double* psd, const int64_t* edges, int Np, double* F,
                         double* Fpart, int nthreads) {
    if (B < 0 || Np < 1 || nch < 1 || !models || models[0].n < 1) return -1;
    const int64_t n = models[0].n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; b++) {
        const or_params* P = params + b;
        long double* Nb = (long double*)malloc(sizeof(long double) * 4 * Np);
        long double* Mb = (long double*)malloc(sizeof(long double) * 16 * Np);
        long double* Nc = (long double*)malloc(sizeof(long double) * 4 * Np);
        long double* Mc = (long double*)malloc(sizeof(long double) * 16 * Np);
        int64_t* nb = (int64_t*)malloc(sizeof(int64_t) * Np);
        long double tot = 0.0L;
        if (!or_params_finite(P)) {
            tot = NAN;
            if (Fpart)
                for (int p = 0; p < Np; p++) Fpart[(int64_t)b * Np + p] = NAN;
        } else {
            for (int i = 0; i < 4 * Np; i++) Nb[i] = 0.0L;
            for (int i = 0; i < 16 * Np; i++) Mb[i] = 0.0L;
            for (int c = 0; c < nch; c++) {
                or_segment_sums_ld(P, models + c, d_re + (int64_t)c * n, d_im + (int64_t)c * n, psd + (int64_t)c * n,
                                   edges, Np, Nc, Mc, nb);
                for (int i = 0; i < 4 * Np; i++) Nb[i] += Nc[i];
                for (int i = 0; i < 16 * Np; i++) Mb[i] += Mc[i];
            }
            for (int p = 0; p < Np; p++) {
                long double Fp = or_segment_F_ld(Nb + 4 * p, Mb + 16 * p, nb[p]);
                if (Fpart) Fpart[(int64_t)b * Np + p] = (double)Fp;
                tot += Fp;
            }
        }
        F[b] = (double)tot;
        free(Nb);
        free(Mb);
        free(Nc);
        free(Mc);
        free(nb);
    }
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- Appendix B --------------------------------------------------------- */
/* Eq. (B1): amplitudes a_i from (D_L, psi, iota, phi_c). */
void or_extrinsic_to_a(double DL, double psi, double iota, double phic, double a[4]) {
    double c2p = cos(2.0 * psi), s2p = sin(2.0 * psi), ci = cos(iota);
    double ap = 0.5 * (1.0 + ci * ci), cf = cos(phic), sf = sin(phic);
    a[0] = (c2p * ap * cf - s2p * ci * sf) / DL;
    a[1] = -(s2p * ap * cf + c2p * ci * sf) / DL;
    a[2] = -(c2p * ap * sf + s2p * ci * cf) / DL;
    a[3] = (s2p * ap * sf - c2p * ci * cf) / DL;
}

/* Eqs. (B2)-(B3): (D_L, iota, psi, phi_c) from a_i. */
void or_a_to_extrinsic(const double a[4], double* DL, double* iota, double* psi, double* phic) {
    double r1 = sqrt((a[0] + a[3]) * (a[0] + a[3]) + (a[1] - a[2]) * (a[1] - a[2]));
    double r2 = sqrt((a[0] - a[3]) * (a[0] - a[3]) + (a[1] + a[2]) * (a[1] + a[2]));
    double Ap = r1 + r2, Ax = r1 - r2;
    double A = Ap + sqrt(Ap * Ap - Ax * Ax);
    *DL = 2.0 / A;
    *iota = acos(-Ax / (Ap + sqrt(Ap * Ap - Ax * Ax)));
    double ps = 0.5 * atan2(Ap * a[3] - Ax * a[0], -(Ax * a[1] + Ap * a[2]));
    *psi = ps;
    double c = (sin(2.0 * ps) > 0.0) ? 1.0 : ((sin(2.0 * ps) < 0.0) ? -1.0 : 0.0);
    *phic = atan2(c * (Ap * a[3] - Ax * a[0]), -c * (Ax * a[2] + Ap * a[1]));
}

/* ---- Philox4x32-10 (Salmon et al. 2011), written from its definition ---- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static double or_u53(uint32_t lo, uint32_t hi) {
    uint64_t w = ((uint64_t)hi << 32) | lo;
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

/* ---- PSO (Sec. III.A) ---------------------------------------------------- */
/* Initial positions x ~ U[0,1]^D and velocities v ~ U[-x, 1-x] in the
 * normalised search space; Philox counter (0xFFFFFFFF, particle, dim, run). */
void or_pso_init(int R, int Npart, int D, uint64_t seed, double* x, double* v) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int r = 0; r < R; r++)
        for (int i = 0; i < Npart; i++)
            for (int j = 0; j < D; j++) {
                uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)i, (uint32_t)j, (uint32_t)r}, o[4];
                or_philox4x32_10(ctr, key, o);
                int64_t idx = ((int64_t)r * Npart + i) * D + j;
                double u1 = or_u53(o[0], o[1]), u2 = or_u53(o[2], o[3]);
                x[idx] = u1;
                v[idx] = u2 - u1;
            }
}

/* One PSO iteration for R independent runs of Npart particles in D dims.
 * fit[r*Npart+i] is the fitness of the current position (NaN counts as -inf).
 *  1. personal best: replaced only on a strictly greater fitness;
 *  2. local best: best personal best on the ring {i-1, i, i+1}, ties to the
 *     lowest particle index;
 *  3. v <- w v + c1 r1 (p - x) + c2 r2 (l - x), r1, r2 ~ U[0,1) from Philox
 *     counter (iteration, particle, dim, run), key = seed;
 *  4. v clamped to [-vmax, vmax]; 5. x <- x + v.
 * Evaluated in this exact order with no fused multiply-add. */
void or_pso_step(int R, int Npart, int D, double* x, double* v, double* pbest_x, double* pbest_f,
                 const double* fit, uint64_t seed, uint32_t iteration, double w, double c1, double c2,
                 double vmax, int* lbest_idx_out) {
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int r = 0; r < R; r++)
        for (int i = 0; i < Npart; i++) {
            int64_t pi = (int64_t)r * Npart + i;
            double f = fit[pi];
            if (f > pbest_f[pi]) { /* NaN compares false */
                pbest_f[pi] = f;
                for (int j = 0; j < D; j++) pbest_x[pi * D + j] = x[pi * D + j];
            }
        }
    int* lb = (int*)malloc(sizeof(int) * (size_t)R * Npart);
    for (int r = 0; r < R; r++)
        for (int i = 0; i < Npart; i++) {
            int cand[3] = {(i + Npart - 1) % Npart, i, (i + 1) % Npart};
            int best = -1;
            for (int c = 0; c < 3; c++) {
                int j = cand[c];
                if (best < 0) { best = j; continue; }
                double fj = pbest_f[(int64_t)r * Npart + j], fb = pbest_f[(int64_t)r * Npart + best];
                if (fj > fb || (fj == fb && j < best)) best = j;
            }
            lb[r * Npart + i] = best;
        }
    for (int r = 0; r < R; r++)
        for (int i = 0; i < Npart; i++) {
            int64_t pi = (int64_t)r * Npart + i;
            int64_t li = (int64_t)r * Npart + lb[r * Npart + i];
            if (lbest_idx_out) lbest_idx_out[pi] = lb[r * Npart + i];
            for (int j = 0; j < D; j++) {
                uint32_t ctr[4] = {iteration, (uint32_t)i, (uint32_t)j, (uint32_t)r}, o[4];
                or_philox4x32_10(ctr, key, o);
                double r1 = or_u53(o[0], o[1]), r2 = or_u53(o[2], o[3]);
                double xv = x[pi * D + j];
                double cog = c1 * r1;
                cog = cog * (pbest_x[pi * D + j] - xv);
                double soc = c2 * r2;
                soc = soc * (pbest_x[li * D + j] - xv);
                double nv = w * v[pi * D + j];
                nv = nv + cog;
                nv = nv + soc;
                if (nv > vmax) nv = vmax;
                if (nv < -vmax) nv = -vmax;
                v[pi * D + j] = nv;
                x[pi * D + j] = xv + nv;
            }
        }
    free(lb);
}
