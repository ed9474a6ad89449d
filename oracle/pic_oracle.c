/*
 * pic_oracle.c -- plain FP64 CPU oracle for the particle-in-cell step of
 * arXiv 2602.15939 (shearing box KSB-OA, expanding box KEB, leaky box).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU baseline of bench.py to check and time the CUDA path.  Written for a
 * reader who checks it against the paper by eye: every operation follows the
 * paper's notation and order, one particle and one grid point at a time, with
 * no blocking, fusion or reordering.  Conventions are in pic_oracle.h.
 *
 * Readings of points the paper leaves open (each listed in the design notes):
 *  - Yee staggering for the "central-difference scheme in space" (Sec. 2.2);
 *  - field and current shapes of order 1 or 2, each component gathered at its
 *    own staggered location; charge-conserving deposit after Esirkepov for
 *    both orders (the paper cites Villasenor-Buneman, Sec. 2.2);
 *  - standard-PIC field update: B half step, E full step, B half step;
 *  - shearing box: x measured from the box centre; fractional shear shifts
 *    interpolated linearly in y (ghost values) and folded with the adjoint
 *    weights (currents); the particle crossing x_o gets y += Dy_s, crossing
 *    x_i gets y -= Dy_s, u' unchanged; the fixed-point Maxwell solve uses a
 *    fixed number of sweeps; each advection term is upwinded with respect to
 *    its own transport velocity (V for B and E'_y, -V for E'_x and E'_z);
 *    terms off their component's stagger are centred and averaged in y;
 *  - expanding box: l_i(t) = exp(rate_i t); L at each field's own time level,
 *    L^{-1} at t^{n+1/2} for positions, Lambda at t^n;
 *  - leaky box: the displacement uses the velocity that moved the particle,
 *    u^{n+1/2}/gamma^{n+1/2}; the reinjection distribution is a Maxwell-Juettner
 *    at theta_inj, sampled with Philox4x32-10 keyed on (id, seed).
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "pic_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define FOUR_PI (4.0 * 3.14159265358979323846)
#define TWO_PI (2.0 * 3.14159265358979323846)

/* ======================================================================== */
/* Small vector helpers                                                      */
/* ======================================================================== */

static void cross3(const double a[3], const double b[3], double r[3])
{
    double t0 = a[1] * b[2] - a[2] * b[1];
    double t1 = a[2] * b[0] - a[0] * b[2];
    double t2 = a[0] * b[1] - a[1] * b[0];
    r[0] = t0;
    r[1] = t1;
    r[2] = t2;
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Boris operator B(nu) = nu + 2 (nu x t + (nu x t) x t) / (1 + t^2)   (Sec. 2.2) */
static void boris_op(const double nu[3], const double t[3], double out[3])
{
    double a[3], b[3];
    double den = 1.0 + dot3(t, t);
    cross3(nu, t, a);
    cross3(a, t, b);
    for (int i = 0; i < 3; ++i) out[i] = nu[i] + 2.0 * (a[i] + b[i]) / den;
}

/* half-Boris operator R(nu) = nu + (nu x t + (nu x t) x t) / (1 + t^2)   (Sec. 2.2) */
static void half_boris_op(const double nu[3], const double t[3], double out[3])
{
    double a[3], b[3];
    double den = 1.0 + dot3(t, t);
    cross3(nu, t, a);
    cross3(a, t, b);
    for (int i = 0; i < 3; ++i) out[i] = nu[i] + (a[i] + b[i]) / den;
}

/* ======================================================================== */
/* Particle pushers                                                          */
/* ======================================================================== */

/* Standard Boris push (the S = 0 reduction of Sec. 2.2, and the Lambda = 0
 * reduction of Sec. 3.2): u^- = u + eps, gamma^- from u^-,
 * tau = q dt B / (2 m c gamma^-), u^+ = B(u^-), u^{n+1/2} = u^+ + eps. */
void ora_push_boris(double q, double m, double c, const double E[3], const double B[3], double u[3])
{
    double eps[3], um[3], tau[3], up[3];
    for (int i = 0; i < 3; ++i) eps[i] = q * E[i] / (2.0 * m);
    for (int i = 0; i < 3; ++i) um[i] = u[i] + eps[i];
    double gm = sqrt(1.0 + dot3(um, um) / (c * c));
    for (int i = 0; i < 3; ++i) tau[i] = q * B[i] / (2.0 * m * c * gm);
    boris_op(um, tau, up);
    for (int i = 0; i < 3; ++i) u[i] = up[i] + eps[i];
}

/* Midpoint Lorentz factor of the shearing-box push (Sec. 2.2): the real root
 * gbar >= 1 of gbar^2 = 1 + [u^2 + 2 a1 ux uy + 2 a2 (u.eps) uy / gbar] / c^2,
 * i.e. gbar^3 - A gbar - C = 0.  Newton iteration started from the paper's
 * small-Omega0 approximation, run to convergence. */
double ora_ksb_gamma_bar(double c, double alpha1, double alpha2, const double um[3],
                         const double eps[3], double *residual)
{
    double c2 = c * c;
    double u2 = dot3(um, um);
    double ue = dot3(um, eps);
    double A = 1.0 + (u2 + 2.0 * alpha1 * um[0] * um[1]) / c2;
    double C = 2.0 * alpha2 * ue * um[1] / c2;
    double gminus = sqrt(1.0 + u2 / c2);
    /* small-Omega0 approximation printed in Sec. 2.2 */
    double g = gminus + (alpha1 * um[0] * um[1] * gminus + alpha2 * ue * um[1]) / (c2 * gminus * gminus);
    for (int it = 0; it < 60; ++it) {
        double f = g * g * g - A * g - C;
        double df = 3.0 * g * g - A;
        double dg = f / df;
        g -= dg;
        if (fabs(dg) <= 1e-16 * g) break;
    }
    if (residual) {
        /* residual of the defining relation, relative to gbar^2 */
        double rhs = 1.0 + (u2 + 2.0 * alpha1 * um[0] * um[1] + 2.0 * alpha2 * ue * um[1] / g) / c2;
        *residual = fabs(g * g - rhs) / (g * g);
    }
    return g;
}

/* Shearing-box (KSB-OA) Boris-like push, Sec. 2.2: solves
 *   u+ - u+ x tt - a1 u+_x e_y - a2 (u+.et) e_y = u- + u- x tt + a1 u-_x e_y + a2 (u-.et) e_y
 * with eps = q dt E'/(2m), et = eps/(c gbar), tau = q dt B/(2 m c),
 * tt = tau/gbar + dt Omega0 e_z, a1 = s Omega0 dt/2, a2 = s Omega0 x^n / c,
 * through u+ = B(u-) + R(S u-) + R(S (B(u-) + R(S u-))) / (1 - g),
 * g = S_2 . R(e_y), then u'^{n+1/2} = u+ + eps.  xc is x^n from the box centre. */
void ora_push_ksb(double q, double m, double c, double s, double Omega0, double xc,
                  const double E[3], const double B[3], double u[3], double *gbar_out)
{
    double eps[3], um[3];
    for (int i = 0; i < 3; ++i) eps[i] = q * E[i] / (2.0 * m);
    for (int i = 0; i < 3; ++i) um[i] = u[i] + eps[i];
    double alpha1 = s * Omega0 / 2.0;
    double alpha2 = s * Omega0 * xc / c;
    double gbar = ora_ksb_gamma_bar(c, alpha1, alpha2, um, eps, NULL);
    if (gbar_out) *gbar_out = gbar;

    double et[3], tt[3];
    for (int i = 0; i < 3; ++i) et[i] = eps[i] / (c * gbar);
    for (int i = 0; i < 3; ++i) tt[i] = q * B[i] / (2.0 * m * c) / gbar;
    tt[2] += Omega0;

    /* second row of the rank-1 matrix S */
    double S2[3] = {alpha1 + alpha2 * et[0], alpha2 * et[1], alpha2 * et[2]};
    const double ey[3] = {0.0, 1.0, 0.0};
    double Rey[3];
    half_boris_op(ey, tt, Rey);
    double g = dot3(S2, Rey);

    /* w = B(u-) + R(S u-) */
    double Bu[3], Su[3], RSu[3], w[3];
    boris_op(um, tt, Bu);
    Su[0] = 0.0;
    Su[1] = dot3(S2, um);
    Su[2] = 0.0;
    half_boris_op(Su, tt, RSu);
    for (int i = 0; i < 3; ++i) w[i] = Bu[i] + RSu[i];

    /* u+ = w + R(S w) / (1 - g) */
    double Sw[3], RSw[3], up[3];
    Sw[0] = 0.0;
    Sw[1] = dot3(S2, w);
    Sw[2] = 0.0;
    half_boris_op(Sw, tt, RSw);
    for (int i = 0; i < 3; ++i) up[i] = w[i] + RSw[i] / (1.0 - g);
    for (int i = 0; i < 3; ++i) u[i] = up[i] + eps[i];
}

/* Solve the 3x3 system M x = b by Cramer's rule. */
static void solve3(const double M[3][3], const double b[3], double x[3])
{
    double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
               - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
               + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    for (int col = 0; col < 3; ++col) {
        double A[3][3];
        memcpy(A, M, sizeof(A));
        for (int r = 0; r < 3; ++r) A[r][col] = b[r];
        double d = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
                 - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
                 + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
        x[col] = d / det;
    }
}

/* Expanding-box (KEB) modified Boris push, Sec. 3.2, for the diagonal
 * Lambda = -(dt/2) L^{-1} dL/dt (passed as its three diagonal entries):
 *   gbar = sqrt(1 + ((1 + Lambda) u-)^2 / c^2),  tau = q dt B / (2 gbar m c),
 *   tt_i = tau_i / (1 - Lambda_ii),  Lt_ii = (1 + Lambda_ii) / (1 - Lambda_ii),
 *   u+ = Lt nu + ((1+Lt) nu x tt + ((1+Lt) nu x tt) x tt) / (1 + tt^2).
 * exact != 0 instead solves u+ - Lambda u+ - u+ x tau = u- + Lambda u- + u- x tau
 * directly (the two agree when Lambda is isotropic). */
void ora_push_keb(double q, double m, double c, const double Lambda[3], const double E[3],
                  const double B[3], double u[3], int exact)
{
    double eps[3], um[3], up[3];
    for (int i = 0; i < 3; ++i) eps[i] = q * E[i] / (2.0 * m);
    for (int i = 0; i < 3; ++i) um[i] = u[i] + eps[i];
    double lu[3];
    for (int i = 0; i < 3; ++i) lu[i] = (1.0 + Lambda[i]) * um[i];
    double gbar = sqrt(1.0 + dot3(lu, lu) / (c * c));
    double tau[3];
    for (int i = 0; i < 3; ++i) tau[i] = q * B[i] / (2.0 * gbar * m * c);

    if (!exact) {
        double tt[3], Lt[3], a[3], b[3], ax[3];
        for (int i = 0; i < 3; ++i) tt[i] = tau[i] / (1.0 - Lambda[i]);
        for (int i = 0; i < 3; ++i) Lt[i] = (1.0 + Lambda[i]) / (1.0 - Lambda[i]);
        double den = 1.0 + dot3(tt, tt);
        for (int i = 0; i < 3; ++i) a[i] = (1.0 + Lt[i]) * um[i];
        cross3(a, tt, ax);
        cross3(ax, tt, b);
        for (int i = 0; i < 3; ++i) up[i] = Lt[i] * um[i] + (ax[i] + b[i]) / den;
    } else {
        /* (I - Lambda - T) u+ = (I + Lambda + T) u-, with T v = v x tau */
        double M[3][3], rhs[3], ut[3];
        cross3(um, tau, ut);
        for (int i = 0; i < 3; ++i) rhs[i] = um[i] + Lambda[i] * um[i] + ut[i];
        /* v x tau = (v1 t2 - v2 t1, v2 t0 - v0 t2, v0 t1 - v1 t0) as a matrix acting on v */
        double T[3][3] = {{0.0, tau[2], -tau[1]}, {-tau[2], 0.0, tau[0]}, {tau[1], -tau[0], 0.0}};
        for (int r = 0; r < 3; ++r)
            for (int col = 0; col < 3; ++col)
                M[r][col] = (r == col ? 1.0 - Lambda[r] : 0.0) - T[r][col];
        solve3(M, rhs, up);
    }
    for (int i = 0; i < 3; ++i) u[i] = up[i] + eps[i];
}

/* Solve the 3x3 system M x = b by Gaussian elimination with partial pivoting. */
static void solve3_gauss(const double M0[3][3], const double b0[3], double x[3])
{
    double M[3][3], b[3];
    memcpy(M, M0, sizeof(M));
    memcpy(b, b0, sizeof(b));
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int r = col + 1; r < 3; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (piv != col) {
            for (int k = 0; k < 3; ++k) {
                double tmp = M[col][k];
                M[col][k] = M[piv][k];
                M[piv][k] = tmp;
            }
            double tb = b[col];
            b[col] = b[piv];
            b[piv] = tb;
        }
        for (int r = col + 1; r < 3; ++r) {
            double f = M[r][col] / M[col][col];
            for (int k = col; k < 3; ++k) M[r][k] -= f * M[col][k];
            b[r] -= f * b[col];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < 3; ++k) acc -= M[r][k] * x[k];
        x[r] = acc / M[r][r];
    }
}

/* Combined shearing + expanding box (the combination Sec. 5 leaves for future
 * work; this library's formulation).  The KSB-OA momentum equation (eq. OAu)
 * in the coordinates xi = L^{-1} x of the expanding box gains the KEB term
 * -L^{-1} dL/dt u' (eq. EBu).  Discretised like eqs. OAu_disc and EBu_disc
 * together:
 *   (I - Lambda - T - S) u+ = (I + Lambda + T + S) u-,
 * T v = v x tt, tt = tau/gbar + dt Omega0 e_z, S v = (S_2 . v) e_y with the
 * alpha terms of Sec. 2.2 (a2 = s Omega0 x^n / c, x^n the physical radial
 * coordinate from the box centre), Lambda = -(dt/2) L^{-1} dL/dt (diagonal).
 * gbar: the root >= 1 of
 *   gbar^2 = 1 + [((I + Lambda) u-)^2 + 2 a1 u-_x u-_y + 2 a2 (u-.eps) u-_y / gbar] / c^2,
 * which is Sec. 2.2's relation for Lambda = 0 and Sec. 3.2's definition for
 * Omega0 = 0.  The 3x3 system is solved directly.  u'^{n+1/2} = u+ + eps. */
void ora_push_sxe(double q, double m, double c, double s, double Omega0, double xc, const double Lambda[3],
                  const double E[3], const double B[3], double u[3], double *gbar_out)
{
    double eps[3], um[3];
    for (int i = 0; i < 3; ++i) eps[i] = q * E[i] / (2.0 * m);
    for (int i = 0; i < 3; ++i) um[i] = u[i] + eps[i];
    double alpha1 = s * Omega0 / 2.0;
    double alpha2 = s * Omega0 * xc / c;
    double c2 = c * c;
    double lu[3];
    for (int i = 0; i < 3; ++i) lu[i] = (1.0 + Lambda[i]) * um[i];
    double ue = dot3(um, eps);
    double A = 1.0 + (dot3(lu, lu) + 2.0 * alpha1 * um[0] * um[1]) / c2;
    double C = 2.0 * alpha2 * ue * um[1] / c2;
    /* Newton on gbar^3 - A gbar - C = 0 from the Lambda-corrected Lorentz factor */
    double g = sqrt(1.0 + dot3(lu, lu) / c2);
    for (int it = 0; it < 60; ++it) {
        double f = g * g * g - A * g - C;
        double dg = f / (3.0 * g * g - A);
        g -= dg;
        if (fabs(dg) <= 1e-16 * g) break;
    }
    if (gbar_out) *gbar_out = g;
    double et[3], tt[3];
    for (int i = 0; i < 3; ++i) et[i] = eps[i] / (c * g);
    for (int i = 0; i < 3; ++i) tt[i] = q * B[i] / (2.0 * m * c) / g;
    tt[2] += Omega0;
    double S2[3] = {alpha1 + alpha2 * et[0], alpha2 * et[1], alpha2 * et[2]};
    /* rows of K = Lambda + T + S: (K v)_r = Lambda_r v_r + (v x tt)_r + [r == y] S_2 . v */
    double K[3][3] = {{Lambda[0], tt[2], -tt[1]}, {-tt[2], Lambda[1], tt[0]}, {tt[1], -tt[0], Lambda[2]}};
    for (int k = 0; k < 3; ++k) K[1][k] += S2[k];
    double M[3][3], rhs[3];
    for (int r = 0; r < 3; ++r) {
        rhs[r] = um[r];
        for (int k = 0; k < 3; ++k) {
            M[r][k] = (r == k ? 1.0 : 0.0) - K[r][k];
            rhs[r] += K[r][k] * um[k];
        }
    }
    double up[3];
    solve3_gauss(M, rhs, up);
    for (int i = 0; i < 3; ++i) u[i] = up[i] + eps[i];
}

/* ======================================================================== */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the samplers        */
/* ======================================================================== */

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Stream tags in the third counter word, so the draws never overlap. */
#define ORA_TAG_ESCAPE 0x45534350u /* "ESCP" */
#define ORA_TAG_ENERGY 0x494E4A54u /* "INJT" */
#define ORA_TAG_DIRECT 0x44495243u /* "DIRC" */

static void ora_draw(uint32_t id, uint32_t seed, int64_t step, uint32_t tag, uint32_t word3,
                     uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32), tag, word3};
    uint32_t key[2] = {id, seed};
    ora_philox4x32_10(ctr, key, out);
}

/* open-interval uniform (0,1) from a 32-bit word */
static double u01(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Probabilistic escape: escape iff the first Philox word is below
 * floor(p 2^32), an integer comparison so every implementation agrees. */
int ora_escape_draw(uint32_t id, uint32_t seed, int64_t step, double p)
{
    double pc = p < 0.0 ? 0.0 : p;
    uint32_t thresh = pc >= 1.0 ? 0xFFFFFFFFu : (uint32_t)floor(pc * 4294967296.0);
    uint32_t r[4];
    ora_draw(id, seed, step, ORA_TAG_ESCAPE, 0u, r);
    return r[0] < thresh;
}

/* Maxwell-Juettner sample, u = c * gamma*beta, isotropic.
 * The kinetic energy e = gamma - 1 has density proportional to
 *   (1 + e) sqrt(e (e + 2)) exp(-e/theta).
 * Since sqrt(e + 2) <= sqrt(2) + sqrt(e), this is bounded by
 *   (sqrt2 e^1/2 + e + sqrt2 e^3/2 + e^2) exp(-e/theta),
 * a mixture of Gamma(3/2), Gamma(2), Gamma(5/2), Gamma(3) laws of scale theta.
 * Draw from the mixture and accept with probability
 *   sqrt(e + 2) / (sqrt2 + sqrt(e))  (>= 1/sqrt2 for every e).
 * Attempt a uses counters (step, ENERGY, 2a) and (step, ENERGY, 2a+1); after
 * 64 rejections (probability < 1e-34) the last draw is kept.  The direction
 * uses counter (step, DIRECT, 0).  Returns the number of attempts used. */
int ora_sample_mj(uint32_t id, uint32_t seed, int64_t step, double theta, double c, double u[3])
{
    const double sqrt2 = sqrt(2.0), sqrtpi = sqrt(3.14159265358979323846);
    double w[4];
    w[0] = sqrt2 * (sqrtpi / 2.0) * pow(theta, 1.5);        /* Gamma(3/2) */
    w[1] = 1.0 * theta * theta;                            /* Gamma(2)   */
    w[2] = sqrt2 * (3.0 * sqrtpi / 4.0) * pow(theta, 2.5); /* Gamma(5/2) */
    w[3] = 2.0 * theta * theta * theta;                    /* Gamma(3)   */
    double wsum = w[0] + w[1] + w[2] + w[3];

    double e = 0.0;
    int attempt;
    for (attempt = 0; attempt < 64; ++attempt) {
        uint32_t r0[4], r1[4];
        ora_draw(id, seed, step, ORA_TAG_ENERGY, 2u * (uint32_t)attempt, r0);
        ora_draw(id, seed, step, ORA_TAG_ENERGY, 2u * (uint32_t)attempt + 1u, r1);
        double pick = u01(r0[0]) * wsum;
        double ex1 = -log(u01(r0[1]));
        double ex2 = -log(u01(r0[2]));
        double ex3 = -log(u01(r0[3]));
        double cb = cos(TWO_PI * u01(r1[1]));
        double half = -log(u01(r1[0])) * cb * cb; /* Gamma(1/2) of unit scale: Z^2/2 */
        if (pick < w[0])
            e = theta * (ex1 + half);
        else if (pick < w[0] + w[1])
            e = theta * (ex1 + ex2);
        else if (pick < w[0] + w[1] + w[2])
            e = theta * (ex1 + ex2 + half);
        else
            e = theta * (ex1 + ex2 + ex3);
        double accept = sqrt(e + 2.0) / (sqrt2 + sqrt(e));
        if (u01(r1[2]) < accept) break;
    }
    if (attempt == 64) attempt = 63;

    uint32_t rd[4];
    ora_draw(id, seed, step, ORA_TAG_DIRECT, 0u, rd);
    double mu = 2.0 * u01(rd[0]) - 1.0;
    double phi = TWO_PI * u01(rd[1]);
    double umag = c * sqrt(e * (e + 2.0));
    double st = sqrt(1.0 - mu * mu);
    u[0] = umag * st * cos(phi);
    u[1] = umag * st * sin(phi);
    u[2] = umag * mu;
    return attempt + 1;
}

/* ======================================================================== */
/* Grid access with periodic / shearing-periodic identification              */
/* ======================================================================== */

static int64_t floordiv(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

static int64_t wrapi(int64_t a, int64_t n)
{
    int64_t r = a % n;
    return r < 0 ? r + n : r;
}

static int64_t gidx(const ora_params *p, int comp, int64_t i, int64_t j, int64_t k)
{
    return ((comp * (int64_t)p->nz + k) * p->ny + j) * p->nx + i;
}

/* Displacement along y of the shearing-periodic boundary,
 * Dy_s = s Omega0 (x_o - x_i) t (Sec. 2.1), reduced modulo the box length. */
double ora_shear_shift(const ora_params *p, double t)
{
    double d;
    if (p->box == ORA_BOX_SHEAR) {
        d = p->s * p->Omega0 * (double)p->nx * t;
    } else if (p->box == ORA_BOX_SHEAR_EXPAND) {
        /* In the expanding coordinates xi = L^{-1} x the two x faces slide
         * apart along xi_y at s Omega0 (l_1 nx) / l_2, so
         * Dxi_s(t) = s Omega0 nx int_0^t l_1/l_2 dt' with l_i = exp(rate_i t). */
        double dr = p->rate[0] - p->rate[1];
        double I = dr == 0.0 ? t : expm1(dr * t) / dr;
        d = p->s * p->Omega0 * (double)p->nx * I;
    } else {
        return 0.0;
    }
    d = fmod(d, (double)p->ny);
    if (d < 0.0) d += (double)p->ny;
    return d;
}

/* Value of component comp of field F at array index (i,j,k), which may lie
 * outside the box.  Periodic in y and z; across x the shearing-periodic
 * condition X(x_i, y) = X(x_o, y - Dy_s) identifies a point w box lengths to
 * the right with the interior point shifted by w Dy_s in y (linear
 * interpolation for a fractional shift). */
static double fetch(const ora_params *p, const double *F, int comp, int64_t i, int64_t j, int64_t k,
                    double dys)
{
    int64_t w = floordiv(i, p->nx);
    int64_t ii = i - w * p->nx;
    int64_t kk = wrapi(k, p->nz);
    if (w != 0 && dys != 0.0) {
        double yy = (double)j + (double)w * dys;
        double y0 = floor(yy);
        double f = yy - y0;
        int64_t j0 = wrapi((int64_t)y0, p->ny), j1 = wrapi((int64_t)y0 + 1, p->ny);
        return (1.0 - f) * F[gidx(p, comp, ii, j0, kk)] + f * F[gidx(p, comp, ii, j1, kk)];
    }
    return F[gidx(p, comp, ii, wrapi(j, p->ny), kk)];
}

/* Add v to component comp of F at index (i,j,k), possibly outside the box:
 * the adjoint of fetch(), so the total added is v whatever the shift. */
static void accumulate(const ora_params *p, double *F, int comp, int64_t i, int64_t j, int64_t k,
                       double dys, double v)
{
    int64_t w = floordiv(i, p->nx);
    int64_t ii = i - w * p->nx;
    int64_t kk = wrapi(k, p->nz);
    if (w != 0 && dys != 0.0) {
        double yy = (double)j + (double)w * dys;
        double y0 = floor(yy);
        double f = yy - y0;
        int64_t j0 = wrapi((int64_t)y0, p->ny), j1 = wrapi((int64_t)y0 + 1, p->ny);
        F[gidx(p, comp, ii, j0, kk)] += (1.0 - f) * v;
        F[gidx(p, comp, ii, j1, kk)] += f * v;
        return;
    }
    F[gidx(p, comp, ii, wrapi(j, p->ny), kk)] += v;
}

/* ======================================================================== */
/* Shape functions, gather and charge-conserving deposit                     */
/* ======================================================================== */

/* B-spline shape of order 1 (linear) or 2 (quadratic) at distance d from a grid point. */
static double shape(int order, double d)
{
    double a = fabs(d);
    if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
    if (a <= 0.5) return 0.75 - a * a;
    if (a < 1.5) return 0.5 * (1.5 - a) * (1.5 - a);
    return 0.0;
}

/* stagger (in cells) of each field component along x, y, z */
static const double E_STAG[3][3] = {{0.5, 0.0, 0.0}, {0.0, 0.5, 0.0}, {0.0, 0.0, 0.5}};
static const double B_STAG[3][3] = {{0.0, 0.5, 0.5}, {0.5, 0.0, 0.5}, {0.5, 0.5, 0.0}};

static double gather_one(const ora_params *p, const double *F, int comp, const double stag[3],
                         const double x[3], double dys)
{
    /* a wide stencil of 6 points per axis; points outside the support weigh zero */
    int64_t base[3];
    double w[3][6];
    for (int a = 0; a < 3; ++a) {
        base[a] = (int64_t)floor(x[a] - stag[a]) - 2;
        for (int m = 0; m < 6; ++m) w[a][m] = shape(p->order, x[a] - ((double)(base[a] + m) + stag[a]));
    }
    double sum = 0.0;
    for (int n = 0; n < 6; ++n)
        for (int m = 0; m < 6; ++m)
            for (int l = 0; l < 6; ++l) {
                double ww = w[0][l] * w[1][m] * w[2][n];
                if (ww == 0.0) continue;
                sum += ww * fetch(p, F, comp, base[0] + l, base[1] + m, base[2] + n, dys);
            }
    return sum;
}

/* Interpolate E and B to the particle position x at time t (shape of the
 * configured order at each component's own staggered location). */
void ora_gather(const ora_params *p, const double *E, const double *B, double t,
                const double x[3], double Ep[3], double Bp[3])
{
    double dys = ora_shear_shift(p, t);
    for (int c = 0; c < 3; ++c) {
        Ep[c] = gather_one(p, E, c, E_STAG[c], x, dys);
        Bp[c] = gather_one(p, B, c, B_STAG[c], x, dys);
    }
}

/* Charge-conserving current of one particle of charge q moving on a straight
 * line from x0 to x1 (less than one cell per axis), after Esirkepov:
 *   W_x = (S1x - S0x) (S1y S1z / 3 + S0y S1z / 6 + S1y S0z / 6 + S0y S0z / 3),
 * similarly W_y, W_z; J_x(i+1/2) = J_x(i-1/2) - q W_x(i) (dx = dt = 1).
 * Points across the x boundary are folded with the shift at time t. */
void ora_deposit_current(const ora_params *p, double *J, double t, double q,
                         const double x0[3], const double x1[3])
{
    double dys = ora_shear_shift(p, t);
    int64_t base[3];
    double S0[3][6], S1[3][6];
    for (int a = 0; a < 3; ++a) {
        double lo = x0[a] < x1[a] ? x0[a] : x1[a];
        base[a] = (int64_t)floor(lo) - 2;
        for (int m = 0; m < 6; ++m) {
            S0[a][m] = shape(p->order, x0[a] - (double)(base[a] + m));
            S1[a][m] = shape(p->order, x1[a] - (double)(base[a] + m));
        }
    }
    double W[3][6][6][6]; /* [component][n(z)][m(y)][l(x)] */
    for (int n = 0; n < 6; ++n)
        for (int m = 0; m < 6; ++m)
            for (int l = 0; l < 6; ++l) {
                double dSx = S1[0][l] - S0[0][l];
                double dSy = S1[1][m] - S0[1][m];
                double dSz = S1[2][n] - S0[2][n];
                W[0][n][m][l] = dSx * (S1[1][m] * S1[2][n] / 3.0 + S0[1][m] * S1[2][n] / 6.0
                                       + S1[1][m] * S0[2][n] / 6.0 + S0[1][m] * S0[2][n] / 3.0);
                W[1][n][m][l] = dSy * (S1[0][l] * S1[2][n] / 3.0 + S0[0][l] * S1[2][n] / 6.0
                                       + S1[0][l] * S0[2][n] / 6.0 + S0[0][l] * S0[2][n] / 3.0);
                W[2][n][m][l] = dSz * (S1[0][l] * S1[1][m] / 3.0 + S0[0][l] * S1[1][m] / 6.0
                                       + S1[0][l] * S0[1][m] / 6.0 + S0[0][l] * S0[1][m] / 3.0);
            }
    /* J_x: running sum along x; J_x at array index i sits at i + 1/2 */
    for (int n = 0; n < 6; ++n)
        for (int m = 0; m < 6; ++m) {
            double run = 0.0;
            for (int l = 0; l < 6; ++l) {
                run -= q * W[0][n][m][l];
                if (run != 0.0) accumulate(p, J, 0, base[0] + l, base[1] + m, base[2] + n, dys, run);
            }
        }
    for (int n = 0; n < 6; ++n)
        for (int l = 0; l < 6; ++l) {
            double run = 0.0;
            for (int m = 0; m < 6; ++m) {
                run -= q * W[1][n][m][l];
                if (run != 0.0) accumulate(p, J, 1, base[0] + l, base[1] + m, base[2] + n, dys, run);
            }
        }
    for (int m = 0; m < 6; ++m)
        for (int l = 0; l < 6; ++l) {
            double run = 0.0;
            for (int n = 0; n < 6; ++n) {
                run -= q * W[2][n][m][l];
                if (run != 0.0) accumulate(p, J, 2, base[0] + l, base[1] + m, base[2] + n, dys, run);
            }
        }
}

/* Node charge density of one particle (used by the continuity checks). */
void ora_deposit_rho(const ora_params *p, double *rho, double t, double q, const double x[3])
{
    double dys = ora_shear_shift(p, t);
    int64_t base[3];
    double S[3][6];
    for (int a = 0; a < 3; ++a) {
        base[a] = (int64_t)floor(x[a]) - 2;
        for (int m = 0; m < 6; ++m) S[a][m] = shape(p->order, x[a] - (double)(base[a] + m));
    }
    for (int n = 0; n < 6; ++n)
        for (int m = 0; m < 6; ++m)
            for (int l = 0; l < 6; ++l) {
                double v = q * S[0][l] * S[1][m] * S[2][n];
                if (v != 0.0) accumulate(p, rho, 0, base[0] + l, base[1] + m, base[2] + n, dys, v);
            }
}

/* Shearing box: the current collected from x^n -> x' is J'(x'); the comoving
 * current on the lab grid follows by advecting it along y by v_{s,y} dt / 2 =
 * -s Omega0 x dt / 2 (Sec. 2.2), x of each component's own location measured
 * from the box centre.  Linear interpolation per x column, periodic in y. */
void ora_ksb_advect_current(const ora_params *p, double *J)
{
    int64_t ny = p->ny;
    double *col = (double *)malloc(sizeof(double) * (size_t)ny);
    for (int comp = 0; comp < 3; ++comp)
        for (int64_t k = 0; k < p->nz; ++k)
            for (int64_t i = 0; i < p->nx; ++i) {
                double xc = (double)i + E_STAG[comp][0] - 0.5 * (double)p->nx;
                double d = -p->s * p->Omega0 * xc / 2.0; /* content moves by d along y */
                for (int64_t j = 0; j < ny; ++j) col[j] = J[gidx(p, comp, i, j, k)];
                for (int64_t j = 0; j < ny; ++j) {
                    double ys = (double)j - d;
                    double y0 = floor(ys);
                    double f = ys - y0;
                    int64_t j0 = wrapi((int64_t)y0, ny), j1 = wrapi((int64_t)y0 + 1, ny);
                    J[gidx(p, comp, i, j, k)] = (1.0 - f) * col[j0] + f * col[j1];
                }
            }
    free(col);
}

/* ======================================================================== */
/* Field solvers                                                             */
/* ======================================================================== */

static int64_t ncell(const ora_params *p) { return (int64_t)p->nx * p->ny * p->nz; }

/* Yee curl of E (result at B locations) and of B (result at E locations),
 * optionally scaling component c of the input by sc[c] first. */
static void curl_E(const ora_params *p, const double *E, const double sc[3], double *out, double dys)
{
    for (int64_t k = 0; k < p->nz; ++k)
        for (int64_t j = 0; j < p->ny; ++j)
            for (int64_t i = 0; i < p->nx; ++i) {
#define EV(c, di, dj, dk) (sc[c] * fetch(p, E, c, i + (di), j + (dj), k + (dk), dys))
                out[gidx(p, 0, i, j, k)] = (EV(2, 0, 1, 0) - EV(2, 0, 0, 0)) - (EV(1, 0, 0, 1) - EV(1, 0, 0, 0));
                out[gidx(p, 1, i, j, k)] = (EV(0, 0, 0, 1) - EV(0, 0, 0, 0)) - (EV(2, 1, 0, 0) - EV(2, 0, 0, 0));
                out[gidx(p, 2, i, j, k)] = (EV(1, 1, 0, 0) - EV(1, 0, 0, 0)) - (EV(0, 0, 1, 0) - EV(0, 0, 0, 0));
#undef EV
            }
}

static void curl_B(const ora_params *p, const double *B, const double sc[3], double *out, double dys)
{
    for (int64_t k = 0; k < p->nz; ++k)
        for (int64_t j = 0; j < p->ny; ++j)
            for (int64_t i = 0; i < p->nx; ++i) {
#define BV(c, di, dj, dk) (sc[c] * fetch(p, B, c, i + (di), j + (dj), k + (dk), dys))
                out[gidx(p, 0, i, j, k)] = (BV(2, 0, 0, 0) - BV(2, 0, -1, 0)) - (BV(1, 0, 0, 0) - BV(1, 0, 0, -1));
                out[gidx(p, 1, i, j, k)] = (BV(0, 0, 0, 0) - BV(0, 0, 0, -1)) - (BV(2, 0, 0, 0) - BV(2, -1, 0, 0));
                out[gidx(p, 2, i, j, k)] = (BV(1, 0, 0, 0) - BV(1, -1, 0, 0)) - (BV(0, 0, 0, 0) - BV(0, 0, -1, 0));
#undef BV
            }
}

/* Standard leapfrog (periodic and leaky boxes):
 * B^{n+1/2} = B^n - (c/2) curl E^n;  E^{n+1} = E^n + c curl B^{n+1/2} - 4 pi J;
 * B^{n+1} = B^{n+1/2} - (c/2) curl E^{n+1}. */
void ora_yee_update(const ora_params *p, double *E, double *B, const double *J)
{
    int64_t N = 3 * ncell(p);
    double *cu = (double *)malloc(sizeof(double) * (size_t)N);
    const double one[3] = {1.0, 1.0, 1.0};
    curl_E(p, E, one, cu, 0.0);
    for (int64_t q = 0; q < N; ++q) B[q] -= 0.5 * p->c * cu[q];
    curl_B(p, B, one, cu, 0.0);
    for (int64_t q = 0; q < N; ++q) E[q] += p->c * cu[q] - FOUR_PI * J[q];
    curl_E(p, E, one, cu, 0.0);
    for (int64_t q = 0; q < N; ++q) B[q] -= 0.5 * p->c * cu[q];
    free(cu);
}

/* Expanding box (Sec. 3.2): lab fields E, B are carried; at each time level
 * X' = ell L^{-1} X; the leapfrog advances B', E' with the curls acting on
 * L^2 X' / ell = L X and the source -4 pi (ell J'), which the deposit in x'
 * gives directly; the result is transformed back with L at the new level.
 * J here is the deposited ell J'.  t is t^n. */
void ora_keb_field_update(const ora_params *p, double *E, double *B, const double *J, double t)
{
    int64_t nc = ncell(p), N = 3 * nc;
    double *cu = (double *)malloc(sizeof(double) * (size_t)N);
    double l0[3], lh[3], l1[3];
    for (int a = 0; a < 3; ++a) {
        l0[a] = exp(p->rate[a] * t);
        lh[a] = exp(p->rate[a] * (t + 0.5));
        l1[a] = exp(p->rate[a] * (t + 1.0));
    }
    double ell0 = l0[0] * l0[1] * l0[2], ellh = lh[0] * lh[1] * lh[2], ell1 = l1[0] * l1[1] * l1[2];

    /* B'^{n+1/2} = B'^n - (c/2) curl(L^n E^n);  B^{n+1/2} = L B' / ell at n+1/2 */
    curl_E(p, E, l0, cu, 0.0);
    for (int c = 0; c < 3; ++c)
        for (int64_t q = 0; q < nc; ++q) {
            double Bp = ell0 / l0[c] * B[c * nc + q] - 0.5 * p->c * cu[c * nc + q];
            B[c * nc + q] = lh[c] / ellh * Bp;
        }
    /* E'^{n+1} = E'^n + c curl(L B^{n+1/2}) - 4 pi ell J';  E^{n+1} = L E' / ell at n+1 */
    curl_B(p, B, lh, cu, 0.0);
    for (int c = 0; c < 3; ++c)
        for (int64_t q = 0; q < nc; ++q) {
            double Ep = ell0 / l0[c] * E[c * nc + q] + p->c * cu[c * nc + q] - FOUR_PI * J[c * nc + q];
            E[c * nc + q] = l1[c] / ell1 * Ep;
        }
    /* B'^{n+1} = B'^{n+1/2} - (c/2) curl(L^{n+1} E^{n+1});  B^{n+1} = L B' / ell at n+1 */
    curl_E(p, E, l1, cu, 0.0);
    for (int c = 0; c < 3; ++c)
        for (int64_t q = 0; q < nc; ++q) {
            double Bp = ellh / lh[c] * B[c * nc + q] - 0.5 * p->c * cu[c * nc + q];
            B[c * nc + q] = l1[c] / ell1 * Bp;
        }
    free(cu);
}

/* Right-hand sides of the shearing-box field equations (Sec. 2.1) on the Yee
 * grid, with V(x) = -s Omega0 x (x from the box centre):
 *   F_B  = -c curl E' - V d_y B - s Omega0 B_x e_y
 *   F_Ex = (c curl B)_x - 4 pi J'_x + V d_y E'_x - V d_x E'_y
 *   F_Ey = (c curl B)_y - 4 pi J'_y - V d_y E'_y - V (d_x E'_x + d_z E'_z)
 *   F_Ez = (c curl B)_z - 4 pi J'_z + V d_y E'_z - V d_z E'_y
 * d_y of the advected component: first-order upwind for its transport
 * velocity (V in the B and E'_y rows, -V in the E'_x and E'_z rows); other
 * V-terms: centred difference, averaged in y onto the component's location;
 * B_x in the B_y row: average of the four surrounding B_x.  Ghost values
 * across x use the shear shift at time t. */
static void ksb_rhs_scaled(const ora_params *p, const double *E, const double *B, const double *J, double t,
                           const double sig[3], double vf, double rx, double rz, double *FE, double *FB);

void ora_ksb_rhs(const ora_params *p, const double *E, const double *B, const double *J,
                 double t, double *FE, double *FB)
{
    const double one[3] = {1.0, 1.0, 1.0};
    ksb_rhs_scaled(p, E, B, J, t, one, 1.0, 1.0, 1.0, FE, FB);
}

/* The right-hand sides above with the factors of the expanding coordinates
 * (see ora_sxe_rhs): the curls act on sig (.) X, the shear velocity and the
 * shear term carry vf, the -V dx E'_y and -V dz E'_y terms rx and rz.  With
 * all factors one this is ora_ksb_rhs exactly. */
static void ksb_rhs_scaled(const ora_params *p, const double *E, const double *B, const double *J, double t,
                           const double sig[3], double vf, double rx, double rz, double *FE, double *FB)
{
    double dys = ora_shear_shift(p, t);
    double sO = p->s * p->Omega0 * vf, c = p->c;
    for (int64_t k = 0; k < p->nz; ++k)
        for (int64_t j = 0; j < p->ny; ++j)
            for (int64_t i = 0; i < p->nx; ++i) {
#define Ef(cc, di, dj, dk) fetch(p, E, cc, i + (di), j + (dj), k + (dk), dys)
#define Bf(cc, di, dj, dk) fetch(p, B, cc, i + (di), j + (dj), k + (dk), dys)
                double VN = -sO * ((double)i - 0.5 * p->nx);       /* at x-nodes */
                double VH = -sO * ((double)i + 0.5 - 0.5 * p->nx); /* at x half-points */
#define SEf(cc, di, dj, dk) (sig[cc] * Ef(cc, di, dj, dk))
#define SBf(cc, di, dj, dk) (sig[cc] * Bf(cc, di, dj, dk))
                double curlEx = (SEf(2, 0, 1, 0) - SEf(2, 0, 0, 0)) - (SEf(1, 0, 0, 1) - SEf(1, 0, 0, 0));
                double curlEy = (SEf(0, 0, 0, 1) - SEf(0, 0, 0, 0)) - (SEf(2, 1, 0, 0) - SEf(2, 0, 0, 0));
                double curlEz = (SEf(1, 1, 0, 0) - SEf(1, 0, 0, 0)) - (SEf(0, 0, 1, 0) - SEf(0, 0, 0, 0));
                double curlBx = (SBf(2, 0, 0, 0) - SBf(2, 0, -1, 0)) - (SBf(1, 0, 0, 0) - SBf(1, 0, 0, -1));
                double curlBy = (SBf(0, 0, 0, 0) - SBf(0, 0, 0, -1)) - (SBf(2, 0, 0, 0) - SBf(2, -1, 0, 0));
                double curlBz = (SBf(1, 0, 0, 0) - SBf(1, -1, 0, 0)) - (SBf(0, 0, 0, 0) - SBf(0, 0, -1, 0));
#undef SEf
#undef SBf
                /* upwinded d_y for transport velocity v */
#define UPB(cc, v) ((v) > 0.0 ? Bf(cc, 0, 0, 0) - Bf(cc, 0, -1, 0) : Bf(cc, 0, 1, 0) - Bf(cc, 0, 0, 0))
#define UPE(cc, v) ((v) > 0.0 ? Ef(cc, 0, 0, 0) - Ef(cc, 0, -1, 0) : Ef(cc, 0, 1, 0) - Ef(cc, 0, 0, 0))
                double bx4 = 0.25 * (Bf(0, 0, 0, 0) + Bf(0, 1, 0, 0) + Bf(0, 0, -1, 0) + Bf(0, 1, -1, 0));
                FB[gidx(p, 0, i, j, k)] = -c * curlEx - VN * UPB(0, VN);
                FB[gidx(p, 1, i, j, k)] = -c * curlEy - VH * UPB(1, VH) - sO * bx4;
                FB[gidx(p, 2, i, j, k)] = -c * curlEz - VH * UPB(2, VH);

                double dxEy = 0.5 * ((Ef(1, 1, 0, 0) - Ef(1, 0, 0, 0)) + (Ef(1, 1, -1, 0) - Ef(1, 0, -1, 0)));
                double divxz = 0.5 * ((Ef(0, 0, 0, 0) - Ef(0, -1, 0, 0)) + (Ef(0, 0, 1, 0) - Ef(0, -1, 1, 0))
                                      + (Ef(2, 0, 0, 0) - Ef(2, 0, 0, -1)) + (Ef(2, 0, 1, 0) - Ef(2, 0, 1, -1)));
                double dzEy = 0.5 * ((Ef(1, 0, 0, 1) - Ef(1, 0, 0, 0)) + (Ef(1, 0, -1, 1) - Ef(1, 0, -1, 0)));
                FE[gidx(p, 0, i, j, k)] = c * curlBx - FOUR_PI * J[gidx(p, 0, i, j, k)]
                                          + VH * UPE(0, -VH) - VH * (rx * dxEy);
                FE[gidx(p, 1, i, j, k)] = c * curlBy - FOUR_PI * J[gidx(p, 1, i, j, k)]
                                          - VN * UPE(1, VN) - VN * divxz;
                FE[gidx(p, 2, i, j, k)] = c * curlBz - FOUR_PI * J[gidx(p, 2, i, j, k)]
                                          + VN * UPE(2, -VN) - VN * (rz * dzEy);
#undef UPB
#undef UPE
#undef Ef
#undef Bf
            }
}

/* Shearing-box Maxwell solve (Sec. 2.2): implicit midpoint in time,
 * X^{n+1} = X^n + dt F((X^n + X^{n+1})/2), by fixed-point iteration
 * X^(0) = X^n, X^(k+1) = X^n + dt F((X^n + X^(k))/2), fp_iters sweeps.
 * The midpoint state sits at t^{n+1/2}; t is t^n. */
void ora_ksb_field_solve(const ora_params *p, double *E, double *B, const double *J, double t)
{
    int64_t N = 3 * ncell(p);
    size_t sz = sizeof(double) * (size_t)N;
    double *E0 = (double *)malloc(sz), *B0 = (double *)malloc(sz);
    double *Em = (double *)malloc(sz), *Bm = (double *)malloc(sz);
    double *FE = (double *)malloc(sz), *FB = (double *)malloc(sz);
    memcpy(E0, E, sz);
    memcpy(B0, B, sz);
    for (int it = 0; it < p->fp_iters; ++it) {
        for (int64_t q = 0; q < N; ++q) {
            Em[q] = 0.5 * (E0[q] + E[q]);
            Bm[q] = 0.5 * (B0[q] + B[q]);
        }
        ora_ksb_rhs(p, Em, Bm, J, t + 0.5, FE, FB);
        for (int64_t q = 0; q < N; ++q) {
            E[q] = E0[q] + FE[q];
            B[q] = B0[q] + FB[q];
        }
    }
    free(E0); free(B0); free(Em); free(Bm); free(FE); free(FB);
}

/* Combined shearing + expanding box, fields.  The shearing-box equations
 * (eqs. OAB, OAE) in the expanding coordinates xi = L^{-1} x, with the
 * expanding-frame fields X^ = ell L^{-1} X of Sec. 3.1 (X = E', B):
 *   F_B^  = -c curl(L^2 E^/ell) - V^ d_y B^ - s Omega0 (l_1/l_2) B^_x e_y
 *   F_E^x = [c curl(L^2 B^/ell)]_x - 4 pi ell J^_x + V^ d_y E^_x - V^ (l_2/l_1)^2 d_x E^_y
 *   F_E^y = [c curl(L^2 B^/ell)]_y - 4 pi ell J^_y - V^ d_y E^_y - V^ (d_x E^_x + d_z E^_z)
 *   F_E^z = [c curl(L^2 B^/ell)]_z - 4 pi ell J^_z + V^ d_y E^_z - V^ (l_2/l_3)^2 d_z E^_y
 * all derivatives along xi, V^ = -s Omega0 (l_1/l_2)(xi_x - nx/2): each
 * shear term of Sec. 2.1 multiplied by ell L^{-1} with X = L X^/ell and
 * d/dx_a = (1/l_a) d/dxi_a.  L at time t (the midpoint state's level). */
void ora_sxe_rhs(const ora_params *p, const double *Eh, const double *Bh, const double *J,
                 double t, double *FE, double *FB)
{
    double l[3];
    for (int a = 0; a < 3; ++a) l[a] = exp(p->rate[a] * t);
    double ell = l[0] * l[1] * l[2];
    double sig[3] = {l[0] * l[0] / ell, l[1] * l[1] / ell, l[2] * l[2] / ell};
    double rx = (l[1] / l[0]) * (l[1] / l[0]), rz = (l[1] / l[2]) * (l[1] / l[2]);
    ksb_rhs_scaled(p, Eh, Bh, J, t, sig, l[0] / l[1], rx, rz, FE, FB);
}

/* Combined box: J' collected in xi is advected along xi_y by
 * v_{s,y} dt / (2 l_2) = -s Omega0 (l_1/l_2) (xi_x - nx/2) dt / 2 at t^{n+1/2}. */
static void advect_y(const ora_params *p, double *J, double vf)
{
    int64_t ny = p->ny;
    double *col = (double *)malloc(sizeof(double) * (size_t)ny);
    for (int comp = 0; comp < 3; ++comp)
        for (int64_t k = 0; k < p->nz; ++k)
            for (int64_t i = 0; i < p->nx; ++i) {
                double xc = (double)i + E_STAG[comp][0] - 0.5 * (double)p->nx;
                double d = -p->s * p->Omega0 * vf * xc / 2.0; /* content moves by d along y */
                for (int64_t j = 0; j < ny; ++j) col[j] = J[gidx(p, comp, i, j, k)];
                for (int64_t j = 0; j < ny; ++j) {
                    double ys = (double)j - d; /* the value now at j came from j - d */
                    double y0 = floor(ys);
                    double f = ys - y0;
                    int64_t j0 = wrapi((int64_t)y0, ny), j1 = wrapi((int64_t)y0 + 1, ny);
                    J[gidx(p, comp, i, j, k)] = (1.0 - f) * col[j0] + f * col[j1];
                }
            }
    free(col);
}

void ora_sxe_advect_current(const ora_params *p, double *J, double t)
{
    advect_y(p, J, exp((p->rate[0] - p->rate[1]) * (t + 0.5)));
}

/* Combined box: implicit midpoint on the expanding-frame fields, N
 * fixed-point sweeps as in Sec. 2.2, X^ = ell L^{-1} X at t^n, the
 * right-hand sides at t^{n+1/2}, back to X = L X^ / ell at t^{n+1}.
 * J is the collected ell J^ (deposited in xi).  t is t^n. */
void ora_sxe_field_solve(const ora_params *p, double *E, double *B, const double *J, double t)
{
    int64_t nc = ncell(p), N = 3 * nc;
    size_t sz = sizeof(double) * (size_t)N;
    double l0[3], l1[3];
    for (int a = 0; a < 3; ++a) {
        l0[a] = exp(p->rate[a] * t);
        l1[a] = exp(p->rate[a] * (t + 1.0));
    }
    double ell0 = l0[0] * l0[1] * l0[2], ell1 = l1[0] * l1[1] * l1[2];
    double *E0 = (double *)malloc(sz), *B0 = (double *)malloc(sz);
    double *Em = (double *)malloc(sz), *Bm = (double *)malloc(sz);
    double *FE = (double *)malloc(sz), *FB = (double *)malloc(sz);
    for (int c = 0; c < 3; ++c)
        for (int64_t q = 0; q < nc; ++q) {
            E0[c * nc + q] = ell0 / l0[c] * E[c * nc + q];
            B0[c * nc + q] = ell0 / l0[c] * B[c * nc + q];
        }
    memcpy(E, E0, sz); /* E, B hold the iterate X^(k) in expanding-frame form */
    memcpy(B, B0, sz);
    for (int it = 0; it < p->fp_iters; ++it) {
        for (int64_t q = 0; q < N; ++q) {
            Em[q] = 0.5 * (E0[q] + E[q]);
            Bm[q] = 0.5 * (B0[q] + B[q]);
        }
        ora_sxe_rhs(p, Em, Bm, J, t + 0.5, FE, FB);
        for (int64_t q = 0; q < N; ++q) {
            E[q] = E0[q] + FE[q];
            B[q] = B0[q] + FB[q];
        }
    }
    for (int c = 0; c < 3; ++c)
        for (int64_t q = 0; q < nc; ++q) {
            E[c * nc + q] *= l1[c] / ell1;
            B[c * nc + q] *= l1[c] / ell1;
        }
    free(E0); free(B0); free(Em); free(Bm); free(FE); free(FB);
}

/* ======================================================================== */
/* The step                                                                  */
/* ======================================================================== */

static void wrap_coord(double *x, int64_t n)
{
    if (*x >= (double)n) *x -= (double)n;
    if (*x < 0.0) {
        *x += (double)n;
        if (*x >= (double)n) *x = 0.0; /* -tiny + n rounded up to n: same point as 0 */
    }
}

/* One PIC step n -> n+1 of the configured box.
 *  periodic / leaky (standard PIC, Sec. 1 and Sec. 4.1):
 *    gather E^n, B^n at x^n; Boris u^{n-1/2} -> u^{n+1/2}; x^{n+1} = x^n + u/gamma;
 *    deposit J^{n+1/2}; [leaky: Dr += u/gamma, escape test, reinjection];
 *    leapfrog field update.
 *  shearing box (KSB-OA, the five steps of Sec. 2.2):
 *    gather E'^n, B^n at x^n, KSB push; x' = x^n + u'/gamma'; deposit J' from
 *    x^n -> x', advect it along y; x^{n+1} = x' - s Omega0 (x'+x^n)/2 dt e_y;
 *    implicit-midpoint Maxwell solve.
 *  expanding box (KEB, the four steps of Sec. 3.2):
 *    gather lab E, B at x'^n; modified Boris; x'^{n+1} = x'^n + L^{-1}u/gamma
 *    with L at t^{n+1/2}; deposit ell J'; transformed leapfrog. */
/* One particle's part of a step n -> n+1 (see ora_step): gather at x^n,
 * push, position update with the box's boundary identification, current
 * deposit into J (skipped when J is NULL), and the leaky box's escape test and
 * reinjection.  x, u (and dr for the displacement rule) are updated in place;
 * the escape and superluminal counters of *loc are incremented. */
void ora_advance_particle(const ora_params *p, const double *E, const double *B, double *J, int64_t n,
                          double q, double m, uint32_t id, double x[3], double u[3], double dr[3],
                          ora_stepinfo *loc)
{
    double t = (double)n;
    double half_nx = 0.5 * (double)p->nx;
    double Ep[3], Bp[3], x1[3];
    ora_gather(p, E, B, t, x, Ep, Bp);

    if (p->box == ORA_BOX_SHEAR) {
        double dys_end = ora_shear_shift(p, t + 1.0);
        double xc = x[0] - half_nx;
        ora_push_ksb(q, m, p->c, p->s, p->Omega0, xc, Ep, Bp, u, NULL);
        double gp = sqrt(1.0 + dot3(u, u) / (p->c * p->c));
        for (int a = 0; a < 3; ++a) x1[a] = x[a] + u[a] / gp; /* x' */
        {
            double vy = u[1] / gp - p->s * p->Omega0 * xc;
            double v2 = (u[0] / gp) * (u[0] / gp) + vy * vy + (u[2] / gp) * (u[2] / gp);
            if (v2 >= p->c * p->c) loc->superluminal++;
        }
        if (J) ora_deposit_current(p, J, t + 0.5, q, x, x1);
        double xpc = x1[0] - half_nx;
        x1[1] -= p->s * p->Omega0 * (xpc + xc) / 2.0;
        /* shearing-periodic crossing of x: y shifts by Dy_s at t^{n+1} */
        if (x1[0] >= (double)p->nx) {
            x1[0] -= (double)p->nx;
            x1[1] += dys_end;
        } else if (x1[0] < 0.0) {
            x1[0] += (double)p->nx;
            x1[1] -= dys_end;
            if (x1[0] >= (double)p->nx) x1[0] = 0.0;
        }
        x1[1] = fmod(x1[1], (double)p->ny);
        wrap_coord(&x1[1], p->ny);
        wrap_coord(&x1[2], p->nz);
    } else if (p->box == ORA_BOX_SHEAR_EXPAND) {
        /* positions are the expanding coordinates xi; u is the comoving u' */
        double dys_end = ora_shear_shift(p, t + 1.0);
        double Lambda[3], lh[3];
        for (int a = 0; a < 3; ++a) {
            Lambda[a] = -0.5 * p->rate[a];
            lh[a] = exp(p->rate[a] * (t + 0.5));
        }
        double xic = x[0] - half_nx;                 /* xi_x from the box centre */
        double xc = exp(p->rate[0] * t) * xic;       /* physical radial coordinate at t^n */
        ora_push_sxe(q, m, p->c, p->s, p->Omega0, xc, Lambda, Ep, Bp, u, NULL);
        double gp = sqrt(1.0 + dot3(u, u) / (p->c * p->c));
        for (int a = 0; a < 3; ++a) x1[a] = x[a] + u[a] / (gp * lh[a]); /* xi' = xi^n + L^{-1} u'/gamma' */
        {
            double vy = u[1] / gp - p->s * p->Omega0 * xc;
            double v2 = (u[0] / gp) * (u[0] / gp) + vy * vy + (u[2] / gp) * (u[2] / gp);
            if (v2 >= p->c * p->c) loc->superluminal++;
        }
        if (J) ora_deposit_current(p, J, t + 0.5, q, x, x1);
        /* the shear motion along xi_y: v_{s,y} / l_2 at t^{n+1/2} */
        double vf = lh[0] / lh[1];
        x1[1] -= p->s * p->Omega0 * vf * ((x1[0] - half_nx) + xic) / 2.0;
        if (x1[0] >= (double)p->nx) {
            x1[0] -= (double)p->nx;
            x1[1] += dys_end;
        } else if (x1[0] < 0.0) {
            x1[0] += (double)p->nx;
            x1[1] -= dys_end;
            if (x1[0] >= (double)p->nx) x1[0] = 0.0;
        }
        x1[1] = fmod(x1[1], (double)p->ny);
        wrap_coord(&x1[1], p->ny);
        wrap_coord(&x1[2], p->nz);
    } else if (p->box == ORA_BOX_EXPAND) {
        double Lambda[3], lh[3];
        for (int a = 0; a < 3; ++a) {
            Lambda[a] = -0.5 * p->rate[a]; /* -(dt/2) L^{-1} dL/dt for l = exp(rate t) */
            lh[a] = exp(p->rate[a] * (t + 0.5));
        }
        ora_push_keb(q, m, p->c, Lambda, Ep, Bp, u, p->keb_exact);
        double g = sqrt(1.0 + dot3(u, u) / (p->c * p->c));
        for (int a = 0; a < 3; ++a) x1[a] = x[a] + u[a] / (g * lh[a]);
        if (J) ora_deposit_current(p, J, t + 0.5, q, x, x1);
        wrap_coord(&x1[0], p->nx);
        wrap_coord(&x1[1], p->ny);
        wrap_coord(&x1[2], p->nz);
    } else {
        ora_push_boris(q, m, p->c, Ep, Bp, u);
        double g = sqrt(1.0 + dot3(u, u) / (p->c * p->c));
        for (int a = 0; a < 3; ++a) x1[a] = x[a] + u[a] / g;
        if (J) ora_deposit_current(p, J, t + 0.5, q, x, x1);
        wrap_coord(&x1[0], p->nx);
        wrap_coord(&x1[1], p->ny);
        wrap_coord(&x1[2], p->nz);
        if (p->box == ORA_BOX_LEAKY && p->esc_mode == ORA_ESC_DISPLACEMENT) {
            /* Sec. 4.1: the displacement since the last (re)injection */
            for (int a = 0; a < 3; ++a) dr[a] += u[a] / g;
        }
    }
    if (p->esc_mode == ORA_ESC_PROBABILISTIC || (p->box == ORA_BOX_LEAKY && p->esc_mode == ORA_ESC_DISPLACEMENT)) {
        /* Sec. 4.1: end-of-step escape test and reinjection.  The displacement
         * rule is the leaky box's; the probabilistic rule runs in every box
         * (the leaky box combined with the others, Sec. 5), where the
         * reinjected momentum replaces the momentum variable that box
         * evolves (the peculiar u' of the shearing box, the comoving u of
         * the expanding box) and the position is kept. */
        int esc;
        if (p->esc_mode == ORA_ESC_DISPLACEMENT) {
            double mx = fabs(dr[0]) > fabs(dr[1]) ? fabs(dr[0]) : fabs(dr[1]);
            if (p->esc_dims == 3 && fabs(dr[2]) > mx) mx = fabs(dr[2]);
            esc = mx >= p->l_esc;
        } else {
            esc = ora_escape_draw(id, p->seed, n, p->p_esc);
        }
        if (esc) {
            ora_sample_mj(id, p->seed, n, p->theta_inj, p->c, u);
            if (dr) dr[0] = dr[1] = dr[2] = 0.0;
            loc->escaped++;
        }
    }
    x[0] = x1[0];
    x[1] = x1[1];
    x[2] = x1[2];
}

/* Threads of the particle loop of ora_step (1: the plain loop).  Tests use
 * one thread; the timed CPU baseline may use every host core. */
static int g_threads = 1;

void ora_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

int ora_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ora_step(const ora_params *p, ora_fields *f, int nsp, ora_species *sp, ora_stepinfo *info)
{
    int64_t n = f->step;
    double t = (double)n;
    int64_t N = 3 * ncell(p);
    memset(f->J, 0, sizeof(double) * (size_t)N);
    ora_stepinfo loc = {0, 0};
    int nt = 1;
#ifdef _OPENMP
    nt = g_threads;
#endif
    if (nt <= 1) {
        for (int s = 0; s < nsp; ++s) {
            ora_species *S = &sp[s];
            for (int64_t ip = 0; ip < S->n; ++ip)
                ora_advance_particle(p, f->E, f->B, f->J, n, S->q, S->m, S->id[ip], &S->x[3 * ip], &S->u[3 * ip],
                                     S->dr ? &S->dr[3 * ip] : NULL, &loc);
        }
    } else {
#ifdef _OPENMP
        /* the same per-particle step on nt threads: each thread deposits into
         * its own current array; the arrays are then added in thread order */
        double *Jt = (double *)calloc((size_t)nt * (size_t)N, sizeof(double));
        ora_stepinfo *lt = (ora_stepinfo *)calloc((size_t)nt, sizeof(ora_stepinfo));
#pragma omp parallel num_threads(nt)
        {
            int tid = omp_get_thread_num();
            double *Jl = Jt + (size_t)tid * (size_t)N;
            for (int s = 0; s < nsp; ++s) {
                ora_species *S = &sp[s];
#pragma omp for schedule(static)
                for (int64_t ip = 0; ip < S->n; ++ip)
                    ora_advance_particle(p, f->E, f->B, Jl, n, S->q, S->m, S->id[ip], &S->x[3 * ip], &S->u[3 * ip],
                                         S->dr ? &S->dr[3 * ip] : NULL, &lt[tid]);
            }
        }
        for (int k = 0; k < nt; ++k) {
            const double *Jl = Jt + (size_t)k * (size_t)N;
            for (int64_t q = 0; q < N; ++q) f->J[q] += Jl[q];
            loc.escaped += lt[k].escaped;
            loc.superluminal += lt[k].superluminal;
        }
        free(Jt);
        free(lt);
#endif
    }

    if (p->box == ORA_BOX_SHEAR) {
        ora_ksb_advect_current(p, f->J);
        ora_ksb_field_solve(p, f->E, f->B, f->J, t);
    } else if (p->box == ORA_BOX_SHEAR_EXPAND) {
        ora_sxe_advect_current(p, f->J, t);
        ora_sxe_field_solve(p, f->E, f->B, f->J, t);
    } else if (p->box == ORA_BOX_EXPAND) {
        ora_keb_field_update(p, f->E, f->B, f->J, t);
    } else {
        ora_yee_update(p, f->E, f->B, f->J);
    }
    f->step = n + 1;
    if (info) *info = loc;
}
