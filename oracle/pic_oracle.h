/*
 * pic_oracle.h -- plain FP64 CPU oracle for the particle-in-cell step of
 * "Particle-in-Cell Methods for Simulations of Sheared, Expanding, or
 * Escaping Astrophysical Plasma" (arXiv 2602.15939).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path; it is
 * never called by the product library.  Only tests/, __graft_entry__.smoke()
 * and bench.py (its cpu_baseline leg and --impl reference) may load it.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * Conventions (all in code units, dx = dt = 1, c = Courant number):
 *  - grid nx*ny*nz cells; a 2D run sets its ignorable axis to one cell, which
 *    makes every derivative along it vanish and every shape sum along it one;
 *  - node (i,j,k) sits at position (i,j,k); Yee staggering: Ex at (i+1/2,j,k),
 *    Ey at (i,j+1/2,k), Ez at (i,j,k+1/2), Bx at (i,j+1/2,k+1/2),
 *    By at (i+1/2,j,k+1/2), Bz at (i+1/2,j+1/2,k); J like E; rho on nodes;
 *  - field arrays are [3][nz][ny][nx], index ((c*nz+k)*ny+j)*nx+i, no guards;
 *  - particle momentum u is the spatial part of the four-velocity, u = gamma v,
 *    in cells/step; gamma = sqrt(1 + (u/c)^2);
 *  - positions are absolute, x in [0,nx) etc.; for the shearing box the
 *    radial coordinate entering v_s = -s Omega0 x e_y is measured from the
 *    box centre, x - nx/2.
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_BOX_PERIODIC = 0, ORA_BOX_SHEAR = 1, ORA_BOX_EXPAND = 2, ORA_BOX_LEAKY = 3,
       ORA_BOX_SHEAR_EXPAND = 4 /* shearing box in expanding coordinates (see pic_oracle.c) */ };
enum { ORA_ESC_NONE = 0, ORA_ESC_DISPLACEMENT = 1, ORA_ESC_PROBABILISTIC = 2 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t order;          /* shape order, 1 (linear) or 2 (quadratic) */
    int32_t box;            /* ORA_BOX_* */
    int32_t fp_iters;       /* shearing box: fixed-point sweeps of the Maxwell solve */
    int32_t keb_exact;      /* expanding box: 0 = closed-form modified Boris, 1 = 3x3 solve */
    int32_t esc_mode;       /* ORA_ESC_*: the displacement rule in the leaky box; the probabilistic rule in any box */
    int32_t esc_dims;       /* 2: max(|dx|,|dy|); 3: max over x,y,z */
    uint32_t seed;          /* low word of the Philox key */
    double c;
    double s;               /* shear parameter (3/2 Keplerian) */
    double Omega0;          /* rotation frequency, per step */
    double rate[3];         /* expanding box: l_i(t) = exp(rate_i t) */
    double l_esc;           /* displacement escape distance (cells) */
    double p_esc;           /* escape probability per step (dt / t_esc) */
    double theta_inj;       /* temperature of the reinjection Maxwell-Juettner */
} ora_params;

typedef struct {
    double *E, *B, *J;      /* [3][nz][ny][nx] each */
    int64_t step;           /* n: fields are at t^n = n */
} ora_fields;

typedef struct {
    int64_t n;
    double q, m;
    double *x;              /* [n][3] */
    double *u;              /* [n][3] */
    uint32_t *id;           /* [n] */
    double *dr;             /* [n][3], leaky box displacement (may be NULL otherwise) */
} ora_species;

typedef struct {
    int64_t escaped;        /* particles reinjected in the last step */
    int64_t superluminal;   /* shearing box: |u'/gamma' + v_s| >= c occurrences */
} ora_stepinfo;

/* ---- single-particle operators ---------------------------------------- */
void ora_push_boris(double q, double m, double c, const double E[3], const double B[3], double u[3]);
void ora_push_ksb(double q, double m, double c, double s, double Omega0, double xc,
                  const double E[3], const double B[3], double u[3], double *gbar_out);
double ora_ksb_gamma_bar(double c, double alpha1, double alpha2, const double um[3],
                         const double eps[3], double *residual);
void ora_push_keb(double q, double m, double c, const double Lambda[3], const double E[3],
                  const double B[3], double u[3], int exact);
void ora_push_sxe(double q, double m, double c, double s, double Omega0, double xc, const double Lambda[3],
                  const double E[3], const double B[3], double u[3], double *gbar_out);

/* ---- random numbers ----------------------------------------------------- */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
int ora_escape_draw(uint32_t id, uint32_t seed, int64_t step, double p);
int ora_sample_mj(uint32_t id, uint32_t seed, int64_t step, double theta, double c, double u[3]);

/* ---- grid operators ------------------------------------------------------ */
double ora_shear_shift(const ora_params *p, double t);
void ora_gather(const ora_params *p, const double *E, const double *B, double t,
                const double x[3], double Ep[3], double Bp[3]);
void ora_deposit_current(const ora_params *p, double *J, double t, double q,
                         const double x0[3], const double x1[3]);
void ora_deposit_rho(const ora_params *p, double *rho, double t, double q, const double x[3]);
void ora_ksb_advect_current(const ora_params *p, double *J);
void ora_yee_update(const ora_params *p, double *E, double *B, const double *J);
void ora_keb_field_update(const ora_params *p, double *E, double *B, const double *J, double t);
void ora_ksb_field_solve(const ora_params *p, double *E, double *B, const double *J, double t);
void ora_ksb_rhs(const ora_params *p, const double *E, const double *B, const double *J,
                 double t, double *FE, double *FB);
void ora_sxe_rhs(const ora_params *p, const double *Eh, const double *Bh, const double *J,
                 double t, double *FE, double *FB);
void ora_sxe_advect_current(const ora_params *p, double *J, double t);
void ora_sxe_field_solve(const ora_params *p, double *E, double *B, const double *J, double t);

/* ---- one particle's part of a step (gather, push, move, deposit when J is
 * non-NULL, escape); the whole step ------------------------------------------ */
void ora_advance_particle(const ora_params *p, const double *E, const double *B, double *J, int64_t n,
                          double q, double m, uint32_t id, double x[3], double u[3], double dr[3],
                          ora_stepinfo *loc);
void ora_step(const ora_params *p, ora_fields *f, int nsp, ora_species *sp, ora_stepinfo *info);

/* ---- threads of ora_step's particle loop (default 1; needs an OpenMP build) -- */
void ora_set_threads(int n);
int ora_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
