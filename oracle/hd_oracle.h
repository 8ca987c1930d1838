/*
 * hd_oracle.h -- plain CPU FP64 oracle for the batched hyperdynamics path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py load this library.  The CUDA library shares
 * no code, header, table or helper with it.
 *
 * What it computes (Kim & Falk, "Accelerated molecular dynamics simulation
 * of low-velocity frictional sliding"):
 *   - LJ 12-6 pair potential with type-pair parameters, Eq. 9, cut at rc and
 *     shifted so that it is zero there;
 *   - the local slope sigma = grad V . s (Eq. 5), the distance d (Eq. 7) and
 *     the direction s = (r - r_O)/d defined after Eq. 7;
 *   - the slope bias DeltaV_1(sigma), Eq. 14, alone (Eq. 13 with DeltaV_2 = 0)
 *     or combined by Eq. 13 with the eigenvalue bias DeltaV_2(epsilon),
 *     Eq. 15, epsilon the lowest eigenvalue of the Hessian;
 *   - the boosted clock sum of exp(beta DeltaV) dt, Eq. 3;
 *   - optional harmonic bonds between tip atoms in place of their LJ term,
 *     Eq. 12 (the 3-D model of Sec. 3.2.1);
 *   - the rigid top layer pulled by the slider spring and the normal load
 *     (Sec. 3.1.1, Sec. 3.2.1), lateral force F_R = k (x_S - x_T), Eq. 10;
 *   - Langevin BAOAB dynamics with Philox4x32-10 noise, or a Nose-Hoover
 *     chain (Sec. 3.1.1); the slider held still (stepped sliding) or moving
 *     at a set velocity (continuous sliding, Sec. 3.1.1);
 *   - steepest-descent and FIRE quenches to the basin minimum r_O (after
 *     Eq. 7) and a transition test by displacement from r_O (Sec. 2.3).
 *
 * Pins (tests/test_oracle_*.py) tie each function to closed forms, finite
 * differences, brute force or invariants.  One quantity has no pin against
 * the paper: time averages of F_R (Eq. 10), parity unpinned; the paper prints
 * no value for them, so they are checked GPU against oracle only.
 *
 * Every array is caller-owned.  Positions are [n][3] (z = 0 in 2-D) and are
 * never wrapped into the periodic box; minimum images are taken where two
 * positions are differenced.
 */
#ifndef HD_ORACLE_H
#define HD_ORACLE_H
#include <stdint.h>

typedef struct {
    /* settings (inputs) */
    int dim, n, rep_id, m_exp;
    double L[3];
    int periodic[3];
    double kT, gamma, kspring, fnormal, slider[2];
    double dvmax, sig_lo, sig_hi;
    double eps[2][2], sig[2][2];
    /* caller-owned arrays */
    double *x, *v, *xo;               /* [n][3] */
    const uint8_t *role, *type;       /* [n]: role 0 fixed 1 mobile 2 rigid; type 0 s 1 t */
    int maxnb;
    int *nnb, *nbr;                   /* [n], [n][maxnb]; rows sorted by j */
    double *xb;                       /* [n][3] positions at the last list build */
    double *f_lj, *hdr, *e_atom;      /* [n][3], [n][3], [n] */
    double *ftot;                     /* [n][3] total force incl. bias */
    /* scalar state */
    double t_h, t_md;
    int64_t step, n_rebuild, nb_overflow;
    double vbody[3];
    /* scalars at the current positions */
    double V, V_lj, K, dV, dVp, sigma, d, G, xT[3], fbody[3], FR;
    /* eigenvalue bias, Eq. 13 and Eq. 15 (eig_on = 0: the slope bias alone) */
    int eig_on, eig_maxit;            /* Lanczos steps per evaluation, at most */
    double eig_lo, eig_hi;            /* epsilon_L, epsilon_U */
    double *veig;                     /* [n][3] lowest eigenvector, kept as the next start */
    double eig, dV1, dV2, dVe;        /* epsilon, DeltaV_1, DeltaV_2, dDeltaV/depsilon */
    /* continuous sliding (Sec. 3.1.1, method 1): with vslide != 0 the slider
     * moves along x every step, x_S = slide_x0 + k (vslide dt) after the k-th
     * step since slide_step0; vslide = 0 keeps it where it is */
    double vslide, slide_x0;
    int64_t slide_step0;
    /* harmonic tip bonds, Eq. 12 (Sec. 3.2.1): nbond pairs i, j bonded by
     * kbond (r - rbond)^2 / 2; with nbond > 0 tip-tip pairs have no LJ term */
    int nbond;
    const int *bonds;                 /* [nbond][2] */
    double kbond, rbond;
    /* Nose-Hoover chain thermostat (Sec. 3.1.1) in place of Langevin when
     * nhc_len > 0: chain length (<= 8), period tau of the thermostat masses
     * Q_1 = N_f kT tau^2, Q_j = kT tau^2, positions xi and velocities v of
     * the chain; it acts on the mobile atoms (N_f = dim n_mobile) */
    int nhc_len;
    double nhc_tau;
    double nhc_xi[8], nhc_v[8];
} or_rep;

typedef struct {
    double dt, rc, skin;
    int bias_on;
    uint64_t seed;
} or_params;

void   or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_unif(uint32_t a, uint32_t b);
void   or_normals(uint64_t seed, int rep_id, int64_t step, int atom, int call, double out[2]);
void   or_lj(double r, double eps, double sig, double rc, double out[3]);
void   or_dv1(const or_rep *R, double sigma, double out[2]);

int    or_nlist_brute(or_rep *R, double rl);
int    or_nlist_cells(or_rep *R, double rl);
double or_forces(or_rep *R, const or_params *P);
double or_forces_brute(const or_rep *R, const or_params *P, double *f, double *e_atom);
double or_potential(const or_rep *R, const or_params *P, const double *x);
void   or_gradient(const or_rep *R, const or_params *P, const double *x, double *g);
void   or_hessvec(const or_rep *R, const or_params *P, const double *x, const double *u, double *out);
double or_bias_potential(const or_rep *R, const or_params *P, const double *x);
void   or_bias_eval(or_rep *R, const or_params *P);
void   or_init(or_rep *R, const or_params *P, int draw_velocities);
void   or_run(or_rep *R, const or_params *P, int nsteps);
void   or_run_batch(or_rep *reps, int nrep, const or_params *P, int nsteps);
int    or_quench(or_rep *R, const or_params *P, int method, double ftol, int max_iter,
                 double step_size, double *xq, double *fmax_out);
int    or_quench_batch(or_rep *reps, int nrep, const or_params *P, int method, double ftol,
                       int max_iter, double step_size, double **xq, double *fmax_out, int *iters);
int    or_quench_gated(or_rep *R, const or_params *P, int method, double ftol, double ftol_stay, double keep,
                       int max_iter, double step_size, double *xq, double *fmax_out);
int    or_quench_batch_gated(or_rep *reps, int nrep, const or_params *P, int method, double ftol,
                             double ftol_stay, double keep, int max_iter, double step_size, double **xq,
                             double *fmax_out, int *iters);
int    or_transition(const or_rep *R, const double *xq, double theta, double *maxdisp);
double or_lj3(double r, double eps, double sig);
void   or_project(const or_rep *R, double *u);
double or_lowest_eig(const or_rep *R, const or_params *P, const double *x, double *v, int maxit, double tol);
void   or_eig_grad(const or_rep *R, const or_params *P, const double *x, const double *v, double *g);
void   or_dv2(const or_rep *R, double e, double out[2]);
void   or_dv13(const or_rep *R, double dv1, double dv2, double out[3]);
double or_nhc_energy(const or_rep *R);
int    or_num_threads(void);

#endif
