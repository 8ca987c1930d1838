/*
 * hd_oracle.c -- plain CPU FP64 oracle for the batched hyperdynamics path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py.  It shares no code with the CUDA library.
 * Built with -O2 -ffp-contract=off so that every product and sum is rounded
 * separately, in the order written.
 *
 * Each function states the passage of Kim & Falk it follows.  Where the paper
 * is silent the reading used is stated beside the code.  Written for a reader
 * checking it against the paper: no blocking, no fusion, no reordering.
 */
#include "hd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the
 * round multipliers 0xD2511F53 and 0xCD9E8D57; the key is bumped by the
 * Weyl constants 0x9E3779B9 and 0xBB67AE85 before every round but the first.
 * ---------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform strictly inside (0,1) from two 32-bit words: the 26 high bits of
 * a and of b form k < 2^52, and u = (k + 1/2) 2^-52 is exact in FP64. */
double or_unif(uint32_t a, uint32_t b) {
    return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * 0x1p-52;
}

/* Two standard normals (Box-Muller) for (step, atom, replica, call).
 * Counter = (step low word, atom, replica, call | step high word << 8);
 * key = the 64-bit seed.  Calls 0 and 1 feed the thermostat (Sec. 3.1.1
 * replaced by Langevin, see the reading in or_run); calls 2 and 3 draw the
 * initial Maxwell-Boltzmann velocities. */
void or_normals(uint64_t seed, int rep_id, int64_t step, int atom, int call, double out[2]) {
    uint32_t ctr[4], key[2], w[4];
    ctr[0] = (uint32_t)(uint64_t)step;
    ctr[1] = (uint32_t)atom;
    ctr[2] = (uint32_t)rep_id;
    ctr[3] = (uint32_t)call | ((uint32_t)((uint64_t)step >> 32) << 8);
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
    or_philox4x32_10(ctr, key, w);
    double u1 = or_unif(w[0], w[1]);
    double u2 = or_unif(w[2], w[3]);
    double rad = sqrt(-2.0 * log(u1));
    double ang = 2.0 * M_PI * u2;
    out[0] = rad * cos(ang);
    out[1] = rad * sin(ang);
}

/* ------------------------------------------------------------------------
 * Eq. 9: V(r) = 4 eps [(sig/r)^12 - (sig/r)^6], cut at rc and shifted by its
 * value there (reading: energy-shifted, forces not shifted).
 * out = { phi(r), phi'(r), phi''(r) } for r < rc.
 * ---------------------------------------------------------------------- */
void or_lj(double r, double eps, double sig, double rc, double out[3]) {
    double sr6 = pow(sig / r, 6.0);
    double sr12 = sr6 * sr6;
    double sc6 = pow(sig / rc, 6.0);
    double shift = 4.0 * eps * (sc6 * sc6 - sc6);
    out[0] = 4.0 * eps * (sr12 - sr6) - shift;
    out[1] = 4.0 * eps * (-12.0 * sr12 + 6.0 * sr6) / r;
    out[2] = 4.0 * eps * (156.0 * sr12 - 42.0 * sr6) / (r * r);
}

/* Eq. 14 (and Eq. 13 with DeltaV_2 = 0): out = { DeltaV_1(sigma), dDeltaV_1/dsigma }.
 * Orientation as printed: DeltaV_max above sigma_U, 0 below sigma_L. */
void or_dv1(const or_rep *R, double s, double out[2]) {
    double lo = R->sig_lo, hi = R->sig_hi, dvm = R->dvmax;
    int m = R->m_exp;
    if (s >= hi) { out[0] = dvm; out[1] = 0.0; return; }
    if (s <= lo) { out[0] = 0.0; out[1] = 0.0; return; }
    double t = (s - hi) / (lo - hi);              /* in (0,1) */
    double tm1 = pow(t, (double)(m - 1));
    double q = 1.0 - tm1 * t;                      /* 1 - t^m */
    out[0] = dvm * q * q;
    /* d/dsigma: 2 dvm q (-m t^(m-1)) dt/dsigma, dt/dsigma = 1/(lo - hi) */
    out[1] = 2.0 * dvm * q * (-(double)m * tm1) / (lo - hi);
}

/* Minimum image along one axis (periodic in-plane directions, Sec. 3.1.1). */
static double or_mi(double d, double L, int per) {
    return per ? d - L * rint(d / L) : d;
}

static double or_rij(const or_rep *R, const double *x, int i, int j, double r[3]) {
    for (int a = 0; a < 3; ++a)
        r[a] = or_mi(x[3 * i + a] - x[3 * j + a], R->L[a], R->periodic[a]);
    return r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
}

static void or_disp(const or_rep *R, const double *x, int i, double dr[3]) {
    for (int a = 0; a < 3; ++a)
        dr[a] = or_mi(x[3 * i + a] - R->xo[3 * i + a], R->L[a], R->periodic[a]);
}

/* Eq. 12: out = { phi, phi', phi'' } of the harmonic bond; phi''' = 0. */
static void or_bond(const or_rep *R, double r, double out[3]) {
    double d = r - R->rbond;
    out[0] = 0.5 * R->kbond * d * d;
    out[1] = R->kbond * d;
    out[2] = R->kbond;
}

/* The LJ term acts between i and j unless both are atoms of a bonded tip. */
static int or_lj_on(const or_rep *R, int i, int j) {
    return !(R->nbond > 0 && R->type[i] == 1 && R->type[j] == 1);
}

/* ------------------------------------------------------------------------
 * Rigid top layer, slider spring and normal load (Sec. 3.1.1, Sec. 3.2.1).
 * x_T is the centre of the rigid layer.  The spring pulls x_T toward x_S
 * (and, in 3-D, y_T toward y_S: reading, the paper names only the sliding
 * direction); the load F_N pushes the layer down along the vertical axis
 * (y in 2-D, z in 3-D).  The potential energy includes both terms, since
 * "the potential energy is a function of the slider position" (Sec. 2.3).
 * ---------------------------------------------------------------------- */
static int or_nrig(const or_rep *R) {
    int c = 0;
    for (int i = 0; i < R->n; ++i) c += (R->role[i] == 2);
    return c;
}

static void or_tip_centre(const or_rep *R, const double *x, double xt[3]) {
    int c = 0;
    xt[0] = xt[1] = xt[2] = 0.0;
    for (int i = 0; i < R->n; ++i)
        if (R->role[i] == 2) {
            for (int a = 0; a < 3; ++a) xt[a] += x[3 * i + a];
            ++c;
        }
    if (c > 0)
        for (int a = 0; a < 3; ++a) xt[a] /= (double)c;
}

static double or_ext_energy(const or_rep *R, const double xt[3]) {
    double e = 0.5 * R->kspring * (xt[0] - R->slider[0]) * (xt[0] - R->slider[0]);
    if (R->dim == 3) e += 0.5 * R->kspring * (xt[1] - R->slider[1]) * (xt[1] - R->slider[1]);
    e += R->fnormal * xt[R->dim - 1];
    return e;
}

/* gradient of the spring + load energy with respect to the tip centre */
static void or_ext_grad(const or_rep *R, const double xt[3], double gs[3]) {
    gs[0] = R->kspring * (xt[0] - R->slider[0]);
    gs[1] = 0.0;
    gs[2] = 0.0;
    if (R->dim == 3) gs[1] = R->kspring * (xt[1] - R->slider[1]);
    gs[R->dim - 1] = R->fnormal;
}

/* ------------------------------------------------------------------------
 * Neighbour list.  Definition: j is in row i iff j != i and the minimum-image
 * squared distance (x, then y, then z, each product rounded) is < rl^2, with
 * rl = rc + skin; each row in ascending j.
 * ---------------------------------------------------------------------- */
static int or_list_brute(const or_rep *R, const double *x, double rl, int *nnb, int *nbr) {
    double rl2 = rl * rl, r[3];
    int over = 0;
    for (int i = 0; i < R->n; ++i) {
        int cnt = 0;
        for (int j = 0; j < R->n; ++j) {
            if (j == i) continue;
            if (or_rij(R, x, i, j, r) < rl2) {
                if (cnt < R->maxnb) nbr[(size_t)i * R->maxnb + cnt] = j;
                ++cnt;
            }
        }
        if (cnt > R->maxnb) { ++over; cnt = R->maxnb; }
        nnb[i] = cnt;
    }
    return over;
}

static int or_cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Same list through a cell grid (cells at least rl wide), then each row sorted. */
static int or_list_cells(const or_rep *R, const double *x, double rl, int *nnb, int *nbr) {
    int n = R->n, nc[3], bad = 0;
    double lo[3], w[3];
    for (int a = 0; a < 3; ++a) {
        if (R->periodic[a]) {
            nc[a] = (int)floor(R->L[a] / (rl * (1.0 + 1e-12)));
            if (nc[a] < 3) nc[a] = 1;
            lo[a] = 0.0;
            w[a] = R->L[a] / nc[a];
            for (int i = 0; i < n; ++i) bad |= !isfinite(x[3 * i + a]);
        } else {
            double mn = x[a], mx = x[a];
            for (int i = 1; i < n; ++i) {
                if (x[3 * i + a] < mn) mn = x[3 * i + a];
                if (x[3 * i + a] > mx) mx = x[3 * i + a];
            }
            lo[a] = mn;
            w[a] = rl * (1.0 + 1e-12);
            double span = (mx - mn) / w[a];
            if (!(span < 65536.0)) { bad = 1; span = 0.0; }
            nc[a] = (int)floor(span) + 1;
        }
    }
    /* a runaway configuration (a diverged quench: non-finite or wildly
     * spread coordinates) gets empty rows and -1, instead of an unbounded
     * cell grid */
    if (bad) {
        for (int i = 0; i < n; ++i) nnb[i] = 0;
        return -1;
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int *cid = malloc(sizeof(int) * n), *start = calloc(ncell + 1, sizeof(int)), *list = malloc(sizeof(int) * n);
    int *cc = malloc(sizeof(int) * n * 3);
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double p = x[3 * i + a];
            if (R->periodic[a]) p = p - R->L[a] * floor(p / R->L[a]);
            int c = (int)floor((p - lo[a]) / w[a]);
            if (c < 0) c = 0;
            if (c >= nc[a]) c = nc[a] - 1;
            cc[3 * i + a] = c;
        }
        cid[i] = (cc[3 * i + 2] * nc[1] + cc[3 * i + 1]) * nc[0] + cc[3 * i];
        start[cid[i] + 1]++;
    }
    for (long c = 0; c < ncell; ++c) start[c + 1] += start[c];
    int *fill = malloc(sizeof(int) * (ncell + 1));
    memcpy(fill, start, sizeof(int) * (ncell + 1));
    for (int i = 0; i < n; ++i) list[fill[cid[i]]++] = i;
    int over = 0, cap = 4096;
    int *row = malloc(sizeof(int) * cap);
    double rl2 = rl * rl, r[3];
    for (int i = 0; i < n; ++i) {
        int cnt = 0;
        int off[3][3], noff[3];
        for (int a = 0; a < 3; ++a) {
            noff[a] = 0;
            for (int d = -1; d <= 1; ++d) {
                int c = cc[3 * i + a] + d;
                if (R->periodic[a]) c = (c + nc[a]) % nc[a];
                else if (c < 0 || c >= nc[a]) continue;
                int dup = 0;
                for (int k = 0; k < noff[a]; ++k) dup |= (off[a][k] == c);
                if (!dup) off[a][noff[a]++] = c;
            }
        }
        for (int iz = 0; iz < noff[2]; ++iz)
            for (int iy = 0; iy < noff[1]; ++iy)
                for (int ix = 0; ix < noff[0]; ++ix) {
                    long c = ((long)off[2][iz] * nc[1] + off[1][iy]) * nc[0] + off[0][ix];
                    for (int k = start[c]; k < start[c + 1]; ++k) {
                        int j = list[k];
                        if (j == i) continue;
                        if (or_rij(R, x, i, j, r) < rl2) {
                            if (cnt == cap) { cap *= 2; row = realloc(row, sizeof(int) * cap); }
                            row[cnt++] = j;
                        }
                    }
                }
        qsort(row, cnt, sizeof(int), or_cmp_int);
        if (cnt > R->maxnb) { ++over; cnt = R->maxnb; }
        memcpy(nbr + (size_t)i * R->maxnb, row, sizeof(int) * cnt);
        nnb[i] = cnt;
    }
    free(row); free(fill); free(cc); free(list); free(start); free(cid);
    return over;
}

int or_nlist_brute(or_rep *R, double rl) {
    int over = or_list_brute(R, R->x, rl, R->nnb, R->nbr);
    memcpy(R->xb, R->x, sizeof(double) * 3 * R->n);
    R->nb_overflow += over;
    return over;
}

int or_nlist_cells(or_rep *R, double rl) {
    int over = or_list_cells(R, R->x, rl, R->nnb, R->nbr);
    if (over < 0) over = R->n;                /* runaway positions: no usable list */
    memcpy(R->xb, R->x, sizeof(double) * 3 * R->n);
    R->nb_overflow += over;
    return over;
}

/* ------------------------------------------------------------------------
 * LJ forces, per-atom energies and the Hessian-vector product H.dr with
 * dr = r - r_O (needed by grad sigma of Eq. 5 with s from Eq. 7), summed over
 * each list row in row order.  For one pair, with A = phi'/r and
 * B = (phi'' - phi'/r)/r^2, the Hessian block is A I + B r r^T.
 * The spring adds k/n_rig^2 to every (rigid x, rigid x) Hessian entry
 * (and y in 3-D); the load is linear and adds nothing.
 * ---------------------------------------------------------------------- */
static double or_pairs_on_list(const or_rep *R, const double *x, const int *nnb, const int *nbr,
                               double rc, double *f, double *hdr, double *e_atom) {
    int n = R->n;
    double rc2 = rc * rc, r[3], dri[3], drj[3], ph[3];
    memset(f, 0, sizeof(double) * 3 * n);
    if (hdr) memset(hdr, 0, sizeof(double) * 3 * n);
    if (e_atom) memset(e_atom, 0, sizeof(double) * n);
    double vtot = 0.0;
    for (int i = 0; i < n; ++i) {
        int ti = R->type[i];
        if (hdr) or_disp(R, x, i, dri);
        for (int k = 0; k < nnb[i]; ++k) {
            int j = nbr[(size_t)i * R->maxnb + k];
            double r2 = or_rij(R, x, i, j, r);
            if (!(r2 < rc2) || !or_lj_on(R, i, j)) continue;
            int tj = R->type[j];
            double rr = sqrt(r2);
            or_lj(rr, R->eps[ti][tj], R->sig[ti][tj], rc, ph);
            double A = ph[1] / rr;
            double B = (ph[2] - A) / r2;
            for (int a = 0; a < 3; ++a) f[3 * i + a] -= A * r[a];
            if (e_atom) e_atom[i] += 0.5 * ph[0];
            if (hdr) {
                or_disp(R, x, j, drj);
                double du[3] = {dri[0] - drj[0], dri[1] - drj[1], dri[2] - drj[2]};
                double rdu = r[0] * du[0] + r[1] * du[1] + r[2] * du[2];
                for (int a = 0; a < 3; ++a) hdr[3 * i + a] += A * du[a] + B * rdu * r[a];
            }
        }
    }
    /* bonds (Eq. 12), each pair once, both atoms updated */
    for (int b = 0; b < R->nbond; ++b) {
        int i = R->bonds[2 * b], j = R->bonds[2 * b + 1];
        double r2 = or_rij(R, x, i, j, r), rr = sqrt(r2);
        or_bond(R, rr, ph);
        double A = ph[1] / rr, B = (ph[2] - A) / r2;
        for (int a = 0; a < 3; ++a) {
            f[3 * i + a] -= A * r[a];
            f[3 * j + a] += A * r[a];
        }
        if (e_atom) { e_atom[i] += 0.5 * ph[0]; e_atom[j] += 0.5 * ph[0]; }
        if (hdr) {
            or_disp(R, x, i, dri);
            or_disp(R, x, j, drj);
            double du[3] = {dri[0] - drj[0], dri[1] - drj[1], dri[2] - drj[2]};
            double rdu = r[0] * du[0] + r[1] * du[1] + r[2] * du[2];
            for (int a = 0; a < 3; ++a) {
                double h = A * du[a] + B * rdu * r[a];
                hdr[3 * i + a] += h;
                hdr[3 * j + a] -= h;
            }
        }
    }
    if (e_atom)
        for (int i = 0; i < n; ++i) vtot += e_atom[i];
    if (hdr) {
        int nr = or_nrig(R);
        if (nr > 0) {
            double sx = 0.0, sy = 0.0, d[3];
            for (int i = 0; i < n; ++i)
                if (R->role[i] == 2) {
                    or_disp(R, x, i, d);
                    sx += d[0];
                    sy += d[1];
                }
            double kk = R->kspring / ((double)nr * (double)nr);
            for (int i = 0; i < n; ++i)
                if (R->role[i] == 2) {
                    hdr[3 * i + 0] += kk * sx;
                    if (R->dim == 3) hdr[3 * i + 1] += kk * sy;
                }
        }
    }
    return vtot;
}

double or_forces(or_rep *R, const or_params *P) {
    R->V_lj = or_pairs_on_list(R, R->x, R->nnb, R->nbr, P->rc, R->f_lj, R->hdr, R->e_atom);
    return R->V_lj;
}

/* All pairs i < j directly, third law applied; independent of the list. */
double or_forces_brute(const or_rep *R, const or_params *P, double *f, double *e_atom) {
    int n = R->n;
    double rc2 = P->rc * P->rc, r[3], ph[3], vtot = 0.0;
    memset(f, 0, sizeof(double) * 3 * n);
    if (e_atom) memset(e_atom, 0, sizeof(double) * n);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r2 = or_rij(R, R->x, i, j, r);
            if (!(r2 < rc2) || !or_lj_on(R, i, j)) continue;
            double rr = sqrt(r2);
            or_lj(rr, R->eps[R->type[i]][R->type[j]], R->sig[R->type[i]][R->type[j]], P->rc, ph);
            for (int a = 0; a < 3; ++a) {
                double fa = -ph[1] * r[a] / rr;
                f[3 * i + a] += fa;
                f[3 * j + a] -= fa;
            }
            vtot += ph[0];
            if (e_atom) { e_atom[i] += 0.5 * ph[0]; e_atom[j] += 0.5 * ph[0]; }
        }
    for (int b = 0; b < R->nbond; ++b) {
        int i = R->bonds[2 * b], j = R->bonds[2 * b + 1];
        double rr = sqrt(or_rij(R, R->x, i, j, r));
        or_bond(R, rr, ph);
        for (int a = 0; a < 3; ++a) {
            double fa = -ph[1] * r[a] / rr;
            f[3 * i + a] += fa;
            f[3 * j + a] -= fa;
        }
        vtot += ph[0];
        if (e_atom) { e_atom[i] += 0.5 * ph[0]; e_atom[j] += 0.5 * ph[0]; }
    }
    return vtot;
}

/* Total potential V (LJ pairs + spring + load) at positions x, all pairs. */
double or_potential(const or_rep *R, const or_params *P, const double *x) {
    int n = R->n;
    double rc2 = P->rc * P->rc, r[3], ph[3], v = 0.0, xt[3];
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r2 = or_rij(R, x, i, j, r);
            if (!(r2 < rc2) || !or_lj_on(R, i, j)) continue;
            or_lj(sqrt(r2), R->eps[R->type[i]][R->type[j]], R->sig[R->type[i]][R->type[j]], P->rc, ph);
            v += ph[0];
        }
    for (int b = 0; b < R->nbond; ++b) {
        or_bond(R, sqrt(or_rij(R, x, R->bonds[2 * b], R->bonds[2 * b + 1], r)), ph);
        v += ph[0];
    }
    if (or_nrig(R) > 0) {
        or_tip_centre(R, x, xt);
        v += or_ext_energy(R, xt);
    }
    return v;
}

/* g = grad V over all 3N coordinates (Eq. 2 notation), all pairs. */
void or_gradient(const or_rep *R, const or_params *P, const double *x, double *g) {
    int n = R->n, nr = or_nrig(R);
    double rc2 = P->rc * P->rc, r[3], ph[3];
    memset(g, 0, sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r2 = or_rij(R, x, i, j, r);
            if (!(r2 < rc2) || !or_lj_on(R, i, j)) continue;
            double rr = sqrt(r2);
            or_lj(rr, R->eps[R->type[i]][R->type[j]], R->sig[R->type[i]][R->type[j]], P->rc, ph);
            for (int a = 0; a < 3; ++a) {
                double ga = ph[1] * r[a] / rr;
                g[3 * i + a] += ga;
                g[3 * j + a] -= ga;
            }
        }
    for (int b = 0; b < R->nbond; ++b) {
        int i = R->bonds[2 * b], j = R->bonds[2 * b + 1];
        double rr = sqrt(or_rij(R, x, i, j, r));
        or_bond(R, rr, ph);
        for (int a = 0; a < 3; ++a) {
            double ga = ph[1] * r[a] / rr;
            g[3 * i + a] += ga;
            g[3 * j + a] -= ga;
        }
    }
    if (nr > 0) {
        double xt[3], gs[3];
        or_tip_centre(R, x, xt);
        or_ext_grad(R, xt, gs);
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 2)
                for (int a = 0; a < 3; ++a) g[3 * i + a] += gs[a] / (double)nr;
    }
}

/* out = H u for an arbitrary 3N vector u, all pairs, plus the spring term. */
void or_hessvec(const or_rep *R, const or_params *P, const double *x, const double *u, double *out) {
    int n = R->n, nr = or_nrig(R);
    double rc2 = P->rc * P->rc, r[3], ph[3];
    memset(out, 0, sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r2 = or_rij(R, x, i, j, r);
            if (!(r2 < rc2) || !or_lj_on(R, i, j)) continue;
            double rr = sqrt(r2);
            or_lj(rr, R->eps[R->type[i]][R->type[j]], R->sig[R->type[i]][R->type[j]], P->rc, ph);
            double A = ph[1] / rr, B = (ph[2] - A) / r2;
            double du[3] = {u[3 * i] - u[3 * j], u[3 * i + 1] - u[3 * j + 1], u[3 * i + 2] - u[3 * j + 2]};
            double rdu = r[0] * du[0] + r[1] * du[1] + r[2] * du[2];
            for (int a = 0; a < 3; ++a) {
                double h = A * du[a] + B * rdu * r[a];
                out[3 * i + a] += h;
                out[3 * j + a] -= h;
            }
        }
    for (int b = 0; b < R->nbond; ++b) {
        int i = R->bonds[2 * b], j = R->bonds[2 * b + 1];
        double r2 = or_rij(R, x, i, j, r), rr = sqrt(r2);
        or_bond(R, rr, ph);
        double A = ph[1] / rr, B = (ph[2] - A) / r2;
        double du[3] = {u[3 * i] - u[3 * j], u[3 * i + 1] - u[3 * j + 1], u[3 * i + 2] - u[3 * j + 2]};
        double rdu = r[0] * du[0] + r[1] * du[1] + r[2] * du[2];
        for (int a = 0; a < 3; ++a) {
            double h = A * du[a] + B * rdu * r[a];
            out[3 * i + a] += h;
            out[3 * j + a] -= h;
        }
    }
    if (nr > 0) {
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 2) { sx += u[3 * i]; sy += u[3 * i + 1]; }
        double kk = R->kspring / ((double)nr * (double)nr);
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 2) {
                out[3 * i] += kk * sx;
                if (R->dim == 3) out[3 * i + 1] += kk * sy;
            }
    }
}

/* ------------------------------------------------------------------------
 * Eigenvalue bias (Eq. 13, Eq. 15).  epsilon is the lowest eigenvalue of the
 * Hessian of V over the motions the model allows.  Reading: fixed atoms do
 * not move and the rigid layer moves as one body, measured in the same 3N
 * metric as d and sigma (Eq. 5, Eq. 7: each rigid atom carries the body's
 * displacement).  The projector P onto those motions zeroes fixed atoms (and
 * z in 2-D) and replaces every rigid atom's displacement by the layer mean;
 * epsilon is the lowest eigenvalue of P H P on the range of P.  It is found
 * by Lanczos iteration with full reorthogonalisation; the lowest eigenvalue
 * of the tridiagonal matrix by bisection on its Sturm count, its eigenvector
 * by inverse iteration.  The gradient follows from first-order perturbation
 * theory: for the unit eigenvector v, grad epsilon = grad (v^T H(r) v) with v
 * held fixed, a sum over pairs of the third derivative of the pair term.
 * ---------------------------------------------------------------------- */

/* phi'''(r) of the LJ pair (the shift does not enter). */
double or_lj3(double r, double eps, double sig) {
    double sr6 = pow(sig / r, 6.0);
    double sr12 = sr6 * sr6;
    return 4.0 * eps * (-2184.0 * sr12 + 336.0 * sr6) / (r * r * r);
}

void or_project(const or_rep *R, double *u) {
    int n = R->n, nr = or_nrig(R);
    double m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i)
        if (R->role[i] == 2)
            for (int a = 0; a < 3; ++a) m[a] += u[3 * i + a];
    if (nr > 0)
        for (int a = 0; a < 3; ++a) m[a] /= (double)nr;
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (R->role[i] == 0 || a >= R->dim) u[3 * i + a] = 0.0;
            else if (R->role[i] == 2) u[3 * i + a] = m[a];
        }
}

static double or_dot(const double *a, const double *b, int N) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += a[k] * b[k];
    return s;
}

/* number of eigenvalues of the tridiagonal (alpha, beta) below lam */
static int or_sturm(const double *al, const double *be, int m, double lam) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
        d = (al[i] - lam) - (i > 0 ? b2 / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

/* lowest eigenvalue of the tridiagonal matrix and its unit eigenvector y */
static double or_tri_lowest(const double *al, const double *be, int m, double *y) {
    double lo = al[0], hi = al[0];
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
        lo = fmin(lo, al[i] - r);
        hi = fmax(hi, al[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(1.0, fabs(lo) + fabs(hi)); ++it) {
        double mid = 0.5 * (lo + hi);
        if (or_sturm(al, be, m, mid) >= 1) hi = mid;
        else lo = mid;
    }
    double lam = 0.5 * (lo + hi);
    /* inverse iteration with T - (lam - delta) I, positive definite */
    double delta = 1e-10 * fmax(1.0, fabs(lam));
    double *c = malloc(sizeof(double) * m), *dd = malloc(sizeof(double) * m);
    for (int i = 0; i < m; ++i) y[i] = 1.0;
    for (int rep = 0; rep < 3; ++rep) {
        /* forward elimination of the symmetric tridiagonal system */
        double s = lam - delta;
        dd[0] = al[0] - s;
        c[0] = y[0];
        for (int i = 1; i < m; ++i) {
            double l = be[i - 1] / dd[i - 1];
            dd[i] = (al[i] - s) - l * be[i - 1];
            c[i] = y[i] - l * c[i - 1];
        }
        y[m - 1] = c[m - 1] / dd[m - 1];
        for (int i = m - 2; i >= 0; --i) y[i] = (c[i] - be[i] * y[i + 1]) / dd[i];
        double nrm = sqrt(or_dot(y, y, m));
        for (int i = 0; i < m; ++i) y[i] /= nrm;
    }
    free(c);
    free(dd);
    return lam;
}

double or_lowest_eig(const or_rep *R, const or_params *P, const double *x, double *v, int maxit, double tol) {
    int n = R->n, N = 3 * n, nr = or_nrig(R), nmob = 0;
    for (int i = 0; i < n; ++i) nmob += R->role[i] == 1;
    int dimP = R->dim * nmob + (nr > 0 ? R->dim : 0);
    if (maxit > dimP) maxit = dimP;
    if (maxit < 1) return 0.0;
    double *Q = malloc(sizeof(double) * (size_t)N * (size_t)(maxit + 1));
    double *w = malloc(sizeof(double) * N);
    double *al = malloc(sizeof(double) * maxit), *be = malloc(sizeof(double) * maxit);
    double *y = malloc(sizeof(double) * maxit);
    /* start: the given vector (the last eigenvector) plus a fixed generic
     * vector, so that a new lowest mode after a level crossing is never
     * missing from the Krylov space; the generic vector alone without one */
    double *gen = malloc(sizeof(double) * N);
    for (int k = 0; k < N; ++k) gen[k] = 1.0 + 0.5 * sin(0.7 * (double)k + 0.3 * (double)(k % 7));
    or_project(R, gen);
    double ng = sqrt(or_dot(gen, gen, N));
    memcpy(Q, v, sizeof(double) * N);
    or_project(R, Q);
    double nv = sqrt(or_dot(Q, Q, N));
    for (int k = 0; k < N; ++k) Q[k] = (nv > 1e-12 ? Q[k] / nv : 0.0) + 0.3 * gen[k] / ng;
    free(gen);
    double nrm = sqrt(or_dot(Q, Q, N));
    for (int k = 0; k < N; ++k) Q[k] /= nrm;
    int m = 0;
    double lam = 0.0;
    for (int j = 0; j < maxit; ++j) {
        double *qj = Q + (size_t)j * N;
        or_hessvec(R, P, x, qj, w);
        or_project(R, w);
        al[j] = or_dot(qj, w, N);
        for (int k = 0; k < N; ++k) w[k] -= al[j] * qj[k] + (j > 0 ? be[j - 1] * Q[(size_t)(j - 1) * N + k] : 0.0);
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i <= j; ++i) {
                double *qi = Q + (size_t)i * N;
                double c = or_dot(qi, w, N);
                for (int k = 0; k < N; ++k) w[k] -= c * qi[k];
            }
        be[j] = sqrt(or_dot(w, w, N));
        m = j + 1;
        lam = or_tri_lowest(al, be, m, y);
        if (be[j] * fabs(y[m - 1]) <= tol * fmax(1.0, fabs(lam)) || be[j] < 1e-14 || m == maxit) break;
        double *qn = Q + (size_t)(j + 1) * N;
        for (int k = 0; k < N; ++k) qn[k] = w[k] / be[j];
    }
    memset(v, 0, sizeof(double) * N);
    for (int i = 0; i < m; ++i)
        for (int k = 0; k < N; ++k) v[k] += y[i] * Q[(size_t)i * N + k];
    nrm = sqrt(or_dot(v, v, N));
    for (int k = 0; k < N; ++k) v[k] /= nrm;
    free(Q); free(w); free(al); free(be); free(y);
    return lam;
}

/* g = grad over all 3N coordinates of v^T H(x) v, v held fixed.  Per pair,
 * with r = x_i - x_j, rho = |r|, w = v_i - v_j, the pair's share is
 * A |w|^2 + B (r.w)^2 with A = phi'/rho and B = (phi'' - A)/rho^2; since
 * dA/drho = B rho and dB/drho = (phi''' - 3 B rho)/rho^2, its gradient with
 * respect to r is r [B |w|^2 + (phi''' - 3 B rho) (r.w)^2 / rho^3]
 * + 2 B (r.w) w.  The spring's Hessian is constant. */
static void or_eig_grad_pair(const double r[3], double r2, const double ph[3], double p3, const double *v, int i,
                             int j, double *g) {
    double rho = sqrt(r2);
    double A = ph[1] / rho, B = (ph[2] - A) / r2;
    double w[3] = {v[3 * i] - v[3 * j], v[3 * i + 1] - v[3 * j + 1], v[3 * i + 2] - v[3 * j + 2]};
    double ww = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double rw = r[0] * w[0] + r[1] * w[1] + r[2] * w[2];
    double cr = B * ww + (p3 - 3.0 * B * rho) * rw * rw / (r2 * rho);
    for (int a = 0; a < 3; ++a) {
        double ga = cr * r[a] + 2.0 * B * rw * w[a];
        g[3 * i + a] += ga;
        g[3 * j + a] -= ga;
    }
}

void or_eig_grad(const or_rep *R, const or_params *P, const double *x, const double *v, double *g) {
    int n = R->n;
    double rc2 = P->rc * P->rc, r[3], ph[3];
    memset(g, 0, sizeof(double) * 3 * n);
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double r2 = or_rij(R, x, i, j, r);
            if (!(r2 < rc2) || !or_lj_on(R, i, j)) continue;
            double rho = sqrt(r2);
            int ti = R->type[i], tj = R->type[j];
            or_lj(rho, R->eps[ti][tj], R->sig[ti][tj], P->rc, ph);
            or_eig_grad_pair(r, r2, ph, or_lj3(rho, R->eps[ti][tj], R->sig[ti][tj]), v, i, j, g);
        }
    for (int b = 0; b < R->nbond; ++b) {            /* Eq. 12: phi''' = 0 */
        int i = R->bonds[2 * b], j = R->bonds[2 * b + 1];
        double r2 = or_rij(R, x, i, j, r);
        or_bond(R, sqrt(r2), ph);
        or_eig_grad_pair(r, r2, ph, 0.0, v, i, j, g);
    }
}

/* Eq. 15: out = { DeltaV_2(epsilon), dDeltaV_2/depsilon }, the shape of Eq. 14
 * with epsilon_L, epsilon_U. */
void or_dv2(const or_rep *R, double e, double out[2]) {
    double lo = R->eig_lo, hi = R->eig_hi, dvm = R->dvmax;
    int m = R->m_exp;
    if (e >= hi) { out[0] = dvm; out[1] = 0.0; return; }
    if (e <= lo) { out[0] = 0.0; out[1] = 0.0; return; }
    double t = (e - hi) / (lo - hi);
    double tm1 = pow(t, (double)(m - 1));
    double q = 1.0 - tm1 * t;
    out[0] = dvm * q * q;
    out[1] = 2.0 * dvm * q * (-(double)m * tm1) / (lo - hi);
}

/* Eq. 13: out = { DeltaV, dDeltaV/dDeltaV_1, dDeltaV/dDeltaV_2 }. */
void or_dv13(const or_rep *R, double dv1, double dv2, double out[3]) {
    double dvm = R->dvmax;
    if (!(dvm > 0.0)) { out[0] = 0.0; out[1] = out[2] = 0.0; return; }
    out[0] = dv1 + dv2 - dv1 * dv2 / dvm;
    out[1] = 1.0 - dv2 / dvm;
    out[2] = 1.0 - dv1 / dvm;
}

/* ------------------------------------------------------------------------
 * Bias.  Eq. 7: d = |r - r_O| over all 3N coordinates (fixed atoms give 0;
 * every rigid atom contributes its own coordinates), s = (r - r_O)/d.
 * Eq. 5: sigma = grad V . s.  Eq. 14: DeltaV = DeltaV_1(sigma).
 * Its gradient: grad sigma = (H dr + g)/d - sigma dr/d^2, so the bias force
 * is F_b = -DeltaV_1'(sigma) grad sigma.
 * ---------------------------------------------------------------------- */
double or_bias_potential(const or_rep *R, const or_params *P, const double *x) {
    int n = R->n;
    double *g = malloc(sizeof(double) * 3 * n), dr[3], d2 = 0.0, G = 0.0, out[2];
    or_gradient(R, P, x, g);
    for (int i = 0; i < n; ++i) {
        or_disp(R, x, i, dr);
        for (int a = 0; a < 3; ++a) { d2 += dr[a] * dr[a]; G += g[3 * i + a] * dr[a]; }
    }
    free(g);
    double d = sqrt(d2);
    double s = d > 0.0 ? G / d : 0.0;
    or_dv1(R, s, out);
    if (!P->bias_on) return 0.0;
    if (!R->eig_on) return out[0];
    /* Eq. 13 with epsilon at x, Lanczos run to convergence from a copy of
     * the kept eigenvector */
    double *v = calloc((size_t)3 * n, sizeof(double)), b2[2], c[3];
    if (R->veig) memcpy(v, R->veig, sizeof(double) * 3 * n);
    double e = or_lowest_eig(R, P, x, v, 3 * n, 1e-13);
    free(v);
    or_dv2(R, e, b2);
    or_dv13(R, out[0], b2[0], c);
    return c[0];
}

void or_bias_eval(or_rep *R, const or_params *P) {
    int n = R->n, nr = or_nrig(R);
    double xt[3] = {0, 0, 0}, gs[3] = {0, 0, 0}, dr[3];
    if (nr > 0) {
        or_tip_centre(R, R->x, xt);
        or_ext_grad(R, xt, gs);
    }
    double d2 = 0.0, G = 0.0;
    for (int i = 0; i < n; ++i) {
        or_disp(R, R->x, i, dr);
        for (int a = 0; a < 3; ++a) {
            double g = -R->f_lj[3 * i + a] + (R->role[i] == 2 ? gs[a] / (double)nr : 0.0);
            d2 += dr[a] * dr[a];
            G += g * dr[a];
        }
    }
    double d = sqrt(d2);
    double s = d > 0.0 ? G / d : 0.0;
    double bv[2] = {0.0, 0.0};
    if (P->bias_on) or_dv1(R, s, bv);
    R->d = d; R->G = G; R->sigma = s; R->dV = bv[0]; R->dVp = bv[1];
    R->dV1 = bv[0]; R->dV2 = 0.0; R->dVe = 0.0;
    /* Eq. 13: DeltaV = DeltaV_1 + DeltaV_2 - DeltaV_1 DeltaV_2 / DeltaV_max,
     * its force -(dDeltaV/dsigma) grad sigma - (dDeltaV/depsilon) grad epsilon */
    double *ge = NULL;
    if (P->bias_on && R->eig_on) {
        double b2[2], c[3];
        int maxit = R->eig_maxit > 0 ? R->eig_maxit : 3 * R->n;   /* to convergence: capped at the allowed dimension */
        R->eig = or_lowest_eig(R, P, R->x, R->veig, maxit, 1e-10);
        or_dv2(R, R->eig, b2);
        or_dv13(R, bv[0], b2[0], c);
        R->dV2 = b2[0];
        R->dV = c[0];
        R->dVp = c[1] * bv[1];
        R->dVe = c[2] * b2[1];
        if (R->dVe != 0.0) {
            ge = malloc(sizeof(double) * 3 * n);
            or_eig_grad(R, P, R->x, R->veig, ge);
        }
    }
    R->fbody[0] = R->fbody[1] = R->fbody[2] = 0.0;
    for (int i = 0; i < n; ++i) {
        or_disp(R, R->x, i, dr);
        for (int a = 0; a < 3; ++a) {
            double g = -R->f_lj[3 * i + a] + (R->role[i] == 2 ? gs[a] / (double)nr : 0.0);
            double gsig = d > 0.0 ? (R->hdr[3 * i + a] + g) / d - s * dr[a] / (d * d) : 0.0;
            double ft = -g - R->dVp * gsig - (ge ? R->dVe * ge[3 * i + a] : 0.0);
            R->ftot[3 * i + a] = ft;
            if (R->role[i] == 2) R->fbody[a] += ft;
        }
    }
    free(ge);
    for (int a = 0; a < 3; ++a) R->xT[a] = xt[a];
    R->V = R->V_lj + (nr > 0 ? or_ext_energy(R, xt) : 0.0);
    R->FR = R->kspring * (R->slider[0] - xt[0]);          /* Eq. 10 */
}

static void or_kinetic(or_rep *R) {
    int nr = or_nrig(R);
    double k = 0.0;
    for (int i = 0; i < R->n; ++i)
        if (R->role[i] == 1)
            for (int a = 0; a < 3; ++a) k += 0.5 * R->v[3 * i + a] * R->v[3 * i + a];
    for (int a = 0; a < 3; ++a) k += 0.5 * (double)nr * R->vbody[a] * R->vbody[a];
    R->K = k;
}

/* Set up the cached state: list, forces, bias; optionally Maxwell-Boltzmann
 * velocities for the mobile atoms (rigid layer starts at rest). */
void or_init(or_rep *R, const or_params *P, int draw_velocities) {
    int n = R->n;
    if (draw_velocities) {
        double sd = sqrt(R->kT), z[2], z2[2];
        R->vbody[0] = R->vbody[1] = R->vbody[2] = 0.0;
        for (int i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a) R->v[3 * i + a] = 0.0;
            if (R->role[i] != 1) continue;
            or_normals(P->seed, R->rep_id, R->step, i, 2, z);
            R->v[3 * i + 0] = sd * z[0];
            R->v[3 * i + 1] = sd * z[1];
            if (R->dim == 3) {
                or_normals(P->seed, R->rep_id, R->step, i, 3, z2);
                R->v[3 * i + 2] = sd * z2[0];
            }
        }
    } else {
        R->vbody[0] = R->vbody[1] = R->vbody[2] = 0.0;
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 2) {
                for (int a = 0; a < 3; ++a) R->vbody[a] = R->v[3 * i + a];
                break;
            }
    }
    or_nlist_cells(R, P->rc + P->skin);
    or_forces(R, P);
    or_bias_eval(R, P);
    or_kinetic(R);
}

/* ------------------------------------------------------------------------
 * Dynamics.  Reading: the paper's Nose-Hoover chain with modified velocity
 * Verlet (Sec. 3.1.1) is replaced by Langevin dynamics in the BAOAB splitting
 * (Leimkuhler & Matthews): B = half kick, A = half drift, O = exact
 * Ornstein-Uhlenbeck step v <- c v + sqrt((1-c^2) kT/m) xi, c = exp(-gamma dt).
 * The thermostat acts on the mobile atoms only; fixed atoms never move; the
 * rigid layer moves as one body of mass n_rig (m = 1) under the sum of its
 * members' forces (LJ and bias), the spring and the load.
 * The boosted clock (Eq. 3) advances by dt exp(beta DeltaV) per step with the
 * DeltaV of the configuration the step starts from.
 * Verlet list rebuilt when any atom has moved more than skin/2.
 * ---------------------------------------------------------------------- */
/* ------------------------------------------------------------------------
 * Nose-Hoover chain (Sec. 3.1.1 names the chain thermostat; the integrator
 * is the reversible Trotter splitting of Martyna, Tuckerman, Tobias & Klein,
 * Mol. Phys. 87 (1996) 1117, one stage): a half step of the chain before the
 * first kick and after the last.  Thermostat j has mass Q_j, position xi_j,
 * velocity v_j and force G_1 = (2K_m - N_f kT)/Q_1 (K_m the kinetic energy
 * of the mobile atoms), G_j = (Q_{j-1} v_{j-1}^2 - kT)/Q_j; the chain end
 * is updated first, each v_j between two damping factors exp(-v_{j+1} dt/8)
 * from the end down to 1, the mobile velocities are scaled by
 * exp(-v_1 dt/2), the xi advance by v dt/2, and the sweep is repeated from
 * 1 back up to the end.  The extended energy K + V + DeltaV + sum Q v^2/2
 * + N_f kT xi_1 + kT sum_{j>1} xi_j is conserved.
 * ---------------------------------------------------------------------- */
static int or_nmobile(const or_rep *R) {
    int c = 0;
    for (int i = 0; i < R->n; ++i) c += (R->role[i] == 1);
    return c;
}

static void or_nhc_masses(const or_rep *R, double *Q) {
    double t2 = R->nhc_tau * R->nhc_tau;
    for (int j = 0; j < R->nhc_len; ++j) Q[j] = (j == 0 ? (double)(R->dim * or_nmobile(R)) : 1.0) * R->kT * t2;
}

double or_nhc_energy(const or_rep *R) {
    double Q[8], e = 0.0;
    if (R->nhc_len <= 0) return 0.0;
    or_nhc_masses(R, Q);
    double nf = (double)(R->dim * or_nmobile(R));
    for (int j = 0; j < R->nhc_len; ++j) {
        e += 0.5 * Q[j] * R->nhc_v[j] * R->nhc_v[j];
        e += (j == 0 ? nf : 1.0) * R->kT * R->nhc_xi[j];
    }
    return e;
}

static double or_nhc_force(const or_rep *R, const double *Q, double k2, double nf, int j) {
    if (j == 0) return (k2 - nf * R->kT) / Q[0];
    return (Q[j - 1] * R->nhc_v[j - 1] * R->nhc_v[j - 1] - R->kT) / Q[j];
}

static void or_nhc_half(or_rep *R, double h) {
    int M = R->nhc_len, D = R->dim;
    double Q[8], nf = (double)(D * or_nmobile(R)), k2 = 0.0;
    double *v = R->nhc_v;
    or_nhc_masses(R, Q);
    for (int i = 0; i < R->n; ++i)
        if (R->role[i] == 1)
            for (int a = 0; a < D; ++a) k2 += R->v[3 * i + a] * R->v[3 * i + a];
    v[M - 1] += 0.25 * h * or_nhc_force(R, Q, k2, nf, M - 1);
    for (int j = M - 2; j >= 0; --j) {
        double damp = exp(-0.125 * h * v[j + 1]);
        v[j] *= damp;
        v[j] += 0.25 * h * or_nhc_force(R, Q, k2, nf, j);
        v[j] *= damp;
    }
    double s = exp(-0.5 * h * v[0]);
    for (int i = 0; i < R->n; ++i)
        if (R->role[i] == 1)
            for (int a = 0; a < D; ++a) R->v[3 * i + a] *= s;
    k2 *= s * s;
    for (int j = 0; j < M; ++j) R->nhc_xi[j] += 0.5 * h * v[j];
    for (int j = 0; j < M - 1; ++j) {
        double damp = exp(-0.125 * h * v[j + 1]);
        v[j] *= damp;
        v[j] += 0.25 * h * or_nhc_force(R, Q, k2, nf, j);
        v[j] *= damp;
    }
    v[M - 1] += 0.25 * h * or_nhc_force(R, Q, k2, nf, M - 1);
}

void or_run(or_rep *R, const or_params *P, int nsteps) {
    int n = R->n, nr = or_nrig(R), D = R->dim;
    double h = P->dt;
    double c = exp(-R->gamma * h);
    double s = sqrt((1.0 - c * c) * R->kT);
    double half_skin2 = 0.25 * P->skin * P->skin;
    double z[2], z2[2];
    for (int it = 0; it < nsteps; ++it) {
        R->t_h += h * exp(R->dV / R->kT);
        R->t_md += h;
        if (R->nhc_len > 0) or_nhc_half(R, h);            /* chain half step (instead of O) */
        /* B */
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 1)
                for (int a = 0; a < D; ++a) R->v[3 * i + a] += 0.5 * h * R->ftot[3 * i + a];
        if (nr > 0)
            for (int a = 0; a < D; ++a) R->vbody[a] += 0.5 * h * R->fbody[a] / (double)nr;
        /* A */
        for (int i = 0; i < n; ++i) {
            if (R->role[i] == 1)
                for (int a = 0; a < D; ++a) R->x[3 * i + a] += 0.5 * h * R->v[3 * i + a];
            else if (R->role[i] == 2)
                for (int a = 0; a < D; ++a) R->x[3 * i + a] += 0.5 * h * R->vbody[a];
        }
        /* O (Langevin only) */
        for (int i = 0; i < n && R->nhc_len == 0; ++i) {
            if (R->role[i] != 1) continue;
            or_normals(P->seed, R->rep_id, R->step, i, 0, z);
            R->v[3 * i + 0] = c * R->v[3 * i + 0] + s * z[0];
            R->v[3 * i + 1] = c * R->v[3 * i + 1] + s * z[1];
            if (D == 3) {
                or_normals(P->seed, R->rep_id, R->step, i, 1, z2);
                R->v[3 * i + 2] = c * R->v[3 * i + 2] + s * z2[0];
            }
        }
        /* A */
        for (int i = 0; i < n; ++i) {
            if (R->role[i] == 1)
                for (int a = 0; a < D; ++a) R->x[3 * i + a] += 0.5 * h * R->v[3 * i + a];
            else if (R->role[i] == 2)
                for (int a = 0; a < D; ++a) R->x[3 * i + a] += 0.5 * h * R->vbody[a];
        }
        /* list check, forces at the new positions, bias */
        double mx = 0.0;
        for (int i = 0; i < n; ++i) {
            double dd = 0.0;
            for (int a = 0; a < 3; ++a) {
                double q = R->x[3 * i + a] - R->xb[3 * i + a];
                dd += q * q;
            }
            if (dd > mx) mx = dd;
        }
        if (mx > half_skin2) {
            or_nlist_cells(R, P->rc + P->skin);
            R->n_rebuild += 1;
        }
        if (R->vslide != 0.0)          /* continuous sliding: the slider at the step's end */
            R->slider[0] = R->slide_x0 + (double)(R->step + 1 - R->slide_step0) * (R->vslide * h);
        or_forces(R, P);
        or_bias_eval(R, P);
        /* B */
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 1)
                for (int a = 0; a < D; ++a) R->v[3 * i + a] += 0.5 * h * R->ftot[3 * i + a];
        if (nr > 0)
            for (int a = 0; a < D; ++a) R->vbody[a] += 0.5 * h * R->fbody[a] / (double)nr;
        for (int i = 0; i < n; ++i)
            if (R->role[i] == 2)
                for (int a = 0; a < 3; ++a) R->v[3 * i + a] = R->vbody[a];
        if (R->nhc_len > 0) or_nhc_half(R, h);
        R->step += 1;
    }
    or_kinetic(R);
}

void or_run_batch(or_rep *reps, int nrep, const or_params *P, int nsteps) {
    int r;
#pragma omp parallel for schedule(dynamic, 1)
    for (r = 0; r < nrep; ++r) or_run(&reps[r], P, nsteps);
}

/* ------------------------------------------------------------------------
 * Quench to the basin minimum r_O (the local minimum after Eq. 7).  The paper
 * does not name the minimiser; readings: unbiased V (LJ + spring + load),
 * slider fixed, fixed atoms frozen, rigid layer as one body.
 *   method 0, steepest descent: x_i += a F_i, X_body += a F_body / n_rig.
 *   method 1, FIRE (Bitzek, Koskinen, Gahler, Moseler, Gumbsch, PRL 97,
 *   170201, 2006) with its published settings N_min = 5, f_inc = 1.1,
 *   f_dec = 0.5, alpha_start = 0.1, f_alpha = 0.99, dt_max = 10 dt_0, and
 *   semi-implicit Euler steps; the body enters the mixing mass-weighted.
 * Converged when max(|F_i| over mobile atoms, |F_body|) < ftol.  Works on the
 * copy xq; the MD state is left untouched.  Returns the number of updates.
 * ---------------------------------------------------------------------- */
static void or_qforce(const or_rep *R, const or_params *P, const double *xq, const int *nnb, const int *nbr,
                      double *f, double fb[3], double *fmax) {
    int n = R->n, nr = or_nrig(R);
    or_pairs_on_list(R, xq, nnb, nbr, P->rc, f, NULL, NULL);
    double m = 0.0;
    fb[0] = fb[1] = fb[2] = 0.0;
    for (int i = 0; i < n; ++i) {
        if (R->role[i] == 1) {
            double q = f[3 * i] * f[3 * i] + f[3 * i + 1] * f[3 * i + 1] + f[3 * i + 2] * f[3 * i + 2];
            if (q > m) m = q;
        } else if (R->role[i] == 2) {
            for (int a = 0; a < 3; ++a) fb[a] += f[3 * i + a];
        }
    }
    if (nr > 0) {
        double xt[3], gs[3];
        or_tip_centre(R, xq, xt);
        or_ext_grad(R, xt, gs);
        for (int a = 0; a < 3; ++a) fb[a] -= gs[a];
        double q = fb[0] * fb[0] + fb[1] * fb[1] + fb[2] * fb[2];
        if (q > m) m = q;
    }
    *fmax = sqrt(m);
}

/* Largest displacement of xq from r_O over all atoms, squared (minimum image). */
static double or_maxdisp2(const or_rep *R, const double *xq) {
    double m = 0.0, dr[3];
    for (int i = 0; i < R->n; ++i) {
        or_disp(R, xq, i, dr);
        double q = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
        if (q > m) m = q;
    }
    return m;
}

/* The quench serves the transition test (Sec. 2.3), whose answer is a
 * displacement from r_O compared with theta.  Reading: a replica whose every
 * atom already lies within keep (< theta) of r_O and whose largest force is
 * below ftol_stay (> ftol) has not left its basin, and its quench stops there;
 * one that has not reached both goes on to ftol.  ftol_stay = 0 turns the
 * early stop off. */
int or_quench_gated(or_rep *R, const or_params *P, int method, double ftol, double ftol_stay, double keep,
                    int max_iter, double step_size, double *xq, double *fmax_out) {
    int n = R->n, nr = or_nrig(R), D = R->dim;
    int *nnb = malloc(sizeof(int) * n), *nbr = malloc(sizeof(int) * (size_t)n * R->maxnb);
    double *xb = malloc(sizeof(double) * 3 * n), *f = malloc(sizeof(double) * 3 * n);
    double *v = calloc((size_t)3 * n, sizeof(double));
    double fb[3], vb[3] = {0, 0, 0}, fmax = 0.0;
    double rl = P->rc + P->skin, half_skin2 = 0.25 * P->skin * P->skin;
    memcpy(xq, R->x, sizeof(double) * 3 * n);
    memcpy(xb, xq, sizeof(double) * 3 * n);
    int listed = or_list_cells(R, xq, rl, nnb, nbr) >= 0;
    /* FIRE state */
    double dt = step_size, dtmax = 10.0 * step_size, alpha = 0.1;
    int npos = 0, it;
    for (it = 0; listed && it < max_iter; ++it) {
        double mx = 0.0;
        for (int i = 0; i < n; ++i) {
            double dd = 0.0;
            for (int a = 0; a < 3; ++a) { double q = xq[3 * i + a] - xb[3 * i + a]; dd += q * q; }
            if (dd > mx) mx = dd;
        }
        if (mx > half_skin2) {
            if (or_list_cells(R, xq, rl, nnb, nbr) < 0) { fmax = NAN; break; }
            memcpy(xb, xq, sizeof(double) * 3 * n);
        }
        or_qforce(R, P, xq, nnb, nbr, f, fb, &fmax);
        if (fmax < ftol) break;
        if (ftol_stay > 0.0 && fmax < ftol_stay && or_maxdisp2(R, xq) < keep * keep) break;
        if (!(fmax < 1e30)) break;            /* diverged (step too large for the stiffest mode) */
        if (method == 0) {
            for (int i = 0; i < n; ++i) {
                if (R->role[i] == 1)
                    for (int a = 0; a < D; ++a) xq[3 * i + a] += step_size * f[3 * i + a];
                else if (R->role[i] == 2)
                    for (int a = 0; a < D; ++a) xq[3 * i + a] += step_size * fb[a] / (double)nr;
            }
        } else {
            double pw = 0.0, vv = 0.0, ff = 0.0;
            for (int i = 0; i < n; ++i)
                if (R->role[i] == 1)
                    for (int a = 0; a < D; ++a) {
                        pw += f[3 * i + a] * v[3 * i + a];
                        vv += v[3 * i + a] * v[3 * i + a];
                        ff += f[3 * i + a] * f[3 * i + a];
                    }
            if (nr > 0)
                for (int a = 0; a < D; ++a) {
                    pw += fb[a] * vb[a];
                    vv += (double)nr * vb[a] * vb[a];
                    ff += fb[a] * fb[a] / (double)nr;
                }
            if (pw > 0.0) {
                double mix = ff > 0.0 ? alpha * sqrt(vv) / sqrt(ff) : 0.0;
                for (int i = 0; i < n; ++i)
                    if (R->role[i] == 1)
                        for (int a = 0; a < D; ++a)
                            v[3 * i + a] = (1.0 - alpha) * v[3 * i + a] + mix * f[3 * i + a];
                if (nr > 0)
                    for (int a = 0; a < D; ++a) vb[a] = (1.0 - alpha) * vb[a] + mix * fb[a] / (double)nr;
                npos += 1;
                if (npos > 5) {
                    dt = dt * 1.1 < dtmax ? dt * 1.1 : dtmax;
                    alpha *= 0.99;
                }
            } else {
                for (int i = 0; i < 3 * n; ++i) v[i] = 0.0;
                vb[0] = vb[1] = vb[2] = 0.0;
                dt *= 0.5;
                alpha = 0.1;
                npos = 0;
            }
            for (int i = 0; i < n; ++i) {
                if (R->role[i] == 1)
                    for (int a = 0; a < D; ++a) {
                        v[3 * i + a] += dt * f[3 * i + a];
                        xq[3 * i + a] += dt * v[3 * i + a];
                    }
            }
            if (nr > 0) {
                for (int a = 0; a < D; ++a) vb[a] += dt * fb[a] / (double)nr;
                for (int i = 0; i < n; ++i)
                    if (R->role[i] == 2)
                        for (int a = 0; a < D; ++a) xq[3 * i + a] += dt * vb[a];
            }
        }
    }
    if (!listed) fmax = NAN;
    if (fmax_out) *fmax_out = fmax;
    free(v); free(f); free(xb); free(nbr); free(nnb);
    return it;
}

int or_quench(or_rep *R, const or_params *P, int method, double ftol, int max_iter,
              double step_size, double *xq, double *fmax_out) {
    return or_quench_gated(R, P, method, ftol, 0.0, 0.0, max_iter, step_size, xq, fmax_out);
}

int or_quench_batch(or_rep *reps, int nrep, const or_params *P, int method, double ftol,
                    int max_iter, double step_size, double **xq, double *fmax_out, int *iters) {
    return or_quench_batch_gated(reps, nrep, P, method, ftol, 0.0, 0.0, max_iter, step_size, xq, fmax_out, iters);
}

int or_quench_batch_gated(or_rep *reps, int nrep, const or_params *P, int method, double ftol, double ftol_stay,
                          double keep, int max_iter, double step_size, double **xq, double *fmax_out, int *iters) {
    int r;
#pragma omp parallel for schedule(dynamic, 1)
    for (r = 0; r < nrep; ++r)
        iters[r] = or_quench_gated(&reps[r], P, method, ftol, ftol_stay, keep, max_iter, step_size, xq[r],
                                   &fmax_out[r]);
    return 0;
}

/* Transition test (Sec. 2.3: a transition is a change of basin): the
 * quenched configuration is compared with r_O; reading: flag when any atom
 * has moved by more than theta (minimum image). */
int or_transition(const or_rep *R, const double *xq, double theta, double *maxdisp) {
    double m = 0.0, dr[3];
    for (int i = 0; i < R->n; ++i) {
        or_disp(R, xq, i, dr);
        double q = dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];
        if (q > m) m = q;
    }
    if (maxdisp) *maxdisp = sqrt(m);
    return sqrt(m) > theta;
}
