// hd_eig.cu -- the eigenvalue bias of Eq. 13 and Eq. 15 on the GPU (FP64).
//
// epsilon is the lowest eigenvalue of the Hessian of V over the motions the
// model allows: fixed atoms frozen, the rigid layer moving as one body, in the
// same 3N metric as d and sigma (each rigid atom carries the body's
// displacement).  So epsilon is the lowest eigenvalue of P H P on the range of
// the projector P, which zeroes fixed atoms (and z in 2-D) and sets the rigid
// atoms to their mean.  The spring adds k / n_rig^2 to every (rigid, rigid)
// Hessian entry along x (and y in 3-D); the load is linear and adds nothing.
//
// k_eig: one CTA per replica runs Lanczos on P H P.  The start vector is the
// last step's eigenvector plus 0.3 times a fixed generic vector (both
// projected and normalised), so that a mode that becomes lowest at a level
// crossing is never missing from the Krylov space.  Each step takes the
// Hessian-vector product on the neighbour list, the three-term recurrence and
// a full reorthogonalisation against every earlier Lanczos vector (classical
// Gram-Schmidt, two passes).  The lowest eigenvalue of the tridiagonal matrix
// is found by multisection on Sturm counts (one warp, 32 points a round), its
// eigenvector by inverse iteration; the iteration stops when the Ritz
// residual beta_j |y_m| is below 1e-10 max(1, |lambda|), when beta_j < 1e-14,
// or at the allowed dimension (capped by eig_maxit).
//
// k_eig_grad: grad epsilon = grad (v^T H(r) v) at the fixed unit eigenvector v
// (first-order perturbation theory), summed per atom over its list from
// phi''' of the pair: with A = phi'/rho and B = (phi'' - A)/rho^2 the pair's
// share of v^T H v is A |w|^2 + B (r.w)^2 (w = v_i - v_j), with gradient
// r [B |w|^2 + (phi''' - 3 B rho)(r.w)^2 / rho^3] + 2 B (r.w) w.
#include "hd_internal.cuh"
#include "hd_launch.h"

namespace hd {

namespace {

constexpr int EIG_THREADS = 512;

__device__ __forceinline__ int role_of(const Dev &D, int i) { return (D.rec[i].p.w >> 8) & 0xff; }

// Sum of NV values over the CTA; every thread receives the sums.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*red)[NV], double *out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[w][q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        double a = 0.0;
        for (int k = 0; k < nw; ++k) a += red[k][threadIdx.x];
        out[threadIdx.x] = a;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = out[q];
    __syncthreads();
}

// P u at one atom, given the rigid layer's mean m of u.
__device__ __forceinline__ dbl4 project(int role, int dim, dbl4 u, const double m[3]) {
    if (role == ROLE_FIXED) return make_dbl4(0, 0, 0, 0);
    if (role == ROLE_RIGID) u = make_dbl4(m[0], m[1], m[2], 0.0);
    if (dim == 2) u.z = 0.0;
    u.w = 0.0;
    return u;
}

__device__ __forceinline__ double dot3(dbl4 a, dbl4 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Generic start vector of the oracle: 1 + 0.5 sin(0.7 k + 0.3 (k mod 7)) for
// the coordinate k = 3 (input index) + axis.
__device__ __forceinline__ dbl4 generic(int orig) {
    double g[3];
    for (int a = 0; a < 3; ++a) {
        const int k = 3 * orig + a;
        g[a] = 1.0 + 0.5 * sin(0.7 * (double)k + 0.3 * (double)(k % 7));
    }
    return make_dbl4(g[0], g[1], g[2], 0.0);
}

// (H u)_i on the list (pairs within rc, LJ and bonds) plus the spring term.
__device__ __forceinline__ dbl4 hessvec_atom(const Dev &D, const RepDev &R, int i, const dbl4 *u, int a0) {
    const dbl4 xi = D.x[i];
    const int ti = (int)xi.w;
    const dbl4 ui = u[i - a0];
    double hx = 0, hy = 0, hz = 0;
    const int nn = D.nnb[i];
    for (int k = 0; k < nn; ++k) {
        const int j = D.nbr[(size_t)k * D.natom + i];
        const dbl4 xj = D.x[j];
        const double dx = mi64(R, 0, xi.x - xj.x), dy = mi64(R, 1, xi.y - xj.y), dz = mi64(R, 2, xi.z - xj.z);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < D.rc2)) continue;
        const int tj = (int)xj.w;
        const double eps = R.eps[ti][tj];
        const double ir2 = 1.0 / r2;
        const double s2 = R.sig2[ti][tj] * ir2;
        const double s6 = s2 * s2 * s2;
        const double A = -24.0 * eps * ir2 * s6 * (2.0 * s6 - 1.0);       // phi'/r
        const double B = 96.0 * eps * ir2 * ir2 * s6 * (7.0 * s6 - 2.0);  // (phi'' - phi'/r)/r^2
        const dbl4 uj = u[j - a0];
        const double ux = ui.x - uj.x, uy = ui.y - uj.y, uz = ui.z - uj.z;
        const double rdu = dx * ux + dy * uy + dz * uz;
        hx += A * ux + B * rdu * dx;
        hy += A * uy + B * rdu * dy;
        hz += A * uz + B * rdu * dz;
    }
    if (R.nbond > 0)
        for (int b = D.bond_off[i]; b < D.bond_off[i + 1]; ++b) {
            const int j = D.bond_j[b];
            const dbl4 xj = D.x[j];
            const double dx = mi64(R, 0, xi.x - xj.x), dy = mi64(R, 1, xi.y - xj.y), dz = mi64(R, 2, xi.z - xj.z);
            const double r2 = dx * dx + dy * dy + dz * dz, rr = sqrt(r2);
            const double A = R.kbond * (rr - R.rbond) / rr;
            const double B = (R.kbond - A) / r2;
            const dbl4 uj = u[j - a0];
            const double ux = ui.x - uj.x, uy = ui.y - uj.y, uz = ui.z - uj.z;
            const double rdu = dx * ux + dy * uy + dz * uz;
            hx += A * ux + B * rdu * dx;
            hy += A * uy + B * rdu * dy;
            hz += A * uz + B * rdu * dz;
        }
    if (role_of(D, i) == ROLE_RIGID) {
        // k / n_rig^2 times the sum over the layer, whose atoms all carry u_i
        hx += R.kr_n * ui.x;
        if (R.dim == 3) hy += R.kr_n * ui.y;
    }
    return make_dbl4(hx, hy, hz, 0.0);
}

// Number of eigenvalues of the tridiagonal (al, be) below x.
__device__ __forceinline__ int sturm(const double *al, const double *be, int m, double x) {
    int c = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
        d = (al[i] - x) - (i > 0 ? b2 / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++c;
    }
    return c;
}

}  // namespace

__global__ void __launch_bounds__(EIG_THREADS) k_eig(Dev D) {
    const int r = blockIdx.x;
    const RepDev &R = D.rep[r];
    if (!D.bias_on || !R.eig_on) return;
    __shared__ double red[32][6];
    __shared__ double bc[6];
    __shared__ double s_lam;
    __shared__ int s_stop;
    const int n = R.n, a0 = R.atom0, dim = R.dim, kmax = R.eig_kmax, nr = R.nrig;
    dbl4 *Q = D.eq + R.eig_qoff;
    dbl4 *w = D.ew + a0;
    dbl4 *v = D.ev + a0;
    double *al = D.ealpha + R.eig_toff, *be = D.ebeta + R.eig_toff, *y = D.ey + R.eig_toff,
           *cf = D.ecoef + R.eig_toff;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double inr = nr > 0 ? 1.0 / (double)nr : 0.0;
    // ---- start vector
    {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int il = threadIdx.x; il < n; il += blockDim.x)
            if (role_of(D, a0 + il) == ROLE_RIGID) {
                const dbl4 a = v[il], g = generic(D.orig[a0 + il]);
                s[0] += a.x; s[1] += a.y; s[2] += a.z;
                s[3] += g.x; s[4] += g.y; s[5] += g.z;
            }
        block_sum<6>(s, red, bc);
        const double mv[3] = {s[0] * inr, s[1] * inr, s[2] * inr}, mg[3] = {s[3] * inr, s[4] * inr, s[5] * inr};
        double t[2] = {0, 0};
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            const int ro = role_of(D, a0 + il);
            const dbl4 pv = project(ro, dim, v[il], mv), pg = project(ro, dim, generic(D.orig[a0 + il]), mg);
            t[0] += dot3(pv, pv);
            t[1] += dot3(pg, pg);
        }
        block_sum<2>(t, reinterpret_cast<double (*)[2]>(red), bc);
        const double nv = sqrt(t[0]), ng = sqrt(t[1]);
        double q2[1] = {0};
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            const int ro = role_of(D, a0 + il);
            const dbl4 pv = project(ro, dim, v[il], mv), pg = project(ro, dim, generic(D.orig[a0 + il]), mg);
            dbl4 q = make_dbl4((nv > 1e-12 ? pv.x / nv : 0.0) + 0.3 * pg.x / ng,
                               (nv > 1e-12 ? pv.y / nv : 0.0) + 0.3 * pg.y / ng,
                               (nv > 1e-12 ? pv.z / nv : 0.0) + 0.3 * pg.z / ng, 0.0);
            Q[il] = q;
            q2[0] += dot3(q, q);
        }
        block_sum<1>(q2, reinterpret_cast<double (*)[1]>(red), bc);
        const double nrm = sqrt(q2[0]);
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            dbl4 q = Q[il];
            q.x /= nrm; q.y /= nrm; q.z /= nrm;
            Q[il] = q;
        }
        __syncthreads();
    }
    int m = 0;
    for (int j = 0; j < kmax; ++j) {
        const dbl4 *qj = Q + (size_t)j * n;
        // w = H q_j, then w = P w (rigid mean)
        double s[3] = {0, 0, 0};
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            const dbl4 h = hessvec_atom(D, R, a0 + il, qj, a0);
            w[il] = h;
            if (role_of(D, a0 + il) == ROLE_RIGID) { s[0] += h.x; s[1] += h.y; s[2] += h.z; }
        }
        block_sum<3>(s, reinterpret_cast<double (*)[3]>(red), bc);
        const double mw[3] = {s[0] * inr, s[1] * inr, s[2] * inr};
        double a[1] = {0};
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            const dbl4 pw = project(role_of(D, a0 + il), dim, w[il], mw);
            w[il] = pw;
            a[0] += dot3(qj[il], pw);
        }
        block_sum<1>(a, reinterpret_cast<double (*)[1]>(red), bc);
        const double alpha = a[0];
        const double bprev = j > 0 ? be[j - 1] : 0.0;
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            dbl4 x = w[il];
            const dbl4 q = qj[il];
            if (j > 0) {
                const dbl4 p = Q[(size_t)(j - 1) * n + il];
                x.x -= alpha * q.x + bprev * p.x;
                x.y -= alpha * q.y + bprev * p.y;
                x.z -= alpha * q.z + bprev * p.z;
            } else {
                x.x -= alpha * q.x;
                x.y -= alpha * q.y;
                x.z -= alpha * q.z;
            }
            w[il] = x;
        }
        if (threadIdx.x == 0) al[j] = alpha;
        __syncthreads();
        // full reorthogonalisation, two passes of classical Gram-Schmidt:
        // warps take Lanczos vectors i = wid, wid + nw, ...; then every atom
        // subtracts sum_i c_i q_i
        for (int pass = 0; pass < 2; ++pass) {
            for (int i = wid; i <= j; i += nw) {
                const dbl4 *qi = Q + (size_t)i * n;
                double c = 0.0;
                for (int il = lane; il < n; il += 32) c += dot3(qi[il], w[il]);
                c = warp_sum(c);
                if (lane == 0) cf[i] = c;
            }
            __syncthreads();
            for (int il = threadIdx.x; il < n; il += blockDim.x) {
                dbl4 x = w[il];
                for (int i = 0; i <= j; ++i) {
                    const double c = cf[i];
                    const dbl4 q = Q[(size_t)i * n + il];
                    x.x -= c * q.x;
                    x.y -= c * q.y;
                    x.z -= c * q.z;
                }
                w[il] = x;
            }
            __syncthreads();
        }
        double b2[1] = {0};
        for (int il = threadIdx.x; il < n; il += blockDim.x) b2[0] += dot3(w[il], w[il]);
        block_sum<1>(b2, reinterpret_cast<double (*)[1]>(red), bc);
        const double beta = sqrt(b2[0]);
        m = j + 1;
        // lowest eigenpair of the m x m tridiagonal matrix (warp 0)
        if (wid == 0) {
            if (lane == 0) be[j] = beta;
            __syncwarp();
            double lo = 1e300, hi = -1e300;
            for (int i = lane; i < m; i += 32) {
                const double rr = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i + 1 < m ? fabs(be[i]) : 0.0);
                lo = fmin(lo, al[i] - rr);
                hi = fmax(hi, al[i] + rr);
            }
            for (int o = 16; o > 0; o >>= 1) {
                lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            // multisection: 32 interior points a round; the bracket keeps
            // count(lo) = 0 and count(hi) >= 1
            for (int it = 0; it < 64 && hi - lo > 1e-15 * fmax(1.0, fabs(lo) + fabs(hi)); ++it) {
                const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
                const unsigned up = __ballot_sync(0xffffffffu, sturm(al, be, m, x) >= 1);
                const int first = up ? __ffs(up) - 1 : 32;      // first point with an eigenvalue below
                const double nlo = first > 0 ? lo + (hi - lo) * (double)first / 33.0 : lo;
                const double nhi = first < 32 ? lo + (hi - lo) * (double)(first + 1) / 33.0 : hi;
                lo = nlo;
                hi = nhi;
            }
            if (lane == 0) {
                const double lam = 0.5 * (lo + hi);
                // inverse iteration with T - (lam - delta) I (positive definite)
                const double delta = 1e-10 * fmax(1.0, fabs(lam)), sft = lam - delta;
                for (int i = 0; i < m; ++i) y[i] = 1.0;
                for (int rep = 0; rep < 3; ++rep) {
                    // forward elimination in place: cf holds the pivots d_i,
                    // y the right-hand side c_i
                    cf[0] = al[0] - sft;
                    for (int i = 1; i < m; ++i) {
                        const double l = be[i - 1] / cf[i - 1];
                        cf[i] = (al[i] - sft) - l * be[i - 1];
                        y[i] = y[i] - l * y[i - 1];
                    }
                    y[m - 1] = y[m - 1] / cf[m - 1];
                    for (int i = m - 2; i >= 0; --i) y[i] = (y[i] - be[i] * y[i + 1]) / cf[i];
                    double nrm = 0.0;
                    for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
                    nrm = sqrt(nrm);
                    for (int i = 0; i < m; ++i) y[i] /= nrm;
                }
                s_lam = lam;
                s_stop = (beta * fabs(y[m - 1]) <= 1e-10 * fmax(1.0, fabs(lam))) || beta < 1e-14 || m == kmax;
            }
        }
        __syncthreads();
        if (s_stop) break;
        dbl4 *qn = Q + (size_t)(j + 1) * n;
        for (int il = threadIdx.x; il < n; il += blockDim.x) {
            const dbl4 x = w[il];
            qn[il] = make_dbl4(x.x / beta, x.y / beta, x.z / beta, 0.0);
        }
        __syncthreads();
    }
    // v = sum_i y_i q_i, normalised
    double s1[1] = {0};
    for (int il = threadIdx.x; il < n; il += blockDim.x) {
        double x = 0, yv = 0, z = 0;
        for (int i = 0; i < m; ++i) {
            const dbl4 q = Q[(size_t)i * n + il];
            const double c = y[i];
            x += c * q.x;
            yv += c * q.y;
            z += c * q.z;
        }
        const dbl4 vv = make_dbl4(x, yv, z, 0.0);
        v[il] = vv;
        s1[0] += dot3(vv, vv);
    }
    block_sum<1>(s1, reinterpret_cast<double (*)[1]>(red), bc);
    const double nrm = sqrt(s1[0]);
    for (int il = threadIdx.x; il < n; il += blockDim.x) {
        dbl4 vv = v[il];
        vv.x /= nrm; vv.y /= nrm; vv.z /= nrm;
        v[il] = vv;
    }
    if (threadIdx.x == 0) {
        D.st[r].eig = s_lam;
        D.st[r].eig_iters = m;
    }
}

// grad epsilon per atom and the per-tile sums of its rigid part.
__global__ void __launch_bounds__(128) k_eig_grad(Dev D) {
    const int t = blockIdx.x, r = D.tile_rep[t];
    const RepDev &R = D.rep[r];
    if (!D.bias_on || !R.eig_on) return;
    __shared__ double red[32][3];
    __shared__ double out[3];
    const bool act = threadIdx.x < D.tile_n[t];
    const int i = D.tile_start[t] + (act ? threadIdx.x : 0);
    double gx = 0, gy = 0, gz = 0;
    if (act) {
        const dbl4 xi = D.x[i], vi = D.ev[i];
        const int ti = (int)xi.w;
        auto pair = [&](double dx, double dy, double dz, double r2, double A, double B, double p3, const dbl4 &vj) {
            const double rho = sqrt(r2);
            const double wx = vi.x - vj.x, wy = vi.y - vj.y, wz = vi.z - vj.z;
            const double ww = wx * wx + wy * wy + wz * wz, rw = dx * wx + dy * wy + dz * wz;
            const double cr = B * ww + (p3 - 3.0 * B * rho) * rw * rw / (r2 * rho);
            gx += cr * dx + 2.0 * B * rw * wx;
            gy += cr * dy + 2.0 * B * rw * wy;
            gz += cr * dz + 2.0 * B * rw * wz;
        };
        const int nn = D.nnb[i];
        for (int k = 0; k < nn; ++k) {
            const int j = D.nbr[(size_t)k * D.natom + i];
            const dbl4 xj = D.x[j];
            const double dx = mi64(R, 0, xi.x - xj.x), dy = mi64(R, 1, xi.y - xj.y), dz = mi64(R, 2, xi.z - xj.z);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < D.rc2)) continue;
            const int tj = (int)xj.w;
            const double eps = R.eps[ti][tj];
            const double ir2 = 1.0 / r2;
            const double s2 = R.sig2[ti][tj] * ir2;
            const double s6 = s2 * s2 * s2;
            const double A = -24.0 * eps * ir2 * s6 * (2.0 * s6 - 1.0);
            const double B = 96.0 * eps * ir2 * ir2 * s6 * (7.0 * s6 - 2.0);
            const double rho = sqrt(r2);
            const double p3 = 4.0 * eps * (-2184.0 * s6 * s6 + 336.0 * s6) / (rho * rho * rho);   // phi'''
            pair(dx, dy, dz, r2, A, B, p3, D.ev[j]);
        }
        if (R.nbond > 0)
            for (int b = D.bond_off[i]; b < D.bond_off[i + 1]; ++b) {
                const int j = D.bond_j[b];
                const dbl4 xj = D.x[j];
                const double dx = mi64(R, 0, xi.x - xj.x), dy = mi64(R, 1, xi.y - xj.y), dz = mi64(R, 2, xi.z - xj.z);
                const double r2 = dx * dx + dy * dy + dz * dz, rr = sqrt(r2);
                const double A = R.kbond * (rr - R.rbond) / rr;
                pair(dx, dy, dz, r2, A, (R.kbond - A) / r2, 0.0, D.ev[j]);          // phi''' = 0
            }
        D.eg[i] = make_dbl4(gx, gy, gz, 0.0);
    }
    // rigid part of grad epsilon, summed per tile in FP64
    const bool rig = act && role_of(D, i) == ROLE_RIGID;
    double v[3] = {rig ? gx : 0.0, rig ? gy : 0.0, rig ? gz : 0.0};
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = warp_sum(v[q]);
    if (lane == 0)
        for (int q = 0; q < 3; ++q) red[w][q] = v[q];
    __syncthreads();
    if (threadIdx.x < 3) {
        double a = 0.0;
        for (int k = 0; k < nw; ++k) a += red[k][threadIdx.x];
        D.epart[(size_t)t * 4 + threadIdx.x] = a;
    }
}

void launch_eig(const Dev &D, cudaStream_t s) {
    if (!D.any_eig) return;
    k_eig<<<D.nrep, EIG_THREADS, 0, s>>>(D);
    k_eig_grad<<<D.ntile, D.block, 0, s>>>(D);
}

}  // namespace hd
