// hd_internal.cuh -- device-side data layout and helpers of libhdslide.
//
// Layout in HBM (one caller-owned workspace, 256-byte aligned blocks):
//   per atom, all replicas back to back; inside a replica atoms are held in
//   cell-major order of the initial configuration (orig[] maps a slot to the
//   atom's input index, which is also its Philox counter word):
//     x      dbl4  FP64 position, w = LJ type           (never wrapped)
//     xo     dbl4  basin minimum r_O
//     v      dbl4     velocity (FP64 in both forms)
//     po     int4 (split form)  fixed-point image of r_O
//     f      dbl4 | float4   LJ force, w = per-atom energy (half of each pair)
//     h      dbl4 | float4   H.(r - r_O), spring term included
//     dr     dbl4 | float4   r - r_O
//     rec    AtomRec  32-bit fixed-point position (w = type | role << 8) and,
//                     in the split form, r - r_O as the difference of the
//                     images of r and r_O, 32 bytes
//     pfixb  int4     pfix at the last list build (displacement check)
//     nbr    int32 [maxnb][natom] column-major Verlet list (global j), nnb int32
//   per cell: count int32, atoms int32 [cell_cap]
//   per tile (block atoms of one replica): NPART FP64 partial sums, FP64 K part
//   per replica: RepDev (settings), RepState (clocks, body), Scal (scalars)
//
// Fixed point: on a periodic axis x_fix = rint(x * 2^(32+k) / L) taken modulo
// 2^32 (k = fine_shift >= 0), so the int32 difference of two images is the
// exact minimum image of every pair closer than L / 2^(k+1); k is chosen so
// that this covers every pair the list build tests (at most two cell widths
// apart).  On the open axis x_fix = rint((x - origin) * 2^(32+k) / span) with
// span >= L.  Cells are computed from the FP64 positions (exact integer map
// x * 2^32 / L on periodic axes, FP64 quotient on the open axis), and
// |x - origin| stays below span / 2 - 4 (checked every step).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hd.h"

namespace hd {

// 32-byte aligned FP64 quadruple (one 256-bit access per atom)
typedef double4_32a dbl4;
__host__ __device__ __forceinline__ dbl4 make_dbl4(double x, double y, double z, double w) {
    return make_double4_32a(x, y, z, w);
}

constexpr int NPART = 16;        // per-tile partial sums (see PART_*)
constexpr int MAXNB_CAP = 160;   // largest neighbour-row capacity a build supports
constexpr int QPART = 12;        // per-tile partial sums of the quench

enum {
    PART_D2 = 0, PART_G = 1, PART_V = 2, PART_FRIG = 3, PART_HRIG = 6, PART_DRRIG = 9,
    PART_XRIG = 12, PART_PAD = 15
};
enum { QP_FMAX2 = 0, QP_P = 1, QP_VV = 2, QP_FF = 3, QP_FRIG = 4, QP_XRIG = 7, QP_PAD = 10 };

// KIN: kinetic energy only.  NHC: scale the mobile velocities by the chain's
// factor before the opening kick and take no Langevin noise.  SCALE: only
// scale the mobile velocities by the chain's factor (closing chain half step
// of the last step of a call), kinetic energy after it.
enum { MODE_CLOSE = 1, MODE_OPEN = 2, MODE_KIN = 4, MODE_NHC = 8, MODE_SCALE = 16 };
enum { ROLE_FIXED = 0, ROLE_MOBILE = 1, ROLE_RIGID = 2 };

// Per-atom record read by the pair sweep: fixed-point position (w = type |
// role << 8) and, in the split form, r - r_O on the same fixed-point grid (w
// unused); one 32-byte sector.  Differences of two atoms' r - r_O, which the
// Hessian-vector term takes, are then exact integers.
struct __align__(32) AtomRec {
    int4 p;
    int4 d;
};

struct RepDev {
    int dim, n, atom0, tile0, ntile, nrig, m_exp, rep_id;
    int cell0, ncell, vert, pad0;
    int nc[3], periodic[3];
    double L[3], invL[3];
    double kT, beta, c_ou, s_ou, kspring, fnormal, slider[2];
    double v_slide;              // continuous sliding: x_S = slider[0] + (step - slide_step0) (v_slide dt)
    long long slide_step0;       // step count of the configuration at which slider[0] was set
    double dvmax, sig_lo, sig_hi;
    double eps[2][2], sig2[2][2], shift[2][2];
    float epsf[2][2], sig2f[2][2], shiftf[2][2];
    // fine fixed point of the pair sweep: q = rint(x * scale - origin * scale)
    // mod 2^32, taken as the low word of fma(x, scale, fx_add) with
    // fx_add = 1.5 2^52 - origin * scale (a common offset of at most half a
    // unit per axis, which every difference of images cancels)
    double fx_scale[3], fx_origin[3], fx_add[3];
    float fx_lsb[3];
    int fine_shift;              // periodic axes count 2^(32 + fine_shift) units per L
    double bin_scale[3];         // periodic axes: 2^32 / L, the exact integer cell map
    double cell_lo, cell_inv_w;  // open axis: origin and inverse width of the cell grid
    double open_lim;             // escape bound |x - origin| on the open axis
    double kr_n;                 // k / n_rig (spring Hessian per rigid atom)
    float kr_nf, c_ouf, s_ouf, pad1;
    // exact squared distances: all axes share one fixed-point unit u (the open
    // axis counts 2^zshift units per step); u^2 = lsb2_hi + lsb2_lo
    int exact_r2, zshift, shift_y, shift_z;
    float u2_42, u2_21, u2_0, u2lo_42;     // u^2 2^42, u^2 2^21, u^2 (FP32) and the low part of u^2 2^42
    float lsb_rel[3];            // (unit - fl32(unit)) / fl32(unit) per axis
    float pad2;
    float r0sq_hi[2][2], r0sq_lo[2][2];  // 2^(1/3) sigma_ab^2 (LJ minimum, squared) as hi + lo
    float eps24f[2][2], eps96f[2][2];    // 24 eps_ab, 96 eps_ab (FP32 rounding) ...
    float eps24l[2][2], eps96l[2][2];    // ... and the remainders (hi + lo = the FP64 value)
    float rA2f;                  // list class A (first shell): FP32 r^2 below this at build time
    float kbondf;                // Eq. 12 bonds: stiffness (FP32)
    double kbond, rbond;         // Eq. 12 bonds: stiffness, rest length
    float rbond_hi, rbond_lo;    // rest length as FP32 hi + lo
    int nbond;                   // bonds of this replica (0: none; then every pair is LJ)
    int nhc_len;                 // Nose-Hoover chain length (0: Langevin)
    double nhc_nf, nhc_Q[8];     // chain: degrees of freedom, masses
    // eigenvalue bias (Eq. 13, Eq. 15): band of epsilon, Lanczos steps at most,
    // offsets of this replica's Krylov basis (dbl4 units) and tridiagonal arrays
    int eig_on, eig_kmax;
    double eig_lo, eig_hi;
    long long eig_qoff, eig_toff;
};

struct RepState {
    double t_h, t_md, vbody[3], vbody_full[3], K;
    long long step, n_rebuild;
    long long n_dv[3];           // steps with DeltaV = 0, inside the band, at DeltaV_max
    double nhc_xi[8], nhc_v[8];  // Nose-Hoover chain positions and velocities
    double nhc_k2;               // sum of m v^2 over mobile atoms after the last chain half step
    double eig;                  // lowest eigenvalue epsilon of the constrained Hessian (Eq. 15)
    int eig_iters, pad_st;       // Lanczos steps the last evaluation took
    // quench
    double q_dt, q_alpha, q_vb[3], q_fmax, q_disp;
    int q_npos, q_iter, q_done, q_flag;
    int q_stay, pad_q;           // the quench stopped inside its basin (at ftol_stay, not ftol)
};

struct Scal {
    double d, sigma, dV, dVp, G, V, Vlj, xT[3], fbody[3], FR, xS;
    double ca, cb;
    double vb_mid[3], vb_new[3];
    long long step_cur;
    // quench scalars of the current iteration
    double q_fbody[3], q_mix, q_alpha, q_dt, q_vb[3];
    int q_zero, q_active;
    double nhc_scale;            // chain: scale of the mobile velocities before the next kick
    double ce;                   // eigenvalue bias: F_tot += ce grad(epsilon), ce = -dDeltaV/depsilon
    double dV1, dV2;             // the two terms of Eq. 13
};

struct Dev {
    int nrep, ntile, natom, maxnb, cell_cap, ncell, prec, bias_on, block;
    int q_method, max_cells;        // max_cells: largest cell count of one replica
    double dt, rc2, rl2, half_skin2, q_ftol, q_step, q_theta;
    double q_ftol_stay, q_keep2;    // quench: early stop inside the basin (0: off), (theta/2)^2
    float rc2f, rl2_lo_f, rl2_hi_f, half_skin2_f;
    float rc2_lo_f, rc2_hi_f;    // rc^2 (1 -+ 2^-20): band decided in FP64
    uint32_t seed_lo, seed_hi;
    const RepDev *rep;
    RepState *st;
    Scal *sc;
    const int *tile_rep, *tile_start, *tile_n;
    double *part, *kpart;
    dbl4 *x, *xo;
    dbl4 *v64, *f64, *h64, *dr64;
    float4 *v32, *f32, *h32;     // v32: the quench's FIRE velocities (split form)
    int4 *po;                    // split form: fixed-point image of r_O (r - r_O = image difference)
    AtomRec *rec;                // fixed-point position + FP32 r - r_O
    int4 *pfixb;
    int *cellid, *nnb, *nbr, *cell_cnt, *cell_atoms;
    int *rebuild;                // per replica: list rebuild requested
    int *err;                    // [0] first error code, [1] atom, [2] replica
    unsigned int *bar;           // per replica barrier counters (persistent driver)
    unsigned long long *qdisp;   // per replica max |x_q - r_O|^2 (bits of the double)
    unsigned long long *qgate;   // per replica max |x_q - r_O|^2 of the current quench iterate
    const int *orig;             // per slot: index of the atom in its replica's input
    int *rb_list;                // replicas whose list is rebuilt, ascending (count rb_meta[0])
    int *rb_off, *rb_aoff;       // [count + 1] first compacted cell / atom of each of them
    int *rb_meta;                // {count, compacted cells, compacted atoms}
    const int *cta_rep;          // persistent launch: replica of each CTA (-1: spare)
    const int *pg_first, *pg_count;  // persistent launch: first CTA and CTA count of each replica
    const int *bond_off, *bond_j;    // per slot: bond partners (slots) in bond_j[bond_off[i] .. bond_off[i+1])
    int fault_rep;               // test hook (-1 off): a CTA of this replica skips one barrier arrival
    int nl_pow2, nl_grid;        // neighbour-row buffer (power of two >= maxnb), k_nlist CTAs
    int any_nhc;                 // some replica runs a Nose-Hoover chain: the update splits around it
    int any_eig;                 // some replica has the eigenvalue bias
    int pair_x2;                 // split form: the packed FP32x2 pair sweep (tiles <= 128 atoms)
    dbl4 *eq, *ev, *ew, *eg;     // eigenvalue bias: Krylov bases, eigenvector, work vector, grad epsilon
    double *ealpha, *ebeta, *ey, *ecoef;  // tridiagonal (alpha, beta), its eigenvector, coefficients
    double *epart;               // per tile: sum of grad epsilon over rigid atoms (4 doubles)
};

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ void set_err(const Dev &D, int code, int atom, int rep) {
    if (atomicCAS(D.err, 0, code) == 0) {
        D.err[1] = atom;
        D.err[2] = rep;
    }
}

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_draw(const Dev &D, long long step, int atom, int rep_id, int call) {
    uint4 c = make_uint4((uint32_t)(unsigned long long)step, (uint32_t)atom, (uint32_t)rep_id,
                         (uint32_t)call | ((uint32_t)((unsigned long long)step >> 32) << 8));
    return philox10(c, D.seed_lo, D.seed_hi);
}

// (k + 1/2) 2^-52 with k = (a>>6) 2^26 + (b>>6): strictly inside (0,1), exact in FP64.
__device__ __forceinline__ double unif64(uint32_t a, uint32_t b) {
    return ((double)(a >> 6) * 67108864.0 + (double)(b >> 6) + 0.5) * 0x1p-52;
}
// FP32 rounding of the same uniform, with full relative precision near 0.
__device__ __forceinline__ float unif32(uint32_t a, uint32_t b) {
    return fmaf((float)(a >> 6), 0x1p-26f, ((float)(b >> 6) + 0.5f) * 0x1p-52f);
}

__device__ __forceinline__ void normals64(uint4 w, double &n0, double &n1) {
    double u1 = unif64(w.x, w.y), u2 = unif64(w.z, w.w);
    double rad = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    n0 = rad * c;
    n1 = rad * s;
}
// FP32 Box-Muller from the same 52-bit uniforms u = (k + 1/2) 2^-52: u is
// split into its top 24 bits (head, exact in FP32) and the rest (tail); the
// tails enter to first order (log u = log fl(u) + (u - fl(u)) / fl(u), and
// the angle is rotated by 2 pi tail), so the normals are FP32-accurate with
// respect to the FP64 draw rather than to a 24-bit uniform.
__device__ __forceinline__ void normals32(uint4 w, float &n0, float &n1) {
    const float h1 = (float)(w.x >> 8) * 0x1p-24f;
    const float t1 = ((float)((((w.x >> 6) & 3u) << 26) | (w.y >> 6)) + 0.5f) * 0x1p-52f;
    const float u1 = h1 + t1;
    const float r1 = (h1 - u1) + t1;                      // u1 - fl(u1), exact to FP32
    const float l = logf(u1) + __fdividef(r1, u1);
    const float rad = sqrtf(-2.0f * l);
    const float h2 = (float)(w.z >> 8) * 0x1p-24f;
    const float t2 = ((float)((((w.z >> 6) & 3u) << 26) | (w.w >> 6)) + 0.5f) * 0x1p-52f;
    float s, c;
    sincospif(2.0f * h2, &s, &c);
    const float da = 6.28318530717958648f * t2;
    n0 = rad * fmaf(-s, da, c);
    n1 = rad * fmaf(c, da, s);
}

// Fixed-point image of one coordinate in one FP64 instruction: for
// |x scale - origin scale| < 2^51 the fused x * scale + fx_add lies in
// [2^52, 2^53), where doubles are the integers, so it is 1.5 2^52 plus the
// rounded (nearest even) image, and 1.5 2^52 is a multiple of 2^32: the low
// word is the image mod 2^32.  An axis without a grid has scale 0 and
// fx_add = 1.5 2^52, so its image is 0.
__device__ __forceinline__ int fix_coord(const RepDev &R, int a, double x) {
    return __double2loint(fma(x, R.fx_scale[a], R.fx_add[a]));
}

__device__ __forceinline__ int4 fix_pos(const RepDev &R, dbl4 x, int w) {
    return make_int4(fix_coord(R, 0, x.x), fix_coord(R, 1, x.y), fix_coord(R, 2, x.z), w);
}

// Difference of two fixed-point images, per axis, modulo 2^32 (w = 0).
__device__ __forceinline__ int4 img_diff(int4 a, int4 b) {
    return make_int4((int)((unsigned)a.x - (unsigned)b.x), (int)((unsigned)a.y - (unsigned)b.y),
                     (int)((unsigned)a.z - (unsigned)b.z), 0);
}

// Cell of an FP64 coordinate: exact integer map on periodic axes (the image
// rint(x 2^32 / L) mod 2^32 times nc, top 32 bits), clamped FP64 quotient on
// the open axis.
__device__ __forceinline__ int cell_of(const RepDev &R, int a, double x) {
    const int nc = R.nc[a];
    if (nc <= 1) return 0;
    if (R.periodic[a]) {
        const unsigned q = (unsigned)(unsigned long long)__double2ll_rn(x * R.bin_scale[a]);
        return (int)(((unsigned long long)q * (unsigned long long)nc) >> 32);
    }
    const int c = (int)floor((x - R.cell_lo) * R.cell_inv_w);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// The oracle's squared distance, op for op: minimum image per axis as
// d - L k with k the nearest integer to d / L, then ((dx dx + dy dy) + dz dz),
// every operation rounded.  k is taken as rint(d * (1/L)): for any pair
// within the list radius (L >= 3 (rc + skin)) d / L is far from a half
// integer, so k, and with it every rounded operation after it, is the same
// as the oracle's rint(d / L).
__device__ __forceinline__ double exact_r2(const RepDev &R, dbl4 a, dbl4 b) {
    double d0 = __dsub_rn(a.x, b.x), d1 = __dsub_rn(a.y, b.y), d2 = __dsub_rn(a.z, b.z);
    if (R.periodic[0]) d0 = __dsub_rn(d0, __dmul_rn(R.L[0], rint(d0 * R.invL[0])));
    if (R.periodic[1]) d1 = __dsub_rn(d1, __dmul_rn(R.L[1], rint(d1 * R.invL[1])));
    if (R.periodic[2]) d2 = __dsub_rn(d2, __dmul_rn(R.L[2], rint(d2 * R.invL[2])));
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

__device__ __forceinline__ double mi64(const RepDev &R, int a, double d) {
    return R.periodic[a] ? d - R.L[a] * rint(d * R.invL[a]) : d;
}

// Exact squared distance of an interacting pair as FP32 hi + lo, from its
// integer separations (ix, iy, iz) in the common fixed-point unit u (the open
// axis counts 2^zshift units per step).  q = sum of squares is exact in 64-bit
// integers (three 32x32->64 multiply-adds); q is cut into three 21-bit pieces,
// each turned into an exact float by the 2^23 bias trick, and
// u^2 q = hi + lo with hi the FP32 rounding of u^2 q and lo the remainder
// (TwoProduct by FMA, Fast2Sum).  Integer and FP32 pipes only.
__device__ __forceinline__ float exact_f23(unsigned int p) {
    return __int_as_float(0x4B000000u | p) - 8388608.0f;  // exact for p < 2^23
}
__device__ __forceinline__ void r2_split(const RepDev &R, int ix, int iy, int iz, float &hi, float &lo) {
    const int sy = iy << R.shift_y, sz = iz << R.shift_z;
    unsigned long long q = (unsigned long long)((long long)ix * (long long)ix);
    q += (unsigned long long)((long long)sy * (long long)sy);
    q += (unsigned long long)((long long)sz * (long long)sz);
    const float f0 = exact_f23((unsigned int)q & 0x1FFFFFu);
    const float f1 = exact_f23((unsigned int)(q >> 21) & 0x1FFFFFu);
    const float f2 = exact_f23((unsigned int)(q >> 42));
    // hi = fl(u^2 q): the top piece plus the middle one (Fast2Sum, |a| >= |b|);
    // lo = both rounding errors plus the small terms
    const float a = f2 * R.u2_42;
    const float ea = fmaf(f2, R.u2_42, -a);
    const float b = f1 * R.u2_21;
    hi = a + b;
    const float eb = (a - hi) + b;
    lo = (ea + eb) + fmaf(f0, R.u2_0, f2 * R.u2lo_42);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Slider x of the configuration reached after `step` steps: fixed (stepped
// sliding, Sec. 2.3) or moving at v_slide (continuous sliding, Sec. 3.1.1),
// written in closed form so that it does not accumulate rounding.
__device__ __forceinline__ double slider_x(const RepDev &R, long long step, double dt) {
    if (R.v_slide == 0.0) return R.slider[0];
    return R.slider[0] + (double)(step - R.slide_step0) * (R.v_slide * dt);
}

// Eq. 15: value and derivative of DeltaV_2(epsilon), the shape of Eq. 14 on
// the band [eps_L, eps_U] of the lowest Hessian eigenvalue.
__device__ __forceinline__ void dv2(const RepDev &R, double e, double &dv, double &dvp) {
    if (e >= R.eig_hi) { dv = R.dvmax; dvp = 0.0; return; }
    if (e <= R.eig_lo) { dv = 0.0; dvp = 0.0; return; }
    double t = (e - R.eig_hi) / (R.eig_lo - R.eig_hi);
    double tm1 = 1.0;
    for (int k = 1; k < R.m_exp; ++k) tm1 *= t;
    double q = 1.0 - tm1 * t;
    dv = R.dvmax * q * q;
    dvp = 2.0 * R.dvmax * q * (-(double)R.m_exp * tm1) / (R.eig_lo - R.eig_hi);
}

// Eq. 14: value and derivative of DeltaV_1(sigma).
__device__ __forceinline__ void dv1(const RepDev &R, double s, double &dv, double &dvp) {
    if (s >= R.sig_hi) { dv = R.dvmax; dvp = 0.0; return; }
    if (s <= R.sig_lo) { dv = 0.0; dvp = 0.0; return; }
    double t = (s - R.sig_hi) / (R.sig_lo - R.sig_hi);
    double tm1 = 1.0;
    for (int k = 1; k < R.m_exp; ++k) tm1 *= t;
    double q = 1.0 - tm1 * t;
    dv = R.dvmax * q * q;
    dvp = 2.0 * R.dvmax * q * (-(double)R.m_exp * tm1) / (R.sig_lo - R.sig_hi);
}

}  // namespace hd
