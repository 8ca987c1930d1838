// hd_api.cu -- host side of the C ABI declared in include/hd.h.
//
// Plans the workspace layout, uploads the replicas, and drives the per-phase
// kernels (captured in CUDA graphs) or the persistent kernel.  Every call
// returns an hd_status; the first error is kept on the context.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "hd_internal.cuh"
#include "hd_launch.h"

using namespace hd;

namespace {

constexpr size_t ALIGN = 256;

struct Plan {
    int nrep = 0, natom = 0, ntile = 0, maxnb = 0, cell_cap = 0, ncell = 0, block = 128, prec = 0;
    std::vector<RepDev> rep;
    std::vector<int> tile_rep, tile_start, tile_n;
    // storage order: atoms of a replica are held cell-major (cells of the
    // initial configuration, z then y then x, input order inside a cell);
    // slot_orig[global slot] = the atom's index in the replica's input arrays
    std::vector<int> slot_orig;
    // bond partners per slot (Eq. 12), CSR over all replicas' slots
    std::vector<int> bond_off, bond_j;
    size_t bytes = 0;
    // offsets
    size_t o_rep, o_st, o_sc, o_trep, o_tstart, o_tn, o_part, o_qpart, o_kpart;
    size_t o_x, o_xo, o_xq, o_v, o_vq, o_f, o_fq, o_h, o_dr;
    size_t o_pfix, o_pfixb, o_qpfix, o_qpfixb, o_cellid, o_nnb, o_nbr, o_ccnt, o_catoms;
    size_t o_rebuild, o_qrebuild, o_err, o_bar, o_qdisp, o_qgate, o_drawvel, o_adopt, o_orig, o_rboff, o_rbaoff, o_rblist, o_rbmeta;
    size_t o_ctarep, o_pgfirst, o_pgcount, o_boff, o_bj;
    size_t o_eq, o_ev, o_ew, o_eg, o_ealpha, o_ebeta, o_ey, o_ecoef, o_epart, o_po;
    long long eig_q = 0, eig_t = 0;     // dbl4 entries of all Krylov bases, doubles of all tridiagonals
    bool any_eig = false;
};

size_t take(size_t &cur, size_t bytes) {
    size_t o = (cur + ALIGN - 1) / ALIGN * ALIGN;
    cur = o + bytes;
    return o;
}

bool valid_desc(const hd_replica_desc &d, std::string &why) {
    char b[160];
    if (d.dim != 2 && d.dim != 3) { why = "dim must be 2 or 3"; return false; }
    if (d.n_atoms <= 0 || !d.pos || !d.role || !d.type) { why = "empty replica or NULL arrays"; return false; }
    if (d.kT <= 0.0 || d.gamma < 0.0) { why = "kT must be > 0 and gamma >= 0"; return false; }
    if (d.m_exp < 1) { why = "m_exp must be >= 1"; return false; }
    if (!std::isfinite(d.v_slide)) { why = "v_slide must be finite"; return false; }
    if (d.n_bonds < 0 || (d.n_bonds > 0 && !d.bonds)) { why = "n_bonds < 0 or NULL bonds"; return false; }
    if (d.nhc_len < 0 || d.nhc_len > 8) { why = "nhc_len must be in [0, 8]"; return false; }
    if (d.nhc_len > 0 && !(d.nhc_tau > 0.0 && std::isfinite(d.nhc_tau))) { why = "nhc_tau must be > 0"; return false; }
    if (d.eig_on && !(std::isfinite(d.eig_lo) && std::isfinite(d.eig_hi) && d.eig_lo < d.eig_hi)) {
        why = "the eigenvalue band needs eig_lo < eig_hi";
        return false;
    }
    if (d.eig_maxit < 0) { why = "eig_maxit must be >= 0"; return false; }
    if (d.n_bonds > 0 && !(d.k_bond >= 0.0 && std::isfinite(d.k_bond) && d.r_bond > 0.0 && std::isfinite(d.r_bond))) {
        why = "k_bond must be >= 0 and r_bond > 0";
        return false;
    }
    for (int b = 0; b < d.n_bonds; ++b) {
        const int i = d.bonds[2 * b], j = d.bonds[2 * b + 1];
        if (i < 0 || j < 0 || i >= d.n_atoms || j >= d.n_atoms || i == j) { why = "bond with a bad atom index"; return false; }
    }
    for (int a = 0; a < d.dim - 1; ++a)
        if (!d.periodic[a] || !(d.box[a] > 0.0)) {
            snprintf(b, sizeof b, "in-plane axis %d must be periodic with a positive length", a);
            why = b;
            return false;
        }
    if (d.periodic[d.dim - 1] || (d.dim == 2 && d.periodic[2])) { why = "the vertical axis must be open"; return false; }
    for (int i = 0; i < d.n_atoms; ++i) {
        if (d.role[i] > 2 || d.type[i] > 1) { why = "role must be 0..2 and type 0..1"; return false; }
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(d.pos[3 * i + a])) { why = "non-finite position"; return false; }
        if (d.dim == 2 && d.pos[3 * i + 2] != 0.0) { why = "2-D replicas need z == 0"; return false; }
    }
    return true;
}

bool make_plan(const hd_replica_desc *reps, int n_rep, const hd_params *p, Plan &P, std::string &why) {
    if (!reps || n_rep <= 0 || !p) { why = "no replicas or no params"; return false; }
    if (p->prec != HD_FP64 && p->prec != HD_FP32_SPLIT) { why = "prec must be HD_FP64 or HD_FP32_SPLIT"; return false; }
    if (!(p->dt > 0.0) || !(p->rc > 0.0) || !(p->skin > 0.0)) { why = "dt, rc and skin must be > 0"; return false; }
    P.block = p->block > 0 ? p->block : 128;
    if (p->pair_kernel < 0 || p->pair_kernel > 1) { why = "pair_kernel must be 0 or 1"; return false; }
    if (P.block % 32 != 0 || P.block > 256) { why = "block must be a multiple of 32, at most 256"; return false; }
    P.prec = p->prec;
    P.nrep = n_rep;
    const double rl = p->rc + p->skin;
    bool any3 = false;
    for (int r = 0; r < n_rep; ++r) {
        if (!valid_desc(reps[r], why)) {
            why = "replica " + std::to_string(r) + ": " + why;
            return false;
        }
        any3 |= reps[r].dim == 3;
    }
    P.maxnb = p->maxnb > 0 ? p->maxnb : (any3 ? 112 : 32);
    if (P.maxnb > MAXNB_CAP) { why = "maxnb above the build's capacity of 160"; return false; }
    P.rep.resize(n_rep);
    int max_occ = 0;
    long long natom = 0, ntile = 0, ncell = 0;
    for (int r = 0; r < n_rep; ++r) {
        const hd_replica_desc &d = reps[r];
        RepDev R;
        memset(&R, 0, sizeof R);
        R.dim = d.dim;
        R.n = d.n_atoms;
        R.atom0 = (int)natom;
        R.tile0 = (int)ntile;
        R.ntile = (d.n_atoms + P.block - 1) / P.block;
        R.m_exp = d.m_exp;
        R.rep_id = d.rep_id;
        R.vert = d.dim - 1;
        int nrig = 0;
        for (int i = 0; i < d.n_atoms; ++i) nrig += d.role[i] == 2;
        R.nrig = nrig;
        // geometry, fixed point and cells.  The pair sweep's fixed point counts
        // 2^(32+k) units per periodic length L, k = max(0, floor(log2(L / (8 rl)))):
        // the int32 difference of two images is then the exact minimum image of
        // every pair closer than L / 2^(k+1) >= 4 rl, which covers every pair the
        // list build tests (at most two cell widths apart) while the unit stays
        // at L / 2^(32+k) <= 16 rl / 2^32 whatever the box length.
        auto kfine = [&](double len) {
            int k = 0;
            while (k < 16 && len / std::ldexp(1.0, k + 1) >= 8.0 * rl) ++k;
            return k;
        };
        bool same = true;
        for (int q = 0; q < d.dim - 1; ++q) same &= d.box[q] == d.box[0];
        for (int a = 0; a < 3; ++a) {
            R.periodic[a] = (a < d.dim && d.periodic[a]) ? 1 : 0;
            if (R.periodic[a]) {
                const int k = kfine(d.box[a]);
                const double units = std::ldexp(4294967296.0, k);
                R.L[a] = d.box[a];
                R.invL[a] = 1.0 / d.box[a];
                R.fx_scale[a] = units / d.box[a];
                R.fx_origin[a] = 0.0;
                R.fx_lsb[a] = (float)(d.box[a] / units);
                R.bin_scale[a] = 4294967296.0 / d.box[a];
                if (a == 0) R.fine_shift = k;
                int nc = (int)std::floor(d.box[a] / (rl * (1.0 + 1e-6)));
                R.nc[a] = nc >= 3 ? nc : 1;
            } else if (a < d.dim) {
                double mn = d.pos[a], mx = d.pos[a];
                for (int i = 1; i < d.n_atoms; ++i) {
                    mn = std::min(mn, d.pos[3 * i + a]);
                    mx = std::max(mx, d.pos[3 * i + a]);
                }
                // Common fixed-point unit: when every periodic axis has the same
                // length L, the open axis uses span = L 2^z (z >= 0) per 2^(32+k)
                // units, so squared distances are exact integer sums in units of
                // (L / 2^(32+k))^2.
                const double need = 2.0 * (mx - mn) + 24.0;
                double span;
                int k;
                if (same && d.box[0] > 2.0 * (p->rc + 0.5)) {
                    int z = 0;
                    span = d.box[0];
                    while (span < need) { span *= 2.0; ++z; }
                    k = kfine(d.box[0]);
                    R.exact_r2 = 1;
                    R.zshift = z;
                    R.shift_y = a == 1 ? z : 0;
                    R.shift_z = a == 2 ? z : 0;
                    const double u = d.box[0] / std::ldexp(4294967296.0, k), u2 = u * u;
                    R.u2_42 = (float)(u2 * 4398046511104.0);
                    R.u2lo_42 = (float)(u2 * 4398046511104.0 - (double)R.u2_42);
                    R.u2_21 = (float)(u2 * 2097152.0);
                    R.u2_0 = (float)u2;
                } else {
                    span = 64.0;
                    while (span < need) span *= 2.0;
                    k = kfine(span);
                }
                const double units = std::ldexp(4294967296.0, k);
                R.fx_origin[a] = 0.5 * (mn + mx);
                R.fx_scale[a] = units / span;
                R.fx_lsb[a] = (float)(span / units);
                R.open_lim = 0.5 * span - 4.0;
                const double w = rl * (1.0 + 1e-4), lo = mn - 2.0;
                R.nc[a] = std::max(1, (int)std::ceil((mx + 2.0 - lo) / w));
                R.cell_lo = lo;
                R.cell_inv_w = 1.0 / w;
            } else {
                R.nc[a] = 1;
            }
            if (R.nc[a] >= 1024) { why = "replica " + std::to_string(r) + ": more than 1023 cells along an axis"; return false; }
        }
        for (int a = 0; a < 3; ++a) {
            R.fx_add[a] = 6755399441055744.0 - R.fx_origin[a] * R.fx_scale[a];   // 1.5 2^52 - origin scale
            const double u = R.fx_scale[a] != 0.0 ? 1.0 / R.fx_scale[a] : 0.0;
            R.lsb_rel[a] = R.fx_lsb[a] != 0.f ? (float)((u - (double)R.fx_lsb[a]) / (double)R.fx_lsb[a]) : 0.f;
        }
        R.ncell = R.nc[0] * R.nc[1] * R.nc[2];
        R.cell0 = (int)ncell;
        // occupancy estimate of the initial configuration and the storage order
        {
            std::vector<int> occ(R.ncell, 0), key(d.n_atoms);
            for (int i = 0; i < d.n_atoms; ++i) {
                int c[3];
                for (int a = 0; a < 3; ++a) {
                    if (R.nc[a] == 1) { c[a] = 0; continue; }
                    double x = d.pos[3 * i + a];
                    double t;
                    if (R.periodic[a]) t = (x - R.L[a] * std::floor(x / R.L[a])) / R.L[a] * R.nc[a];
                    else t = (x - R.cell_lo) * R.cell_inv_w;
                    c[a] = std::min(R.nc[a] - 1, std::max(0, (int)std::floor(t)));
                }
                key[i] = (c[2] * R.nc[1] + c[1]) * R.nc[0] + c[0];
                max_occ = std::max(max_occ, ++occ[key[i]]);
            }
            std::vector<int> order(d.n_atoms);
            for (int i = 0; i < d.n_atoms; ++i) order[i] = i;
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key[a] < key[b]; });
            P.slot_orig.insert(P.slot_orig.end(), order.begin(), order.end());
        }
        // interaction constants (Eq. 9 with the shift at rc)
        R.kT = d.kT;
        R.beta = 1.0 / d.kT;
        R.c_ou = std::exp(-d.gamma * p->dt);
        R.s_ou = std::sqrt((1.0 - R.c_ou * R.c_ou) * d.kT);
        R.c_ouf = (float)R.c_ou;
        R.s_ouf = (float)R.s_ou;
        R.kspring = d.k_spring;
        R.fnormal = d.f_normal;
        R.slider[0] = d.slider[0];
        R.slider[1] = d.slider[1];
        R.v_slide = d.v_slide;
        R.slide_step0 = d.step0;
        R.dvmax = d.dvmax;
        R.sig_lo = d.sig_lo;
        R.sig_hi = d.sig_hi;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                const double eps = d.eps[a][b], sig = d.sig[a][b];
                const double sc6 = std::pow(sig / p->rc, 6.0);
                R.eps[a][b] = eps;
                R.sig2[a][b] = sig * sig;
                R.shift[a][b] = 4.0 * eps * (sc6 * sc6 - sc6);
                R.epsf[a][b] = (float)eps;
                R.sig2f[a][b] = (float)(sig * sig);
                R.shiftf[a][b] = (float)R.shift[a][b];
                const double r0sq = std::cbrt(2.0) * sig * sig;   // LJ minimum 2^(1/6) sigma, squared
                R.r0sq_hi[a][b] = (float)r0sq;
                R.r0sq_lo[a][b] = (float)(r0sq - (double)R.r0sq_hi[a][b]);
                R.eps24f[a][b] = (float)(24.0 * eps);
                R.eps96f[a][b] = (float)(96.0 * eps);
                R.eps24l[a][b] = (float)(24.0 * eps - (double)R.eps24f[a][b]);
                R.eps96l[a][b] = (float)(96.0 * eps - (double)R.eps96f[a][b]);
                // the pair sweep takes the exact r^2 where |r_0^2 - r^2| < r^2 / 4,
                // i.e. r^2 < (4/3) r_0^2; class A of the list holds the pairs within
                // that radius plus 0.1 sigma at build time
                const double rA = std::sqrt(r0sq * 4.0 / 3.0) + 0.1 * sig;
                R.rA2f = std::max(R.rA2f, (float)(rA * rA));
            }
        R.kr_n = nrig > 0 ? d.k_spring / nrig : 0.0;
        R.kr_nf = (float)R.kr_n;
        // eigenvalue bias: Lanczos steps at most, capped at the dimension of the
        // allowed motions (dim x mobile atoms, plus dim for the rigid body)
        R.eig_on = d.eig_on ? 1 : 0;
        if (R.eig_on) {
            int nmob = 0;
            for (int i = 0; i < d.n_atoms; ++i) nmob += d.role[i] == 1;
            const int dimP = d.dim * nmob + (nrig > 0 ? d.dim : 0);
            int kmax = d.eig_maxit > 0 ? d.eig_maxit : 3 * d.n_atoms;
            kmax = std::max(1, std::min(kmax, dimP));
            R.eig_kmax = kmax;
            R.eig_lo = d.eig_lo;
            R.eig_hi = d.eig_hi;
            R.eig_qoff = P.eig_q;
            R.eig_toff = P.eig_t;
            P.eig_q += (long long)(kmax + 1) * d.n_atoms;
            P.eig_t += kmax;
            P.any_eig = true;
        }
        // Nose-Hoover chain masses: Q_1 = N_f kT tau^2, Q_j = kT tau^2
        R.nhc_len = d.nhc_len;
        if (d.nhc_len > 0) {
            int nmob = 0;
            for (int i = 0; i < d.n_atoms; ++i) nmob += d.role[i] == 1;
            R.nhc_nf = (double)(d.dim * nmob);
            const double t2 = d.nhc_tau * d.nhc_tau;
            for (int j = 0; j < d.nhc_len; ++j) R.nhc_Q[j] = (j == 0 ? R.nhc_nf : 1.0) * d.kT * t2;
        }
        // Eq. 12 bonds: with any bond, tip-tip pairs have no LJ term (zero
        // eps_tt and shift; the bond table carries their interaction)
        R.nbond = d.n_bonds;
        if (d.n_bonds > 0) {
            R.kbond = d.k_bond;
            R.rbond = d.r_bond;
            R.kbondf = (float)d.k_bond;
            R.rbond_hi = (float)d.r_bond;
            R.rbond_lo = (float)(d.r_bond - (double)R.rbond_hi);
            R.eps[1][1] = 0.0;
            R.shift[1][1] = 0.0;
            R.epsf[1][1] = 0.f;
            R.shiftf[1][1] = 0.f;
            R.eps24f[1][1] = 0.f;
            R.eps96f[1][1] = 0.f;
            R.eps24l[1][1] = 0.f;
            R.eps96l[1][1] = 0.f;
        }
        P.rep[r] = R;
        for (int k = 0; k < R.ntile; ++k) {
            P.tile_rep.push_back(r);
            P.tile_start.push_back(R.atom0 + k * P.block);
            P.tile_n.push_back(std::min(P.block, d.n_atoms - k * P.block));
        }
        natom += d.n_atoms;
        ntile += R.ntile;
        ncell += R.ncell;
        if (natom > (1LL << 30)) { why = "more than 2^30 atoms"; return false; }
    }
    P.natom = (int)natom;
    P.ntile = (int)ntile;
    P.ncell = (int)ncell;
    {
        // bond partners per slot, both directions, in the replicas' storage order
        std::vector<int> deg(P.natom, 0), slot_of;
        std::vector<std::vector<int>> part(P.natom);
        for (int r = 0; r < n_rep; ++r) {
            const hd_replica_desc &d = reps[r];
            if (d.n_bonds <= 0) continue;
            const int a0 = P.rep[r].atom0;
            slot_of.assign(d.n_atoms, 0);
            for (int sl = 0; sl < d.n_atoms; ++sl) slot_of[P.slot_orig[a0 + sl]] = a0 + sl;
            for (int b = 0; b < d.n_bonds; ++b) {
                const int i = slot_of[d.bonds[2 * b]], j = slot_of[d.bonds[2 * b + 1]];
                part[i].push_back(j);
                part[j].push_back(i);
            }
        }
        P.bond_off.assign(P.natom + 1, 0);
        for (int i = 0; i < P.natom; ++i) P.bond_off[i + 1] = P.bond_off[i] + (int)part[i].size();
        P.bond_j.clear();
        for (int i = 0; i < P.natom; ++i) P.bond_j.insert(P.bond_j.end(), part[i].begin(), part[i].end());
    }
    P.cell_cap = p->cell_cap > 0 ? p->cell_cap : ((2 * max_occ + 8 + 7) / 8) * 8;
    // layout
    const size_t N = P.natom, T = P.ntile, R = P.nrep;
    const size_t v4 = P.prec == HD_FP64 ? sizeof(dbl4) : sizeof(float4);
    size_t cur = 0;
    P.o_rep = take(cur, R * sizeof(RepDev));
    P.o_st = take(cur, R * sizeof(RepState));
    P.o_sc = take(cur, R * sizeof(Scal));
    P.o_trep = take(cur, T * 4);
    P.o_tstart = take(cur, T * 4);
    P.o_tn = take(cur, T * 4);
    P.o_part = take(cur, T * NPART * 8);
    P.o_qpart = take(cur, T * NPART * 8);
    P.o_kpart = take(cur, T * 8);
    P.o_x = take(cur, N * sizeof(dbl4));
    P.o_xo = take(cur, N * sizeof(dbl4));
    P.o_xq = take(cur, N * sizeof(dbl4));
    P.o_v = take(cur, N * sizeof(dbl4));     // velocities are FP64 in both forms
    P.o_vq = take(cur, N * v4);
    P.o_f = take(cur, N * v4);
    P.o_fq = take(cur, N * v4);
    P.o_h = take(cur, N * v4);
    P.o_dr = take(cur, N * v4);
    P.o_pfix = take(cur, N * sizeof(AtomRec));
    P.o_pfixb = take(cur, N * 16);
    P.o_qpfix = take(cur, N * sizeof(AtomRec));
    P.o_qpfixb = take(cur, N * 16);
    P.o_cellid = take(cur, N * 4);
    P.o_nnb = take(cur, N * 4);
    P.o_nbr = take(cur, N * (size_t)P.maxnb * 4);
    P.o_ccnt = take(cur, (size_t)P.ncell * 4);
    P.o_catoms = take(cur, (size_t)P.ncell * P.cell_cap * 4);
    P.o_rebuild = take(cur, R * 4);
    P.o_qrebuild = take(cur, R * 4);
    P.o_err = take(cur, 4 * 4);
    P.o_bar = take(cur, R * 2 * 4);
    P.o_qdisp = take(cur, R * 8);
    P.o_qgate = take(cur, R * 8);
    P.o_drawvel = take(cur, R * 4);
    P.o_adopt = take(cur, R * 4);
    P.o_orig = take(cur, N * 4);
    P.o_rboff = take(cur, (R + 1) * 4);
    P.o_rbaoff = take(cur, (R + 1) * 4);
    P.o_rblist = take(cur, R * 4);
    P.o_rbmeta = take(cur, 4 * 4);
    P.o_ctarep = take(cur, T * 4);       // at most one CTA per tile
    P.o_pgfirst = take(cur, R * 4);
    P.o_pgcount = take(cur, R * 4);
    P.o_po = take(cur, (P.prec == HD_FP64 ? 1 : N) * 16);   // split form: fixed-point image of r_O
    P.o_boff = take(cur, (N + 1) * 4);
    P.o_bj = take(cur, std::max<size_t>(1, P.bond_j.size()) * 4);
    {
        const size_t nv = P.any_eig ? N : 1, nq = std::max<long long>(1, P.eig_q), nt = std::max<long long>(1, P.eig_t);
        P.o_eq = take(cur, nq * sizeof(dbl4));
        P.o_ev = take(cur, nv * sizeof(dbl4));
        P.o_ew = take(cur, nv * sizeof(dbl4));
        P.o_eg = take(cur, nv * sizeof(dbl4));
        P.o_ealpha = take(cur, nt * 8);
        P.o_ebeta = take(cur, nt * 8);
        P.o_ey = take(cur, nt * 8);
        P.o_ecoef = take(cur, nt * 8);
        P.o_epart = take(cur, T * 4 * 8);
    }
    P.bytes = (cur + ALIGN - 1) / ALIGN * ALIGN;
    return true;
}

}  // namespace

struct hd_ctx {
    Plan P;
    Dev D{}, Q{};
    cudaStream_t s = nullptr;
    char *ws = nullptr;
    hd_status status = HD_OK;
    std::string err;
    int driver = HD_DRIVER_KERNELS;
    int persistent_ctas = 0;
    long long launches = 0;
    std::map<int, cudaGraphExec_t> graphs;
    std::map<std::string, cudaGraphExec_t> qgraphs;
    bool persist_graph_ok = true;
    std::vector<double> qdisp;
    std::vector<int> qflag, qconv;
    long long steps_done = 0;             // hd_step advances every replica alike
    std::vector<long long> step0;
    long long h2d = 0, d2h = 0;
    // timing: events recorded around phases; harvested at hd_timing / next step
    int timing = 0;
    struct Span { cudaEvent_t a, b; int cat; };
    std::vector<Span> pending;            // recorded directly on the stream
    std::map<int, std::vector<Span>> graph_spans;  // event nodes inside graph n
    std::vector<int> graph_pending;       // graphs launched, spans not yet harvested
    double tsum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long tcnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    std::vector<cudaEvent_t> free_events;
};

namespace {

hd_status fail(hd_ctx *c, hd_status st, const char *fmt, ...) {
    char b[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b, sizeof b, fmt, ap);
    va_end(ap);
    if (c && c->status == HD_OK) {
        c->status = st;
        c->err = b;
    }
    return st;
}

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(c, HD_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                         \
    } while (0)

template <typename T>
T *at(char *base, size_t off) { return reinterpret_cast<T *>(base + off); }

enum { T_PAIR = 0, T_UPDATE = 1, T_REBUILD = 2, T_SCALAR = 3, T_NLIST = 4, T_EIG = 5, T_NCAT = 8 };

cudaEvent_t get_event(hd_ctx *c) {
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

// Record a start event if timing is on; returns the span index or -1.
struct Timed {
    hd_ctx *c;
    std::vector<hd_ctx::Span> *sink;
    hd_ctx::Span sp;
    bool on;
    bool capturing = false;
    Timed(hd_ctx *c_, std::vector<hd_ctx::Span> *sink_, int cat) : c(c_), sink(sink_), on(c_->timing && sink_) {
        if (on) {
            sp.a = get_event(c);
            sp.b = get_event(c);
            sp.cat = cat;
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            cudaStreamIsCapturing(c->s, &cs);
            capturing = cs == cudaStreamCaptureStatusActive;
            // inside a capture only an external record becomes an event node
            if (capturing) cudaEventRecordWithFlags(sp.a, c->s, cudaEventRecordExternal);
            else cudaEventRecord(sp.a, c->s);
        }
    }
    ~Timed() {
        if (on) {
            if (capturing) cudaEventRecordWithFlags(sp.b, c->s, cudaEventRecordExternal);
            else cudaEventRecord(sp.b, c->s);
            sink->push_back(sp);
        }
    }
};

void harvest(hd_ctx *c, std::vector<hd_ctx::Span> &v, bool recycle) {
    for (auto &sp : v) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, sp.a, sp.b) == cudaSuccess) {
            c->tsum[sp.cat] += ms;
            c->tcnt[sp.cat] += 1;
        } else {
            (void)cudaGetLastError();  // an unrecorded span is skipped, not reported later
        }
        if (recycle) {
            c->free_events.push_back(sp.a);
            c->free_events.push_back(sp.b);
        }
    }
    if (recycle) v.clear();
}

void harvest_all(hd_ctx *c) {
    cudaStreamSynchronize(c->s);
    harvest(c, c->pending, true);
    for (int n : c->graph_pending) harvest(c, c->graph_spans[n], false);
    c->graph_pending.clear();
}

void fill_dev(hd_ctx *c) {
    Plan &P = c->P;
    char *b = c->ws;
    Dev &D = c->D;
    D.nrep = P.nrep;
    D.ntile = P.ntile;
    D.natom = P.natom;
    D.maxnb = P.maxnb;
    D.cell_cap = P.cell_cap;
    D.ncell = P.ncell;
    D.max_cells = 0;
    for (const RepDev &R : P.rep) D.max_cells = std::max(D.max_cells, R.ncell);
    D.prec = P.prec;
    D.block = P.block;
    D.rep = at<RepDev>(b, P.o_rep);
    D.st = at<RepState>(b, P.o_st);
    D.sc = at<Scal>(b, P.o_sc);
    D.tile_rep = at<int>(b, P.o_trep);
    D.tile_start = at<int>(b, P.o_tstart);
    D.tile_n = at<int>(b, P.o_tn);
    D.part = at<double>(b, P.o_part);
    D.kpart = at<double>(b, P.o_kpart);
    D.x = at<dbl4>(b, P.o_x);
    D.xo = at<dbl4>(b, P.o_xo);
    D.v64 = at<dbl4>(b, P.o_v);
    D.po = at<int4>(b, P.o_po);
    if (P.prec == HD_FP64) {
        D.f64 = at<dbl4>(b, P.o_f);
        D.h64 = at<dbl4>(b, P.o_h);
        D.dr64 = at<dbl4>(b, P.o_dr);
    } else {
        D.f32 = at<float4>(b, P.o_f);
        D.h32 = at<float4>(b, P.o_h);
    }
    D.rec = at<AtomRec>(b, P.o_pfix);
    D.pfixb = at<int4>(b, P.o_pfixb);
    D.cellid = at<int>(b, P.o_cellid);
    D.nnb = at<int>(b, P.o_nnb);
    D.nbr = at<int>(b, P.o_nbr);
    D.cell_cnt = at<int>(b, P.o_ccnt);
    D.cell_atoms = at<int>(b, P.o_catoms);
    D.rebuild = at<int>(b, P.o_rebuild);
    D.err = at<int>(b, P.o_err);
    D.bar = at<unsigned int>(b, P.o_bar);
    D.qdisp = at<unsigned long long>(b, P.o_qdisp);
    D.qgate = at<unsigned long long>(b, P.o_qgate);
    D.orig = at<int>(b, P.o_orig);
    D.rb_off = at<int>(b, P.o_rboff);
    D.rb_aoff = at<int>(b, P.o_rbaoff);
    D.rb_list = at<int>(b, P.o_rblist);
    D.rb_meta = at<int>(b, P.o_rbmeta);
    D.cta_rep = at<int>(b, P.o_ctarep);
    // test hook for the barrier time-out path: HD_TEST_SKIP_ARRIVE=<replica>
    D.fault_rep = -1;
    if (const char *e = getenv("HD_TEST_SKIP_ARRIVE")) D.fault_rep = atoi(e);
    D.pg_first = at<int>(b, P.o_pgfirst);
    D.pg_count = at<int>(b, P.o_pgcount);
    D.bond_off = at<int>(b, P.o_boff);
    D.bond_j = at<int>(b, P.o_bj);
    D.any_eig = P.any_eig ? 1 : 0;
    D.eq = at<dbl4>(b, P.o_eq);
    D.ev = at<dbl4>(b, P.o_ev);
    D.ew = at<dbl4>(b, P.o_ew);
    D.eg = at<dbl4>(b, P.o_eg);
    D.ealpha = at<double>(b, P.o_ealpha);
    D.ebeta = at<double>(b, P.o_ebeta);
    D.ey = at<double>(b, P.o_ey);
    D.ecoef = at<double>(b, P.o_ecoef);
    D.epart = at<double>(b, P.o_epart);
    D.nl_pow2 = 32;
    while (D.nl_pow2 < P.maxnb) D.nl_pow2 <<= 1;
    {
        int dev = 0, nsm = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        D.nl_grid = nsm * 4;
    }
    // quench view: the copy of the positions and its own velocity, force,
    // fixed-point image, rebuild flags and tile sums
    Dev &Q = c->Q;
    Q = D;
    Q.x = at<dbl4>(b, P.o_xq);
    if (P.prec == HD_FP64) {
        Q.v64 = at<dbl4>(b, P.o_vq);
        Q.f64 = at<dbl4>(b, P.o_fq);
    } else {
        Q.v32 = at<float4>(b, P.o_vq);
        Q.f32 = at<float4>(b, P.o_fq);
    }
    Q.rec = at<AtomRec>(b, P.o_qpfix);
    Q.pfixb = at<int4>(b, P.o_qpfixb);
    Q.rebuild = at<int>(b, P.o_qrebuild);
    Q.part = at<double>(b, P.o_qpart);
}

void set_scalars(Dev &D, const hd_params *p) {
    D.bias_on = p->bias_on ? 1 : 0;
    D.dt = p->dt;
    D.rc2 = p->rc * p->rc;
    const double rl = p->rc + p->skin;
    D.rl2 = rl * rl;
    D.half_skin2 = 0.25 * p->skin * p->skin;
    D.rc2f = (float)D.rc2;
    D.rl2_lo_f = (float)(D.rl2 * (1.0 - 1.0 / 4096.0));
    D.rl2_hi_f = (float)(D.rl2 * (1.0 + 1.0 / 4096.0));
    // FP32 r^2 of the split sweep is within ~3e-7 (relative) of the oracle's
    // FP64 r^2 (fixed-point rounding of positions plus FP32 rounding); the
    // band decided in FP64 is 2^-20 ~ 9.5e-7 wide on each side
    D.rc2_lo_f = (float)(D.rc2 * (1.0 - 1.0 / 1048576.0));
    D.rc2_hi_f = (float)(D.rc2 * (1.0 + 1.0 / 1048576.0));
    D.half_skin2_f = (float)(D.half_skin2 * (1.0 - 1e-4));
    D.seed_lo = (uint32_t)p->seed;
    D.seed_hi = (uint32_t)(p->seed >> 32);
    D.pair_x2 = p->pair_kernel == 1 ? 1 : 0;
}

hd_status check_device(hd_ctx *c) {
    CK(cudaStreamSynchronize(c->s));
    CK(cudaGetLastError());
    int e[4];
    CK(cudaMemcpy(e, c->D.err, sizeof e, cudaMemcpyDeviceToHost));
    c->d2h += sizeof e;
    if (e[0] != 0) {
        const char *what = e[0] == HD_ERR_OVERFLOW ? "neighbour row or cell over capacity"
                         : e[0] == HD_ERR_NUMERIC ? "non-finite position or atom outside the open-axis range"
                         : e[0] == HD_ERR_TIMEOUT ? "device barrier wait ran out"
                                                  : "device error";
        return fail(c, (hd_status)e[0], "%s (atom %d, replica %d)", what, e[1], e[2]);
    }
    return HD_OK;
}

hd_status upload_reps(hd_ctx *c) {
    CK(cudaMemcpyAsync((void *)c->D.rep, c->P.rep.data(), c->P.rep.size() * sizeof(RepDev), cudaMemcpyHostToDevice, c->s));
    c->h2d += (long long)(c->P.rep.size() * sizeof(RepDev));
    return HD_OK;
}

// Kernels of one BAOAB step after the opening half (list, pair, scalars, update).
void queue_step(hd_ctx *c, int mode, std::vector<hd_ctx::Span> *sink) {
    // per-atom energies are observables only: computed on the last step of a call
    const bool last = !(mode & MODE_OPEN);
    { Timed t(c, sink, T_REBUILD); launch_rebuild_prep(c->D, c->s); }
    { Timed t(c, sink, T_NLIST); launch_nlist(c->D, c->s); }
    { Timed t(c, sink, T_PAIR); launch_pair(c->D, false, last, c->s); }
    if (c->D.any_eig) { Timed t(c, sink, T_EIG); launch_eig(c->D, c->s); }
    { Timed t(c, sink, T_SCALAR); launch_scalar(c->D, mode, c->s); }
    c->launches += c->D.any_eig ? 2 : 0;
    if (!c->D.any_nhc) {
        { Timed t(c, sink, T_UPDATE); launch_update(c->D, mode, c->s); }
        c->launches += 8;
        return;
    }
    // a Nose-Hoover chain needs the kinetic sums of the closing kick before
    // the velocities are scaled, so the update splits around the chain
    { Timed t(c, sink, T_UPDATE); launch_update(c->D, MODE_CLOSE, c->s); }
    launch_nhc(c->D, mode, c->s);
    { Timed t(c, sink, T_UPDATE); launch_update(c->D, (mode & MODE_OPEN) ? (MODE_OPEN | MODE_NHC) : MODE_SCALE, c->s); }
    c->launches += 10;
}

void queue_steps(hd_ctx *c, int n, std::vector<hd_ctx::Span> *sink) {
    { Timed t(c, sink, T_SCALAR); launch_scalar(c->D, MODE_OPEN, c->s); }
    if (c->D.any_nhc) {
        launch_nhc(c->D, MODE_OPEN, c->s);
        c->launches += 1;
    }
    { Timed t(c, sink, T_UPDATE); launch_update(c->D, c->D.any_nhc ? (MODE_OPEN | MODE_NHC) : MODE_OPEN, c->s); }
    c->launches += 2;
    for (int k = 1; k <= n; ++k) queue_step(c, k < n ? (MODE_CLOSE | MODE_OPEN) : MODE_CLOSE, sink);
}

hd_status refresh_md(hd_ctx *c, bool relist) {
    // recompute list (optional), forces, H.dr and scalars at the MD positions
    if (relist) {
        std::vector<int> two(c->P.nrep, 2);
        CK(cudaMemcpyAsync(c->D.rebuild, two.data(), two.size() * 4, cudaMemcpyHostToDevice, c->s));
        c->h2d += (long long)two.size() * 4;
        launch_rebuild(c->D, c->s);
        c->launches += 5;
        CK(cudaStreamSynchronize(c->s));
    }
    launch_pair(c->D, false, true, c->s);
    launch_eig(c->D, c->s);
    launch_scalar(c->D, 0, c->s);
    c->launches += 2 + (c->D.any_eig ? 2 : 0);
    CK(cudaGetLastError());
    return HD_OK;
}

// Persistent launch: CTAs per replica in proportion to its pair work (3-D
// atoms have ~4x the neighbours of 2-D ones), at least one and at most one
// per tile, all resident at once.  Returns false when the batch has more
// replicas than resident CTAs.
bool setup_persistent(hd_ctx *c) {
    const Plan &P = c->P;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (P.block > 128) return false;  // the persistent kernel is built for tiles of <= 128 atoms
    if (P.any_eig) return false;      // the eigenvalue bias runs on the per-phase kernels only
    const int bps = persist_blocks_per_sm(c->D);
    const long long maxg = (long long)bps * nsm;
    if (!coop || bps <= 0 || P.nrep > maxg) return false;
    std::vector<double> w(P.nrep);
    double wsum = 0.0;
    for (int r = 0; r < P.nrep; ++r) {
        w[r] = (double)P.rep[r].n * (P.rep[r].dim == 3 ? 1.0 : 0.25);
        wsum += w[r];
    }
    std::vector<int> cnt(P.nrep);
    long long tot = 0;
    for (int r = 0; r < P.nrep; ++r) {
        int k = (int)std::floor(w[r] / wsum * (double)maxg);
        k = std::max(1, std::min(k, P.rep[r].ntile));
        cnt[r] = k;
        tot += k;
    }
    while (tot > maxg) {
        int big = 0;
        for (int r = 1; r < P.nrep; ++r)
            if (cnt[r] > cnt[big]) big = r;
        if (cnt[big] <= 1) return false;
        --cnt[big];
        --tot;
    }
    std::vector<int> first(P.nrep), ctarep;
    for (int r = 0; r < P.nrep; ++r) {
        first[r] = (int)ctarep.size();
        for (int k = 0; k < cnt[r]; ++k) ctarep.push_back(r);
    }
    if (cudaMemcpyAsync((void *)c->D.cta_rep, ctarep.data(), ctarep.size() * 4, cudaMemcpyHostToDevice, c->s) !=
            cudaSuccess ||
        cudaMemcpyAsync((void *)c->D.pg_first, first.data(), P.nrep * 4, cudaMemcpyHostToDevice, c->s) !=
            cudaSuccess ||
        cudaMemcpyAsync((void *)c->D.pg_count, cnt.data(), P.nrep * 4, cudaMemcpyHostToDevice, c->s) != cudaSuccess)
        return false;
    c->persistent_ctas = (int)ctarep.size();
    return true;
}

}  // namespace

extern "C" {

size_t hd_workspace_bytes(const hd_replica_desc *reps, int n_rep, const hd_params *p) {
    Plan P;
    std::string why;
    if (!make_plan(reps, n_rep, p, P, why)) return 0;
    return P.bytes;
}

hd_status hd_create(const hd_replica_desc *reps, int n_rep, const hd_params *p, void *d_workspace, size_t ws_bytes,
                    void *cuda_stream, hd_ctx **out) {
    if (!out) return HD_ERR_ARG;
    *out = nullptr;
    hd_ctx *c = new hd_ctx();
    *out = c;
    std::string why;
    if (!make_plan(reps, n_rep, p, c->P, why)) return fail(c, HD_ERR_ARG, "%s", why.c_str());
    if (!d_workspace) return fail(c, HD_ERR_ARG, "NULL workspace");
    if ((uintptr_t)d_workspace % ALIGN) return fail(c, HD_ERR_ARG, "workspace not 256-byte aligned");
    if (ws_bytes < c->P.bytes)
        return fail(c, HD_ERR_NOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, c->P.bytes);
    c->ws = (char *)d_workspace;
    c->s = (cudaStream_t)cuda_stream;
    c->driver = HD_DRIVER_KERNELS;
    fill_dev(c);
    set_scalars(c->D, p);
    set_scalars(c->Q, p);
    {
        int nb = 0;
        CK(nl_configure(c->D, &nb));
        if (nb > 0) {
            c->D.nl_grid = c->D.nl_grid / 4 * nb;    // nl_grid starts at 4 CTAs per SM
            c->Q.nl_grid = c->D.nl_grid;
        }
    }
    c->D.any_nhc = 0;
    for (int r = 0; r < n_rep; ++r) c->D.any_nhc |= reps[r].nhc_len > 0;
    c->Q.any_nhc = c->D.any_nhc;
    Plan &P = c->P;
    const size_t N = P.natom;
    CK(cudaMemsetAsync(c->ws, 0, P.bytes, c->s));
    // host staging
    std::vector<dbl4> hx(N), hxo(N);
    std::vector<AtomRec> hp(N);
    std::vector<char> hv(N * sizeof(dbl4));
    std::vector<RepState> hst(P.nrep);
    std::vector<int> draw(P.nrep), two(P.nrep, 2);
    memset(hst.data(), 0, hst.size() * sizeof(RepState));
    for (int r = 0; r < P.nrep; ++r) {
        const hd_replica_desc &d = reps[r];
        const int a0 = P.rep[r].atom0;
        draw[r] = d.vel == nullptr;
        hst[r].t_h = d.t_h0;
        hst[r].t_md = d.t_md0;
        hst[r].step = d.step0;
        if (d.vel)
            for (int i = 0; i < d.n_atoms; ++i)
                if (d.role[i] == 2) {  // the body starts with the first rigid atom's velocity
                    for (int a = 0; a < d.dim; ++a) hst[r].vbody[a] = hst[r].vbody_full[a] = d.vel[3 * i + a];
                    break;
                }
        for (int sl = 0; sl < d.n_atoms; ++sl) {
            const int i = P.slot_orig[a0 + sl];
            const double *x = d.pos + 3 * i;
            const double *xo = d.pos_ref ? d.pos_ref + 3 * i : x;
            hx[a0 + sl] = make_dbl4(x[0], x[1], x[2], (double)d.type[i]);
            hxo[a0 + sl] = make_dbl4(xo[0], xo[1], xo[2], 0.0);
            hp[a0 + sl].p = make_int4(0, 0, 0, (int)d.type[i] | ((int)d.role[i] << 8));
            hp[a0 + sl].d = make_int4(0, 0, 0, 0);
            double v[3] = {0, 0, 0};
            if (d.vel && d.role[i] != 0)
                for (int a = 0; a < 3; ++a) v[a] = d.vel[3 * i + a];
            if (d.dim == 2) v[2] = 0.0;
            reinterpret_cast<dbl4 *>(hv.data())[a0 + sl] = make_dbl4(v[0], v[1], v[2], 0.0);
        }
    }
    if (upload_reps(c) != HD_OK) return c->status;
    CK(cudaMemcpyAsync(c->D.st, hst.data(), hst.size() * sizeof(RepState), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync((void *)c->D.tile_rep, P.tile_rep.data(), P.ntile * 4, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync((void *)c->D.tile_start, P.tile_start.data(), P.ntile * 4, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync((void *)c->D.tile_n, P.tile_n.data(), P.ntile * 4, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->D.x, hx.data(), N * sizeof(dbl4), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->D.xo, hxo.data(), N * sizeof(dbl4), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->D.rec, hp.data(), N * sizeof(AtomRec), cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync((void *)c->D.orig, P.slot_orig.data(), N * 4, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync((void *)c->D.bond_off, P.bond_off.data(), (N + 1) * 4, cudaMemcpyHostToDevice, c->s));
    if (!P.bond_j.empty())
        CK(cudaMemcpyAsync((void *)c->D.bond_j, P.bond_j.data(), P.bond_j.size() * 4, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->ws + P.o_v, hv.data(), hv.size(), cudaMemcpyHostToDevice, c->s));
    int *d_draw = at<int>(c->ws, P.o_drawvel);
    CK(cudaMemcpyAsync(d_draw, draw.data(), P.nrep * 4, cudaMemcpyHostToDevice, c->s));
    CK(cudaMemcpyAsync(c->D.rebuild, two.data(), P.nrep * 4, cudaMemcpyHostToDevice, c->s));
    launch_init(c->D, d_draw, c->s);
    launch_rebuild(c->D, c->s);
    launch_pair(c->D, false, true, c->s);
    launch_eig(c->D, c->s);
    launch_scalar(c->D, 0, c->s);
    launch_update(c->D, MODE_KIN, c->s);  // kinetic energy of the initial velocities
    launch_nhc(c->D, MODE_KIN, c->s);     // the chains start from it
    launch_obs(c->D, c->s);
    c->launches += 11 + (c->D.any_eig ? 2 : 0);
    CK(cudaGetLastError());
    c->qdisp.assign(P.nrep, 0.0);
    c->qflag.assign(P.nrep, 0);
    c->qconv.assign(P.nrep, 0);
    c->step0.resize(P.nrep);
    for (int r = 0; r < P.nrep; ++r) c->step0[r] = reps[r].step0;
    if (p->driver == HD_DRIVER_PERSISTENT && setup_persistent(c)) c->driver = HD_DRIVER_PERSISTENT;
    return check_device(c);
}

hd_status hd_set_slider(hd_ctx *c, const double *slider, int requench_ref) {
    if (!c) return HD_ERR_ARG;
    if (c->status != HD_OK) return HD_ERR_STATE;
    if (!slider) return fail(c, HD_ERR_ARG, "NULL slider array");
    for (int r = 0; r < c->P.nrep; ++r) {
        if (!std::isfinite(slider[2 * r]) || !std::isfinite(slider[2 * r + 1]))
            return fail(c, HD_ERR_ARG, "replica %d: non-finite slider position", r);
        c->P.rep[r].slider[0] = slider[2 * r];
        c->P.rep[r].slider[1] = slider[2 * r + 1];
        c->P.rep[r].slide_step0 = c->step0[r] + c->steps_done;   // a moving slider restarts from here
    }
    if (upload_reps(c) != HD_OK) return c->status;
    launch_scalar(c->D, 0, c->s);
    c->launches += 1;
    CK(cudaGetLastError());
    // FIRE from dt0 = 0.005 (fastest on thermal LJ states); the rigid body's
    // force, a sum over its atoms' FP32 pair forces, levels off near 4e-4 in
    // the split form, so that form quenches to 1e-3
    if (requench_ref) return hd_quench(c, 1, c->P.prec == HD_FP64 ? 1e-6 : 1e-3, 20000, 0.005, 1e300, 0.0, 2, nullptr);
    return HD_OK;
}

hd_status hd_set_bias(hd_ctx *c, const double *bias) {
    if (!c) return HD_ERR_ARG;
    if (c->status != HD_OK) return HD_ERR_STATE;
    if (!bias) return fail(c, HD_ERR_ARG, "NULL bias array");
    for (int r = 0; r < c->P.nrep; ++r) {
        if (!(bias[4 * r + 3] >= 1.0)) return fail(c, HD_ERR_ARG, "replica %d: m must be >= 1", r);
        c->P.rep[r].dvmax = bias[4 * r];
        c->P.rep[r].sig_lo = bias[4 * r + 1];
        c->P.rep[r].sig_hi = bias[4 * r + 2];
        c->P.rep[r].m_exp = (int)bias[4 * r + 3];
    }
    if (upload_reps(c) != HD_OK) return c->status;
    launch_scalar(c->D, 0, c->s);
    c->launches += 1;
    CK(cudaGetLastError());
    return HD_OK;
}

hd_status hd_step(hd_ctx *c, int n_steps) {
    if (!c) return HD_ERR_ARG;
    if (c->status != HD_OK) return HD_ERR_STATE;
    if (n_steps < 0) return fail(c, HD_ERR_ARG, "n_steps < 0");
    if (n_steps == 0) return HD_OK;
    c->steps_done += n_steps;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(c->s, &cs));
    const bool can_graph = c->s != nullptr && cs == cudaStreamCaptureStatusNone;
    if (c->timing && !c->graph_pending.empty()) harvest_all(c);
    if (c->driver == HD_DRIVER_PERSISTENT) {
        // one cooperative launch for all n steps, replayed from a graph when the
        // runtime captures it; launched directly otherwise
        if (can_graph && c->persist_graph_ok) {
            auto it = c->graphs.find(n_steps);
            if (it == c->graphs.end()) {
                if (c->graphs.size() >= 8) {  // keep at most 8 step counts, as on the per-phase path
                    for (auto &gx : c->graphs) cudaGraphExecDestroy(gx.second);
                    c->graphs.clear();
                }
                cudaGraph_t g = nullptr;
                cudaGraphExec_t ge = nullptr;
                bool ok = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
                cudaError_t le = ok ? launch_persist(c->D, c->persistent_ctas, n_steps, c->s) : cudaErrorUnknown;
                cudaError_t ee = ok ? cudaStreamEndCapture(c->s, &g) : cudaErrorUnknown;
                ok = ok && le == cudaSuccess && ee == cudaSuccess && g &&
                     cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
                if (g) cudaGraphDestroy(g);
                (void)cudaGetLastError();
                if (!ok) {
                    c->persist_graph_ok = false;
                } else {
                    it = c->graphs.emplace(n_steps, ge).first;
                }
            }
            if (c->persist_graph_ok) {
                CK(cudaGraphLaunch(it->second, c->s));
                c->launches += 1;
                return HD_OK;
            }
        }
        CK(launch_persist(c->D, c->persistent_ctas, n_steps, c->s));
        c->launches += 1;
        return HD_OK;
    }
    if (!can_graph) {
        queue_steps(c, n_steps, &c->pending);
        CK(cudaGetLastError());
        return HD_OK;
    }
    const int key = c->timing ? -n_steps : n_steps;
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
        if (c->graphs.size() >= 8) {
            harvest_all(c);
            for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
            c->graphs.clear();
            for (auto &kv : c->graph_spans)
                for (auto &sp : kv.second) {
                    c->free_events.push_back(sp.a);
                    c->free_events.push_back(sp.b);
                }
            c->graph_spans.clear();
        }
        cudaGraph_t g;
        long long before = c->launches;
        std::vector<hd_ctx::Span> spans;
        CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
        queue_steps(c, n_steps, c->timing ? &spans : nullptr);
        CK(cudaStreamEndCapture(c->s, &g));
        c->launches = before;
        cudaGraphExec_t ge;
        CK(cudaGraphInstantiate(&ge, g, 0));
        cudaGraphDestroy(g);
        it = c->graphs.emplace(key, ge).first;
        if (c->timing) c->graph_spans[key] = spans;
    }
    CK(cudaGraphLaunch(it->second, c->s));
    if (c->timing) c->graph_pending.push_back(key);
    c->launches += (c->D.any_nhc ? 3 + 10LL * n_steps : 2 + 8LL * n_steps) + (c->D.any_eig ? 2LL * n_steps : 0);
    return HD_OK;
}

hd_status hd_quench(hd_ctx *c, int method, double ftol, int max_iter, double step_size, double theta,
                    double ftol_stay, int adopt, int32_t *h_flags) {
    if (!c) return HD_ERR_ARG;
    if (c->status != HD_OK) return HD_ERR_STATE;
    if ((method != 0 && method != 1) || !(ftol > 0.0) || max_iter < 0 || !(step_size > 0.0) || adopt < 0 || adopt > 2)
        return fail(c, HD_ERR_ARG, "bad quench arguments");
    if (!(ftol_stay == 0.0 || (ftol_stay > ftol && theta > 0.0 && std::isfinite(theta))))
        return fail(c, HD_ERR_ARG, "ftol_stay must be 0, or above ftol with a finite theta > 0");
    Dev &Q = c->Q;
    Q.q_method = method;
    Q.q_ftol = ftol;
    Q.q_step = step_size;
    Q.q_theta = theta;
    Q.q_ftol_stay = ftol_stay;
    Q.q_keep2 = 0.25 * theta * theta;
    const int R = c->P.nrep;
    if (ftol_stay > 0.0) CK(cudaMemsetAsync(Q.qgate, 0, (size_t)R * 8, c->s));
    launch_qinit(Q, c->D, c->s);
    c->launches += 1;
    std::vector<RepState> st(R);
    const int chunk = 32;
    // one CUDA graph per quench setting replays `chunk` iterations
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(c->s, &cs));
    cudaGraphExec_t qg = nullptr;
    if (c->s != nullptr && cs == cudaStreamCaptureStatusNone) {
        char key[128];
        snprintf(key, sizeof key, "%d/%.17g/%.17g/%d/%.17g/%.17g", method, ftol, step_size, max_iter, ftol_stay, theta);
        auto it = c->qgraphs.find(key);
        if (it == c->qgraphs.end()) {
            if (c->qgraphs.size() >= 8) {
                for (auto &g : c->qgraphs) cudaGraphExecDestroy(g.second);
                c->qgraphs.clear();
            }
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
            for (int k = 0; k < chunk; ++k) launch_qiter(Q, max_iter, c->s);
            CK(cudaStreamEndCapture(c->s, &g));
            cudaGraphExec_t ge;
            CK(cudaGraphInstantiate(&ge, g, 0));
            cudaGraphDestroy(g);
            it = c->qgraphs.emplace(key, ge).first;
        }
        qg = it->second;
    }
    for (int done_iters = 0; done_iters <= max_iter;) {
        if (qg) CK(cudaGraphLaunch(qg, c->s));
        else
            for (int k = 0; k < chunk; ++k) launch_qiter(Q, max_iter, c->s);
        c->launches += 8LL * chunk;
        done_iters += chunk;
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(st.data(), c->D.st, R * sizeof(RepState), cudaMemcpyDeviceToHost, c->s));
        c->d2h += (long long)(R * sizeof(RepState));
        CK(cudaStreamSynchronize(c->s));
        bool all = true;
        for (int r = 0; r < R; ++r) all &= st[r].q_done != 0;
        if (all) break;
    }
    launch_qdisp(Q, c->s);
    c->launches += 1;
    std::vector<unsigned long long> qd(R);
    CK(cudaMemcpyAsync(qd.data(), c->D.qdisp, R * 8, cudaMemcpyDeviceToHost, c->s));
    c->d2h += 8LL * R;
    CK(cudaStreamSynchronize(c->s));
    std::vector<int> ad(R);
    bool any = false;
    for (int r = 0; r < R; ++r) {
        double m;
        memcpy(&m, &qd[r], 8);
        c->qdisp[r] = std::sqrt(m);
        c->qflag[r] = std::sqrt(m) > theta;
        // st[] holds the state after the last chunk: q_fmax is that of the
        // final positions (the iteration that found fmax < ftol moved nothing)
        c->qconv[r] = st[r].q_fmax < ftol ? 1 : (st[r].q_stay ? 2 : 0);
        if (h_flags) h_flags[r] = c->qflag[r];
        // an unconverged quench is no basin minimum: it never becomes r_O
        ad[r] = c->qconv[r] == 1 && (adopt == 2 || (adopt == 1 && c->qflag[r]));
        any |= ad[r] != 0;
    }
    if (any) {
        int *d_ad = at<int>(c->ws, c->P.o_adopt);
        CK(cudaMemcpyAsync(d_ad, ad.data(), R * 4, cudaMemcpyHostToDevice, c->s));
        c->h2d += 4LL * R;
        launch_adopt(Q, c->D, d_ad, c->s);
        c->launches += 1;
    }
    if (refresh_md(c, true) != HD_OK) return c->status;
    return check_device(c);
}

hd_status hd_read(hd_ctx *c, int field, int replica, void *h_dst, size_t bytes) {
    if (!c) return HD_ERR_ARG;
    if (!h_dst) return fail(c, HD_ERR_ARG, "NULL destination");
    const Plan &P = c->P;
    if (field == HD_FIELD_OBS && replica == -1) {
        if (bytes != (size_t)P.nrep * HD_OBS_LEN * 8) return fail(c, HD_ERR_ARG, "OBS: %zu bytes expected", (size_t)P.nrep * HD_OBS_LEN * 8);
        for (int r = 0; r < P.nrep; ++r) {
            hd_status s = hd_read(c, field, r, (char *)h_dst + (size_t)r * HD_OBS_LEN * 8, HD_OBS_LEN * 8);
            if (s != HD_OK) return s;
        }
        return HD_OK;
    }
    if (replica < 0 || replica >= P.nrep) return fail(c, HD_ERR_ARG, "replica %d out of range", replica);
    if (c->status == HD_OK) {
        if (field == HD_FIELD_OBS) {
            launch_obs(c->D, c->s);
            c->launches += 1;
        }
        check_device(c);
    }
    const RepDev &R = P.rep[replica];
    const size_t n = R.n, a0 = R.atom0;
    auto need = [&](size_t b) { return bytes == b; };
    auto vec3 = [&](const void *dptr, bool fp64, int comp_w) -> hd_status {
        // comp_w < 0: xyz into [n][3]; comp_w = 3: the w component into [n]
        const size_t es = fp64 ? sizeof(dbl4) : sizeof(float4);
        std::vector<char> buf(n * es);
        CK(cudaMemcpy(buf.data(), (const char *)dptr + a0 * es, n * es, cudaMemcpyDeviceToHost));
        c->d2h += (long long)(n * es);
        double *o = (double *)h_dst;
        for (size_t sl = 0; sl < n; ++sl) {
            const size_t i = (size_t)P.slot_orig[a0 + sl], si = sl;
            double q[4];
            if (fp64) {
                const dbl4 v = reinterpret_cast<const dbl4 *>(buf.data())[si];
                q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
            } else {
                const float4 v = reinterpret_cast<const float4 *>(buf.data())[si];
                q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
            }
            if (comp_w == 3) o[i] = q[3];
            else for (int a = 0; a < 3; ++a) o[3 * i + a] = q[a];
        }
        return HD_OK;
    };
    const bool f64 = P.prec == HD_FP64;
    switch (field) {
    case HD_FIELD_POS:
        if (!need(n * 24)) break;
        return vec3(c->D.x, true, -1);
    case HD_FIELD_REF:
        if (!need(n * 24)) break;
        return vec3(c->D.xo, true, -1);
    case HD_FIELD_QPOS:
        if (!need(n * 24)) break;
        return vec3(c->Q.x, true, -1);
    case HD_FIELD_VEL:
        if (!need(n * 24)) break;
        return vec3(c->ws + P.o_v, true, -1);
    case HD_FIELD_FORCE:
        if (!need(n * 24)) break;
        return vec3(c->ws + P.o_f, f64, -1);
    case HD_FIELD_ENERGY:
        if (!need(n * 8)) break;
        return vec3(c->ws + P.o_f, f64, 3);
    case HD_FIELD_HDR:
        if (!need(n * 24)) break;
        return vec3(c->ws + P.o_h, f64, -1);
    case HD_FIELD_NBR_COUNT:
    case HD_FIELD_CELL: {
        if (!need(n * 4)) break;
        std::vector<int> tmp(n);
        CK(cudaMemcpy(tmp.data(), (field == HD_FIELD_CELL ? c->D.cellid : c->D.nnb) + a0, n * 4,
                      cudaMemcpyDeviceToHost));
        c->d2h += 4LL * n;
        int *o = (int *)h_dst;
        for (size_t sl = 0; sl < n; ++sl) o[P.slot_orig[a0 + sl]] = tmp[sl];
        return HD_OK;
    }
    case HD_FIELD_NBR: {
        // rows in input numbering, ascending in j
        if (!need(n * P.maxnb * 4)) break;
        std::vector<int> cnt(n), slab(n * P.maxnb);
        CK(cudaMemcpy(cnt.data(), c->D.nnb + a0, n * 4, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy2D(slab.data(), n * 4, c->D.nbr + a0, (size_t)P.natom * 4, n * 4, P.maxnb, cudaMemcpyDeviceToHost));
        c->d2h += 4LL * n * (1 + P.maxnb);
        int *o = (int *)h_dst;
        std::vector<int> row;
        for (size_t sl = 0; sl < n; ++sl) {
            const int i = P.slot_orig[a0 + sl];
            row.clear();
            for (int k = 0; k < cnt[sl] && k < P.maxnb; ++k) row.push_back(P.slot_orig[slab[(size_t)k * n + sl]]);
            std::sort(row.begin(), row.end());
            for (int k = 0; k < P.maxnb; ++k) o[(size_t)i * P.maxnb + k] = k < (int)row.size() ? row[k] : -1;
        }
        return HD_OK;
    }
    case HD_FIELD_OBS: {
        if (!need(HD_OBS_LEN * 8)) break;
        RepState S;
        Scal C;
        CK(cudaMemcpy(&S, c->D.st + replica, sizeof S, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(&C, c->D.sc + replica, sizeof C, cudaMemcpyDeviceToHost));
        c->d2h += (long long)(sizeof S + sizeof C);
        double *o = (double *)h_dst;
        memset(o, 0, HD_OBS_LEN * 8);
        o[HD_OBS_STEP] = (double)S.step;
        o[HD_OBS_TMD] = S.t_md;
        o[HD_OBS_TH] = S.t_h;
        o[HD_OBS_V] = C.V;
        o[HD_OBS_K] = S.K;
        o[HD_OBS_DV] = C.dV;
        o[HD_OBS_SIGMA] = C.sigma;
        o[HD_OBS_D] = C.d;
        o[HD_OBS_FR] = C.FR;
        o[HD_OBS_XT] = C.xT[0];
        o[HD_OBS_YT] = C.xT[1];
        o[HD_OBS_ZT] = C.xT[2];
        o[HD_OBS_NREBUILD] = (double)S.n_rebuild;
        o[HD_OBS_BOOST] = std::exp(C.dV / R.kT);
        o[HD_OBS_QITER] = S.q_iter;
        o[HD_OBS_QFMAX] = S.q_fmax;
        o[HD_OBS_G] = C.G;
        for (int a = 0; a < 3; ++a) {
            o[HD_OBS_FBODY + a] = C.fbody[a];
            o[HD_OBS_VBODY + a] = S.vbody_full[a];
        }
        o[HD_OBS_QDISP] = c->qdisp.empty() ? 0.0 : c->qdisp[replica];
        for (int a = 0; a < 3; ++a) o[HD_OBS_NDV_ZERO + a] = (double)S.n_dv[a];
        o[HD_OBS_QCONV] = c->qconv.empty() ? 0.0 : (double)c->qconv[replica];
        o[HD_OBS_XS] = C.xS;
        if (R.eig_on) {
            o[HD_OBS_EIG] = S.eig;
            o[HD_OBS_EIG_ITERS] = (double)S.eig_iters;
        }
        if (R.nhc_len > 0) {
            double e = 0.0;
            for (int j = 0; j < R.nhc_len; ++j)
                e += 0.5 * R.nhc_Q[j] * S.nhc_v[j] * S.nhc_v[j] + (j == 0 ? R.nhc_nf : 1.0) * R.kT * S.nhc_xi[j];
            o[HD_OBS_NHC_E] = e;
        }
        return HD_OK;
    }
    default:
        return fail(c, HD_ERR_ARG, "unknown field %d", field);
    }
    return fail(c, HD_ERR_ARG, "field %d of replica %d: wrong byte count %zu", field, replica, bytes);
}

hd_status hd_info(const hd_ctx *c, int64_t out[12]) {
    if (!c || !out) return HD_ERR_ARG;
    out[8] = c->h2d;
    out[9] = c->d2h;
    out[10] = (int64_t)c->P.bytes;
    out[11] = 0;
    out[0] = c->P.nrep;
    out[1] = c->P.natom;
    out[2] = c->P.maxnb;
    out[3] = c->P.cell_cap;
    out[4] = c->P.ntile;
    out[5] = c->driver;
    out[6] = c->persistent_ctas;
    out[7] = c->launches;
    return HD_OK;
}

hd_status hd_sync(hd_ctx *c) {
    if (!c) return HD_ERR_ARG;
    if (c->status != HD_OK) return HD_ERR_STATE;
    return check_device(c);
}

hd_status hd_timing(hd_ctx *c, int enable, double out[16]) {
    if (!c) return HD_ERR_ARG;
    if (enable < -1 || enable > 2) return fail(c, HD_ERR_ARG, "timing mode %d", enable);
    harvest_all(c);
    if (enable == 2) {
        for (int k = 0; k < T_NCAT; ++k) { c->tsum[k] = 0.0; c->tcnt[k] = 0; }
    } else if (enable >= 0) {
        c->timing = enable;
    }
    if (out)
        for (int k = 0; k < T_NCAT; ++k) {
            out[2 * k] = c->tsum[k];
            out[2 * k + 1] = (double)c->tcnt[k];
        }
    return HD_OK;
}

void hd_destroy(hd_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->s);
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
    for (auto &g : c->qgraphs) cudaGraphExecDestroy(g.second);
    for (auto &sp : c->pending) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
    for (auto &kv : c->graph_spans)
        for (auto &sp : kv.second) { cudaEventDestroy(sp.a); cudaEventDestroy(sp.b); }
    for (auto e : c->free_events) cudaEventDestroy(e);
    delete c;
}

const char *hd_last_error(const hd_ctx *c) { return c ? c->err.c_str() : "NULL context"; }

}  // extern "C"
