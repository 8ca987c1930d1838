// hd_kernels.cu -- per-phase kernels of libhdslide (sm_103a).
//
// One step of the batched path, per replica (Kim & Falk, Sec. 2.2-2.3):
//   [k_cell_clear, k_bin, k_nlist]  Verlet list rebuild, only for replicas
//                                   whose rebuild flag is set
//   k_pair{64,32}                   LJ force + energy (Eq. 9) and H.(r - r_O)
//                                   in one sweep of the list; per-tile sums
//   k_scalar                        per replica: d (Eq. 7), sigma (Eq. 5),
//                                   DeltaV_1 (Eq. 14), rigid-body force, clocks
//   k_update{64,32}                 bias force + BAOAB kicks/drifts/noise
// The quench (steepest descent / FIRE) reuses the list and pair kernels on a
// copy of the positions (k_pair<true>, k_qscalar, k_qupdate).
//
// Tiles: a CTA handles one tile = up to blockDim atoms of ONE replica, so any
// per-replica quantity is a fixed-order sum of per-tile sums (deterministic).
#include "hd_internal.cuh"
#include "hd_launch.h"

namespace hd {

// ---------------------------------------------------------------- reductions
// Sums NV per-thread values over the CTA in a fixed order and writes them to
// out[0..NV).  Slot `maxslot` (if >= 0) is reduced with max instead of +.
template <int NV>
__device__ __forceinline__ void cta_reduce(double (&v)[NV], double *out, int maxslot) {
    __shared__ double sm[32][NV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = (q == maxslot) ? warp_max(v[q]) : warp_sum(v[q]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sm[w][q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        const int q = threadIdx.x;
        double a = sm[0][q];
        for (int k = 1; k < nw; ++k) a = (q == maxslot) ? fmax(a, sm[k][q]) : a + sm[k][q];
        out[q] = a;
    }
    __syncthreads();
}

// Tile sums of the split form: slots PART_D2, PART_G, PART_V are per-atom
// FP64 values (products of FP32 factors, exact in FP64) summed in FP64, since
// sigma = G / d (Eq. 5) feeds the bias; slots [3, nf) are FP32 per-atom values
// summed in FP32 within each warp; xr (rigid positions, FP64) go to slots
// PART_XRIG..+2 when some lane holds a rigid atom.  Warp results are added in
// FP64 in warp order.  Slots never written by a warp count as zero.
__device__ __forceinline__ void tile_reduce_mixed(double (&d3)[3], float (&v)[12], int nf, double (&xr)[3],
                                                  bool anyrig, double *out) {
    __shared__ double sm[32][NPART];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double wsum[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) wsum[q] = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) wsum[q] = warp_sum(d3[q]);
#pragma unroll
    for (int q = 3; q < 12; ++q)
        if (q < nf) wsum[q] = (double)warp_sum(v[q]);
    if (anyrig)
#pragma unroll
        for (int a = 0; a < 3; ++a) wsum[PART_XRIG + a] = warp_sum(xr[a]);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NPART; ++q) sm[w][q] = wsum[q];
    __syncthreads();
    if (threadIdx.x < NPART) {
        const int q = threadIdx.x;
        double a = sm[0][q];
        for (int k = 1; k < nw; ++k) a += sm[k][q];
        out[q] = a;
    }
    __syncthreads();
}

// Quench tile sums: slot QP_FMAX2 is a max; FIRE's power F.v, v.v and F.F
// (pvf, FP64 per-atom products of FP32 factors) are summed in FP64, since the
// sign of the power near convergence is a small difference of large sums; the
// rigid forces are FP32 sums within warps.
__device__ __forceinline__ void tile_reduce_quench(float (&v)[12], double (&pvf)[3], double (&xr)[3], bool anyrig,
                                                   double *out) {
    __shared__ double sm[32][NPART];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double wsum[NPART];
#pragma unroll
    for (int q = 0; q < NPART; ++q) wsum[q] = 0.0;
    float m = v[QP_FMAX2];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    wsum[QP_FMAX2] = (double)m;
    wsum[QP_P] = warp_sum(pvf[0]);
    wsum[QP_VV] = warp_sum(pvf[1]);
    wsum[QP_FF] = warp_sum(pvf[2]);
    if (anyrig) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            wsum[QP_FRIG + a] = (double)warp_sum(v[QP_FRIG + a]);
            wsum[QP_XRIG + a] = warp_sum(xr[a]);
        }
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NPART; ++q) sm[w][q] = wsum[q];
    __syncthreads();
    if (threadIdx.x < NPART) {
        const int q = threadIdx.x;
        double a = sm[0][q];
        for (int k = 1; k < nw; ++k) a = (q == QP_FMAX2) ? fmax(a, sm[k][q]) : a + sm[k][q];
        out[q] = a;
    }
    __syncthreads();
}

// ---------------------------------------------------------------- init
// Fixed-point image, r - r_O, and (where asked) Maxwell-Boltzmann velocities
// from Philox calls 2 and 3 at the current step.
__global__ void k_init(Dev D, const int *draw_vel) {
    const int t = blockIdx.x, r = D.tile_rep[t];
    if (threadIdx.x >= D.tile_n[t]) return;
    const int i = D.tile_start[t] + threadIdx.x;
    const RepDev &R = D.rep[r];
    dbl4 x = D.x[i], xo = D.xo[i];
    int4 p = D.rec[i].p;  // w (type | role << 8) preset by the host
    p = fix_pos(R, x, p.w);
    D.rec[i].p = p;
    D.pfixb[i] = p;
    const int role = (p.w >> 8) & 0xff;
    if (D.prec == HD_FP64) {
        D.dr64[i] = make_dbl4(x.x - xo.x, x.y - xo.y, x.z - xo.z, 0.0);
    } else {
        const int4 po = fix_pos(R, xo, 0);
        D.po[i] = po;
        D.rec[i].d = img_diff(p, po);
    }
    if (draw_vel[r]) {
        double v0 = 0, v1 = 0, v2 = 0;
        if (role == ROLE_MOBILE) {
            const double sd = sqrt(R.kT);
            double z0, z1, z2, z3;
            normals64(philox_draw(D, D.st[r].step, D.orig[i], R.rep_id, 2), z0, z1);
            v0 = sd * z0;
            v1 = sd * z1;
            if (R.dim == 3) {
                normals64(philox_draw(D, D.st[r].step, D.orig[i], R.rep_id, 3), z2, z3);
                v2 = sd * z2;
            }
        }
        D.v64[i] = make_dbl4(v0, v1, v2, 0.0);
    }
}

// ---------------------------------------------------------------- neighbour list
// A list rebuild touches only the replicas whose flag is set.  k_rebuild_plan
// (one warp) compacts them: rb_list[k] is the k-th such replica in ascending
// order, rb_off[k] / rb_aoff[k] its first cell / atom in the compacted range,
// rb_meta = {count, cells, atoms}.  The other rebuild kernels run fixed grids
// that stride over that compacted range, so a step without rebuilds costs a
// few near-empty launches.
__global__ void k_rebuild_plan(Dev D) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x;
    int nrb = 0, coff = 0, aoff = 0;
    for (int base = 0; base < D.nrep; base += 32) {
        const int r = base + lane;
        const bool f = r < D.nrep && D.rebuild[r] != 0;
        const int nc = f ? D.rep[r].ncell : 0, na = f ? D.rep[r].n : 0;
        int c = nc, a = na;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int tc = __shfl_up_sync(full, c, o), ta = __shfl_up_sync(full, a, o);
            if (lane >= o) {
                c += tc;
                a += ta;
            }
        }
        const unsigned m = __ballot_sync(full, f);
        if (f) {
            const int k = nrb + __popc(m & ((1u << lane) - 1u));
            D.rb_list[k] = r;
            D.rb_off[k] = coff + c - nc;
            D.rb_aoff[k] = aoff + a - na;
        }
        nrb += __popc(m);
        coff += __shfl_sync(full, c, 31);
        aoff += __shfl_sync(full, a, 31);
    }
    if (lane == 0) {
        D.rb_off[nrb] = coff;
        D.rb_aoff[nrb] = aoff;
        D.rb_meta[0] = nrb;
        D.rb_meta[1] = coff;
        D.rb_meta[2] = aoff;
    }
}

// Entry k of the compacted replicas that holds compacted index idx.
__device__ __forceinline__ int rb_find(const int *off, int n, int idx) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= idx) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_cell_clear(Dev D) {
    const int n = D.rb_meta[0], total = D.rb_meta[1];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int k = rb_find(D.rb_off, n, idx);
        D.cell_cnt[D.rep[D.rb_list[k]].cell0 + idx - D.rb_off[k]] = 0;
    }
}

__device__ __forceinline__ void dev_bin_atom(const Dev &D, int r, int i) {
    const RepDev &R = D.rep[r];
    const int4 p = D.rec[i].p;
    const dbl4 x = D.x[i];
    const int cx = cell_of(R, 0, x.x), cy = cell_of(R, 1, x.y), cz = cell_of(R, 2, x.z);
    D.cellid[i] = cx | (cy << 10) | (cz << 20);
    const int c = R.cell0 + (cz * R.nc[1] + cy) * R.nc[0] + cx;
    const int slot = atomicAdd(&D.cell_cnt[c], 1);
    if (slot < D.cell_cap) D.cell_atoms[(size_t)c * D.cell_cap + slot] = i;
    else set_err(D, HD_ERR_OVERFLOW, i, r);
    D.pfixb[i] = p;
}
// tile form, for the persistent driver (which rebuilds one replica at a time)
__device__ __forceinline__ void dev_bin(const Dev &D, int t) {
    const int r = D.tile_rep[t];
    if (!D.rebuild[r] || threadIdx.x >= D.tile_n[t]) return;
    dev_bin_atom(D, r, D.tile_start[t] + threadIdx.x);
}
__global__ void k_bin(Dev D) {
    const int n = D.rb_meta[0], total = D.rb_meta[2];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int k = rb_find(D.rb_aoff, n, idx);
        const int r = D.rb_list[k];
        dev_bin_atom(D, r, D.rep[r].atom0 + idx - D.rb_aoff[k]);
    }
}


// Each cell's atom list in ascending slot order: one warp per cell copies the
// list to shared memory and writes every entry at its rank (slot indices are
// distinct).  With atoms stored cell-major, walking the neighbour cells in
// ascending cell order then yields candidates in (almost) ascending j.
__device__ __forceinline__ void dev_cellsort_warp(const Dev &D, const RepDev &R, int c, int *buf) {
    const int lane = threadIdx.x & 31;
    int *a = D.cell_atoms + (size_t)(R.cell0 + c) * D.cell_cap;
    const int m = min(D.cell_cnt[R.cell0 + c], D.cell_cap);
    for (int k = lane; k < m; k += 32) buf[k] = a[k];
    __syncwarp();
    for (int k = lane; k < m; k += 32) {
        const int v = buf[k];
        int rank = 0;
        for (int q = 0; q < m; ++q) rank += buf[q] < v;
        a[rank] = v;
    }
    __syncwarp();
}
__global__ void __launch_bounds__(128) k_cellsort(Dev D) {
    extern __shared__ int cs_buf[];
    const int w = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const int n = D.rb_meta[0], total = D.rb_meta[1];
    for (int idx = blockIdx.x * nwb + w; idx < total; idx += gridDim.x * nwb) {
        const int k = rb_find(D.rb_off, n, idx);
        dev_cellsort_warp(D, D.rep[D.rb_list[k]], idx - D.rb_off[k], cs_buf + w * D.cell_cap);
    }
}

// Row i = every j != i whose FP64 minimum-image squared distance is below
// (rc + skin)^2.  One CTA builds the rows of one cell's atoms.  It first
// stages the candidates of the cell's stencil (the 27, or 9 in 2-D,
// surrounding cells in ascending cell order, each cell's atoms ascending) in
// shared memory: index and fixed-point position.  Then one warp per atom of
// the cell walks the staged candidates 32 at a time.  An FP32 test on the
// exact integer differences decides all but a thin band around the radius,
// where the oracle's FP64 test is repeated operation for operation.  Each
// accepted j gets a class, kept in shared memory:
//   A (first shell) FP32 r^2 < rA^2, the pairs that can come within the
//                   range where the pair sweep takes the exact r^2;
//   B               the rest of the pairs within rc at build time;
//   C (skin shell)  the rest of the row.
// The row is then written as A | B | C, each block in candidate order, so the
// lanes of the pair sweep leave the first shell, and later the cutoff, at
// nearly the same k.  The row order is a deterministic function of the cell
// lists (sorted by k_cellsort); reads return each row ascending in j.
// ballot masks per warp of the list build: three per 32 staged candidates
__host__ __device__ inline int nl_mask_words(const Dev &D) { return 3 * ((27 * D.cell_cap + 31) / 32); }
// Row-build CTA: 8 warps share one staged stencil (the cell's atoms split among them).
constexpr int NL_THREADS = 256;

struct NlSmem {
    int nst, tot, kc;
    int cell[27], off[28];
};

__device__ __forceinline__ void dev_nlist_cell(const Dev &D, int r, int c, NlSmem &M, int4 *sp,
                                               unsigned *smask) {
    const RepDev &R = D.rep[r];
    const int cell0 = R.cell0 + c;
    const int m = min(D.cell_cnt[cell0], D.cell_cap);
    if (m == 0) return;  // uniform: every thread reads the same count
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (w == 0) {
        // lane k < 27: stencil cell (k % 3, k / 3 % 3, k / 9) of the per-axis
        // lists, each list ascending (a periodic wrap puts nc-1 after 0 and 1)
        const int ci[3] = {c % R.nc[0], (c / R.nc[0]) % R.nc[1], c / (R.nc[0] * R.nc[1])};
        int cs[3], ncs[3];
        const int pick[3] = {lane % 3, (lane / 3) % 3, lane / 9};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int nc = R.nc[a], q = pick[a];
            int list[3] = {0, 0, 0}, n = 0;
            if (nc == 1) {
                list[n++] = 0;
            } else {
                const int c0 = ci[a] - 1, c2 = ci[a] + 1;
                if (R.periodic[a]) {
                    if (c0 < 0) { list[0] = 0; list[1] = 1; list[2] = nc - 1; }
                    else if (c2 >= nc) { list[0] = 0; list[1] = nc - 2; list[2] = nc - 1; }
                    else { list[0] = c0; list[1] = ci[a]; list[2] = c2; }
                    n = 3;
                } else {
                    if (c0 >= 0) list[n++] = c0;
                    list[n++] = ci[a];
                    if (c2 < nc) list[n++] = c2;
                }
            }
            ncs[a] = n;
            cs[a] = q < n ? list[q] : 0;
        }
        const bool valid = lane < 27 && pick[0] < ncs[0] && pick[1] < ncs[1] && pick[2] < ncs[2];
        const int nst = ncs[0] * ncs[1] * ncs[2];
        const int k = valid ? (pick[2] * ncs[1] + pick[1]) * ncs[0] + pick[0] : 0;
        const int cc = R.cell0 + (cs[2] * R.nc[1] + cs[1]) * R.nc[0] + cs[0];
        if (valid) {
            M.cell[k] = cc;
            M.off[k] = min(D.cell_cnt[cc], D.cell_cap);   // the count, until the scan below
            if (cc == cell0) M.kc = k;
        }
        __syncwarp();
        // exclusive scan of the counts in stencil order
        const int cnt = lane < nst ? M.off[lane] : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncwarp();
        if (lane < nst) M.off[lane] = incl - cnt;
        if (lane == nst - 1) {
            M.off[nst] = incl;
            M.tot = incl;
            M.nst = nst;
        }
    }
    __syncthreads();
    // stage the stencil: every thread takes candidates idx, idx + blockDim, ...,
    // four at a time so that their loads are in flight together
    {
        const int tot = M.tot, nst = M.nst;
        for (int base = threadIdx.x; base < tot; base += 4 * blockDim.x) {
            int jj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * blockDim.x;
                jj[u] = -1;
                if (idx < tot) {
                    int lo = 0, hi = nst - 1;          // last stencil cell with off <= idx
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (M.off[mid] <= idx) lo = mid;
                        else hi = mid - 1;
                    }
                    jj[u] = D.cell_atoms[(size_t)M.cell[lo] * D.cell_cap + (idx - M.off[lo])];
                }
            }
            int4 pp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) pp[u] = jj[u] >= 0 ? D.rec[jj[u]].p : make_int4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = base + u * blockDim.x;
                if (idx < tot) sp[idx] = make_int4(pp[u].x, pp[u].y, pp[u].z, jj[u]);   // w: the candidate's slot
            }
        }
    }
    __syncthreads();
    const int tot = M.tot, cap = D.maxnb;
    const unsigned full = 0xffffffffu;
    const float lx = R.fx_lsb[0], ly = R.fx_lsb[1], lz = R.fx_lsb[2];
    const size_t stride = (size_t)D.natom;
    // per warp: three ballot masks (classes A, B, C) per 32 candidates
    unsigned *msk = smask + (size_t)w * nl_mask_words(D);
    for (int a = w; a < m; a += nw) {
        const int slot = M.off[M.kc] + a;
        const int4 pi = sp[slot];
        const int i = pi.w;
        int nA = 0, nB = 0, nC = 0;
        // pass 1: classify every candidate, count the classes
        for (int base = 0; base < tot; base += 32) {
            const int q = base + lane;
            int cl = 0;
            if (q < tot) {
                const int4 pj = sp[q];
                const int j = pj.w;
                if (j != i) {
                    const float dx = (float)(int)((unsigned)pi.x - (unsigned)pj.x) * lx;
                    const float dy = (float)(int)((unsigned)pi.y - (unsigned)pj.y) * ly;
                    const float dz = (float)(int)((unsigned)pi.z - (unsigned)pj.z) * lz;
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    bool in;
                    if (r2 < D.rl2_lo_f) in = true;
                    else if (r2 >= D.rl2_hi_f) in = false;
                    else in = exact_r2(R, D.x[i], D.x[j]) < D.rl2;
                    if (in) cl = r2 < R.rA2f ? 1 : (r2 < D.rc2_lo_f ? 2 : 3);
                }
            }
            const unsigned mA = __ballot_sync(full, cl == 1), mB = __ballot_sync(full, cl == 2),
                           mC = __ballot_sync(full, cl == 3);
            if (lane == 0) {
                msk[3 * (base >> 5)] = mA;
                msk[3 * (base >> 5) + 1] = mB;
                msk[3 * (base >> 5) + 2] = mC;
            }
            nA += __popc(mA);
            nB += __popc(mB);
            nC += __popc(mC);
        }
        __syncwarp();
        // pass 2: write the row as A | B | C, each block in candidate order
        int bA = 0, bB = nA, bC = nA + nB;
        const unsigned below = (1u << lane) - 1u, bit = 1u << lane;
        for (int base = 0; base < tot; base += 32) {
            const unsigned mA = msk[3 * (base >> 5)], mB = msk[3 * (base >> 5) + 1], mC = msk[3 * (base >> 5) + 2];
            const int cl = (mA & bit) ? 1 : ((mB & bit) ? 2 : ((mC & bit) ? 3 : 0));
            if (cl) {
                const int pos = cl == 1 ? bA + __popc(mA & below) : (cl == 2 ? bB + __popc(mB & below)
                                                                             : bC + __popc(mC & below));
                if (pos < cap) D.nbr[(size_t)pos * stride + i] = sp[base + lane].w;
            }
            bA += __popc(mA);
            bB += __popc(mB);
            bC += __popc(mC);
        }
        __syncwarp();
        if (lane == 0) {
            const int n = nA + nB + nC;
            D.nnb[i] = min(n, cap);
            if (n > cap) set_err(D, HD_ERR_OVERFLOW, i, r);
        }
    }
    __syncthreads();  // the staging buffers are reused by the next cell
}

__device__ __forceinline__ void nl_smem_carve(const Dev &D, char *base, int4 *&sp, unsigned *&smask) {
    sp = reinterpret_cast<int4 *>(base);
    smask = reinterpret_cast<unsigned *>(base + (size_t)27 * D.cell_cap * sizeof(int4));
}

__global__ void __launch_bounds__(NL_THREADS) k_nlist(Dev D) {
    extern __shared__ __align__(16) char nl_smem[];
    __shared__ NlSmem M;
    int4 *sp;
    unsigned *smask;
    nl_smem_carve(D, nl_smem, sp, smask);
    const int n = D.rb_meta[0], total = D.rb_meta[1];
    for (int idx = blockIdx.x; idx < total; idx += gridDim.x) {
        const int k = rb_find(D.rb_off, n, idx);
        dev_nlist_cell(D, D.rb_list[k], idx - D.rb_off[k], M, sp, smask);
    }
}

// ---------------------------------------------------------------- pair sweep
// F_i = sum_j -phi'(r)/r r_ij; e_i = sum_j phi(r)/2;
// (H dr)_i = sum_j [A (dr_i - dr_j) + B ((dr_i - dr_j) . r_ij) r_ij],
// A = phi'/r, B = (phi'' - phi'/r)/r^2, with s = sigma_ab/r:
//   -A = 24 eps s^6 (2 s^6 - 1)/r^2,   B = 96 eps s^6 (7 s^6 - 2)/r^4.
// Q (quench): positions of the quench copy, no H.dr, quench partial sums.
template <bool Q, bool E>
__device__ __forceinline__ void dev_pair64(const Dev &D, int t) {
    const int r = D.tile_rep[t];
    if (Q && D.st[r].q_done) return;
    const RepDev &R = D.rep[r];
    const bool act = threadIdx.x < D.tile_n[t];
    const int i = D.tile_start[t] + (act ? threadIdx.x : 0);
    const dbl4 xi = D.x[i];
    const int ti = (int)xi.w;
    const dbl4 dri = Q ? make_dbl4(0, 0, 0, 0) : D.dr64[i];
    double fx = 0, fy = 0, fz = 0, e = 0, hx = 0, hy = 0, hz = 0;
    const int nn = act ? D.nnb[i] : 0;
    const double rc2 = D.rc2;
    for (int k = 0; k < nn; ++k) {
        const int j = D.nbr[(size_t)k * D.natom + i];
        const dbl4 xj = D.x[j];
        const double dx = mi64(R, 0, xi.x - xj.x), dy = mi64(R, 1, xi.y - xj.y), dz = mi64(R, 2, xi.z - xj.z);
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < rc2) {
            const int tj = (int)xj.w;
            const double eps = R.eps[ti][tj];
            const double ir2 = 1.0 / r2;
            const double s2 = R.sig2[ti][tj] * ir2;
            const double s6 = s2 * s2 * s2;
            const double fr = 24.0 * eps * ir2 * s6 * (2.0 * s6 - 1.0);
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            if (E) e += 0.5 * (4.0 * eps * s6 * (s6 - 1.0) - R.shift[ti][tj]);
            if (!Q) {
                const dbl4 drj = D.dr64[j];
                const double ux = dri.x - drj.x, uy = dri.y - drj.y, uz = dri.z - drj.z;
                const double rdu = dx * ux + dy * uy + dz * uz;
                const double B = 96.0 * eps * ir2 * ir2 * s6 * (7.0 * s6 - 2.0);
                hx += -fr * ux + B * rdu * dx;
                hy += -fr * uy + B * rdu * dy;
                hz += -fr * uz + B * rdu * dz;
            }
        }
    }
    // harmonic bonds of Eq. 12, phi = k (r - r_b)^2 / 2 at any distance:
    // A = phi'/r = k (r - r_b)/r, B = (phi'' - A)/r^2 = k r_b / r^3
    if (R.nbond > 0 && act) {
        for (int b = D.bond_off[i]; b < D.bond_off[i + 1]; ++b) {
            const int j = D.bond_j[b];
            const dbl4 xj = D.x[j];
            const double dx = mi64(R, 0, xi.x - xj.x), dy = mi64(R, 1, xi.y - xj.y), dz = mi64(R, 2, xi.z - xj.z);
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double rr = sqrt(r2), db = rr - R.rbond;
            const double A = R.kbond * db / rr;
            fx -= A * dx;
            fy -= A * dy;
            fz -= A * dz;
            if (E) e += 0.5 * (0.5 * R.kbond * db * db);
            if (!Q) {
                const dbl4 drj = D.dr64[j];
                const double ux = dri.x - drj.x, uy = dri.y - drj.y, uz = dri.z - drj.z;
                const double rdu = dx * ux + dy * uy + dz * uz;
                const double B = (R.kbond - A) / r2;
                hx += A * ux + B * rdu * dx;
                hy += A * uy + B * rdu * dy;
                hz += A * uz + B * rdu * dz;
            }
        }
    }
    const int role = act ? ((D.rec[i].p.w >> 8) & 0xff) : -1;
    if (!Q && role == ROLE_RIGID) {
        hx += R.kr_n * dri.x;
        if (R.dim == 3) hy += R.kr_n * dri.y;
    }
    if (act) {
        D.f64[i] = make_dbl4(fx, fy, fz, e);
        if (!Q) D.h64[i] = make_dbl4(hx, hy, hz, 0.0);
    }
    const bool rig = role == ROLE_RIGID;
    if (!Q) {
        double v[NPART] = {};
        if (act) {
            v[PART_D2] = dri.x * dri.x + dri.y * dri.y + dri.z * dri.z;
            v[PART_G] = -(fx * dri.x + fy * dri.y + fz * dri.z);
            v[PART_V] = e;
        }
        if (rig) {
            v[PART_FRIG] = fx; v[PART_FRIG + 1] = fy; v[PART_FRIG + 2] = fz;
            v[PART_HRIG] = hx; v[PART_HRIG + 1] = hy; v[PART_HRIG + 2] = hz;
            v[PART_DRRIG] = dri.x; v[PART_DRRIG + 1] = dri.y; v[PART_DRRIG + 2] = dri.z;
            v[PART_XRIG] = xi.x; v[PART_XRIG + 1] = xi.y; v[PART_XRIG + 2] = xi.z;
        }
        cta_reduce<NPART>(v, D.part + (size_t)t * NPART, -1);
    } else {
        double v[QPART] = {};
        if (role == ROLE_MOBILE) {
            const dbl4 vv = D.v64[i];
            v[QP_FMAX2] = fx * fx + fy * fy + fz * fz;
            v[QP_P] = fx * vv.x + fy * vv.y + fz * vv.z;
            v[QP_VV] = vv.x * vv.x + vv.y * vv.y + vv.z * vv.z;
            v[QP_FF] = v[QP_FMAX2];
        }
        if (rig) {
            v[QP_FRIG] = fx; v[QP_FRIG + 1] = fy; v[QP_FRIG + 2] = fz;
            v[QP_XRIG] = xi.x; v[QP_XRIG + 1] = xi.y; v[QP_XRIG + 2] = xi.z;
        }
        cta_reduce<QPART>(v, D.part + (size_t)t * NPART, QP_FMAX2);
    }
}

// Split form: positions are differenced exactly in 32-bit fixed point, the
// pair arithmetic is FP32; per-tile sums are carried in FP64.  Near the LJ
// minimum the force holds the cancelling factor (2 s^6 - 1); it is evaluated
// as (1 + t)^3 - 1 = t (3 + 3t + t^2) with t = (r_0^2 - r^2) / r^2, r_0^2 =
// 2^(1/3) sigma^2, and r^2 carried as hi + lo from the exact integer sum of
// squares, so the FP32 result is accurate relative to the force itself.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// 1/x to FP32 rounding: the hardware approximation refined by one Newton
// step, y (2 - x y), so that its error carries no bias into the forces
// (an unrefined approximation shifts every pair force the same way, and the
// slope sigma of Eq. 5 sums them over the whole replica).
__device__ __forceinline__ float rcp_refined(float x) {
    const float y = rcp_approx(x);
    return fmaf(y, fmaf(-x, y, 1.f), y);
}

// Asynchronous 4-byte copies global -> shared (cp.async): each lane stages
// its own atom's list entries, so a chunk needs no barrier, only the wait.
__device__ __forceinline__ void cp_async4(int *dst, const int *src) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// List entries a lane stages ahead per chunk, double-buffered: a warp keeps
// 2 x NBC x 128 B of its column-major list rows in shared memory, the next
// chunk in flight while the current one is used.
constexpr int NBC = 16;
__host__ __device__ constexpr size_t pair_smem_bytes_for(int block) {
    return (size_t)(block / 32) * 2 * NBC * 32 * sizeof(int);
}

template <bool Q, bool E, bool X2 = false>
__device__ __forceinline__ void dev_pair32(const Dev &D, int t) {
    const int r = D.tile_rep[t];
    if (Q && D.st[r].q_done) return;
    const RepDev &R = D.rep[r];
    const bool act = threadIdx.x < D.tile_n[t];
    const int i = D.tile_start[t] + (act ? threadIdx.x : 0);
    const AtomRec ai = D.rec[i];
    const int4 pi = ai.p;
    const int ti = pi.w & 1;
    const float lx = R.fx_lsb[0], ly = R.fx_lsb[1], lz = R.fx_lsb[2];
    const int4 dfi = Q ? make_int4(0, 0, 0, 0) : ai.d;                 // r - r_O, fixed point
    const float4 dri = make_float4((float)dfi.x * lx, (float)dfi.y * ly, (float)dfi.z * lz, 0.f);
    const float e0 = R.epsf[ti][0], e1 = R.epsf[ti][1];
    // 24 eps and 96 eps as FP32 hi + lo: an eps such as 0.2 is not an FP32
    // number, and its rounding would scale every such pair force alike
    const float a0 = R.eps24f[ti][0], a1 = R.eps24f[ti][1], al0 = R.eps24l[ti][0], al1 = R.eps24l[ti][1];
    const float b0 = R.eps96f[ti][0], b1 = R.eps96f[ti][1], bl0 = R.eps96l[ti][0], bl1 = R.eps96l[ti][1];
    const float h0 = R.shiftf[ti][0], h1 = R.shiftf[ti][1];
    const float q0h = R.r0sq_hi[ti][0], q1h = R.r0sq_hi[ti][1];
    const float q0l = R.r0sq_lo[ti][0], q1l = R.r0sq_lo[ti][1];
    const bool exact = R.exact_r2 != 0;
    const float r2corr = exact ? 2.f * R.lsb_rel[0] : 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
    const int nn = act ? D.nnb[i] : 0;
    const int *nb = D.nbr + i;
    const size_t stride = (size_t)D.natom;
    // The list streams from HBM: each lane stages its row NBC entries at a
    // time through shared memory by cp.async, the next chunk in flight while
    // the current one is used; the record of the next entry is loaded while
    // the current one is used.
    extern __shared__ __align__(16) int pair_smem[];
    const int lane = threadIdx.x & 31;
    int(*sbuf)[NBC][32] = reinterpret_cast<int(*)[NBC][32]>(pair_smem) + 2 * (threadIdx.x >> 5);
    int nmax = nn;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    const int nch = (nmax + NBC - 1) / NBC;
    auto stage = [&](int c) {
        int(*b)[32] = sbuf[c & 1];
#pragma unroll
        for (int u = 0; u < NBC; ++u) {
            const int k = c * NBC + u;
            if (k < nn) cp_async4(&b[u][lane], nb + (size_t)k * stride);
        }
        cp_async_commit();
    };
    if (nch > 0) stage(0);
    // one pair's contribution.  Cancellation-free LJ form: 2 s^6 - 1 = w(tt)
    // with tt = (r_0^2 - r^2) / r^2.  Where |tt| < 1/4 (around the minimum,
    // where w is small and the FP32 r^2 would cost it its relative accuracy)
    // r^2 is taken exactly, as hi + lo, from the integer separations when the
    // replica's axes share one fixed-point unit; elsewhere the FP32 r^2 gives
    // w to a few ulps.  The list builder puts the pairs that can need the
    // exact r^2 at the head of each row, so the branch is nearly uniform.
    auto term = [&](const AtomRec &aj, int ix, int iy, int iz, float dx, float dy, float dz, float r2) {
        const int tj = aj.p.w & 1;
        const float r0h = tj ? q1h : q0h, r0l = tj ? q1l : q0l;
        // the FP32 r^2 with the rounding of the fixed-point unit undone (all
        // axes share its relative rounding when they share the unit)
        const float r2c = fmaf(r2, r2corr, r2);
        float ir2 = rcp_refined(r2c);
        float tt = ((r0h - r2c) + r0l) * ir2;
        if (exact && fabsf(tt) < 0.25f) {
            float r2h, r2l;
            r2_split(R, ix, iy, iz, r2h, r2l);
            ir2 = rcp_refined(r2h);
            tt = ((r0h - r2h) + (r0l - r2l)) * ir2;
        }
        const float u = 1.f + tt;
        const float s6 = 0.5f * u * u * u;
        const float w = tt * fmaf(tt, tt + 3.f, 3.f);          // 2 s^6 - 1
        const float pf = ir2 * s6 * w;
        const float fr = fmaf(pf, tj ? al1 : al0, pf * (tj ? a1 : a0));
        fx = fmaf(fr, dx, fx);
        fy = fmaf(fr, dy, fy);
        fz = fmaf(fr, dz, fz);
        if (E) e = fmaf(0.5f, fmaf(4.f * (tj ? e1 : e0) * s6, s6 - 1.f, -(tj ? h1 : h0)), e);
        if (!Q) {
            const float ux = (float)(int)((unsigned)dfi.x - (unsigned)aj.d.x) * lx;
            const float uy = (float)(int)((unsigned)dfi.y - (unsigned)aj.d.y) * ly;
            const float uz = (float)(int)((unsigned)dfi.z - (unsigned)aj.d.z) * lz;
            const float rdu = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
            const float pb = ir2 * ir2 * s6 * fmaf(7.f, s6, -2.f) * rdu;
            const float B = fmaf(pb, tj ? bl1 : bl0, pb * (tj ? b1 : b0));
            hx = fmaf(-fr, ux, fmaf(B, dx, hx));
            hy = fmaf(-fr, uy, fmaf(B, dy, hy));
            hz = fmaf(-fr, uz, fmaf(B, dz, hz));
        }
    };
    bool band = false;
    if (!X2) {
        for (int c = 0; c < nch; ++c) {
            if (c + 1 < nch) {
                stage(c + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            const int(*b)[32] = sbuf[c & 1];
            const int kend = min(NBC, nn - c * NBC);
            AtomRec an = kend > 0 ? D.rec[b[0][lane]] : ai;
            for (int u = 0; u < kend; ++u) {
                const AtomRec aj = an;
                if (u + 1 < kend) an = D.rec[b[u + 1][lane]];
                const int4 pj = aj.p;
                const int ix = (int)((unsigned)pi.x - (unsigned)pj.x);
                const int iy = (int)((unsigned)pi.y - (unsigned)pj.y);
                const int iz = (int)((unsigned)pi.z - (unsigned)pj.z);
                const float dx = (float)ix * lx, dy = (float)iy * ly, dz = (float)iz * lz;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                if (r2 < D.rc2_lo_f) term(aj, ix, iy, iz, dx, dy, dz, r2);
                else band |= r2 < D.rc2_hi_f;
            }
        }
    } else {
        // Two list entries per iteration in packed FP32x2 arithmetic (one
        // instruction for both halves), with the same operations per entry as
        // term(); an entry outside the cutoff contributes through a select to
        // zero.  Records of the next two entries and the indices of the two
        // after them are in flight while the current two are used.
        const float2 one2 = make_float2(1.f, 1.f), mone2 = make_float2(-1.f, -1.f), half2 = make_float2(0.5f, 0.5f);
        const float2 three2 = make_float2(3.f, 3.f), seven2 = make_float2(7.f, 7.f), mtwo2 = make_float2(-2.f, -2.f);
        const float2 corr2 = make_float2(r2corr, r2corr);
        float2 Fx = make_float2(0.f, 0.f), Fy = Fx, Fz = Fx, Hx = Fx, Hy = Fx, Hz = Fx, Ee = Fx;
        for (int c = 0; c < nch; ++c) {
          if (c + 1 < nch) {
              stage(c + 1);
              cp_async_wait<1>();
          } else {
              cp_async_wait<0>();
          }
          const int(*b)[32] = sbuf[c & 1];
          const int kend = min(NBC, nn - c * NBC);
          AtomRec na = kend > 0 ? D.rec[b[0][lane]] : ai, nbr2 = kend > 1 ? D.rec[b[1][lane]] : ai;
          for (int u = 0; u < kend; u += 2) {
            const AtomRec A = na, B = nbr2;
            const bool vb = u + 1 < kend;
            if (u + 2 < kend) na = D.rec[b[u + 2][lane]];
            if (u + 3 < kend) nbr2 = D.rec[b[u + 3][lane]];
            const int ixa = (int)((unsigned)pi.x - (unsigned)A.p.x), ixb = (int)((unsigned)pi.x - (unsigned)B.p.x);
            const int iya = (int)((unsigned)pi.y - (unsigned)A.p.y), iyb = (int)((unsigned)pi.y - (unsigned)B.p.y);
            const int iza = (int)((unsigned)pi.z - (unsigned)A.p.z), izb = (int)((unsigned)pi.z - (unsigned)B.p.z);
            const float2 dx = __fmul2_rn(make_float2((float)ixa, (float)ixb), make_float2(lx, lx));
            const float2 dy = __fmul2_rn(make_float2((float)iya, (float)iyb), make_float2(ly, ly));
            const float2 dz = __fmul2_rn(make_float2((float)iza, (float)izb), make_float2(lz, lz));
            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
            const bool ina = r2.x < D.rc2_lo_f, inb = vb && r2.y < D.rc2_lo_f;
            band |= (!ina && r2.x < D.rc2_hi_f) || (vb && !inb && r2.y < D.rc2_hi_f);
            if (!(ina || inb)) continue;
            const int ta = A.p.w & 1, tb = B.p.w & 1;
            const float2 r0h = make_float2(ta ? q1h : q0h, tb ? q1h : q0h);
            const float2 r0l = make_float2(ta ? q1l : q0l, tb ? q1l : q0l);
            const float2 r2c = __ffma2_rn(r2, corr2, r2);
            float2 ir2 = make_float2(rcp_approx(r2c.x), rcp_approx(r2c.y));
            ir2 = __ffma2_rn(ir2, __ffma2_rn(r2c, __fmul2_rn(ir2, mone2), one2), ir2);
            float2 tt = __fmul2_rn(__fadd2_rn(__ffma2_rn(r2c, mone2, r0h), r0l), ir2);
            if (exact && ina && fabsf(tt.x) < 0.25f) {
                float h, l;
                r2_split(R, ixa, iya, iza, h, l);
                ir2.x = rcp_refined(h);
                tt.x = ((r0h.x - h) + (r0l.x - l)) * ir2.x;
            }
            if (exact && inb && fabsf(tt.y) < 0.25f) {
                float h, l;
                r2_split(R, ixb, iyb, izb, h, l);
                ir2.y = rcp_refined(h);
                tt.y = ((r0h.y - h) + (r0l.y - l)) * ir2.y;
            }
            const float2 u1 = __fadd2_rn(one2, tt);
            const float2 s6 = __fmul2_rn(__fmul2_rn(half2, u1), __fmul2_rn(u1, u1));
            const float2 w = __fmul2_rn(tt, __ffma2_rn(tt, __fadd2_rn(tt, three2), three2));      // 2 s^6 - 1
            const float2 pf = __fmul2_rn(ir2, __fmul2_rn(s6, w));
            float2 fr = __ffma2_rn(pf, make_float2(ta ? al1 : al0, tb ? al1 : al0),
                                   __fmul2_rn(pf, make_float2(ta ? a1 : a0, tb ? a1 : a0)));
            fr.x = ina ? fr.x : 0.f;
            fr.y = inb ? fr.y : 0.f;
            Fx = __ffma2_rn(fr, dx, Fx);
            Fy = __ffma2_rn(fr, dy, Fy);
            Fz = __ffma2_rn(fr, dz, Fz);
            if (E) {
                float2 ee = __ffma2_rn(__fmul2_rn(make_float2(4.f * (ta ? e1 : e0), 4.f * (tb ? e1 : e0)), s6),
                                       __fadd2_rn(s6, mone2), make_float2(-(ta ? h1 : h0), -(tb ? h1 : h0)));
                ee.x = ina ? ee.x : 0.f;
                ee.y = inb ? ee.y : 0.f;
                Ee = __ffma2_rn(half2, ee, Ee);
            }
            if (!Q) {
                const float2 ux = __fmul2_rn(make_float2((float)(int)((unsigned)dfi.x - (unsigned)A.d.x),
                                                         (float)(int)((unsigned)dfi.x - (unsigned)B.d.x)),
                                             make_float2(lx, lx));
                const float2 uy = __fmul2_rn(make_float2((float)(int)((unsigned)dfi.y - (unsigned)A.d.y),
                                                         (float)(int)((unsigned)dfi.y - (unsigned)B.d.y)),
                                             make_float2(ly, ly));
                const float2 uz = __fmul2_rn(make_float2((float)(int)((unsigned)dfi.z - (unsigned)A.d.z),
                                                         (float)(int)((unsigned)dfi.z - (unsigned)B.d.z)),
                                             make_float2(lz, lz));
                const float2 rdu = __ffma2_rn(dx, ux, __ffma2_rn(dy, uy, __fmul2_rn(dz, uz)));
                const float2 pb = __fmul2_rn(__fmul2_rn(ir2, ir2),
                                             __fmul2_rn(__fmul2_rn(s6, __ffma2_rn(seven2, s6, mtwo2)), rdu));
                float2 Bc = __ffma2_rn(pb, make_float2(ta ? bl1 : bl0, tb ? bl1 : bl0),
                                       __fmul2_rn(pb, make_float2(ta ? b1 : b0, tb ? b1 : b0)));
                Bc.x = ina ? Bc.x : 0.f;
                Bc.y = inb ? Bc.y : 0.f;
                const float2 nfr = __fmul2_rn(fr, mone2);
                Hx = __ffma2_rn(nfr, ux, __ffma2_rn(Bc, dx, Hx));
                Hy = __ffma2_rn(nfr, uy, __ffma2_rn(Bc, dy, Hy));
                Hz = __ffma2_rn(nfr, uz, __ffma2_rn(Bc, dz, Hz));
            }
          }
        }
        fx += Fx.x + Fx.y;
        fy += Fy.x + Fy.y;
        fz += Fz.x + Fz.y;
        if (E) e += Ee.x + Ee.y;
        if (!Q) {
            hx += Hx.x + Hx.y;
            hy += Hy.x + Hy.y;
            hz += Hz.x + Hz.y;
        }
    }
    // Rare: pairs in a thin band around rc are cut by the oracle's FP64 test
    // (same operations), so no pair is cut at a different step than in FP64.
    if (band) {
        const dbl4 xi64 = D.x[i];
        for (int k = 0; k < nn; ++k) {
            const int j = nb[(size_t)k * stride];
            const AtomRec aj = D.rec[j];
            const int ix = (int)((unsigned)pi.x - (unsigned)aj.p.x);
            const int iy = (int)((unsigned)pi.y - (unsigned)aj.p.y);
            const int iz = (int)((unsigned)pi.z - (unsigned)aj.p.z);
            const float dx = (float)ix * lx, dy = (float)iy * ly, dz = (float)iz * lz;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (r2 >= D.rc2_lo_f && r2 < D.rc2_hi_f && exact_r2(R, xi64, D.x[j]) < D.rc2)
                term(aj, ix, iy, iz, dx, dy, dz, r2);
        }
    }
    // harmonic bonds of Eq. 12 at any distance, from the exact r^2 where the
    // axes share one unit (r - r_b is a small difference of two numbers near
    // r_b); A = k (r - r_b)/r, B = k r_b / r^3
    if (R.nbond > 0 && act) {
        for (int b = D.bond_off[i]; b < D.bond_off[i + 1]; ++b) {
            const int j = D.bond_j[b];
            const AtomRec aj = D.rec[j];
            const int ix = (int)((unsigned)pi.x - (unsigned)aj.p.x);
            const int iy = (int)((unsigned)pi.y - (unsigned)aj.p.y);
            const int iz = (int)((unsigned)pi.z - (unsigned)aj.p.z);
            const float dx = (float)ix * lx, dy = (float)iy * ly, dz = (float)iz * lz;
            float r2h = fmaf(dx, dx, fmaf(dy, dy, dz * dz)), r2l = 0.f;
            if (exact) r2_split(R, ix, iy, iz, r2h, r2l);
            const float rh = sqrtf(r2h);
            const float rr = rh + (fmaf(-rh, rh, r2h) + r2l) * (0.5f / rh);
            const float db = (rr - R.rbond_hi) - R.rbond_lo;
            const float ir = 1.f / rr;
            const float A = R.kbondf * db * ir;
            fx = fmaf(-A, dx, fx);
            fy = fmaf(-A, dy, fy);
            fz = fmaf(-A, dz, fz);
            if (E) e = fmaf(0.25f * R.kbondf * db, db, e);
            if (!Q) {
                const float ux = (float)(int)((unsigned)dfi.x - (unsigned)aj.d.x) * lx;
                const float uy = (float)(int)((unsigned)dfi.y - (unsigned)aj.d.y) * ly;
                const float uz = (float)(int)((unsigned)dfi.z - (unsigned)aj.d.z) * lz;
                const float rdu = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
                const float B = (R.kbondf - A) * ir * ir * rdu;
                hx = fmaf(A, ux, fmaf(B, dx, hx));
                hy = fmaf(A, uy, fmaf(B, dy, hy));
                hz = fmaf(A, uz, fmaf(B, dz, hz));
            }
        }
    }
    // undo the FP32 rounding of the per-axis fixed-point unit (uniform per axis)
    fx = fmaf(fx, R.lsb_rel[0], fx);
    fy = fmaf(fy, R.lsb_rel[1], fy);
    fz = fmaf(fz, R.lsb_rel[2], fz);
    const int role = act ? ((pi.w >> 8) & 0xff) : -1;
    if (!Q && role == ROLE_RIGID) {
        hx += R.kr_nf * dri.x;
        if (R.dim == 3) hy += R.kr_nf * dri.y;
    }
    if (act) {
        D.f32[i] = make_float4(fx, fy, fz, e);
        if (!Q) D.h32[i] = make_float4(hx, hy, hz, 0.f);
    }
    const bool rig = role == ROLE_RIGID;
    const bool anyrig = __any_sync(0xffffffffu, rig);
    // FP32 sums inside each warp, FP64 across warps and tiles
    if (!Q) {
        float v[12] = {};
        double d3[3] = {0.0, 0.0, 0.0};
        if (act) {
            const double rx = dri.x, ry = dri.y, rz = dri.z;
            d3[PART_D2] = rx * rx + ry * ry + rz * rz;
            d3[PART_G] = -((double)fx * rx + (double)fy * ry + (double)fz * rz);
            d3[PART_V] = (double)e;
        }
        if (rig) {
            v[PART_FRIG] = fx; v[PART_FRIG + 1] = fy; v[PART_FRIG + 2] = fz;
            v[PART_HRIG] = hx; v[PART_HRIG + 1] = hy; v[PART_HRIG + 2] = hz;
            v[PART_DRRIG] = dri.x; v[PART_DRRIG + 1] = dri.y; v[PART_DRRIG + 2] = dri.z;
        }
        double xr[3] = {0.0, 0.0, 0.0};
        if (rig) {
            const dbl4 xi = D.x[i];
            xr[0] = xi.x; xr[1] = xi.y; xr[2] = xi.z;
        }
        tile_reduce_mixed(d3, v, anyrig ? 12 : 3, xr, anyrig, D.part + (size_t)t * NPART);
    } else {
        float v[12] = {};
        double pvf[3] = {0.0, 0.0, 0.0};
        float fm = 0.f;
        if (role == ROLE_MOBILE) {
            const float4 vv = D.v32[i];
            fm = fx * fx + fy * fy + fz * fz;
            const double gx = fx, gy = fy, gz = fz, ux = vv.x, uy = vv.y, uz = vv.z;
            pvf[0] = gx * ux + gy * uy + gz * uz;
            pvf[1] = ux * ux + uy * uy + uz * uz;
            pvf[2] = gx * gx + gy * gy + gz * gz;
        }
        if (rig) {
            v[QP_FRIG] = fx; v[QP_FRIG + 1] = fy; v[QP_FRIG + 2] = fz;
        }
        double xr[3] = {0.0, 0.0, 0.0};
        if (rig) {
            const dbl4 xi = D.x[i];
            xr[0] = xi.x; xr[1] = xi.y; xr[2] = xi.z;
        }
        v[QP_FMAX2] = fm;
        tile_reduce_quench(v, pvf, xr, anyrig, D.part + (size_t)t * NPART);
    }
}

template <bool Q, bool E>
__global__ void __launch_bounds__(256) k_pair64(Dev D) { dev_pair64<Q, E>(D, blockIdx.x); }
template <bool Q, bool E>
__global__ void __launch_bounds__(256, 4) k_pair32(Dev D) { dev_pair32<Q, E>(D, blockIdx.x); }
// the packed FP32x2 variant: more registers a thread, fewer warps resident
template <bool Q, bool E>
__global__ void __launch_bounds__(128, 5) k_pair32x2(Dev D) { dev_pair32<Q, E, true>(D, blockIdx.x); }

// ---------------------------------------------------------------- per-replica scalars
// Gathers the replica's tile sums (warp q sums slot q over the tiles in a
// fixed order) and evaluates, in FP64:
//   x_T = centre of the rigid layer, spring/load gradient gs;
//   G = grad V . dr (LJ part + gs . sum_rigid dr / n_rig);
//   d = sqrt(sum dr^2) (Eq. 7), sigma = G / d (Eq. 5), DeltaV_1 (Eq. 14);
//   bias coefficients: F_tot = F + ca (H dr - F) + cb dr, ca = -DeltaV'/d,
//   cb = DeltaV' sigma / d^2 (from grad sigma = (H dr + g)/d - sigma dr/d^2);
//   rigid-body force = sum_rigid F - gs - DeltaV' sum_rigid grad sigma;
//   body kicks and the clocks: t_h += dt exp(DeltaV / kT) (Eq. 3).
__device__ void scalar_eval(const Dev &D, int r, int mode, const double *acc, double ksum, RepState &S, Scal &C) {
    const RepDev &R = D.rep[r];
    const int nr = R.nrig, dim = R.dim, vert = R.vert;
    const double xs = slider_x(R, S.step, D.dt);
    double xT[3] = {0, 0, 0}, gs[3] = {0, 0, 0};
    if (nr > 0) {
        for (int a = 0; a < 3; ++a) xT[a] = acc[PART_XRIG + a] / (double)nr;
        gs[0] = R.kspring * (xT[0] - xs);
        if (dim == 3) gs[1] = R.kspring * (xT[1] - R.slider[1]);
        gs[vert] = R.fnormal;
    }
    double G = acc[PART_G];
    if (nr > 0) G += (gs[0] * acc[PART_DRRIG] + gs[1] * acc[PART_DRRIG + 1] + gs[2] * acc[PART_DRRIG + 2]) / (double)nr;
    const double d = sqrt(acc[PART_D2]);
    const double sig = d > 0.0 ? G / d : 0.0;
    double dV = 0.0, dVp = 0.0, dVe = 0.0, d1 = 0.0, d2 = 0.0;
    if (D.bias_on) dv1(R, sig, dV, dVp);
    d1 = dV;
    if (D.bias_on && R.eig_on) {
        // Eq. 13: DeltaV = DeltaV_1 + DeltaV_2 - DeltaV_1 DeltaV_2 / DeltaV_max
        double dvp1 = dVp, dvp2 = 0.0;
        dv2(R, S.eig, d2, dvp2);
        if (R.dvmax > 0.0) {
            dV = d1 + d2 - d1 * d2 / R.dvmax;
            dVp = (1.0 - d2 / R.dvmax) * dvp1;
            dVe = (1.0 - d1 / R.dvmax) * dvp2;
        } else {
            dV = dVp = dVe = 0.0;
        }
    }
    const double ca = d > 0.0 ? -dVp / d : 0.0;
    const double cb = d > 0.0 ? dVp * sig / (d * d) : 0.0;
    double fb[3] = {0, 0, 0};
    if (nr > 0)
        for (int a = 0; a < 3; ++a) {
            const double grig = -acc[PART_FRIG + a] + gs[a];
            const double srig = d > 0.0 ? (acc[PART_HRIG + a] + grig) / d - sig * acc[PART_DRRIG + a] / (d * d) : 0.0;
            fb[a] = acc[PART_FRIG + a] - gs[a] - dVp * srig;
        }
    if (dVe != 0.0 && nr > 0) {
        // the rigid layer's share of -dDeltaV/depsilon grad epsilon, summed per tile
        for (int a = 0; a < 3; ++a) {
            double e = 0.0;
            for (int t = R.tile0; t < R.tile0 + R.ntile; ++t) e += D.epart[(size_t)t * 4 + a];
            fb[a] -= dVe * e;
        }
    }
    C.ce = -dVe;
    C.dV1 = d1;
    C.dV2 = d2;
    double ext = 0.0;
    if (nr > 0) {
        ext = 0.5 * R.kspring * (xT[0] - xs) * (xT[0] - xs);
        if (dim == 3) ext += 0.5 * R.kspring * (xT[1] - R.slider[1]) * (xT[1] - R.slider[1]);
        ext += R.fnormal * xT[vert];
    }
    C.d = d; C.sigma = sig; C.dV = dV; C.dVp = dVp; C.G = G;
    C.Vlj = acc[PART_V];
    C.V = acc[PART_V] + ext;
    C.FR = R.kspring * (xs - xT[0]);
    C.xS = xs;
    C.ca = ca; C.cb = cb;
    for (int a = 0; a < 3; ++a) { C.xT[a] = xT[a]; C.fbody[a] = fb[a]; }
    // clocks and the rigid body
    const double h = D.dt;
    double vb[3] = {S.vbody[0], S.vbody[1], S.vbody[2]};
    if (mode & MODE_CLOSE) {
        if (nr > 0)
            for (int a = 0; a < dim; ++a) vb[a] += 0.5 * h * fb[a] / (double)nr;
        for (int a = 0; a < 3; ++a) S.vbody_full[a] = vb[a];
    }
    for (int a = 0; a < 3; ++a) C.vb_mid[a] = vb[a];
    C.step_cur = S.step;
    if (mode & MODE_OPEN) {
        S.t_h += h * exp(dV / R.kT);
        S.t_md += h;
        S.step += 1;
        S.n_dv[dV <= 0.0 ? 0 : (dV >= R.dvmax ? 2 : 1)] += 1;
        if (nr > 0)
            for (int a = 0; a < dim; ++a) vb[a] += 0.5 * h * fb[a] / (double)nr;
    }
    for (int a = 0; a < 3; ++a) { C.vb_new[a] = vb[a]; S.vbody[a] = vb[a]; }
    S.K = ksum + 0.5 * (double)nr * (S.vbody_full[0] * S.vbody_full[0] + S.vbody_full[1] * S.vbody_full[1] +
                                     S.vbody_full[2] * S.vbody_full[2]);
}

// Tile sums of one replica, slot by slot (slot NPART = kinetic parts): for
// each slot, lane l adds tiles l, l+32, ... in order, then a fixed warp
// tree; the result does not depend on which warp of which CTA computes it.
__device__ __forceinline__ void dev_scalar_acc(const Dev &D, int r, double *acc) {
    const RepDev &R = D.rep[r];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int q = w; q <= NPART; q += nw) {
        double a = 0.0;
        for (int t = R.tile0 + lane; t < R.tile0 + R.ntile; t += 32)
            a += (q < NPART) ? D.part[(size_t)t * NPART + q] : D.kpart[t];
        a = warp_sum(a);
        if (lane == 0) acc[q] = a;
    }
    __syncthreads();
}

// blockDim = 32 * (NPART + 1): warp q < NPART sums partial slot q, warp NPART sums K.
__global__ void k_scalar(Dev D, int mode) {
    const int r = blockIdx.x;
    __shared__ double acc[NPART + 1];
    dev_scalar_acc(D, r, acc);
    if (threadIdx.x == 0) {
        scalar_eval(D, r, mode, acc, acc[NPART], D.st[r], D.sc[r]);
        // the list (if rebuilt this step) has been used; count displacement-triggered builds
        const int f = D.rebuild[r];
        if (f) {
            if (f == 1) D.st[r].n_rebuild += 1;
            D.rebuild[r] = 0;
        }
    }
}

// Kinetic energy of the last full step (observables only).
__global__ void k_obs(Dev D) {
    const int r = blockIdx.x;
    const RepDev &R = D.rep[r];
    RepState &S = D.st[r];
    double a = 0.0;
    for (int t = R.tile0 + (int)threadIdx.x; t < R.tile0 + R.ntile; t += 32) a += D.kpart[t];
    a = warp_sum(a);
    if (threadIdx.x == 0)
        S.K = a + 0.5 * (double)R.nrig * (S.vbody_full[0] * S.vbody_full[0] + S.vbody_full[1] * S.vbody_full[1] +
                                          S.vbody_full[2] * S.vbody_full[2]);
}

// ---------------------------------------------------------------- Nose-Hoover chain
// One half step of the chain (Sec. 3.1.1; the reversible Trotter splitting of
// Martyna, Tuckerman, Tobias and Klein, 1996, one stage): quarter kicks of
// the chain velocities from the top down with exp(-v_{j+1} h/8) damping on
// both sides, the particle scale s = exp(-v_1 h/2), the chain positions by
// h/2, then the kicks from the bottom up.  k2 = sum m v^2 of the mobile atoms
// is updated to its scaled value; returns s.
__device__ double nhc_half(const RepDev &R, RepState &S, double &k2, double h) {
    const int M = R.nhc_len;
    const double kT = R.kT;
    double *v = S.nhc_v;
    auto force = [&](int j) {
        return j == 0 ? (k2 - R.nhc_nf * kT) / R.nhc_Q[0] : (R.nhc_Q[j - 1] * v[j - 1] * v[j - 1] - kT) / R.nhc_Q[j];
    };
    v[M - 1] += 0.25 * h * force(M - 1);
    for (int j = M - 2; j >= 0; --j) {
        const double damp = exp(-0.125 * h * v[j + 1]);
        v[j] *= damp;
        v[j] += 0.25 * h * force(j);
        v[j] *= damp;
    }
    const double sc = exp(-0.5 * h * v[0]);
    k2 *= sc * sc;
    for (int j = 0; j < M; ++j) S.nhc_xi[j] += 0.5 * h * v[j];
    for (int j = 0; j < M - 1; ++j) {
        const double damp = exp(-0.125 * h * v[j + 1]);
        v[j] *= damp;
        v[j] += 0.25 * h * force(j);
        v[j] *= damp;
    }
    v[M - 1] += 0.25 * h * force(M - 1);
    return sc;
}

// The chain between two kicks.  mode KIN: remember k2 of the current
// velocities.  CLOSE: the closing half step of the step that ends (k2 from
// the kinetic sums of the closing kick just made); OPEN: the opening half
// step of the next one (k2 carried over).  C.nhc_scale is the product of the
// particle scales, applied by the next update pass.
__device__ void nhc_eval(const Dev &D, int r, int mode, double ksum, RepState &S, Scal &C) {
    const RepDev &R = D.rep[r];
    C.nhc_scale = 1.0;
    if (R.nhc_len <= 0) return;
    if (mode & MODE_KIN) {
        S.nhc_k2 = 2.0 * ksum;
        return;
    }
    double k2 = (mode & MODE_CLOSE) ? 2.0 * ksum : S.nhc_k2, sc = 1.0;
    if (mode & MODE_CLOSE) sc *= nhc_half(R, S, k2, D.dt);
    if (mode & MODE_OPEN) sc *= nhc_half(R, S, k2, D.dt);
    S.nhc_k2 = k2;
    C.nhc_scale = sc;
}

__global__ void k_nhc(Dev D, int mode) {
    const int r = blockIdx.x;
    const RepDev &R = D.rep[r];
    double a = 0.0;
    for (int t = R.tile0 + (int)threadIdx.x; t < R.tile0 + R.ntile; t += 32) a += D.kpart[t];
    a = warp_sum(a);
    if (threadIdx.x == 0) nhc_eval(D, r, mode, a, D.st[r], D.sc[r]);
}

// ---------------------------------------------------------------- integrator
// BAOAB (reading: Langevin in place of the paper's Nose-Hoover chain):
//   CLOSE: v += dt/2 F_tot                      (end of the previous step)
//   OPEN:  v += dt/2 F_tot; x += dt/2 v; v = c v + s xi; x += dt/2 v
// Mobile atoms only; rigid atoms follow the body velocity; fixed atoms stay.
__device__ __forceinline__ int4 post_move(const Dev &D, const RepDev &R, int r, int i, dbl4 x, int4 p) {
    const int4 q = fix_pos(R, x, p.w);
    D.rec[i].p = q;
    const int4 b = D.pfixb[i];
    const float ex = (float)(int)((unsigned)q.x - (unsigned)b.x) * R.fx_lsb[0];
    const float ey = (float)(int)((unsigned)q.y - (unsigned)b.y) * R.fx_lsb[1];
    const float ez = (float)(int)((unsigned)q.z - (unsigned)b.z) * R.fx_lsb[2];
    if (ex * ex + ey * ey + ez * ez > D.half_skin2_f) D.rebuild[r] = 1;
    const double zv = R.vert == 2 ? x.z : x.y;
    if (!(fabs(zv - R.fx_origin[R.vert]) < R.open_lim) || !isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z))
        set_err(D, HD_ERR_NUMERIC, i, r);
    return q;
}

// Split form: the new fixed-point image and r - r_O as the difference of
// images, in one 32-byte record store; then the checks of post_move.  r - r_O
// wraps at L / 2^(k+1) >= 4 (rc + skin); an atom is reported (HD_ERR_NUMERIC)
// when it has moved 3/4 of that from its r_O.
__device__ __forceinline__ void post_move32(const Dev &D, const RepDev &R, int r, int i, dbl4 x, int4 p) {
    const int4 q = fix_pos(R, x, p.w);
    const int4 d = img_diff(q, D.po[i]);
    AtomRec a;
    a.p = q;
    a.d = d;
    D.rec[i] = a;
    const int4 b = D.pfixb[i];
    const float ex = (float)(int)((unsigned)q.x - (unsigned)b.x) * R.fx_lsb[0];
    const float ey = (float)(int)((unsigned)q.y - (unsigned)b.y) * R.fx_lsb[1];
    const float ez = (float)(int)((unsigned)q.z - (unsigned)b.z) * R.fx_lsb[2];
    if (ex * ex + ey * ey + ez * ez > D.half_skin2_f) D.rebuild[r] = 1;
    const double zv = R.vert == 2 ? x.z : x.y;
    const int lim = 3 << 29;
    if (!(fabs(zv - R.fx_origin[R.vert]) < R.open_lim) || !isfinite(x.x) || !isfinite(x.y) || !isfinite(x.z) ||
        abs(d.x) > lim || abs(d.y) > lim || abs(d.z) > lim)
        set_err(D, HD_ERR_NUMERIC, i, r);
}

__device__ __forceinline__ void dev_update64(const Dev &D, int t, int mode, const Scal &C) {
    const int r = D.tile_rep[t];
    const RepDev &R = D.rep[r];
    const bool act = threadIdx.x < D.tile_n[t];
    const int i = D.tile_start[t] + (act ? threadIdx.x : 0);
    const int4 p = D.rec[i].p;
    const int role = act ? ((p.w >> 8) & 0xff) : ROLE_FIXED;
    double kin = 0.0;
    if (role != ROLE_FIXED) {
        const double h = D.dt;
        dbl4 x = D.x[i], v = D.v64[i];
        if (role == ROLE_MOBILE) {
            const dbl4 F = D.f64[i], H = D.h64[i], dr = D.dr64[i];
            const double ca = C.ca, cb = C.cb;
            double Fx = F.x + ca * (H.x - F.x) + cb * dr.x;
            double Fy = F.y + ca * (H.y - F.y) + cb * dr.y;
            double Fz = F.z + ca * (H.z - F.z) + cb * dr.z;
            if (C.ce != 0.0) {               // eigenvalue bias (Eq. 13, Eq. 15)
                const dbl4 g = D.eg[i];
                Fx += C.ce * g.x;
                Fy += C.ce * g.y;
                Fz += C.ce * g.z;
            }
            const bool three = R.dim == 3;
            const bool chain = R.nhc_len > 0;
            if (mode & MODE_KIN) kin = 0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
            if (mode & MODE_SCALE) {
                if (chain) {
                    v.x *= C.nhc_scale;
                    v.y *= C.nhc_scale;
                    v.z *= C.nhc_scale;
                }
                kin = 0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
            }
            if (mode & MODE_CLOSE) {
                v.x += 0.5 * h * Fx;
                v.y += 0.5 * h * Fy;
                if (three) v.z += 0.5 * h * Fz;
                kin = 0.5 * (v.x * v.x + v.y * v.y + v.z * v.z);
            }
            if (mode & MODE_OPEN) {
                if (chain && (mode & MODE_NHC)) {
                    v.x *= C.nhc_scale;
                    v.y *= C.nhc_scale;
                    v.z *= C.nhc_scale;
                }
                v.x += 0.5 * h * Fx;
                v.y += 0.5 * h * Fy;
                if (three) v.z += 0.5 * h * Fz;
                x.x += 0.5 * h * v.x;
                x.y += 0.5 * h * v.y;
                if (three) x.z += 0.5 * h * v.z;
                if (!chain) {
                    double n0, n1, n2, n3;
                    normals64(philox_draw(D, C.step_cur, D.orig[i], R.rep_id, 0), n0, n1);
                    v.x = R.c_ou * v.x + R.s_ou * n0;
                    v.y = R.c_ou * v.y + R.s_ou * n1;
                    if (three) {
                        normals64(philox_draw(D, C.step_cur, D.orig[i], R.rep_id, 1), n2, n3);
                        v.z = R.c_ou * v.z + R.s_ou * n2;
                    }
                }
                x.x += 0.5 * h * v.x;
                x.y += 0.5 * h * v.y;
                if (three) x.z += 0.5 * h * v.z;
            }
        } else {
            if (mode & MODE_CLOSE) v = make_dbl4(C.vb_mid[0], C.vb_mid[1], C.vb_mid[2], 0.0);
            if (mode & MODE_OPEN) {
                x.x += 0.5 * h * C.vb_new[0];
                x.y += 0.5 * h * C.vb_new[1];
                x.z += 0.5 * h * C.vb_new[2];
                x.x += 0.5 * h * C.vb_new[0];
                x.y += 0.5 * h * C.vb_new[1];
                x.z += 0.5 * h * C.vb_new[2];
                v = make_dbl4(C.vb_new[0], C.vb_new[1], C.vb_new[2], 0.0);
            }
        }
        D.v64[i] = v;
        if (mode & MODE_OPEN) {
            D.x[i] = x;
            const dbl4 xo = D.xo[i];
            D.dr64[i] = make_dbl4(x.x - xo.x, x.y - xo.y, x.z - xo.z, 0.0);
            post_move(D, R, r, i, x, p);
        }
    }
    if (mode & (MODE_CLOSE | MODE_KIN | MODE_SCALE)) {
        double v1[1] = {kin};
        cta_reduce<1>(v1, D.kpart + t, -1);
    }
}

__device__ __forceinline__ void dev_update32(const Dev &D, int t, int mode, const Scal &C) {
    // split form: FP32 forces, FP64 velocities and positions (FP32 velocities
    // would round every kick and thermostat step at 2^-24 of |v|, which after
    // 100 steps puts sigma and the boosted clock beyond 1e-6 of FP64); r - r_O
    // from the fixed-point images of r and r_O
    const int r = D.tile_rep[t];
    const RepDev &R = D.rep[r];
    const bool act = threadIdx.x < D.tile_n[t];
    const int i = D.tile_start[t] + (act ? threadIdx.x : 0);
    const AtomRec ai = D.rec[i];
    const int4 p = ai.p;
    const int role = act ? ((p.w >> 8) & 0xff) : ROLE_FIXED;
    // the closing half kick of one step and the opening one of the next see
    // the same force: between steps of one call a Langevin replica takes one
    // full kick in FP64 (this GPU's FP64 rate is a small fraction of its FP32
    // rate).  The kinetic energy at the half step is an observable there, not
    // an input, and is summed only on the closing half of a call's last step.
    const bool fused = R.nhc_len == 0 && (mode & MODE_CLOSE) && (mode & MODE_OPEN);
    float kin = 0.f;
    if (role != ROLE_FIXED) {
        const double hh = 0.5 * D.dt;
        dbl4 v = D.v64[i];
        dbl4 x = D.x[i];
        if (role == ROLE_MOBILE) {
            const float4 F = D.f32[i], H = D.h32[i];
            const float4 dr = make_float4((float)ai.d.x * R.fx_lsb[0], (float)ai.d.y * R.fx_lsb[1],
                                          (float)ai.d.z * R.fx_lsb[2], 0.f);
            const float ca = (float)C.ca, cb = (float)C.cb;
            double Fx = (double)fmaf(ca, H.x - F.x, fmaf(cb, dr.x, F.x));
            double Fy = (double)fmaf(ca, H.y - F.y, fmaf(cb, dr.y, F.y));
            double Fz = (double)fmaf(ca, H.z - F.z, fmaf(cb, dr.z, F.z));
            if (C.ce != 0.0) {               // eigenvalue bias (Eq. 13, Eq. 15), FP64
                const dbl4 g = D.eg[i];
                Fx += C.ce * g.x;
                Fy += C.ce * g.y;
                Fz += C.ce * g.z;
            }
            const bool three = R.dim == 3;
            const bool chain = R.nhc_len > 0;
            if (fused) {
                v.x = fma(D.dt, Fx, v.x);
                v.y = fma(D.dt, Fy, v.y);
                if (three) v.z = fma(D.dt, Fz, v.z);
            } else {
                if (mode & MODE_KIN) kin = (float)(0.5 * (v.x * v.x + v.y * v.y + v.z * v.z));
                if (mode & MODE_SCALE) {
                    if (chain) {
                        v.x *= C.nhc_scale;
                        v.y *= C.nhc_scale;
                        v.z *= C.nhc_scale;
                    }
                    kin = (float)(0.5 * (v.x * v.x + v.y * v.y + v.z * v.z));
                }
                if (mode & MODE_CLOSE) {
                    v.x += hh * Fx;
                    v.y += hh * Fy;
                    if (three) v.z += hh * Fz;
                    kin = (float)(0.5 * (v.x * v.x + v.y * v.y + v.z * v.z));
                }
                if (mode & MODE_OPEN) {
                    if (chain && (mode & MODE_NHC)) {
                        v.x *= C.nhc_scale;
                        v.y *= C.nhc_scale;
                        v.z *= C.nhc_scale;
                    }
                    v.x += hh * Fx;
                    v.y += hh * Fy;
                    if (three) v.z += hh * Fz;
                }
            }
            if (mode & MODE_OPEN) {
                const double ax = v.x, ay = v.y, az = v.z;
                if (!chain) {
                    float n0, n1, n2, n3;
                    normals32(philox_draw(D, C.step_cur, D.orig[i], R.rep_id, 0), n0, n1);
                    v.x = R.c_ou * v.x + R.s_ou * (double)n0;
                    v.y = R.c_ou * v.y + R.s_ou * (double)n1;
                    if (three) {
                        normals32(philox_draw(D, C.step_cur, D.orig[i], R.rep_id, 1), n2, n3);
                        v.z = R.c_ou * v.z + R.s_ou * (double)n2;
                    }
                }
                x.x += hh * (ax + v.x);
                x.y += hh * (ay + v.y);
                if (three) x.z += hh * (az + v.z);
            }
        } else {
            if (mode & MODE_CLOSE) v = make_dbl4(C.vb_mid[0], C.vb_mid[1], C.vb_mid[2], 0.0);
            if (mode & MODE_OPEN) {
                x.x += hh * C.vb_new[0];
                x.y += hh * C.vb_new[1];
                x.z += hh * C.vb_new[2];
                x.x += hh * C.vb_new[0];
                x.y += hh * C.vb_new[1];
                x.z += hh * C.vb_new[2];
                v = make_dbl4(C.vb_new[0], C.vb_new[1], C.vb_new[2], 0.0);
            }
        }
        D.v64[i] = v;
        if (mode & MODE_OPEN) {
            D.x[i] = x;
            post_move32(D, R, r, i, x, p);
        }
    }
    if ((mode & (MODE_CLOSE | MODE_KIN | MODE_SCALE)) && !fused) {
        double v1[1] = {(double)warp_sum(kin)};
        if ((threadIdx.x & 31) != 0) v1[0] = 0.0;
        cta_reduce<1>(v1, D.kpart + t, -1);
    }
}

__global__ void __launch_bounds__(256) k_update64(Dev D, int mode) {
    dev_update64(D, blockIdx.x, mode, D.sc[D.tile_rep[blockIdx.x]]);
}
__global__ void __launch_bounds__(256) k_update32(Dev D, int mode) {
    dev_update32(D, blockIdx.x, mode, D.sc[D.tile_rep[blockIdx.x]]);
}

// ---------------------------------------------------------------- quench
// |x - r_O|^2 in FP64, in the transition test's operation order.  Positions
// and r_O are never wrapped, so below L/2 per axis this is the minimum-image
// value bit for bit; beyond it it is larger, which only delays an early stop.
__device__ __forceinline__ double disp2(dbl4 a, dbl4 b) {
    const double d0 = __dsub_rn(a.x, b.x), d1 = __dsub_rn(a.y, b.y), d2 = __dsub_rn(a.z, b.z);
    return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

// Split form: |x - r_O|^2 in FP32 from the difference of the fixed-point
// images of x and r_O (exact integers; no FP64 instruction).  A difference
// beyond 3/4 of the image range reads as far.  The early stop compares it
// with (theta/2)^2, where FP32 rounding can only matter within ~1e-7 of it.
__device__ __forceinline__ float disp2_img(const RepDev &R, int4 q, int4 po) {
    const int4 d = img_diff(q, po);
    const int lim = 3 << 29;
    if (abs(d.x) > lim || abs(d.y) > lim || abs(d.z) > lim) return 3.0e38f;
    const float dx = (float)d.x * R.fx_lsb[0], dy = (float)d.y * R.fx_lsb[1], dz = (float)d.z * R.fx_lsb[2];
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Largest m over the CTA into qgate[r] (non-negative doubles order as their
// bit patterns).  Every thread of the CTA calls it.
__device__ __forceinline__ void gate_max(const Dev &D, int r, double m) {
    __shared__ double sm[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    m = warp_max(m);
    if (lane == 0) sm[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = sm[0];
        for (int k = 1; k < nw; ++k) a = fmax(a, sm[k]);
        atomicMax(D.qgate + r, (unsigned long long)__double_as_longlong(a));
    }
}
// The same over FP32 values, converted once per CTA.
__device__ __forceinline__ void gate_max_f(const Dev &D, int r, float m) {
    __shared__ float smf[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if (lane == 0) smf[w] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = smf[0];
        for (int k = 1; k < nw; ++k) a = fmaxf(a, smf[k]);
        atomicMax(D.qgate + r, (unsigned long long)__double_as_longlong((double)a));
    }
}

__global__ void k_qinit(Dev Q, Dev M) {
    // Q: quench view (x = copy), M: MD view
    const int t = blockIdx.x, r = Q.tile_rep[t];
    if (threadIdx.x == 0 && t == Q.rep[r].tile0) {
        RepState &S = Q.st[r];
        S.q_dt = Q.q_step;
        S.q_alpha = 0.1;
        S.q_npos = 0;
        S.q_iter = 0;
        S.q_done = 0;
        S.q_flag = 0;
        S.q_stay = 0;
        S.q_fmax = 0.0;
        S.q_vb[0] = S.q_vb[1] = S.q_vb[2] = 0.0;
        Q.qdisp[r] = 0ull;
        Q.rebuild[r] = 2;
    }
    double m = 0.0;
    float mf = 0.f;
    if (threadIdx.x < Q.tile_n[t]) {
        const int i = Q.tile_start[t] + threadIdx.x;
        const dbl4 x = M.x[i];
        const int4 p = M.rec[i].p;
        Q.x[i] = x;
        Q.rec[i].p = p;
        if (Q.prec == HD_FP64) Q.v64[i] = make_dbl4(0, 0, 0, 0);
        else Q.v32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (Q.q_ftol_stay > 0.0) {
            if (Q.prec == HD_FP64) m = disp2(x, Q.xo[i]);
            else mf = disp2_img(Q.rep[r], p, Q.po[i]);
        }
    }
    if (Q.q_ftol_stay > 0.0) {
        if (Q.prec == HD_FP64) gate_max(Q, r, m);
        else gate_max_f(Q, r, mf);
    }
}

// Convergence test and FIRE bookkeeping (reading of Bitzek et al. 2006: mix
// with the alpha of this step, then grow/shrink dt and alpha).
__global__ void k_qscalar(Dev D, int max_iter) {
    const int r = blockIdx.x;
    const RepDev &R = D.rep[r];
    RepState &S = D.st[r];
    Scal &C = D.sc[r];
    // this iteration's list rebuild (if any) has been used by the pair pass
    __syncthreads();
    if (threadIdx.x == 0) D.rebuild[r] = 0;
    if (S.q_done) return;
    __shared__ double acc[QPART];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < QPART) {
        double a = (w == QP_FMAX2) ? 0.0 : 0.0;
        for (int t = R.tile0 + lane; t < R.tile0 + R.ntile; t += 32) {
            const double v = D.part[(size_t)t * NPART + w];
            a = (w == QP_FMAX2) ? fmax(a, v) : a + v;
        }
        a = (w == QP_FMAX2) ? warp_max(a) : warp_sum(a);
        if (lane == 0) acc[w] = a;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int nr = R.nrig, dim = R.dim;
    double fb[3] = {0, 0, 0};
    double fm2 = acc[QP_FMAX2];
    if (nr > 0) {
        double xT[3], gs[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) xT[a] = acc[QP_XRIG + a] / (double)nr;
        gs[0] = R.kspring * (xT[0] - slider_x(R, S.step, D.dt));   // the slider stands still during a quench
        if (dim == 3) gs[1] = R.kspring * (xT[1] - R.slider[1]);
        gs[R.vert] = R.fnormal;
        for (int a = 0; a < 3; ++a) fb[a] = acc[QP_FRIG + a] - gs[a];
        fm2 = fmax(fm2, fb[0] * fb[0] + fb[1] * fb[1] + fb[2] * fb[2]);
    }
    const double fmax_ = sqrt(fm2);
    S.q_fmax = fmax_;
    // early stop inside the basin: every atom within theta/2 of r_O and the
    // force below ftol_stay rule a transition out (Sec. 2.3 transition test)
    bool stay = false;
    if (D.q_ftol_stay > 0.0) {
        const double g2 = __longlong_as_double((long long)D.qgate[r]);
        D.qgate[r] = 0ull;
        stay = fmax_ < D.q_ftol_stay && g2 < D.q_keep2;
    }
    if (fmax_ < D.q_ftol || stay || S.q_iter >= max_iter) {
        S.q_done = 1;
        S.q_stay = stay && !(fmax_ < D.q_ftol);
        C.q_active = 0;
        return;
    }
    C.q_active = 1;
    for (int a = 0; a < 3; ++a) C.q_fbody[a] = fb[a];
    if (D.q_method == 1) {
        double pw = acc[QP_P], vv = acc[QP_VV], ff = acc[QP_FF];
        if (nr > 0)
            for (int a = 0; a < dim; ++a) {
                pw += fb[a] * S.q_vb[a];
                vv += (double)nr * S.q_vb[a] * S.q_vb[a];
                ff += fb[a] * fb[a] / (double)nr;
            }
        double alpha = S.q_alpha, dt = S.q_dt;
        double vb[3] = {S.q_vb[0], S.q_vb[1], S.q_vb[2]};
        if (pw > 0.0) {
            const double mix = ff > 0.0 ? alpha * sqrt(vv) / sqrt(ff) : 0.0;
            C.q_mix = mix;
            C.q_zero = 0;
            if (nr > 0)
                for (int a = 0; a < dim; ++a) vb[a] = (1.0 - alpha) * vb[a] + mix * fb[a] / (double)nr;
            S.q_npos += 1;
            if (S.q_npos > 5) {
                dt = dt * 1.1 < 10.0 * D.q_step ? dt * 1.1 : 10.0 * D.q_step;
                alpha *= 0.99;
            }
        } else {
            C.q_mix = 0.0;
            C.q_zero = 1;
            vb[0] = vb[1] = vb[2] = 0.0;
            dt *= 0.5;
            alpha = 0.1;
            S.q_npos = 0;
        }
        C.q_alpha = S.q_alpha;   // the alpha this step mixes with
        C.q_dt = dt;             // the dt this step moves with
        S.q_alpha = alpha;
        S.q_dt = dt;
        if (nr > 0)
            for (int a = 0; a < dim; ++a) vb[a] += dt * fb[a] / (double)nr;
        for (int a = 0; a < 3; ++a) { S.q_vb[a] = vb[a]; C.q_vb[a] = vb[a]; }
    }
    S.q_iter += 1;
}

// Per-atom quench move.  SD: x += a F (body: a F_body / n_rig).  FIRE: mix,
// or zero, the velocity, then a semi-implicit Euler step.
template <typename V4>
__device__ __forceinline__ dbl4 qmove(const Dev &D, const RepDev &R, const Scal &C, int r, int i, int4 p, int role,
                                      double fx, double fy, double fz, V4 *vq, int4 *img) {
    dbl4 x = D.x[i];
    const int dim = R.dim;
    if (D.q_method == 0) {
        const double a = D.q_step;
        if (role == ROLE_MOBILE) {
            x.x += a * fx;
            x.y += a * fy;
            if (dim == 3) x.z += a * fz;
        } else {
            const double inr = 1.0 / (double)R.nrig;
            x.x += a * C.q_fbody[0] * inr;
            x.y += a * C.q_fbody[1] * inr;
            if (dim == 3) x.z += a * C.q_fbody[2] * inr;
        }
    } else {
        const double dt = C.q_dt;
        if (role == ROLE_MOBILE) {
            V4 v = vq[i];
            double vx = v.x, vy = v.y, vz = v.z;
            if (C.q_zero) {
                vx = vy = vz = 0.0;
            } else {
                vx = (1.0 - C.q_alpha) * vx + C.q_mix * fx;
                vy = (1.0 - C.q_alpha) * vy + C.q_mix * fy;
                vz = (1.0 - C.q_alpha) * vz + C.q_mix * fz;
            }
            vx += dt * fx;
            vy += dt * fy;
            if (dim == 3) vz += dt * fz;
            else vz = 0.0;
            x.x += dt * vx;
            x.y += dt * vy;
            if (dim == 3) x.z += dt * vz;
            v.x = vx; v.y = vy; v.z = vz;
            vq[i] = v;
        } else {
            x.x += dt * C.q_vb[0];
            x.y += dt * C.q_vb[1];
            if (dim == 3) x.z += dt * C.q_vb[2];
        }
    }
    D.x[i] = x;
    *img = post_move(D, R, r, i, x, p);
    return x;
}

// The split form's FIRE move in FP32 (its velocities are FP32 and its forces
// FP32 already): only the position, kept in FP64, takes FP64 adds.
__device__ __forceinline__ int4 qmove32(const Dev &D, const RepDev &R, const Scal &C, int r, int i, int4 p, int role,
                                        float fx, float fy, float fz) {
    if (D.q_method == 0) {
        int4 q;
        qmove(D, R, C, r, i, p, role, (double)fx, (double)fy, (double)fz, D.v32, &q);
        return q;
    }
    dbl4 x = D.x[i];
    const bool three = R.dim == 3;
    const float dt = (float)C.q_dt;
    if (role == ROLE_MOBILE) {
        float4 v = D.v32[i];
        if (C.q_zero) {
            v.x = v.y = v.z = 0.f;
        } else {
            const float keep = (float)(1.0 - C.q_alpha), mix = (float)C.q_mix;
            v.x = fmaf(keep, v.x, mix * fx);
            v.y = fmaf(keep, v.y, mix * fy);
            v.z = fmaf(keep, v.z, mix * fz);
        }
        v.x = fmaf(dt, fx, v.x);
        v.y = fmaf(dt, fy, v.y);
        v.z = three ? fmaf(dt, fz, v.z) : 0.f;
        x.x += (double)(dt * v.x);
        x.y += (double)(dt * v.y);
        if (three) x.z += (double)(dt * v.z);
        D.v32[i] = v;
    } else {
        x.x += C.q_dt * C.q_vb[0];
        x.y += C.q_dt * C.q_vb[1];
        if (three) x.z += C.q_dt * C.q_vb[2];
    }
    D.x[i] = x;
    return post_move(D, R, r, i, x, p);
}

__global__ void __launch_bounds__(256) k_qupdate(Dev D) {
    const int t = blockIdx.x, r = D.tile_rep[t];
    const Scal &C = D.sc[r];
    if (!C.q_active || D.st[r].q_done) return;        // the same for the whole CTA
    // displacement from r_O of the new iterate (every atom, as in the
    // transition test), for the next convergence test
    const bool gate = D.q_ftol_stay > 0.0;
    double m = 0.0;
    float mf = 0.f;
    if (threadIdx.x < D.tile_n[t]) {
        const int i = D.tile_start[t] + threadIdx.x;
        const RepDev &R = D.rep[r];
        const int4 p = D.rec[i].p;
        const int role = (p.w >> 8) & 0xff;
        if (D.prec == HD_FP64) {
            dbl4 x;
            int4 q;
            if (role == ROLE_FIXED) {
                if (gate) x = D.x[i];
            } else {
                const dbl4 f = D.f64[i];
                x = qmove(D, R, C, r, i, p, role, f.x, f.y, f.z, D.v64, &q);
            }
            if (gate) m = disp2(x, D.xo[i]);
        } else {
            int4 q = p;
            if (role != ROLE_FIXED) {
                const float4 f = D.f32[i];
                q = qmove32(D, R, C, r, i, p, role, f.x, f.y, f.z);
            }
            if (gate) mf = disp2_img(R, q, D.po[i]);
        }
    }
    if (gate) {
        if (D.prec == HD_FP64) gate_max(D, r, m);
        else gate_max_f(D, r, mf);
    }
}

// Largest displacement of the quenched copy from r_O per replica (minimum
// image, FP64, the oracle's operation order); stored as the bits of the
// non-negative double so that an integer max is the FP64 max.
__global__ void k_qdisp(Dev Q) {
    const int t = blockIdx.x, r = Q.tile_rep[t];
    if (threadIdx.x >= Q.tile_n[t]) return;
    const int i = Q.tile_start[t] + threadIdx.x;
    const RepDev &R = Q.rep[r];
    const dbl4 a = Q.x[i], b = Q.xo[i];
    double d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z;
    if (R.periodic[0]) d0 = __dsub_rn(d0, __dmul_rn(R.L[0], rint(__ddiv_rn(d0, R.L[0]))));
    if (R.periodic[1]) d1 = __dsub_rn(d1, __dmul_rn(R.L[1], rint(__ddiv_rn(d1, R.L[1]))));
    if (R.periodic[2]) d2 = __dsub_rn(d2, __dmul_rn(R.L[2], rint(__ddiv_rn(d2, R.L[2]))));
    const double m = __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
    atomicMax(Q.qdisp + r, (unsigned long long)__double_as_longlong(m));
}

// r_O <- quenched copy for replicas with adopt[r] != 0; refresh r - r_O.
__global__ void k_adopt(Dev Q, Dev M, const int *adopt) {
    const int t = blockIdx.x, r = M.tile_rep[t];
    if (!adopt[r] || threadIdx.x >= M.tile_n[t]) return;
    const int i = M.tile_start[t] + threadIdx.x;
    const dbl4 q = Q.x[i];
    M.xo[i] = make_dbl4(q.x, q.y, q.z, 0.0);
    const dbl4 x = M.x[i];
    if (M.prec == HD_FP64) M.dr64[i] = make_dbl4(x.x - q.x, x.y - q.y, x.z - q.z, 0.0);
    else {
        const int4 po = fix_pos(M.rep[r], make_dbl4(q.x, q.y, q.z, 0.0), 0);
        M.po[i] = po;
        M.rec[i].d = img_diff(M.rec[i].p, po);
    }
}

// ---------------------------------------------------------------- persistent driver
// One launch steps every replica n times.  Replica r owns CTAs
// [pg_first[r], pg_first[r] + pg_count[r]); each CTA takes the replica's
// tiles round robin and runs the same per-tile phases as the per-phase
// kernels; the compiler may contract multiply-adds differently where a phase
// is inlined here, so the two drivers agree to rounding.  Phases of one
// replica are separated by that replica's own barrier: a counter in global
// memory (reset before each launch) that CTAs increment and poll.  Polling
// is bounded: after ~2^24 polls the CTA records HD_ERR_TIMEOUT, raises the
// abort word err[3], and every CTA leaves at its next barrier.  The launch
// is cooperative, so all CTAs are resident.  A one-CTA replica uses only
// __syncthreads().
__device__ __forceinline__ bool grp_barrier(const Dev &D, int r, int nc, unsigned &epoch) {
    __shared__ int s_ok;
    __syncthreads();
    if (nc > 1) {
        if (threadIdx.x == 0) {
            int ok = 1;
            __threadfence();
            const unsigned target = (epoch + 1u) * (unsigned)nc;
            // test hook: one CTA of replica fault_rep skips its first arrival
            const bool skip = D.fault_rep == r && epoch == 0 && blockIdx.x == (unsigned)D.pg_first[r];
            if (!skip) atomicAdd(D.bar + r, 1u);
            unsigned polls = 0;
            while (*((volatile unsigned *)(D.bar + r)) < target) {
                if (*((volatile int *)(D.err + 3)) != 0) { ok = 0; break; }
                if (++polls > (1u << 24)) {
                    set_err(D, HD_ERR_TIMEOUT, -1, r);
                    atomicExch(D.err + 3, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
            __threadfence();
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return false;
    }
    ++epoch;
    return true;
}

template <int PREC>
__global__ void __launch_bounds__(128, 4) k_persist(Dev D, int nsteps) {
    const int r = D.cta_rep[blockIdx.x];
    if (r < 0) return;
    const RepDev &R = D.rep[r];
    const int nc = D.pg_count[r], me = blockIdx.x - D.pg_first[r];
    const bool leader = me == 0;
    __shared__ RepState S;
    __shared__ Scal C;
    __shared__ double acc[NPART + 1];
    __shared__ int s_flag;
    __shared__ NlSmem M;
    extern __shared__ __align__(16) char nl_smem[];
    int4 *sp;
    unsigned *smask;
    nl_smem_carve(D, nl_smem, sp, smask);
    if (threadIdx.x == 0) {
        S = D.st[r];
        C = D.sc[r];
    }
    __syncthreads();
    unsigned epoch = 0;
    auto scalars = [&](int mode) {
        dev_scalar_acc(D, r, acc);
        if (threadIdx.x == 0) {
            scalar_eval(D, r, mode, acc, acc[NPART], S, C);
            if (leader) {
                D.st[r] = S;
                D.sc[r] = C;
            }
        }
        __syncthreads();
    };
    auto update = [&](int mode) {
        for (int t = R.tile0 + me; t < R.tile0 + R.ntile; t += nc) {
            if (PREC == HD_FP64) dev_update64(D, t, mode, C);
            else dev_update32(D, t, mode, C);
        }
    };
    // the chain between the kicks (every CTA evaluates it alike from the
    // replica's kinetic sums)
    auto chain = [&](int mode) {
        dev_scalar_acc(D, r, acc);
        if (threadIdx.x == 0) {
            nhc_eval(D, r, mode, acc[NPART], S, C);
            if (leader) {
                D.st[r] = S;
                D.sc[r] = C;
            }
        }
        __syncthreads();
    };
    const bool nhc = D.any_nhc != 0;
    // opening half of the first step, from the forces of the last call
    scalars(MODE_OPEN);
    if (nhc) chain(MODE_OPEN);
    update(nhc ? (MODE_OPEN | MODE_NHC) : MODE_OPEN);
    if (!grp_barrier(D, r, nc, epoch)) return;
    for (int k = 1; k <= nsteps; ++k) {
        if (threadIdx.x == 0) s_flag = *((volatile int *)(D.rebuild + r));
        __syncthreads();
        const int flag = s_flag;
        if (flag) {
            for (int c = me * blockDim.x + threadIdx.x; c < R.ncell; c += nc * blockDim.x) D.cell_cnt[R.cell0 + c] = 0;
            if (!grp_barrier(D, r, nc, epoch)) return;
            for (int t = R.tile0 + me; t < R.tile0 + R.ntile; t += nc) dev_bin(D, t);
            if (!grp_barrier(D, r, nc, epoch)) return;
            {
                const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
                int *buf = reinterpret_cast<int *>(nl_smem) + wib * D.cell_cap;
                for (int c = me * nwb + wib; c < R.ncell; c += nc * nwb) dev_cellsort_warp(D, R, c, buf);
                __syncthreads();
            }
            if (!grp_barrier(D, r, nc, epoch)) return;
            // every CTA has read the flag before the first barrier above
            if (threadIdx.x == 0) {
                if (flag == 1) S.n_rebuild += 1;
                if (leader) D.rebuild[r] = 0;
            }
            // rows are built cell by cell, so a CTA's tiles take rows other CTAs wrote
            for (int c = me; c < R.ncell; c += nc) dev_nlist_cell(D, r, c, M, sp, smask);
            if (!grp_barrier(D, r, nc, epoch)) return;
        }
        for (int t = R.tile0 + me; t < R.tile0 + R.ntile; t += nc) {
            // per-atom energies (observables only) on the last step of the call
            if (PREC == HD_FP64) {
                if (k == nsteps) dev_pair64<false, true>(D, t);
                else dev_pair64<false, false>(D, t);
            } else {
                if (k == nsteps) dev_pair32<false, true>(D, t);
                else dev_pair32<false, false>(D, t);
            }
        }
        if (!grp_barrier(D, r, nc, epoch)) return;
        const int mode = k < nsteps ? (MODE_CLOSE | MODE_OPEN) : MODE_CLOSE;
        scalars(mode);
        if (!nhc) {
            update(mode);
        } else {
            update(MODE_CLOSE);
            if (!grp_barrier(D, r, nc, epoch)) return;
            chain(mode);
            update((mode & MODE_OPEN) ? (MODE_OPEN | MODE_NHC) : MODE_SCALE);
        }
        if (!grp_barrier(D, r, nc, epoch)) return;
    }
    if (leader && threadIdx.x == 0) D.st[r] = S;
}

// ---------------------------------------------------------------- launchers
static inline int nthr(const Dev &D) { return D.block; }

// Dynamic shared memory of the list build: positions, indices and classes
// of up to 27 cells of cell_cap candidates (classes: one byte per candidate
// for each of the warps of a 128-thread CTA).
size_t nl_smem_bytes(const Dev &D, int nwarps) {
    return 27 * (size_t)D.cell_cap * sizeof(int4) + (size_t)nwarps * nl_mask_words(D) * sizeof(unsigned);
}
// the persistent kernel runs the list build and the pair sweep in one launch
static size_t persist_smem_bytes(const Dev &D) {
    const size_t a = nl_smem_bytes(D, (D.block + 31) / 32), b = pair_smem_bytes_for(D.block);
    return a > b ? a : b;
}
cudaError_t nl_configure(const Dev &D, int *nl_blocks_per_sm) {
    const int bytes = (int)nl_smem_bytes(D, NL_THREADS / 32), pbytes = (int)persist_smem_bytes(D);
    cudaError_t e = cudaFuncSetAttribute(k_nlist, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    // the row builder is latency-bound: launch as many CTAs as fit
    *nl_blocks_per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(nl_blocks_per_sm, k_nlist, NL_THREADS, bytes);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_persist<HD_FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, pbytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_persist<HD_FP32_SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, pbytes);
}

void launch_init(const Dev &D, const int *draw_vel, cudaStream_t s) {
    k_init<<<D.ntile, nthr(D), 0, s>>>(D, draw_vel);
}
void launch_rebuild_prep(const Dev &D, cudaStream_t s) {
    k_rebuild_plan<<<1, 32, 0, s>>>(D);
    k_cell_clear<<<D.nl_grid, 256, 0, s>>>(D);
    k_bin<<<D.nl_grid, 256, 0, s>>>(D);
    k_cellsort<<<D.nl_grid, 128, 4 * D.cell_cap * sizeof(int), s>>>(D);
}
void launch_nlist(const Dev &D, cudaStream_t s) {
    k_nlist<<<D.nl_grid, NL_THREADS, nl_smem_bytes(D, NL_THREADS / 32), s>>>(D);
}
void launch_rebuild(const Dev &D, cudaStream_t s) {
    launch_rebuild_prep(D, s);
    launch_nlist(D, s);
}
void launch_pair(const Dev &D, bool quench, bool energy, cudaStream_t s) {
    if (D.prec == HD_FP64) {
        if (quench) k_pair64<true, false><<<D.ntile, nthr(D), 0, s>>>(D);
        else if (energy) k_pair64<false, true><<<D.ntile, nthr(D), 0, s>>>(D);
        else k_pair64<false, false><<<D.ntile, nthr(D), 0, s>>>(D);
    } else if (D.pair_x2 && D.block <= 128) {
        const size_t sm = pair_smem_bytes_for(D.block);
        if (quench) k_pair32x2<true, false><<<D.ntile, nthr(D), sm, s>>>(D);
        else if (energy) k_pair32x2<false, true><<<D.ntile, nthr(D), sm, s>>>(D);
        else k_pair32x2<false, false><<<D.ntile, nthr(D), sm, s>>>(D);
    } else {
        const size_t sm = pair_smem_bytes_for(D.block);
        if (quench) k_pair32<true, false><<<D.ntile, nthr(D), sm, s>>>(D);
        else if (energy) k_pair32<false, true><<<D.ntile, nthr(D), sm, s>>>(D);
        else k_pair32<false, false><<<D.ntile, nthr(D), sm, s>>>(D);
    }
}
void launch_scalar(const Dev &D, int mode, cudaStream_t s) {
    k_scalar<<<D.nrep, 32 * (NPART + 1), 0, s>>>(D, mode);
}
void launch_update(const Dev &D, int mode, cudaStream_t s) {
    if (D.prec == HD_FP64) k_update64<<<D.ntile, nthr(D), 0, s>>>(D, mode);
    else k_update32<<<D.ntile, nthr(D), 0, s>>>(D, mode);
}
void launch_obs(const Dev &D, cudaStream_t s) { k_obs<<<D.nrep, 32, 0, s>>>(D); }
void launch_nhc(const Dev &D, int mode, cudaStream_t s) { k_nhc<<<D.nrep, 32, 0, s>>>(D, mode); }
void launch_qinit(const Dev &Q, const Dev &M, cudaStream_t s) { k_qinit<<<Q.ntile, nthr(Q), 0, s>>>(Q, M); }
void launch_qiter(const Dev &Q, int max_iter, cudaStream_t s) {
    launch_rebuild(Q, s);
    launch_pair(Q, true, false, s);
    k_qscalar<<<Q.nrep, 32 * QPART, 0, s>>>(Q, max_iter);
    k_qupdate<<<Q.ntile, nthr(Q), 0, s>>>(Q);
}
void launch_qdisp(const Dev &Q, cudaStream_t s) { k_qdisp<<<Q.ntile, nthr(Q), 0, s>>>(Q); }
int persist_blocks_per_sm(const Dev &D) {
    int nb = 0;
    const size_t sm = persist_smem_bytes(D);
    if (D.prec == HD_FP64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persist<HD_FP64>, D.block, sm);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persist<HD_FP32_SPLIT>, D.block, sm);
    return nb;
}
cudaError_t launch_persist(const Dev &D, int grid, int nsteps, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(D.bar, 0, sizeof(unsigned) * D.nrep, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(D.err + 3, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(D.block);
    cfg.dynamicSmemBytes = persist_smem_bytes(D);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (D.prec == HD_FP64) return cudaLaunchKernelEx(&cfg, k_persist<HD_FP64>, D, nsteps);
    return cudaLaunchKernelEx(&cfg, k_persist<HD_FP32_SPLIT>, D, nsteps);
}
void launch_adopt(const Dev &Q, const Dev &M, const int *adopt, cudaStream_t s) {
    k_adopt<<<M.ntile, nthr(M), 0, s>>>(Q, M, adopt);
}

}  // namespace hd
