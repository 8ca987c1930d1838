// hd_static.cu -- hd_nlist_static: the neighbour-list build of one replica
// with no device allocation at all.
//
// Some callers cannot let a library allocate device memory: a host program
// that budgets every byte of the GPU itself, or a loop that cannot afford
// the latency or the failure of an allocation.  This entry point takes only
// the caller's input and output buffers and keeps its scratch (fixed-point
// positions, cell ids, cell counts and cell lists, an error word) in one
// file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
//
// The first call on a device looks up that array's device address
// (cudaGetSymbolAddress, with that device current) and keeps it.  Under
// CUDA's lazy module loading that first call is also when the module, and
// with it the array, is committed on the device, so it can itself fail for
// want of memory: make it at start-up, before the program reserves the rest
// of the GPU's memory (or run with CUDA_MODULE_LOADING=EAGER).  Every call
// synchronises its stream (it reads back the error word and, with an open
// axis, the extent of the positions), so no call may be made while that
// stream is being captured into a graph.  Every call shares the array and
// it keeps the last call's contents: the counts, the extent and the error
// word are cleared at the start of each call, and calls that overlap on the
// GPU race.
#include <cmath>
#include <cstring>
#include <mutex>

#include "hd_internal.cuh"

namespace {

constexpr int S_MAX_ATOMS = 65536;
constexpr int S_MAX_CELLS = 16384;
constexpr int S_CELL_CAP = 64;
constexpr int S_MAX_NB = 160;

struct StaticScratch {
    int4 pfix[S_MAX_ATOMS];
    int cellid[S_MAX_ATOMS];
    int cell_cnt[S_MAX_CELLS];
    int cell_atoms[S_MAX_CELLS * S_CELL_CAP];
    unsigned long long ext[6];   // per axis: min then max of the positions, order-preserving bits
    int err[4];
};

static __device__ __align__(256) StaticScratch g_static_scratch;

struct Grid {
    int nc[3], periodic[3];
    double L[3], invL[3], scale[3], origin[3], lo[3], inv_w[3];
    float lsb[3];
    double rl2;
    float rl2_lo, rl2_hi;
};

// Cell along one axis: exact integer map of the fixed-point image on a
// periodic axis; FP64 quotient on an open axis (an FP32 quotient would round
// by more than the cells' 1e-4 width margin near 1000 cells).
__device__ __forceinline__ int s_cell(const Grid &G, int a, int q, double x) {
    if (G.nc[a] <= 1) return 0;
    if (G.periodic[a]) return (int)(((unsigned long long)(unsigned int)q * (unsigned long long)G.nc[a]) >> 32);
    const int c = (int)floor((x - G.lo[a]) * G.inv_w[a]);
    return c < 0 ? 0 : (c >= G.nc[a] ? G.nc[a] - 1 : c);
}

// Order-preserving map of a double onto unsigned 64-bit integers, so that
// integer atomicMin/atomicMax give the FP64 minimum and maximum.
__device__ __forceinline__ unsigned long long ord_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_value(unsigned long long u) {
    const unsigned long long b = (u >> 63) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    double x;
    memcpy(&x, &b, 8);
    return x;
}

// Extent of the positions along every axis (ext must hold +inf / -inf bits:
// all ones for the minima, zero for the maxima).
__global__ void k_s_extent(StaticScratch *S, const double *pos, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int a = 0; a < 3; ++a) {
        const unsigned long long u = ord_bits(pos[3 * i + a]);
        atomicMin(&S->ext[2 * a], u);
        atomicMax(&S->ext[2 * a + 1], u);
    }
}

__device__ __forceinline__ double s_r2(const Grid &G, const double *a, const double *b) {
    double d[3];
    for (int k = 0; k < 3; ++k) {
        d[k] = __dsub_rn(a[k], b[k]);
        if (G.periodic[k]) d[k] = __dsub_rn(d[k], __dmul_rn(G.L[k], rint(d[k] * G.invL[k])));
    }
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}

__global__ void k_s_bin(StaticScratch *S, Grid G, const double *pos, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int q[3];
    for (int a = 0; a < 3; ++a) {
        if (G.scale[a] == 0.0) { q[a] = 0; continue; }
        const long long v = __double2ll_rn((pos[3 * i + a] - G.origin[a]) * G.scale[a]);
        q[a] = (int)(unsigned int)(unsigned long long)v;
    }
    S->pfix[i] = make_int4(q[0], q[1], q[2], 0);
    const int cx = s_cell(G, 0, q[0], pos[3 * i]), cy = s_cell(G, 1, q[1], pos[3 * i + 1]),
              cz = s_cell(G, 2, q[2], pos[3 * i + 2]);
    S->cellid[i] = cx | (cy << 10) | (cz << 20);
    const int c = (cz * G.nc[1] + cy) * G.nc[0] + cx;
    const int slot = atomicAdd(&S->cell_cnt[c], 1);
    if (slot < S_CELL_CAP) S->cell_atoms[c * S_CELL_CAP + slot] = i;
    else atomicCAS(&S->err[0], 0, HD_ERR_OVERFLOW);
}

// Row i: every j != i with FP64 minimum-image r^2 < rl^2 (the FP32 test on
// exact fixed-point differences decides outside a thin band), ascending j.
__global__ void k_s_list(StaticScratch *S, Grid G, const double *pos, int n, int maxnb, int *nbr, int *nnb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 pi = S->pfix[i];
    const int cid = S->cellid[i];
    const int ci[3] = {cid & 1023, (cid >> 10) & 1023, (cid >> 20) & 1023};
    int cs[3][3], ncs[3];
    for (int a = 0; a < 3; ++a) {
        ncs[a] = 0;
        if (G.nc[a] == 1) {
            cs[a][ncs[a]++] = 0;
            continue;
        }
        for (int d = -1; d <= 1; ++d) {
            int c = ci[a] + d;
            if (G.periodic[a]) c = (c + G.nc[a]) % G.nc[a];
            else if (c < 0 || c >= G.nc[a]) continue;
            cs[a][ncs[a]++] = c;
        }
    }
    int *row = nbr + (size_t)i * maxnb;
    int cnt = 0;
    bool over = false;
    for (int iz = 0; iz < ncs[2]; ++iz)
        for (int iy = 0; iy < ncs[1]; ++iy)
            for (int ix = 0; ix < ncs[0]; ++ix) {
                const int c = (cs[2][iz] * G.nc[1] + cs[1][iy]) * G.nc[0] + cs[0][ix];
                const int m = min(S->cell_cnt[c], S_CELL_CAP);
                for (int k = 0; k < m; ++k) {
                    const int j = S->cell_atoms[c * S_CELL_CAP + k];
                    if (j == i) continue;
                    const int4 pj = S->pfix[j];
                    const float dx = (float)(int)((unsigned)pi.x - (unsigned)pj.x) * G.lsb[0];
                    const float dy = (float)(int)((unsigned)pi.y - (unsigned)pj.y) * G.lsb[1];
                    const float dz = (float)(int)((unsigned)pi.z - (unsigned)pj.z) * G.lsb[2];
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    bool in;
                    if (r2 < G.rl2_lo) in = true;
                    else if (r2 >= G.rl2_hi) in = false;
                    else in = s_r2(G, pos + 3 * i, pos + 3 * j) < G.rl2;
                    if (!in) continue;
                    if (cnt < maxnb) {
                        int q = cnt;  // insertion keeps the row ascending
                        while (q > 0 && row[q - 1] > j) {
                            row[q] = row[q - 1];
                            --q;
                        }
                        row[q] = j;
                        ++cnt;
                    } else {
                        over = true;
                    }
                }
            }
    for (int k = cnt; k < maxnb; ++k) row[k] = -1;
    nnb[i] = cnt;
    if (over) atomicCAS(&S->err[0], 0, HD_ERR_OVERFLOW);
}

std::mutex g_mu;
StaticScratch *g_addr[64] = {};

}  // namespace

extern "C" hd_status hd_nlist_static(const double *d_pos, int n_atoms, const double box[3],
                                     const uint8_t periodic[3], double rl, int maxnb, int32_t *d_nbr,
                                     int32_t *d_nnb, void *cuda_stream) {
    if (!d_pos || !d_nbr || !d_nnb || !box || !periodic) return HD_ERR_ARG;
    if (n_atoms <= 0 || n_atoms > S_MAX_ATOMS) return HD_ERR_ARG;
    if (maxnb <= 0 || maxnb > S_MAX_NB || !(rl > 0.0)) return HD_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HD_ERR_CUDA;
    StaticScratch *S;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return HD_ERR_CUDA;
            g_addr[dev] = static_cast<StaticScratch *>(p);
        }
        S = g_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // grid: cells at least rl wide (periodic axes tile the box exactly; the
    // open axis spans the positions of this call, read back to the host)
    Grid G;
    memset(&G, 0, sizeof G);
    G.rl2 = rl * rl;
    G.rl2_lo = (float)(G.rl2 * (1.0 - 1.0 / 4096.0));
    G.rl2_hi = (float)(G.rl2 * (1.0 + 1.0 / 4096.0));
    // the open-axis extent: one reduction kernel into the scratch array, one
    // 48-byte read-back
    double mn[3] = {0, 0, 0}, mx[3] = {0, 0, 0};
    bool need_ext = false;
    for (int a = 0; a < 3; ++a) need_ext |= !periodic[a];
    if (need_ext) {
        if (cudaMemsetAsync(S->ext, 0, sizeof(S->ext), s) != cudaSuccess) return HD_ERR_CUDA;
        for (int a = 0; a < 3; ++a)
            if (cudaMemsetAsync(&S->ext[2 * a], 0xFF, sizeof(unsigned long long), s) != cudaSuccess)
                return HD_ERR_CUDA;
        k_s_extent<<<(n_atoms + 255) / 256, 256, 0, s>>>(S, d_pos, n_atoms);
        unsigned long long e[6];
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(e, S->ext, sizeof e, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return HD_ERR_CUDA;
        for (int a = 0; a < 3; ++a) {
            mn[a] = ord_value(e[2 * a]);
            mx[a] = ord_value(e[2 * a + 1]);
            if (!std::isfinite(mn[a]) || !std::isfinite(mx[a])) return HD_ERR_NUMERIC;
        }
    }
    long long ncell = 1;
    for (int a = 0; a < 3; ++a) {
        G.periodic[a] = periodic[a] ? 1 : 0;
        if (G.periodic[a]) {
            if (!(box[a] > 0.0)) return HD_ERR_ARG;
            G.L[a] = box[a];
            G.invL[a] = 1.0 / box[a];
            G.scale[a] = 4294967296.0 / box[a];
            G.lsb[a] = (float)(box[a] / 4294967296.0);
            const int nc = (int)std::floor(box[a] / (rl * (1.0 + 1e-6)));
            G.nc[a] = nc >= 3 ? nc : 1;
        } else if (mx[a] > mn[a]) {
            double span = 64.0;
            while (span < 4.0 * (mx[a] - mn[a]) + 64.0) span *= 2.0;
            G.origin[a] = 0.5 * (mn[a] + mx[a]);
            G.scale[a] = 4294967296.0 / span;
            G.lsb[a] = (float)(span / 4294967296.0);
            const double w = rl * (1.0 + 1e-4);
            G.inv_w[a] = 1.0 / w;
            G.lo[a] = mn[a] - 1.0;
            G.nc[a] = (int)std::ceil((mx[a] + 1.0 - G.lo[a]) / w);
            if (G.nc[a] < 1) G.nc[a] = 1;
        } else {
            G.nc[a] = 1;
        }
        if (G.nc[a] >= 1024) return HD_ERR_ARG;
        ncell *= G.nc[a];
    }
    if (ncell > S_MAX_CELLS) return HD_ERR_ARG;
    // clear what must start at zero
    if (cudaMemsetAsync(S->cell_cnt, 0, sizeof(int) * ncell, s) != cudaSuccess) return HD_ERR_CUDA;
    if (cudaMemsetAsync(S->err, 0, sizeof(S->err), s) != cudaSuccess) return HD_ERR_CUDA;
    const int nb = (n_atoms + 127) / 128;
    k_s_bin<<<nb, 128, 0, s>>>(S, G, d_pos, n_atoms);
    k_s_list<<<nb, 128, 0, s>>>(S, G, d_pos, n_atoms, maxnb, d_nbr, d_nnb);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    int err[4];
    if (cudaMemcpyAsync(err, S->err, sizeof err, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return HD_ERR_CUDA;
    return err[0] ? (hd_status)err[0] : HD_OK;
}
