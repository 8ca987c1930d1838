/*
 * hd.h -- C ABI of libhdslide: batched hyperdynamics for AFM frictional
 * sliding on one GB300 (sm_103a).
 *
 * Method: Kim & Falk, "Accelerated molecular dynamics simulation of
 * low-velocity frictional sliding".  Many replicas of one Lennard-Jones
 * tip-plus-substrate model, each held at its own slider position (Sec. 2.3,
 * Fig. 2), are stepped together.  One step of one replica does:
 *   - a Verlet-list rebuild when needed (cell binning, then a list of all
 *     pairs closer than rc + skin, rows ascending in j);
 *   - LJ 12-6 forces and energies with type-pair parameters (Eq. 9), cut at
 *     rc and shifted to zero there;
 *   - the slope bias: d = |r - r_O| (Eq. 7), sigma = grad V . (r - r_O)/d
 *     (Eq. 5), DeltaV = DeltaV_1(sigma) (Eq. 14; Eq. 13 with DeltaV_2 = 0)
 *     and its force, which needs the Hessian-vector product H.(r - r_O);
 *   - Langevin BAOAB dynamics with Philox4x32-10 noise; the rigid top layer
 *     of the tip is one body pulled by the slider spring and pushed by the
 *     normal load (Sec. 3.1.1, Sec. 3.2.1);
 *   - the boosted clock t_h += dt exp(DeltaV / kT) (Eq. 3) and the lateral
 *     force F_R = k (x_S - x_T) (Eq. 10).
 * A batched quench (steepest descent or FIRE) finds basin minima r_O and
 * flags transitions (Sec. 2.3).
 *
 * Conventions for every call:
 *   - Host pointers are caller-owned and only read (or written, for
 *     outputs) during the call.  Positions and velocities are [n][3] FP64,
 *     z = 0 for 2-D replicas.  Positions are never wrapped into the box.
 *   - The device workspace is caller-owned: one block of device memory of
 *     at least hd_workspace_bytes() bytes, 256-byte aligned, alive until
 *     hd_destroy().  The library allocates no device memory of its own.
 *   - Work is queued on the caller's CUDA stream; calls that return data
 *     (hd_read, hd_quench flags, hd_sync) synchronise that stream.
 *   - Errors are returned as hd_status codes; nothing is thrown.  The first
 *     error is kept on the context and reported by hd_last_error(); after
 *     it every call but hd_read, hd_last_error and hd_destroy returns
 *     HD_ERR_STATE.  Kernels record device-side faults (list overflow,
 *     non-finite values, an atom leaving the open direction's range, a
 *     barrier wait that ran out) in an error word that is checked when the
 *     stream is synchronised.
 */
#ifndef HD_H
#define HD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hd_ctx hd_ctx;

typedef enum {
    HD_OK = 0,
    HD_ERR_ARG = 1,            /* bad argument (sizes, pointers, field ids)          */
    HD_ERR_CUDA = 2,           /* a CUDA runtime call failed                         */
    HD_ERR_NOMEM = 3,          /* workspace smaller than hd_workspace_bytes()        */
    HD_ERR_NUMERIC = 4,        /* non-finite value or atom outside the open range    */
    HD_ERR_TIMEOUT = 5,        /* a device barrier wait ran out of iterations        */
    HD_ERR_STATE = 6,          /* context holds an earlier error                     */
    HD_ERR_UNIMPLEMENTED = 7,
    HD_ERR_OVERFLOW = 8        /* neighbour row or cell longer than its capacity     */
} hd_status;

typedef enum { HD_FP64 = 0, HD_FP32_SPLIT = 1 } hd_precision;

typedef enum {
    HD_DRIVER_AUTO = 0,        /* the per-phase kernels; pick by measurement instead
                                  (the Python autotuner times both drivers)           */
    HD_DRIVER_KERNELS = 1,     /* one kernel per phase, captured in a CUDA graph     */
    HD_DRIVER_PERSISTENT = 2   /* one cooperative launch steps every replica         */
} hd_driver;

/* One replica.  Roles: 0 fixed (bottom of the substrate, never moves),
 * 1 mobile, 2 rigid (top layer of the tip, moves as one body).  Types select
 * the LJ pair parameters: 0 substrate, 1 tip (Eq. 9). */
typedef struct {
    int dim;                   /* 2 or 3; the vertical (open) axis is dim-1           */
    int n_atoms;
    int rep_id;                /* Philox counter word; keep unique within a batch     */
    int m_exp;                 /* exponent m of Eq. 14 (>= 1; C1 at sigma_U if >= 2)  */
    const double *pos;         /* [n][3] positions                                    */
    const double *vel;         /* [n][3] or NULL: Maxwell-Boltzmann for mobile atoms  */
    const double *pos_ref;     /* [n][3] basin minimum r_O, or NULL: r_O = pos        */
    const uint8_t *role;       /* [n]                                                 */
    const uint8_t *type;       /* [n]                                                 */
    double box[3];             /* periodic lengths (ignored on open axes)             */
    uint8_t periodic[3];       /* 1 on the in-plane axes, 0 on the vertical axis      */
    uint8_t pad_[5];
    double kT;                 /* temperature (k_B = 1)                               */
    double gamma;              /* Langevin friction, 1/tau                            */
    double k_spring;           /* slider spring stiffness k (Eq. 10)                  */
    double f_normal;           /* normal load F_N pushing the rigid layer down        */
    double slider[2];          /* x_S (and y_S, used in 3-D)                          */
    double dvmax, sig_lo, sig_hi;  /* DeltaV_max, sigma_L, sigma_U of Eq. 14          */
    double eps[2][2], sig[2][2];   /* LJ eps_ab, sigma_ab of Eq. 9, by type           */
    double t_h0, t_md0;        /* initial boosted and MD clocks (resume)              */
    int64_t step0;             /* initial step counter (Philox; resume)               */
    double v_slide;            /* continuous sliding (Sec. 3.1.1, method 1): the slider
                                  moves along x at this velocity, x_S = slider[0] +
                                  k (v_slide dt) for a configuration k steps after the
                                  slider was set; 0: stepped sliding, x_S fixed       */
    int n_bonds;               /* harmonic bonds of Eq. 12 (Sec. 3.2.1): k_bond (r -
                                  r_bond)^2 / 2 between the atom pairs of bonds; with
                                  n_bonds > 0 tip-tip pairs (type 1 with type 1) have
                                  no LJ term.  0: every pair is LJ                    */
    int pad2_;
    const int32_t *bonds;      /* [n_bonds][2] input atom indices i != j, or NULL     */
    double k_bond, r_bond;     /* bond stiffness and rest length (paper: 57.2, 1.12)  */
    int nhc_len;               /* Nose-Hoover chain (Sec. 3.1.1) of this length (1..8)
                                  on the mobile atoms in place of the Langevin noise
                                  (gamma unused); 0: Langevin.  The chain starts at
                                  rest; masses Q_1 = N_f kT tau^2, Q_j = kT tau^2 with
                                  N_f = dim x mobile atoms                           */
    int pad3_;
    double nhc_tau;            /* chain period tau                                    */
    int eig_on;                /* 1: Eq. 13 bias, DeltaV_1(sigma) combined with
                                  DeltaV_2(epsilon) of Eq. 15, epsilon the lowest
                                  eigenvalue of the Hessian over the allowed motions
                                  (fixed atoms frozen, rigid layer as one body), by
                                  Lanczos to a Ritz residual of 1e-10 |epsilon|; 0:
                                  the slope bias alone.  Per-phase driver only.     */
    int eig_maxit;             /* Lanczos steps at most (0: 3 n_atoms), capped at the
                                  dimension of the allowed motions                   */
    double eig_lo, eig_hi;     /* epsilon_L, epsilon_U of Eq. 15                      */
} hd_replica_desc;

typedef struct {
    int prec;                  /* hd_precision                                        */
    int bias_on;               /* 0: plain MD (DeltaV = 0), 1: Eq. 14 bias            */
    int driver;                /* hd_driver                                           */
    int block;                 /* atoms per tile / threads per CTA (0: 128)           */
    double dt, rc, skin;       /* time step, LJ cutoff, Verlet skin                   */
    uint64_t seed;             /* Philox key                                          */
    int maxnb;                 /* neighbour row capacity (0: 32 if all 2-D, else 112) */
    int cell_cap;              /* atoms per cell capacity (0: from the input)         */
    int pair_kernel;           /* split form, per-phase driver: 0 the scalar pair
                                  sweep, 1 the packed FP32x2 one (two list entries a
                                  thread per instruction; tiles of <= 128 atoms)      */
    int pad_;
} hd_params;

/* Bytes of device workspace hd_create needs for this batch.  Returns 0 if
 * the arguments are invalid. */
size_t hd_workspace_bytes(const hd_replica_desc *reps, int n_rep, const hd_params *p);

/* Build the batch: copy the replicas into the workspace (replicas back to
 * back), draw Maxwell-Boltzmann velocities where vel == NULL (Philox calls 2
 * and 3 at step0), build the neighbour lists, compute forces, H.dr and the
 * bias at the initial positions.  cuda_stream: a cudaStream_t (NULL: the
 * legacy default stream).  On success *out owns the host-side context. */
hd_status hd_create(const hd_replica_desc *reps, int n_rep, const hd_params *p,
                    void *d_workspace, size_t ws_bytes, void *cuda_stream, hd_ctx **out);

/* Move the sliders: slider[2*r], slider[2*r+1] = (x_S, y_S) of replica r
 * (stepped sliding, Sec. 2.3 and Fig. 1); a replica with v_slide != 0 moves
 * on from there at v_slide, counting steps from the current configuration.  If requench_ref is non-zero, each
 * replica is then quenched (FIRE from dt0 = 0.005, at most 20000 steps, to
 * ftol 1e-6 in the FP64 form and 1e-3 in the split form, whose FP32 pair
 * forces do not resolve the rigid body's summed force much below that) and
 * r_O is set to the result where the quench converged (HD_OBS_QCONV). */
hd_status hd_set_slider(hd_ctx *ctx, const double *slider, int requench_ref);

/* Replace the bias parameters of Eq. 14: bias[4*r .. 4*r+3] =
 * (DeltaV_max, sigma_L, sigma_U, m) of replica r. */
hd_status hd_set_bias(hd_ctx *ctx, const double *bias);

/* Advance every replica by n_steps BAOAB steps (asynchronous). */
hd_status hd_step(hd_ctx *ctx, int n_steps);

/* Quench a copy of every replica's positions to its basin minimum with the
 * unbiased potential (method 0: steepest descent, x += step_size F;
 * method 1: FIRE with initial time step step_size), until the largest force
 * on a mobile atom or the rigid body is below ftol or max_iter updates were
 * made.  A replica whose quenched positions lie more than theta from r_O
 * (any atom, minimum image) is flagged as having made a transition
 * (Sec. 2.3).  ftol_stay > ftol (0: off) stops a replica's quench earlier,
 * once its largest force is below ftol_stay while every atom lies within
 * theta/2 of r_O: the state is then well inside the transition threshold
 * and stays unflagged (HD_OBS_QCONV = 2); a replica that has moved further
 * runs on to ftol.  ftol_stay needs a finite theta > 0.  adopt: 0 keep r_O;
 * 1 set r_O to the quenched positions of flagged replicas; 2 of every
 * replica.  Only a replica whose quench reached ftol adopts: an unconverged
 * quench is no basin minimum.  h_flags [n_rep] (may be NULL) receives the
 * flags; the call synchronises the stream.  The MD state is not changed.
 * HD_ERR_ARG: method not 0 or 1, ftol <= 0, max_iter < 0, step_size <= 0,
 * adopt outside 0..2, or ftol_stay neither 0 nor above ftol. */
hd_status hd_quench(hd_ctx *ctx, int method, double ftol, int max_iter, double step_size,
                    double theta, double ftol_stay, int adopt, int32_t *h_flags);

/* Copy one field of one replica to host memory (synchronises the stream).
 * bytes must equal the field's size for that replica. */
enum {
    HD_FIELD_POS = 0,          /* double [n][3]                                       */
    HD_FIELD_VEL = 1,          /* double [n][3]                                       */
    HD_FIELD_FORCE = 2,        /* double [n][3] LJ force                              */
    HD_FIELD_HDR = 3,          /* double [n][3] H.(r - r_O), spring term included     */
    HD_FIELD_REF = 4,          /* double [n][3] r_O                                   */
    HD_FIELD_NBR = 5,          /* int32 [n][maxnb] replica-local j, -1 padded         */
    HD_FIELD_NBR_COUNT = 6,    /* int32 [n]                                           */
    HD_FIELD_OBS = 7,          /* double [HD_OBS_LEN]; replica -1: [n_rep][HD_OBS_LEN] */
    HD_FIELD_CELL = 8,         /* int32 [n] cell (cx, cy, cz) packed cx|cy<<10|cz<<20  */
    HD_FIELD_QPOS = 9,         /* double [n][3] positions of the last quench          */
    HD_FIELD_ENERGY = 10       /* double [n] per-atom LJ energy (half of each pair)   */
};

/* OBS record, doubles.  K is the kinetic energy at the end of the last step
 * of the last hd_step call (between the steps of one call the library does
 * not form it). */
enum {
    HD_OBS_STEP = 0, HD_OBS_TMD = 1, HD_OBS_TH = 2, HD_OBS_V = 3, HD_OBS_K = 4,
    HD_OBS_DV = 5, HD_OBS_SIGMA = 6, HD_OBS_D = 7, HD_OBS_FR = 8, HD_OBS_XT = 9,
    HD_OBS_YT = 10, HD_OBS_ZT = 11, HD_OBS_NREBUILD = 12, HD_OBS_BOOST = 13,
    HD_OBS_QITER = 14, HD_OBS_QFMAX = 15, HD_OBS_G = 16, HD_OBS_FBODY = 17,
    HD_OBS_VBODY = 20, HD_OBS_QDISP = 23,
    HD_OBS_NDV_ZERO = 24,      /* steps taken so far with DeltaV = 0 (sigma <= sigma_L) */
    HD_OBS_NDV_BAND = 25,      /* ... with 0 < DeltaV < DeltaV_max                    */
    HD_OBS_NDV_MAX = 26,       /* ... with DeltaV = DeltaV_max (sigma >= sigma_U)      */
    HD_OBS_QCONV = 27,         /* last quench: 1 reached ftol, 2 stopped inside its   *
                                *  basin at ftol_stay, 0 stopped at max_iter           */
    HD_OBS_XS = 28,            /* slider x_S of the current configuration             */
    HD_OBS_NHC_E = 29,         /* chain energy sum Q v^2/2 + N_f kT xi_1 + kT sum xi_j */
    HD_OBS_EIG = 30,           /* epsilon of Eq. 15 (eigenvalue bias)                 */
    HD_OBS_EIG_ITERS = 31,     /* Lanczos steps of its last evaluation                */
    HD_OBS_LEN = 32
};

hd_status hd_read(hd_ctx *ctx, int field, int replica, void *h_dst, size_t bytes);

/* Sizes and counters: out[0] n_rep, [1] total atoms, [2] maxnb,
 * [3] cell_cap, [4] tiles, [5] driver in use, [6] CTAs of the persistent
 * launch, [7] device kernel launches made so far, [8] host-to-device bytes
 * copied so far, [9] device-to-host bytes copied so far, [10] workspace
 * bytes in use, [11] reserved (0). */
hd_status hd_info(const hd_ctx *ctx, int64_t out[12]);

/* In-library CUDA-event timers around every launch of the LJ/H.dr pair
 * kernel (and of the other phases), taken on the context's stream; inside a
 * captured CUDA graph they are event nodes.  enable: 1 start timing, 0 stop,
 * 2 zero the totals, -1 leave as is.  out (may be NULL) receives, in ms and
 * counts since the last reset: [0] pair ms, [1] pair launches, [2] update ms,
 * [3] update launches, [4] list-rebuild preparation ms (plan, cell clear,
 * binning, cell sort), [5] its passes, [6] scalar ms, [7] scalar launches,
 * [8] row-build (k_nlist) ms, [9] its launches, [10] eigenvalue-bias ms
 * (Lanczos and grad epsilon), [11] its passes, [12..15] reserved (0).
 * Synchronises the stream. */
hd_status hd_timing(hd_ctx *ctx, int enable, double out[16]);

/* Neighbour list of one replica without any device allocation.  For callers
 * that must not let a library allocate device memory: a program that
 * budgets all of the GPU's memory itself, or a loop that cannot afford the
 * latency or the failure of an allocation.  The paper has no counterpart;
 * it is the list build of hd_create (rows: every j != i with FP64
 * minimum-image r^2 < rl^2, ascending j) run on caller buffers.
 *   d_pos   device, [n_atoms][3] FP64 positions (read)
 *   box, periodic  host, as in hd_replica_desc; rl = list radius (rc + skin)
 *   d_nbr   device, [n_atoms][maxnb] int32 (written; -1 past each row's end)
 *   d_nnb   device, [n_atoms] int32 row lengths (written)
 * Its scratch (fixed-point positions, cells, an error word) lives in one
 * file-scope device array sized for at most 65,536 atoms, 16,384 cells of at
 * most 64 atoms and maxnb <= 160; larger inputs return HD_ERR_ARG.  Each GPU
 * that loads the library holds that array (about 5.4 MB) until the process
 * exits.  The first call on a device looks up the array's address with that
 * device current; under CUDA's lazy module loading that call also commits
 * the module and the array on the device, so it can fail (HD_ERR_CUDA) in a
 * program that has already reserved all of the GPU's memory: make the first
 * call at start-up, before reserving memory, or run with
 * CUDA_MODULE_LOADING=EAGER.  Every call synchronises cuda_stream (it reads
 * back an error word and, with an open axis, the positions' extent), so it
 * cannot be called while that stream is being captured.  Every call shares
 * the array and leaves its contents behind; counts, extent and the error
 * word are cleared at the start of each call, and calls that overlap on the
 * GPU race.  Returns HD_ERR_OVERFLOW if a row or a cell exceeded its
 * capacity, HD_ERR_NUMERIC for a non-finite position on an open axis. */
hd_status hd_nlist_static(const double *d_pos, int n_atoms, const double box[3], const uint8_t periodic[3],
                          double rl, int maxnb, int32_t *d_nbr, int32_t *d_nnb, void *cuda_stream);

/* Wait for queued work and check the device error word. */
hd_status hd_sync(hd_ctx *ctx);

/* Release the host-side context (the workspace stays the caller's). */
void hd_destroy(hd_ctx *ctx);

/* Text of the first error kept on the context ("" if none). */
const char *hd_last_error(const hd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HD_H */
