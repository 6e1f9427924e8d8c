/*
 * vmat.h -- C ABI of libvmat, the GB300 (sm_103a) hot path of column-generation
 * VMAT optimisation (Tian et al., arXiv:1503.01721).
 *
 * Conventions (apply to every entry point unless its comment says otherwise):
 *  - Array arguments are caller-owned DEVICE memory, dense and contiguous
 *    (e.g. PyTorch tensors).  The library keeps no pointer past the call,
 *    except the matrices held inside a vmat_ddc handle (freed by ddc_free).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous on it unless marked "synchronises".
 *  - Every call returns a vmat_status.  Arguments are validated before any
 *    launch (VMAT_EINVAL); CUDA failures return VMAT_ECUDA.  The message of the
 *    last failure on the calling thread is returned by vmat_last_error().
 *    No C++ exception crosses this interface.
 *  - Kernels never trap.  A device-side problem (a bounded wait that ran out,
 *    an index out of range found by a check) sets the library's device status
 *    word, read and cleared by vmat_device_status().
 *  - Beamlet layout (Section 2.2.2 of the paper: beamlets of one control point
 *    (CP) form the MLC rows the pricing step walks):
 *        beamlet j = (k * n_rows + r) * n_cols + c
 *    for CP k, leaf pair (MLC row) r, column c.  An aperture row is the
 *    half-open column interval [L, R); L == R is a closed row.
 */
#ifndef VMAT_H
#define VMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t vmat_status;
#define VMAT_OK 0
#define VMAT_EINVAL (-1)       /* bad argument (pointer, size, index range) */
#define VMAT_ENOMEM (-2)       /* device allocation failed */
#define VMAT_ECUDA (-3)        /* CUDA runtime/launch error */
#define VMAT_ESTATE (-4)       /* handle not in the required state (e.g. not built) */
#define VMAT_ETIMEOUT (-5)     /* a bounded device-side wait ran out */
#define VMAT_EUNSUPPORTED (-6) /* valid request outside what this build supports */

typedef enum { VMAT_F32 = 0, VMAT_BF16 = 1, VMAT_FP8E4M3 = 2 } vmat_dtype;

/* Opaque dose-deposition-coefficient (DDC) matrix D (V voxels x J beamlets),
 * library-owned device memory. */
typedef struct vmat_ddc_s *vmat_ddc;

/* Delivery limits of Eq. 2 (HOST struct; the paper gives no values, so they
 * are parameters).  All finite: cp_step_deg > 0 (gantry angle between adjacent
 * CPs of an arc), 0 <= speed_min <= speed_max, speed_max > 0 (gantry speed
 * bounds S^L, S^U, deg/s), speed_step_max >= 0 (Delta S: the largest change of
 * gantry speed per CP step, deg/s), 0 <= rate_min <= rate_max (dose-rate bounds
 * R^L, R^U, MU/s), leaf_speed_cols > 0 (largest leaf speed, MLC columns/s).
 * The MLC's travel window must be reachable at the slowest gantry speed:
 * travel_cols * speed_min <= cp_step_deg * leaf_speed_cols (else VMAT_EINVAL). */
typedef struct {
    double cp_step_deg;
    double speed_min, speed_max;
    double speed_step_max;
    double rate_min, rate_max;
    double leaf_speed_cols;
} vmat_machine;

/* MLC geometry.  arc_first_cp is HOST memory: n_arcs ascending CP indices,
 * arc_first_cp[0] == 0; arc a spans [arc_first_cp[a], arc_first_cp[a+1]) (the
 * last arc ends at K).  travel_cols: columns a leaf may travel per CP step
 * (the neighbour-compatibility reading of Eq. 2).  interdigitation != 0: the
 * left leaf of a row may not pass the right leaf of an adjacent row,
 * L_r <= min(R_{r-1}, R_{r+1}) (Section 2.2.2, second pricing variant;
 * n_cols <= 88; not in batches).  machine: HOST, or NULL for fixed fluence
 * bounds [0, +inf); with a machine, cg_plan and batches bound every aperture's
 * fluence rate by fluence_bounds before each master problem (Eq. 6). */
typedef struct {
    int32_t K, n_rows, n_cols;
    int32_t n_arcs;
    const int32_t *arc_first_cp;
    int32_t travel_cols;
    int32_t interdigitation;
    const vmat_machine *machine;
} vmat_mlc;

/* Voxel penalty parameters of Eq. 1: per-voxel structure label (device uint8
 * [V]) and per-structure prescription/threshold T, overdose weight w_over and
 * underdose weight w_under (device float [n_struct], n_struct <= 256). */
typedef struct {
    const uint8_t *struct_id;
    int32_t n_struct;
    const float *T;
    const float *w_over;
    const float *w_under;
} vmat_voxels;

/* Build options for ddc_build. */
typedef struct {
    vmat_dtype dtype;   /* stored value type; FP8 uses per-beamlet power-of-two scales */
    int32_t build_D;    /* nonzero: build CSR(D), voxel rows (dose_forward, aperture_dose) */
    int32_t build_Dt;   /* nonzero: build CSR(D^T), beamlet rows (beamlet_price) */
    int32_t tile_cfg;   /* SpMV configuration index of CSR(D) (and of CSR(D^T) when tile_cfg_Dt < 0),
                           -1 = library default */
    int32_t autotune;   /* nonzero: time every tile configuration and keep the fastest */
    int32_t keep_coo;   /* nonzero: keep the COO copy after the build */
    int32_t index16;    /* nonzero: also store 16-bit column indices (rows cut into 128-entry
                           chunks, each with a 32-bit base column) for every CSR whose chunks all
                           span fewer than 65,536 columns; the autotuner then also times the
                           configurations that read them (2 bytes per nonzero instead of 4) */
    int32_t tile_cfg_Dt; /* SpMV configuration index of CSR(D^T), -1 = as tile_cfg (a pair found by
                            the autotuner once, see vmat_ddc_info, can be reused without tuning again) */
    int32_t refine_f32; /* BF16 / FP8 builds: nonzero keeps CSR(D)'s values in FP32 as well (4 more
                           bytes per nonzero), and cg_plan ends with the FP32 refinement described
                           there.  Ignored for F32 builds. */
    int32_t vox_grid[3]; /* {nx, ny, nz} of the voxel grid when voxel i = (z ny + y) nx + x, else all 0.
                            Given, CSR(D^T) numbers its columns in brick order: bricks of 4 x 4 x 2
                            voxels (32 voxels, the 128 bytes of one cache line of g), bricks in x-fastest
                            order, the grid padded up to whole bricks.  A beamlet's 32 consecutive
                            entries then touch about half as many lines of g as in grid order, which
                            the gathers of D^T g pay for (Eq. 3).  beamlet_price and
                            beamlet_price_windowed still take and return vectors in voxel order: they
                            reorder g on the stream first (stream-ordered scratch of 4 bytes per
                            padded voxel); cg_plan and batches write g in brick order directly.
                            nx ny nz must equal V (VMAT_EINVAL otherwise). */
} vmat_build_opts;

/* Master-problem (Eq. 6-10) options.  Stopping rules of Section 2.1:
 * |F_{t-5} - F_t| <= rel_tol5 * F_t, or max|y_t - y_{t-1}| <= step_tol *
 * max(1, max|y_t|), or max_iter iterations.  Steps are clamped to
 * [delta_min, delta_max] times the first (Cauchy) step. */
typedef struct {
    int32_t max_iter;
    double rel_tol5;
    double step_tol;
    double delta_min;
    double delta_max;
} vmat_bb_opts;

#define VMAT_STOP_REL 1
#define VMAT_STOP_STEP 2
#define VMAT_STOP_MAXIT 3
#define VMAT_STOP_GRAD0 4
#define VMAT_STOP_FLAT 5
#define VMAT_STOP_PRICE 10 /* cg_plan: best CP price <= 0 (Section 2.1) */
#define VMAT_STOP_COUNT 11 /* cg_plan: n_apertures generated */

typedef struct {
    int32_t iters;       /* BB iterations run */
    int32_t stop_reason; /* VMAT_STOP_* */
    double F;            /* objective at the returned y */
} vmat_bb_report;

typedef struct {
    int32_t V, J;
    int64_t nnz;
    int32_t n_active_vox;   /* voxels with at least one nonzero (rows of CSR(D)) */
    vmat_dtype dtype;
    int32_t built_D, built_Dt;
    int32_t tile_nnz_D, tile_nnz_Dt; /* nonzeros per SpMV tile */
    int64_t bytes_D, bytes_Dt;       /* device bytes of each CSR (values, columns, row pointers) */
    double build_ms;                 /* device time of the last ddc_build */
    int32_t cfg_D, cfg_Dt;           /* SpMV configuration of each CSR (see vmat_spmv_config_count) */
    int32_t index16_D, index16_Dt;   /* 1: that CSR holds the 16-bit column index */
    int64_t bytes16_D, bytes16_Dt;   /* device bytes of the 16-bit index (offsets, bases, chunk pointers) */
    int32_t refine_f32;              /* 1: CSR(D) also holds FP32 values (build option refine_f32) */
    int32_t vox_brick;               /* 1: CSR(D^T) columns are in brick order (build option vox_grid) */
} vmat_ddc_info;

/* Per-phase device times of cg_plan, named as the paper's Table 2 phases. */
typedef struct {
    double t_total_ms;  /* whole call */
    double t_pp1_ms;    /* gradient + beamlet price (Eq. 3-4) */
    double t_pp2_ms;    /* pricing kernels + choice readback */
    double t_da_ms;     /* aperture dose vectors (Eq. 5) */
    double t_mp_ms;     /* master problems (Eq. 6-10) */
    double t_final_ms;  /* final dose D (A y) and objective */
    double pp1_spmv_ms; /* the D^T g kernels alone */
    int64_t pp1_spmv_launches;
    double pp1_spmv_bytes;  /* algorithmic bytes of those launches (rows inside the leaf-travel windows) */
    double other_spmv_bytes; /* algorithmic bytes of the D x / aperture-dose passes */
    int32_t n_apertures;
    int32_t bb_iters_total;
    int32_t stop_reason;
    int64_t kernel_launches; /* kernels this call launched */
    double pp1_full_bytes;   /* bytes of the same passes over every row of the unoccupied CPs */
    int32_t refined;         /* 1: the plan ended with the FP32 refinement (see cg_plan) */
    int32_t refine_bb_iters; /* BB iterations of the refinement's master problem */
    double t_refine_ms;      /* refinement: FP32 aperture dose vectors and master problem */
    double F_before_refine;  /* objective of the low-precision master problem's dose before it */
    double mp_bytes;         /* bytes the master problems' passes over DA moved (t_mp_ms's work):
                                per pass, each 32-voxel tile in the solve reads its 128-byte label
                                head and its ceil(n/4) four-aperture groups (512 bytes each) and
                                writes (or reads) its 32 doses */
    int32_t pp1_spmv_cfg;    /* SpMV configuration of the windowed D^T g passes: on an autotuned handle
                                the fastest on a pass over half of every MLC row (timed once per
                                handle and MLC shape), else the handle's CSR(D^T) configuration */
} vmat_plan_stats;

/* ---- DDC matrix ---------------------------------------------------------- */

/* Copy a COO DDC matrix into a new handle (Section 2.2.2: the dose engine
 * writes D as COO, value + voxel index + beamlet index).
 * vox[e] in [0, V), blt[e] in [0, J), val[e] finite; nnz >= 0.
 * on_device != 0: the three arrays are device memory; otherwise host memory
 * (pinned or pageable).  Duplicate (voxel, beamlet) pairs are rejected by
 * ddc_build.  On success *out owns device copies; free with ddc_free. */
vmat_status ddc_load_coo(int32_t V, int32_t J, int64_t nnz, const int32_t *vox, const int32_t *blt,
                         const float *val, int32_t on_device, void *stream, vmat_ddc *out);

/* Build the device matrices (Section 2.2.2: CSR of D^T for the beamlet
 * price; the paper converts at initialisation).  CSR(D^T): row j = beamlet j,
 * entries sorted by voxel.  CSR(D): rows = voxels with at least one entry,
 * entries sorted by beamlet.  Values stored as opts->dtype: F32 as given,
 * BF16 round-to-nearest-even, FP8 E4M3 (saturating, nearest-even) of
 * D_ij / s_j with s_j the least power of two with 448 s_j >= max_i |D_ij|.
 * Index checks and the duplicate check report VMAT_EINVAL.  Synchronises. */
vmat_status ddc_build(vmat_ddc h, const vmat_build_opts *opts, void *stream);

/* Release every device buffer of the handle.  NULL is accepted. */
vmat_status ddc_free(vmat_ddc h);

/* Sizes and build facts of a handle (host struct). */
vmat_status ddc_info(vmat_ddc h, vmat_ddc_info *out);

/* ---- Sparse products (hot path) ------------------------------------------ */

/* d = D x (Section 2.1: z_i = sum_j D_ij x_j; Eq. 5 is the case x = the
 * indicator of an aperture).  x: device float [J]; d: device float [V],
 * fully written (voxels without entries get 0).  FP32 accumulation.
 * Needs build_D. */
vmat_status dose_forward(vmat_ddc h, const float *x, float *d, void *stream);

/* pi = D^T g (Eq. 3, beamlet price, with g = -grad F of Eq. 4).
 * g: device float [V]; pi: device float [J].  cp_active: device uint8 [K]
 * or NULL (all CPs); when given, only the beamlets of CPs with
 * cp_active[k] != 0 are priced (the paper prices unoccupied CPs only) and
 * entries of inactive CPs are left unspecified.  beamlets_per_cp =
 * n_rows * n_cols (ignored when cp_active is NULL).  FP32 accumulation.
 * Needs build_Dt.  On a handle built with vox_grid, g is first copied into
 * brick order (stream-ordered scratch of 4 bytes per padded voxel). */
vmat_status beamlet_price(vmat_ddc h, const float *g, float *pi, const uint8_t *cp_active,
                          int32_t beamlets_per_cp, void *stream);

/* pi = D^T g (Eq. 3) on the beamlets that pricing can read: for every CP k with
 * occupied[k] == 0 and MLC row r, the columns [Lmin, Rmax) of the row's
 * leaf-travel window (Section 2.2.2 with the neighbour compatibility of Eq. 2:
 * each leaf within m * travel_cols columns of its position at the nearest
 * occupied CP m steps away in the same arc).  price_apertures reads no other
 * entry; they are left unspecified.  mlc: host; occupied: device uint8 [K];
 * leaves: device int16 [K][n_rows][2], (L, R) of the occupied CPs; g: device
 * float [V]; pi: device float [J] with J = K * n_rows * n_cols.  Needs
 * build_Dt.  Allocates K * n_rows * 8 + 4 bytes of device scratch (stream-ordered; on
 * a handle built with vox_grid also the brick-ordered copy of g, as beamlet_price). */
vmat_status beamlet_price_windowed(vmat_ddc h, const vmat_mlc *mlc, const uint8_t *occupied, const int16_t *leaves,
                                   const float *g, float *pi, void *stream);

/* ---- Objective ------------------------------------------------------------ */

/* F(z) of Eq. 1 and g = -grad F of Eq. 4 for V voxels.
 * z: device float [V]; g: device float [V] (FP32) or NULL; F: device double
 * [1] (FP64 sum, deterministic order) or NULL. */
vmat_status objective_grad(int32_t V, const float *z, const vmat_voxels *vox, float *g, double *F,
                           void *stream);

/* ---- Pricing problem, second step (Section 2.2.2) ------------------------- */

/* For every unoccupied CP k (occupied[k] == 0) and MLC row r, the opening
 * [L, R) maximising the summed price (within leaf-travel windows set by the
 * nearest occupied CP on each side of the same arc, Eq. 2 compatibility),
 * then the CP whose row sum is largest.  Row values are P_R - P_L with P the
 * sequential float64 prefix sum of the float32 prices; ties are broken by
 * (width asc, |L + R - n_cols| asc, L asc); the CP price is the sequential
 * float64 sum over rows; CP ties go to the smallest k.  The result is
 * bit-for-bit reproducible from pi.
 * pi: device float [J]; occupied: device uint8 [K]; leaves: device int16
 * [K][n_rows][2] (read for occupied CPs only).  Outputs (device): best_cp
 * int32 [1] (-1 if no CP is feasible), best_leaves int16 [n_rows][2],
 * best_price double [1].  n_cols <= 1024. */
vmat_status price_apertures(const vmat_mlc *mlc, const float *pi, const uint8_t *occupied, const int16_t *leaves,
                            int32_t *best_cp, int16_t *best_leaves, double *best_price, void *stream);

/* Allocation-free pricing (no counterpart in the paper).  Same inputs, outputs
 * and results, bit for bit, as price_apertures; the difference is that this
 * call allocates no device memory.  It is meant for callers that cannot allocate
 * while they plan: a service that hands all of its GPU memory to its own pool at
 * start-up (an allocation behind that pool's back can fail or fragment it), or
 * a loop that must not touch the allocator after initialisation.
 * Its scratch is one fixed device array inside libvmat of
 * VMAT_NOALLOC_SCRATCH_BYTES (about 0.85 MB), which every GPU that loads the
 * library keeps until the process exits.  Two limits follow from its size:
 *   - K * n_rows at most VMAT_NOALLOC_MAX_ROWS (CP, MLC row) pairs;
 *   - with interdigitation, the chain search also keeps per-CP prices, every
 *     row's prefix sums and every CP's predecessor table there:
 *     K * (9 + 8 n_rows (n_cols + 1) + 2 (n_rows (n_cols + 1)^2 + 1)) + 80
 *     bytes must fit (36 CPs x 20 rows x 20 columns does; the 180 x 64 x 64
 *     geometry does not).
 * Beyond either limit the call returns VMAT_EINVAL (use price_apertures).
 * Every call looks up the array's device address on the current device (a host
 * lookup; the first one on a device also loads the library's device code
 * there, so make that first call outside any stream capture).  All calls share
 * the one array: calls whose work overlaps on the GPU (other streams, other
 * host threads) race on it, so callers must order them.  Nothing needs zeroing
 * between calls. */
#define VMAT_NOALLOC_MAX_ROWS 65536
#define VMAT_NOALLOC_SCRATCH_BYTES ((size_t)VMAT_NOALLOC_MAX_ROWS * 13 + 64)
vmat_status price_apertures_noalloc(const vmat_mlc *mlc, const float *pi, const uint8_t *occupied,
                                    const int16_t *leaves, int32_t *best_cp, int16_t *best_leaves,
                                    double *best_price, void *stream);

/* ---- Apertures <-> beamlets ------------------------------------------------ */

/* DA(A) = sum_{j in A} D_{:,j} (Eq. 5) for the aperture at CP `cp` with
 * leaves (device int16 [n_rows][2]).  da: device float [V], fully written.
 * Needs build_D.  The first call for an MLC shape keeps in the handle a table
 * of where each CP's entries start in every CSR(D) row ((K + 1) x rows 16-bit
 * offsets; cg_plan and batches build it too); it allocates device memory. */
vmat_status aperture_dose(vmat_ddc h, const vmat_mlc *mlc, int32_t cp, const int16_t *leaves, float *da,
                          void *stream);

/* x = A y: x_j = sum of y_n over the apertures n that contain beamlet j (in
 * order of n).  cps: device int32 [n_ap]; leaves: device int16
 * [n_ap][n_rows][2]; y: device float [n_ap]; x: device float [J]. */
vmat_status aperture_fluence(const vmat_mlc *mlc, int32_t n_ap, const int32_t *cps, const int16_t *leaves,
                             const float *y, float *x, void *stream);

/* gy = A^T pi: gy_n = sum of pi over the beamlets of aperture n (FP64
 * accumulation, fixed order).  gy: device float [n_ap]. */
vmat_status aperture_grad(const vmat_mlc *mlc, int32_t n_ap, const int32_t *cps, const int16_t *leaves,
                          const float *pi, float *gy, void *stream);

/* ---- Master problem (Eq. 6-10) -------------------------------------------- */

/* min F(DA y) subject to lo <= y <= hi, by Barzilai-Borwein steps (Eq. 7-8,
 * alternated) with the subspace bound scheme (Eq. 9-10) and the stopping
 * rules of Section 2.1.  DA: device float, column-major [n_ap][ld] (column n
 * = aperture n's dose vector over V voxels, ld >= V).  lo, hi: device float
 * [n_ap] or NULL (0 and +inf).  y: device float [n_ap], warm start in,
 * solution out.  z: device float [V], receives DA y.  opts NULL = defaults
 * (500, 1e-6, 1e-9, 1e-12, 1e12).  rep: HOST struct or NULL.
 * The step lengths, objective and stopping tests use FP64; the products FP32.
 * Synchronises. */
vmat_status mp_bb_solve(const float *DA, int32_t V, int32_t n_ap, int64_t ld, const vmat_voxels *vox,
                        const float *lo, const float *hi, float *y, float *z, const vmat_bb_opts *opts,
                        vmat_bb_report *rep, void *stream);

/* Fluence-rate bounds of Eq. 6 from the delivery limits of Eq. 2, for the
 * apertures placed so far: cps (device int32 [n_ap], distinct CPs; entries < 0
 * are slots not yet placed, which get [0, +inf) and are ignored) and their
 * leaves (device int16 [n_ap][n_rows][2], in the same order).  The gantry speed
 * s_k of a placed CP is the speed from k to the next placed CP k' of its arc,
 * m = k' - k steps: with d the largest leaf move (columns) between the two
 * apertures, s_k <= S^U_{k,k'} = m cp_step_deg leaf_speed_cols / d (no limit if
 * d = 0 or k is the arc's last placed CP).  Speeds of consecutive placed CPs
 * differ by at most m speed_step_max.  S^U_k = min over placed j of the arc of
 * (min(S^U, S^U_{j,j'}) + speed_step_max |k - j|) is the largest speed these
 * constraints allow at k, S^L the smallest; then lo[n] = R^L / S^U_k and
 * hi[n] = R^U / S^L (+inf when S^L = 0), each the float64 quotient rounded to
 * float32.  lo, hi: device float [n_ap].  mlc->machine NULL: [0, +inf).
 * n_ap <= 8192.  Asynchronous on stream. */
vmat_status fluence_bounds(const vmat_mlc *mlc, int32_t n_ap, const int32_t *cps, const int16_t *leaves, float *lo,
                           float *hi, void *stream);

/* ---- Column generation (Section 2.1, Fig. 1a) ---------------------------- */

/* Generate up to n_apertures apertures: repeat { g = -grad F(z); pi = D^T g
 * over unoccupied CPs; best aperture; DA column (Eq. 5); master problem over
 * all apertures (warm start, new y = 0; with mlc->machine, within the bounds
 * fluence_bounds gives for the apertures placed so far) } until n_apertures
 * are generated or the best price is <= 0.  Finally dose = D (A y) in FP32 and F(dose).
 * pi is formed only inside the leaf-travel windows (as beamlet_price_windowed),
 * the only prices pricing reads.  The master problem runs over the 32-voxel
 * tiles that some placed aperture reaches; the other voxels have zero dose for
 * every y, and their penalty enters F as a constant.
 * Outputs may be host or device memory (copied with cudaMemcpyDefault), any
 * may be NULL: cps_out int32 [n_apertures] (unused slots -1), leaves_out
 * int16 [n_apertures][n_rows][2], y_out float [n_apertures], dose_out float
 * [V].  F_out: host double.  stats: host struct or NULL.  Needs build_D and
 * build_Dt.  Synchronises.
 * Device scratch: the call's working arrays (about 2 x the DA matrix plus O(V + J))
 * come from the handle's cache of earlier calls' blocks of the same sizes, else from
 * cudaMalloc, and return to that cache (at most 8 GiB; ddc_free and ddc_build release
 * it) after the call has synchronised its stream.  The first call for an MLC shape
 * also builds the handle's CP tables and, on an autotuned handle, times the windowed
 * D^T g configurations; calls on one handle from several host threads must not
 * overlap.
 * FP32 refinement (BF16 / FP8 handles built with refine_f32): after the last
 * aperture, every placed aperture's dose vector DA (Eq. 5) is recomputed from
 * the FP32 values, the master problem is solved again on those columns (warm
 * start from the plan's y, the same options and bounds), and the final dose
 * D (A y) and F come from the FP32 values.  Pricing stays in the stored type.
 * stats->F_before_refine holds the objective the low-precision master problem
 * reached. */
vmat_status cg_plan(vmat_ddc h, const vmat_mlc *mlc, const vmat_voxels *vox, int32_t n_apertures,
                    const vmat_bb_opts *opts, int32_t *cps_out, int16_t *leaves_out, float *y_out, float *dose_out,
                    double *F_out, vmat_plan_stats *stats, void *stream);

/* ---- Batched plans (independent plans advanced together) ----------------- */

/* One plan of a batch.  ddc: built with CSR(D) and CSR(D^T); every plan of a
 * batch stores its values in the same type.  mlc, vox: as for cg_plan (vox over
 * the plan's V voxels, device arrays).  n_apertures: 0 .. min(K, 96). */
typedef struct {
    vmat_ddc ddc;
    const vmat_mlc *mlc;
    const vmat_voxels *vox;
    int32_t n_apertures;
} vmat_plan_desc;

typedef struct vmat_batch_s *vmat_batch; /* opaque; owns every plan's device state */

typedef struct {
    int32_t n_plans;
    int32_t max_apertures;    /* iterations of the batched loop */
    int32_t spmv_cfg;         /* warp-row SpMV configuration chosen by the autotuner */
    int32_t graph;            /* 1: the run is one CUDA graph launch */
    int64_t graph_nodes;      /* nodes of that graph (0 without a graph) */
    int64_t device_bytes;     /* device memory the batch holds (plan state, tables) */
    double autotune_ms[32];   /* D^T g time of each configuration tried (0 = not a candidate) */
} vmat_batch_info;

/* Column generation (as cg_plan) for n_plans independent plans (1 .. 64)
 * advanced together: iteration t of every plan runs in shared launches (the
 * gradient, D^T g, pricing, the commit, the aperture dose and a persistent
 * master-problem solver whose CTAs are split among the plans), and the whole run
 * is recorded once as a CUDA graph.  Plans with interdigitation set are priced
 * by their own row-chain launches inside that graph; the other plans share one
 * pricing launch.  Plans may differ in MLC, DDC, machine and aperture count, not
 * in the DDC's value type.  The batched D^T g configuration is chosen
 * by timing every warp-row configuration on the batch.  The handles and the
 * descriptors' arrays must stay valid until vmat_batch_free.  opts NULL =
 * defaults.  Synchronises. */
vmat_status vmat_batch_create(int32_t n_plans, const vmat_plan_desc *plans, const vmat_bb_opts *opts, void *stream,
                              vmat_batch *out);

/* Runs every plan once (one graph launch) and synchronises.  F_out: host double
 * [n_plans] or NULL; stats: host [n_plans] or NULL (t_total_ms is the whole
 * batch; phase times are 0). */
vmat_status vmat_batch_run(vmat_batch b, double *F_out, vmat_plan_stats *stats, void *stream);

/* Plan p's results of the last run, as cg_plan's outputs (host or device
 * pointers, any may be NULL).  Synchronises. */
vmat_status vmat_batch_result(vmat_batch b, int32_t p, int32_t *cps_out, int16_t *leaves_out, float *y_out,
                              float *dose_out, void *stream);

vmat_status vmat_batch_info_get(vmat_batch b, vmat_batch_info *info);
vmat_status vmat_batch_free(vmat_batch b);

/* ---- Diagnostics ---------------------------------------------------------- */

/* Message of the last failed call on this thread ("" if none). */
const char *vmat_last_error(void);

/* Device status word (bit 0: a bounded wait ran out; bit 1: an index check
 * failed; bit 2: duplicate COO entry).  reset != 0 clears it.  Synchronises
 * with the device. */
int32_t vmat_device_status(int32_t reset);

/* Library version string. */
const char *vmat_version(void);

/* Number of kernels libvmat has launched in this process (all threads). */
int64_t vmat_launch_count(void);

/* Number of SpMV configurations (valid vmat_build_opts.tile_cfg values are
 * 0 .. count - 1): 0-3 nonzero tiles, 4-8 a warp per row with 4-entry lane
 * chunks, 9-11 a warp per row with consecutive lanes, 12-14 the same reading
 * the 16-bit column index (only where vmat_build_opts.index16 built it). */
int32_t vmat_spmv_config_count(void);

#ifdef __cplusplus
}
#endif

#endif /* VMAT_H */
