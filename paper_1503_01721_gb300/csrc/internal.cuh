// Internal declarations shared by the libvmat translation units (host + device helpers).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <utility>
#include <vector>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/vmat.h"

namespace vmat {

// ---------------------------------------------------------------------------
// Error reporting (host)
// ---------------------------------------------------------------------------
vmat_status set_error(vmat_status st, const char *fmt, ...);
void clear_error();

#define VMAT_CUDA(call)                                                                     \
    do {                                                                                    \
        cudaError_t err__ = (call);                                                         \
        if (err__ != cudaSuccess)                                                           \
            return ::vmat::set_error(err__ == cudaErrorMemoryAllocation ? VMAT_ENOMEM : VMAT_ECUDA, \
                                     "%s failed: %s (%s:%d)", #call, cudaGetErrorString(err__), \
                                     __FILE__, __LINE__);                                  \
    } while (0)

#define VMAT_TRY(expr)                       \
    do {                                     \
        vmat_status st__ = (expr);           \
        if (st__ != VMAT_OK) return st__;    \
    } while (0)

// Kernels launched by this library in this process (each launch site adds one).
extern std::atomic<long long> g_launches;

#define VMAT_LAUNCH_CHECK()                                                  \
    do {                                                                     \
        ::vmat::g_launches.fetch_add(1, std::memory_order_relaxed);          \
        VMAT_CUDA(cudaGetLastError());                                       \
    } while (0)

// Device status word bits (see vmat_device_status).
enum : int32_t { DEV_TIMEOUT = 1, DEV_INDEX = 2, DEV_DUPLICATE = 4 };

// Per-device facts and the device status word.
struct DeviceCtx {
    int device = -1;
    int n_sm = 0;
    int32_t *status = nullptr; // device int32, OR-ed by kernels
};
vmat_status device_ctx(DeviceCtx **out);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Stream-ordered scratch (cudaMallocAsync / cudaFreeAsync).
struct Scratch {
    void *ptr = nullptr;
    cudaStream_t stream = nullptr;
    ~Scratch() {
        if (ptr) cudaFreeAsync(ptr, stream);
    }
    vmat_status alloc(size_t bytes, cudaStream_t s);
};

// Device buffer freed at scope exit unless released (build and set-up steps).
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t b) { return cudaMalloc(&p, b ? b : 16); }
    void *release() {
        void *q = p;
        p = nullptr;
        return q;
    }
};

// ---------------------------------------------------------------------------
// CSR matrix held by a handle
// ---------------------------------------------------------------------------
constexpr int64_t NNZ_PAD = 8192; // value/column arrays padded to a multiple of this

constexpr int ZCHUNK = 128; // entries per chunk of the 16-bit column index

struct CsrMat {
    int32_t n_rows = 0, n_cols = 0;
    int32_t max_row = 0; // longest row
    int64_t nnz = 0, nnz_pad = 0;
    int64_t *rowptr = nullptr;   // [n_rows + 1]
    int32_t *col = nullptr;      // [nnz_pad], padding 0
    void *val = nullptr;         // [nnz_pad] of the stored type, padding 0
    const int32_t *row_ids = nullptr; // output index of each row (CSR(D): compact -> voxel), or null
    // 16-bit column indices, when built: each row is cut into ZCHUNK-entry chunks (from the
    // row's first entry); a chunk stores its first (smallest) column in cbase and every
    // entry its offset from it in col16.  Built only when every chunk spans < 65536 columns.
    uint16_t *col16 = nullptr;   // [nnz_pad], padding 0
    int32_t *cbase = nullptr;    // [n_chunks]
    int64_t *cptr = nullptr;     // [n_rows + 1] first chunk of each row
    int64_t n_chunks = 0;
    // tiles
    int cfg = 0;                 // tile configuration index
    int32_t tile = 0;            // nonzeros per tile
    int32_t n_tiles = 0;
    int32_t *tile_row = nullptr; // [n_tiles + 1]
    float *carry_val = nullptr;  // [n_tiles]
    int32_t *tile_flag = nullptr; // [n_tiles] scratch for active-tile lists
    int32_t *tile_list = nullptr; // [n_tiles]
    int32_t *n_list = nullptr;   // [1]
};

// Brick order of the voxels (build option vox_grid): bricks of 4 x 4 x 2 voxels, one
// 128-byte line of a float vector each, in x-fastest order over the grid padded up to
// whole bricks; inside a brick x fastest, then y, then z.
struct BrickGrid {
    int32_t nx = 0, ny = 0, nz = 0; // 0: voxel order
    int32_t nbx = 0, nby = 0;       // bricks along x and y
    int64_t n_pos = 0;              // positions: whole bricks x 32
    bool on() const { return nx > 0; }
};
__host__ __device__ __forceinline__ int32_t brick_pos(const BrickGrid &b, int32_t v) {
    const int32_t x = v % b.nx, yz = v / b.nx;
    const int32_t y = yz % b.ny, z = yz / b.ny;
    const int32_t brick = ((z >> 1) * b.nby + (y >> 2)) * b.nbx + (x >> 2);
    return brick * 32 + (((z & 1) << 4) | ((y & 3) << 2) | (x & 3));
}

struct Ddc {
    int32_t V = 0, J = 0;
    int64_t nnz = 0;
    int device = -1;
    int32_t *coo_vox = nullptr, *coo_blt = nullptr;
    float *coo_val = nullptr;
    vmat_dtype dtype = VMAT_F32;
    bool built_D = false, built_Dt = false;
    CsrMat D, Dt;
    int32_t n_active = 0;
    int32_t *act_vox = nullptr; // [n_active] compact row -> voxel
    int32_t *vox2act = nullptr; // [V] voxel -> compact row or -1
    // Columns of CSR(D^T) in brick order (BrickGrid) when brick.on(): g vectors for it are
    // indexed by brick_pos, act_gpos maps a compact row to its voxel's position (null: the
    // columns are voxels and act_vox serves)
    BrickGrid brick;
    int32_t *act_gpos = nullptr; // [n_active]
    // SpMV configuration of windowed D^T g passes (ddc_window_config): found for an MLC
    // shape (win_ncols, win_nseg; 0 = none yet) on a handle whose configurations were autotuned
    bool tuned = false;
    int32_t win_cfg = -1, win_ncols = 0, win_nseg = 0;
    // Device blocks (size, pointer) and a pinned host control block of finished cg_plan
    // calls, kept for the next call on this handle (guarded by the plan cache's mutex)
    std::vector<std::pair<size_t, void *>> plan_blocks;
    int32_t *plan_hctl = nullptr;
    // FP32 values of CSR(D) beside the stored BF16 / FP8 ones (build option refine_f32),
    // same order and padding; the FP32 refinement at the end of cg_plan reads them
    float *D_val_f32 = nullptr;
    float *scale = nullptr;     // [J] FP8 per-beamlet scale
    float *xs = nullptr;        // [J] scratch: scaled x for FP8 CSR(D)
    // Offsets of each CP's first entry in each CSR(D) row, [K + 1][n_active], for the
    // aperture dose; built on demand for one MLC shape (cp_tab_bpc beamlets per CP).
    uint16_t *cp_tab = nullptr;
    int32_t cp_tab_K = 0, cp_tab_bpc = 0;
    // CP-major copy of CSR(D) for the aperture dose, built with the CP table: block k holds
    // every compact row's run of CP k's entries, rows in order, each entry as its beamlet's
    // index within the CP (uint16) and its stored value; cpm_base[k * n_grp + g] is the
    // entry where the runs of rows 32 g .. 32 g + 31 start (n_grp = ceil(rows / 32)).  One
    // aperture's dose then reads one contiguous block.  Null when it does not fit in memory.
    uint16_t *cpm_loc = nullptr;
    void *cpm_val = nullptr;
    int64_t *cpm_base = nullptr;
    double build_ms = 0.0;
    void free_all();
};

// Builds (or keeps) the CP offset table of CSR(D) for K CPs of bpc beamlets.  No
// table (and VMAT_OK) when a row is longer than 16-bit offsets reach; the aperture
// dose then searches.  Allocates device memory: not for use while capturing.
vmat_status ddc_cp_table(Ddc &h, int32_t K, int32_t bpc, cudaStream_t s);

inline Ddc *as_ddc(vmat_ddc h) { return reinterpret_cast<Ddc *>(h); }

// Length of a g vector in CSR(D^T)'s column space (act_gpos: where a compact row's g goes).
inline int64_t g_positions(const Ddc &h) { return h.brick.on() ? h.brick.n_pos : (int64_t)h.V; }

// g in CSR(D^T)'s column space: g itself in voxel order, else a brick-ordered copy in
// stream-ordered scratch (ws) written on s.
vmat_status g_for_dt(const Ddc &h, const float *g, Scratch &ws, const float **out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Cross-file entry points (host)
// ---------------------------------------------------------------------------
int value_bytes(vmat_dtype t);

// The rows of a CSR(D^T) pass a caller needs (every row when both pointers are null).
// cp_active: row r belongs to CP r / bpc and is needed only when that CP's flag is set.
// win: row r is beamlet column c = r % n_cols of MLC-row segment q = r / n_cols (CP
// q / n_rows, MLC row q % n_rows) and is needed only when win[q].x <= c < win[q].y:
// the columns that the leaf-travel windows let pricing read (price_windows).
// Rows not needed are not computed: y holds unspecified values there (the tile
// configurations write every row of a tile that holds a needed row).
// woff (may be null, with win): the windows' rows as one list, woff[q] = the rows inside the
// windows of segments 0 .. q - 1 (nseg + 1 entries, window_offsets); the row kernels then
// take list entries in order instead of visiting every row and skipping, so that the
// warps of a launch read neighbouring rows at the same time, as in a full pass.
struct RowMask {
    const uint8_t *cp_active;
    const short2 *win;
    int32_t bpc;
    int32_t n_cols;
    const int32_t *woff;
    int32_t nseg;
};
inline RowMask all_rows() { return RowMask{nullptr, nullptr, 1, 1}; }
__device__ __forceinline__ bool row_needed(const RowMask &m, int64_t r) {
    if (m.cp_active && !m.cp_active[r / m.bpc]) return false;
    if (m.win) {
        const int32_t q = (int32_t)r / m.n_cols, c = (int32_t)r - q * m.n_cols;
        const short2 w = __ldg(m.win + q);
        return c >= w.x && c < w.y;
    }
    return true;
}

// Exclusive scan of the windows' lengths (win[q].y - win[q].x) into woff (nseg + 1
// entries, one block); skip as for the pricing kernels.
vmat_status window_offsets(const short2 *win, int32_t nseg, int32_t *woff, const int32_t *skip, cudaStream_t s);

// SpMV on one CSR; x/y device.  mask: the rows to compute (all_rows(): every row).
// skip (may be null): a device flag; when set at run time the kernels do nothing.
vmat_status spmv_run(const Ddc &h, const CsrMat &m, const float *x, float *y, const float *row_scale, RowMask mask,
                     cudaStream_t s, const int32_t *skip = nullptr);
vmat_status spmv_prepare_tiles(CsrMat &m, int cfg, cudaStream_t s);
// The configuration for D^T g passes over leaf-travel windows of an MLC with n_cols columns and
// nseg = K n_rows rows: the handle's own unless it was autotuned; then every warp-row
// configuration (and the handle's) is timed once on a pass over the middle half of every MLC
// row and the fastest kept for that shape.  Allocates device memory and synchronises the
// first time for a shape: not for use while capturing.
vmat_status ddc_window_config(Ddc &h, int32_t n_cols, int32_t nseg, cudaStream_t s, int *cfg);
// Does configuration cfg read the 16-bit column index (and so need m.col16)?
bool spmv_config_index16(int cfg);
// Builds m.col16 / cbase / cptr when every chunk fits 16 bits (else leaves them null).
vmat_status csr_build_index16(CsrMat &m, int n_sm, cudaStream_t s);
int spmv_n_configs();
int spmv_default_config();
int32_t spmv_config_tile(int cfg);

vmat_status dose_forward_impl(const Ddc &h, const float *x, float *d, bool compact, cudaStream_t s);

// Algorithmic bytes of the matrix part of one SpMV pass over `rows` rows holding
// `nnz` nonzeros and `chunks` 16-bit-index chunks, in the format configuration
// cfg reads: each value (vb bytes) and column index (4, or 2 plus a 4-byte base
// per chunk and an 8-byte chunk pointer per row) once, an 8-byte row pointer
// per row.  Dense inputs, outputs and scales are the caller's.
inline double csr_pass_bytes(int cfg, int vb, double nnz, double rows, double chunks) {
    if (spmv_config_index16(cfg)) return nnz * (vb + 2) + 4.0 * chunks + 16.0 * rows;
    return nnz * (vb + 4) + 8.0 * rows;
}

// ---------------------------------------------------------------------------
// Batched phases: one launch covers every plan of a batch.  Work item g of a
// launch belongs to plan p with off[p] <= g < off[p + 1] (device prefix arrays).
// ---------------------------------------------------------------------------
constexpr int VMAT_MAX_BATCH = 64;

struct SpmvPlan { // one plan's matrix and vectors in a batched warp-row SpMV
    const int64_t *rowptr;
    const int32_t *col;
    const void *val;
    const float *x;
    float *y;
    const float *row_scale; // or null
    const int32_t *row_ids; // or null
    RowMask mask;           // the rows to compute
    const int32_t *skip;    // or null
    int32_t n_rows;
};
bool spmv_batched_config(int cfg);

constexpr int MAX_ARCS = 64;
struct PricingGeom {
    int32_t K, n_rows, n_cols, travel, n_arcs;
    int32_t interdig; // adjacent rows: L_r <= R_{r-1} and L_r <= R_{r+1}
    int32_t arc_first[MAX_ARCS + 1];
};
constexpr int INTERDIG_MAX_COLS = 88; // the chain DP holds (n_cols + 1)^2 states of a row in shared memory
vmat_status pricing_geom(const vmat_mlc *mlc, PricingGeom *g);
size_t pricing_scratch_bytes(const vmat_mlc *mlc);
vmat_status pricing_attributes(); // raises the kernels' shared-memory limits (not a stream operation)
// Leaf-travel windows of every MLC row of every CP (Section 2.2.2, reading R7): win[k *
// n_rows + r] = [Lmin, max(Lmin, Rmax)), the columns any feasible opening of that row
// covers, empty for occupied CPs.  counts (may be null): adds the rows, CSR(D^T)
// nonzeros (rowptr) and 16-bit-index chunks (cptr, may be null) inside the windows to
// counts[0..2].  skip as for the pricing kernels.
vmat_status price_windows(const PricingGeom &g, const uint8_t *occupied, const int16_t *leaves, short2 *win,
                          const int64_t *rowptr, const int64_t *cptr, unsigned long long *counts,
                          const int32_t *skip, cudaStream_t s);
struct WinPlan { // one plan's window inputs and outputs in a batched launch
    PricingGeom g;
    const uint8_t *occupied;
    const int16_t *leaves;
    short2 *win;
    const int64_t *rowptr;
    unsigned long long *counts; // [iterations][3], iteration t at counts + 3 t
    const int32_t *skip;
};
// Iteration t of every plan of a batch (max_K: largest K).
vmat_status price_windows_batched(const WinPlan *plans, int32_t n_plans, int32_t max_K, int32_t t, cudaStream_t s);
// One plan's pricing (either variant) with scratch ws of pricing_scratch_bytes(mlc);
// skip (may be null): a device word, nonzero = leave the outputs untouched.
// ws_has_prefix: ws holds pricing_scratch_bytes_prefix(mlc) bytes, and the row search
// reads prefix sums formed a row per thread (the same values, fewer FP64 instructions).
vmat_status price_apertures_impl(const vmat_mlc *mlc, const float *pi, const uint8_t *occupied, const int16_t *leaves,
                                 int32_t *best_cp, int16_t *best_leaves, double *best_price, void *ws, cudaStream_t s,
                                 const int32_t *skip, bool ws_has_prefix = false);
size_t pricing_scratch_bytes_prefix(const vmat_mlc *mlc);

struct PricePlan { // one plan's pricing inputs, per-row scratch and results
    PricingGeom g;
    const float *pi;
    const uint8_t *occupied;
    const int16_t *leaves;
    double *rb_v;
    int16_t *rb_lr;
    uint8_t *rb_ok;
    int32_t *best_cp;
    int16_t *best_leaves;
    double *best_price;
    const int32_t *skip;
};
// Fluence-rate bounds of Eq. 6 from the delivery limits of Eq. 2 (bounds.cu).
constexpr int BOUNDS_MAX_AP = 8192;
struct BoundsGeom {
    int32_t K, n_rows, n_arcs, has_machine;
    int32_t arc_first[MAX_ARCS + 1];
    double step, s_min, s_max, ds, r_min, r_max, v_leaf;
};
struct BoundsPlan { // one plan's bounds inputs and outputs for the batched kernel
    BoundsGeom g;
    const int32_t *cps;
    const int16_t *leaves;
    float *lo, *hi;
    const int32_t *skip;
};
vmat_status bounds_geom(const vmat_mlc *mlc, BoundsGeom *g);
// lo/hi of the first n slots of (cps, leaves); nothing when *skip != 0.
vmat_status fluence_bounds_enqueue(const BoundsGeom &g, int32_t n, const int32_t *cps, const int16_t *leaves,
                                   float *lo, float *hi, const int32_t *skip, cudaStream_t s);
// One block per plan, the first n slots of each (plans: device array).
vmat_status fluence_bounds_batched(const BoundsPlan *plans, int32_t n_plans, int32_t n, cudaStream_t s);

struct DaPlan { // one plan's CSR(D) and warp-tile DA for the batched aperture dose
    const int64_t *rowptr;
    const int32_t *col;
    const void *val;
    const float *scale; // FP8 column scale, or null
    const uint16_t *cp_tab; // CP offset table of CSR(D) (ddc_cp_table), or null
    int32_t K, n_rrows, n_cols;
    const int32_t *cps;         // the aperture's CP is cps[t]
    const int16_t *leaves;      // its leaves [n_rrows][2]
    float *DA;
    int64_t wstride;
    const int32_t *skip;
};
// off: prefix of the compact row counts over the plans.
vmat_status aperture_dose_batched(vmat_dtype dt, const DaPlan *plans, const int64_t *off, int32_t n_plans,
                                  int64_t total, int32_t t, cudaStream_t s);

struct ObjPlan { // one plan's compact dose and labels for the batched gradient
    const float *z;
    const int32_t *idx;
    const uint8_t *sid;
    const float *T, *wo, *wu;
    float *g_scatter;
    const int32_t *skip;
    const int32_t *gpos; // where g goes in g_scatter (null: at idx, the voxel)
};
vmat_status objective_grad_batched(const ObjPlan *plans, const int64_t *off, int32_t n_plans, int64_t total,
                                   cudaStream_t s);

// off: prefix of K * n_rows over the plans (total entries); max_cols: largest n_cols.
// A plan whose skip word is nonzero, or whose entry range is empty, is left alone
// (interdigitation plans of a batch are priced on their own).
vmat_status price_apertures_batched(const PricePlan *plans, const int64_t *off, int32_t n_plans, int64_t total,
                                    int32_t max_cols, cudaStream_t s);
// cols (host, may be null): the plans' MLC column counts (n_cols entries); the row
// stride is chosen coprime with each so that windowed passes stay balanced.
vmat_status spmv_rows_batched(vmat_dtype dt, int cfg, const SpmvPlan *plans, const int64_t *row_off, int32_t n_plans,
                              int64_t total_rows, cudaStream_t s, const int32_t *cols = nullptr, int n_cols = 0);

// Objective over n voxels.  idx (may be null): voxel i of z is voxel idx[i] of struct_id.
// g_scatter (may be null): write g[i] to g_scatter[idx[i]] instead of g[i].
vmat_status objective_impl(int32_t n, const float *z, const int32_t *idx, const vmat_voxels *vox, float *g,
                           float *g_scatter, double *F, double F_offset, cudaStream_t s);
// The same with caller-owned scratch ws (objective_scratch_bytes) and a skip word.
vmat_status objective_impl_ws(int32_t n, const float *z, const int32_t *idx, const vmat_voxels *vox, float *g,
                              float *g_scatter, double *F, double F_offset, void *ws, cudaStream_t s,
                              const int32_t *skip, const int32_t *gpos = nullptr);
size_t objective_scratch_bytes(int n_sm);
// F0 = the penalty at zero dose of the voxels without DDC entries (their dose is always 0).
vmat_status inactive_objective(const Ddc &h, const vmat_voxels *vox, double *F0, cudaStream_t s);

// compact: write row r of CSR(D) (wstride == 0: at da[r]; else at da[(r / 32) * wstride + (r % 32) * 4],
// the master problem's warp-tile layout with da pointing at the column's first slot);
// otherwise write voxel space da[V] (zero where D has no row).
vmat_status aperture_dose_impl(const Ddc &h, const vmat_mlc *mlc, int32_t cp, const int16_t *leaves, float *da,
                               bool compact, cudaStream_t s, int64_t wstride = 0);
// The same with the CP read from device memory (cp_dev) at run time; skip as for spmv_run.
vmat_status aperture_dose_dev(const Ddc &h, const vmat_mlc *mlc, const int32_t *cp_dev, const int16_t *leaves,
                              float *da, int64_t wstride, const int32_t *skip, cudaStream_t s);

struct BBWork; // defined in mp_bb.cu
// DA layout: column-major (DA[k * ld + i]) when wstride == 0 (copied once, with the
// labels struct_id, into the warp-tile layout), else the warp-tile layout
// DA[(i / 32) * wstride + 32 + (k / 4) * 128 + (i % 32) * 4 + k % 4], wstride = mp_wtile_stride(n_cap),
// whose first 32 bytes of every 32-voxel tile hold the tile's labels (mp_write_labels).
int64_t mp_wtile_stride(int32_t n_cap);
vmat_status mp_write_labels(const uint8_t *sid, int32_t V, int64_t wstride, float *DA, cudaStream_t s);
// Device-driven solve (persistent solver only, n_ap <= n_cap <= 96): no host synchronisation;
// ws holds mp_workspace_bytes(n_cap) bytes; skip and iters_acc as in the solver's arguments.
size_t mp_workspace_bytes(int32_t n_cap);
// Live warp tiles of a plan's master problem.  A voxel that no placed aperture
// reaches has an all-zero row of DA: its dose is 0 whatever y is, and its penalty a
// constant (Eq. 1 at z = 0).  The solver runs over the 32-voxel tiles that some
// placed aperture reaches (in ascending order) and adds the constant of the others.
struct MpLive {
    const float *DA; // the plan's warp-tile DA
    int64_t wstride, n_wtiles;
    uint8_t *flag;        // [n_wtiles] sticky: a placed aperture reaches a voxel of the tile
    const double *c_tile; // [n_wtiles] penalty at zero dose of the tile's voxels (mp_tile_consts)
    int32_t *tiles;       // [n_wtiles] the live tiles, ascending
    int32_t *n_live;      // [1] their number
    double *F_off;        // [1] *F0 + the c_tile of the tiles not live
    const double *F0;     // penalty of the voxels without entries
    const int32_t *skip;  // as for the solver
    int32_t *bcnt;        // [mp_live_blocks(n_wtiles)] scratch: live tiles per block of 1024
    double *bpart;        // [mp_live_blocks(n_wtiles)] scratch: constants of the others per block
    // Packed tiles (all null: the solver reads DA's tiles whole).  gmask[q] bit g: group g
    // (apertures 4g .. 4g + 3) has a nonzero in tile q (sticky).  packed holds every live tile
    // as its 128-byte head (the labels, the group mask at byte 32) followed by its marked
    // groups only (512 bytes each, ascending), live tile i at 128-byte unit poff[i], in list
    // order; poff[n_live] is the total.  Groups left out hold only zeros, whose products
    // add nothing, so the solver's sums are the same bits either way.
    uint32_t *gmask;      // [n_wtiles]
    float *packed;        // [n_wtiles * wstride]
    int32_t *poff;        // [n_wtiles + 1]
    int32_t *bsize;       // [mp_live_blocks(n_wtiles)] scratch: packed units per block
};
constexpr int MP_LIVE_BLOCK = 1024; // tiles per block of the list kernels
__host__ __device__ inline int64_t mp_live_blocks(int64_t n_wtiles) {
    return (n_wtiles + MP_LIVE_BLOCK - 1) / MP_LIVE_BLOCK;
}
vmat_status mp_tile_consts(const uint8_t *sid_c, int32_t NA, const vmat_voxels *vox, int64_t n_wtiles, double *c_tile,
                           cudaStream_t s);
// After column t of DA is written: mark the tiles it reaches, rebuild the list and F_off
// (per-block counts, then ordered writes: the list and the sums are reproducible).
vmat_status mp_live_update(const MpLive &L, int32_t t, cudaStream_t s);
// Copies the live tiles' heads and marked groups into L.packed (L.packed non-null; after
// the list is rebuilt).  The apertures are the first n columns.
vmat_status mp_pack(const MpLive &L, int32_t n, cudaStream_t s);
// The two halves of mp_live_update: mark the tiles column t reaches; rebuild the list and F_off.
vmat_status mp_live_mark(const MpLive &L, int32_t t, cudaStream_t s);
vmat_status mp_live_rebuild(const MpLive &L, cudaStream_t s);
vmat_status mp_live_update_batched(const MpLive *plans, int32_t n_plans, int64_t max_wtiles, int32_t t,
                                   cudaStream_t s);
// live (may be null): solve over the live tiles only, F offset F_offset + *live->F_off.
// bytes_acc (may be null): device double, += the bytes of the solve's passes over DA.
vmat_status mp_bb_enqueue(const float *DA, int32_t V, int32_t n_ap, int32_t n_cap, int64_t wstride,
                          const uint8_t *struct_id, const vmat_voxels *vox, const float *lo, const float *hi, float *y,
                          float *z, const vmat_bb_opts *opts, double F_offset, void *ws, const int32_t *skip,
                          int32_t *iters_acc, cudaStream_t s, const MpLive *live = nullptr,
                          double *bytes_acc = nullptr);
// Batched master problems (persistent solver, one cooperative launch for all plans).
// Per-plan arguments are an opaque mp_args_bytes() record filled by mp_fill_plan_args
// (ws: mp_workspace_bytes(n_cap) bytes); mp_batched_grid gives the launch shape for
// n apertures (every resident CTA; the kernel splits them among the plans).
size_t mp_args_bytes();
vmat_status mp_fill_plan_args(void *out, void *ws, int32_t n_cap, const float *DA, int64_t wstride, int32_t V,
                              const uint8_t *struct_id, const vmat_voxels *vox, const float *lo, const float *hi,
                              float *y, float *z, const vmat_bb_opts *opts, double F_offset, const int32_t *skip,
                              int32_t *iters_acc, const MpLive *live = nullptr);
vmat_status mp_batched_grid(int32_t n, int32_t n_plans, int32_t *grid, int32_t *stages, size_t *smem);
// weight: device [n_plans] (warp tiles of each plan); gctl: device [8] batch barrier, epoch and
// active-set words.
vmat_status mp_bb_enqueue_batched(const void *args, const int64_t *weight, unsigned *gctl, int32_t n_plans, int32_t n,
                                  int32_t grid, int32_t stages, size_t smem, int keep_in_l2, cudaStream_t s);
vmat_status mp_bb_impl(const float *DA, int32_t V, int32_t n_ap, int64_t ld, const uint8_t *struct_id,
                       int64_t wstride, const vmat_voxels *vox, const float *lo, const float *hi, float *y,
                       float *z, const vmat_bb_opts *opts, double F_offset, vmat_bb_report *rep, cudaStream_t s);

vmat_status validate_mlc(const vmat_mlc *mlc);
vmat_status validate_voxels(const vmat_voxels *vox);

// Exclusive scan of int32 counts into int64 offsets (out has n + 1 entries).
vmat_status scan_counts(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);

// Time every SpMV tile configuration on the handle's matrices and keep the fastest.
vmat_status spmv_autotune(Ddc &h, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers: shared-memory addresses, mbarrier and bulk async copy (TMA)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after about `limit_cycles` SM clock cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit_cycles) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > limit_cycles) return false;
    }
}

__device__ __forceinline__ uint64_t l2_evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_evict_last_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 1-D bulk copy global -> shared, completion counted on an mbarrier.
// dst/src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}

constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL; // ~2 s at 2 GHz

// ---------------------------------------------------------------------------
// Device-driven column generation: per-plan control words and the commit step
// ---------------------------------------------------------------------------
enum { CTL_STOPPED = 0, CTL_REASON, CTL_NAP, CTL_BBITERS, CTL_N };

// Commits the aperture priced at iteration t (best_cp, best_leaves), or sets the
// stop flag when no CP has a positive price (Section 2.1).  Called by one block.
__device__ __forceinline__ void commit_aperture_block(int32_t t, int32_t NR, const int32_t *best_cp,
                                                      const double *best_price, const int16_t *best_leaves,
                                                      uint8_t *occupied, uint8_t *active, int16_t *leaves_all,
                                                      int16_t *leaves_seq, int32_t *cps, float *y, int32_t *ctl) {
    if (ctl[CTL_STOPPED]) return;
    const int32_t k = *best_cp;
    const bool stop = k < 0 || !(*best_price > 0.0);
    __syncthreads(); // every thread has read the stop flag before it changes
    if (stop) {
        if (threadIdx.x == 0) {
            ctl[CTL_STOPPED] = 1;
            ctl[CTL_REASON] = VMAT_STOP_PRICE;
        }
        return;
    }
    for (int r = threadIdx.x; r < 2 * NR; r += blockDim.x) {
        leaves_all[(int64_t)k * 2 * NR + r] = best_leaves[r];
        leaves_seq[(int64_t)t * 2 * NR + r] = best_leaves[r];
    }
    if (threadIdx.x == 0) {
        occupied[k] = 1;
        active[k] = 0;
        cps[t] = k;
        y[t] = 0.f;
        ctl[CTL_NAP] = t + 1;
    }
}

} // namespace vmat
