// Batched column generation: many independent plans (Section 2.1, Fig. 1a)
// advanced together.  Iteration t of every plan runs in shared launches:
//   the gradient g = -grad F(z) of every plan's active voxels     (one launch)
//   pi = D^T g over every plan's unoccupied CPs (warp per row)     (one launch)
//   pricing rows of every plan, then one block per plan picks CPs  (two)
//   the commit (or the stop) of every plan                        (one)
//   the new aperture's dose column of every plan (Eq. 5)           (one)
//   the fluence-rate bounds of plans with delivery limits (Eq. 2, 6)  (one)
//   the master problems: one persistent cooperative launch whose
//   CTAs are split among the plans in proportion to their voxels   (two)
// A plan that has all its apertures, or whose best price is <= 0, sets its
// stop flag and every later launch skips its work.  The whole run (state reset,
// the n_max iterations and each plan's final dose) is recorded once as a CUDA
// graph and replayed by vmat_batch_run.  The batched D^T g configuration is
// the fastest warp-row variant on the batch (timed when the batch is made).
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace vmat {


namespace {

struct CommitPlan {
    int32_t NR;
    const int32_t *best_cp;
    const double *best_price;
    const int16_t *best_leaves;
    uint8_t *occupied, *active;
    int16_t *leaves_all, *leaves_seq;
    int32_t *cps;
    float *y;
    int32_t *ctl;
};

__global__ void batch_begin(int32_t t, const int32_t *targets, int32_t *ctl, int32_t n) {
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        int32_t *c = ctl + p * CTL_N;
        if (!c[CTL_STOPPED] && t >= targets[p]) {
            c[CTL_STOPPED] = 1;
            c[CTL_REASON] = VMAT_STOP_COUNT;
        }
    }
}

__global__ void batch_commit(int32_t t, const CommitPlan *plans) {
    const CommitPlan &c = plans[blockIdx.x];
    commit_aperture_block(t, c.NR, c.best_cp, c.best_price, c.best_leaves, c.occupied, c.active, c.leaves_all,
                          c.leaves_seq, c.cps, c.y, c.ctl);
}

__global__ void batch_fill_u8(uint8_t *p, int32_t n, uint8_t v) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

__global__ void batch_fill_i32(int32_t *p, int32_t n, int32_t v) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

__global__ void batch_gather_u8(const uint8_t *src, const int32_t *idx, int32_t n, uint8_t *dst) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

__global__ void batch_cp_offsets(const int64_t *rowptr, int32_t K, int32_t bpc, int64_t *out) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x)
        out[k] = rowptr[(int64_t)k * bpc];
}

struct BPlan {
    Ddc *h = nullptr;
    vmat_mlc mlc = {};
    vmat_machine machine = {}; // the plan's own copy (mlc.machine points here when set)
    std::vector<int32_t> arcs;
    vmat_voxels vox = {}, vox_c = {};
    int32_t n_ap = 0, V = 0, J = 0, K = 0, NR = 0, bpc = 0, NA = 0;
    int64_t n_wtiles = 0, wstride = 0;
    float *z_c = nullptr, *g_full = nullptr, *pi = nullptr, *DA = nullptr, *y = nullptr, *x = nullptr,
          *dose = nullptr, *lo = nullptr, *hi = nullptr;
    uint8_t *occupied = nullptr, *active = nullptr, *sid_c = nullptr;
    int16_t *leaves_all = nullptr, *best_leaves = nullptr, *leaves_seq = nullptr;
    int32_t *best_cp = nullptr, *cps = nullptr, *ctl = nullptr;
    double *best_price = nullptr, *F_dev = nullptr, *F0 = nullptr;
    void *obj_ws = nullptr, *pr_ws = nullptr, *mp_ws = nullptr;
    short2 *win = nullptr;                 // [K * NR] leaf-travel windows of the current iteration
    uint8_t *live_flag = nullptr;          // master-problem live tiles (MpLive)
    double *c_tile = nullptr, *F_off = nullptr;
    int32_t *live_tiles = nullptr, *n_live = nullptr, *live_bcnt = nullptr;
    double *live_bpart = nullptr;
    unsigned long long *wcount = nullptr;  // [iterations][3]: rows, nonzeros (and 0) inside the windows
    double F_offset = 0.0;
    std::vector<int64_t> cpo; // CSR(D^T) rowptr at each CP boundary
};

} // namespace

struct Batch {
    int n = 0;
    vmat_dtype dt = VMAT_F32;
    vmat_bb_opts opts = {500, 1e-6, 1e-9, 1e-12, 1e12};
    int T = 0;
    std::vector<BPlan> P;
    std::vector<void *> allocs;
    int64_t device_bytes = 0;
    SpmvPlan *d_spmv = nullptr;
    int64_t *d_rows_off = nullptr, tot_rows = 0;
    PricePlan *d_price = nullptr;
    int64_t *d_price_off = nullptr, tot_price = 0;
    int32_t max_cols = 1;
    DaPlan *d_da = nullptr;
    ObjPlan *d_obj = nullptr;
    int64_t *d_na_off = nullptr, tot_na = 0;
    CommitPlan *d_commit = nullptr;
    BoundsPlan *d_bounds = nullptr; // null when no plan has a machine
    WinPlan *d_win = nullptr;
    MpLive *d_live = nullptr;
    int64_t max_wtiles = 1;
    int32_t max_K = 1;
    std::vector<int32_t> cols; // the distinct MLC column counts of the plans
    void *d_mpargs = nullptr;
    int64_t *d_weight = nullptr; // [n] warp tiles of each plan (the solver's CTA split)
    unsigned *d_gctl = nullptr;  // [8] batch barrier, epoch and active-set words
    std::vector<int32_t> grid_t, stages_t, keep_t;
    std::vector<size_t> smem_t;
    int32_t *d_ctl = nullptr, *d_targets = nullptr, *h_ctl = nullptr;
    int32_t *d_one = nullptr; // a word holding 1: the batched pricing's skip word of interdigitation plans
    bool any_interdig = false;
    int spmv_cfg = 4;
    double autotune_ms[32] = {0};
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_nodes = 0;
    double last_ms = 0.0;
    bool ran = false;

    ~Batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        if (h_ctl) cudaFreeHost(h_ctl);
        for (void *p : allocs) cudaFree(p);
    }
    template <typename T_> vmat_status get(T_ **out, size_t count) {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(count * sizeof(T_), 16);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess)
            return set_error(e == cudaErrorMemoryAllocation ? VMAT_ENOMEM : VMAT_ECUDA, "vmat_batch: %s",
                             cudaGetErrorString(e));
        allocs.push_back(p);
        device_bytes += (int64_t)bytes;
        *out = static_cast<T_ *>(p);
        return VMAT_OK;
    }
};

// The whole run on stream s: state reset, the batched iterations, final doses.
static vmat_status enqueue_run(Batch &b, cudaStream_t s) {
    const int n = b.n;
    for (BPlan &p : b.P) {
        if (p.NA > 0) VMAT_CUDA(cudaMemsetAsync(p.z_c, 0, (size_t)p.NA * 4, s));
        VMAT_CUDA(cudaMemsetAsync(p.wcount, 0, (size_t)3 * std::max(b.T, 1) * 8, s));
        VMAT_CUDA(cudaMemsetAsync(p.live_flag, 0, (size_t)p.n_wtiles, s));
        VMAT_CUDA(cudaMemsetAsync(p.occupied, 0, p.K, s));
        VMAT_CUDA(cudaMemsetAsync(p.leaves_all, 0, (size_t)p.K * p.NR * 4, s));
        batch_fill_u8<<<std::max(1, (p.K + 255) / 256), 256, 0, s>>>(p.active, p.K, 1);
        VMAT_LAUNCH_CHECK();
        batch_fill_i32<<<1, 256, 0, s>>>(p.cps, std::max(p.n_ap, 1), -1);
        VMAT_LAUNCH_CHECK();
    }
    VMAT_CUDA(cudaMemsetAsync(b.d_ctl, 0, (size_t)n * CTL_N * sizeof(int32_t), s));
    for (int t = 0; t < b.T; ++t) {
        batch_begin<<<1, 64, 0, s>>>(t, b.d_targets, b.d_ctl, n);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(objective_grad_batched(b.d_obj, b.d_na_off, n, b.tot_na, s));
        VMAT_TRY(price_windows_batched(b.d_win, n, b.max_K, t, s));
        VMAT_TRY(spmv_rows_batched(b.dt, b.spmv_cfg, b.d_spmv, b.d_rows_off, n, b.tot_rows, s, b.cols.data(),
                                   (int)b.cols.size()));
        VMAT_TRY(price_apertures_batched(b.d_price, b.d_price_off, n, b.tot_price, b.max_cols, s));
        if (b.any_interdig) // the chain DP over rows (Section 2.2.2), each such plan on its own scratch
            for (BPlan &p : b.P)
                if (p.mlc.interdigitation)
                    VMAT_TRY(price_apertures_impl(&p.mlc, p.pi, p.occupied, p.leaves_all, p.best_cp, p.best_leaves,
                                                  p.best_price, p.pr_ws, s, p.ctl));
        batch_commit<<<n, 128, 0, s>>>(t, b.d_commit);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(aperture_dose_batched(b.dt, b.d_da, b.d_na_off, n, b.tot_na, t, s));
        VMAT_TRY(mp_live_update_batched(b.d_live, n, b.max_wtiles, t, s));
        if (b.d_bounds) VMAT_TRY(fluence_bounds_batched(b.d_bounds, n, t + 1, s));
        VMAT_TRY(mp_bb_enqueue_batched(b.d_mpargs, b.d_weight, b.d_gctl, n, t + 1, b.grid_t[t], b.stages_t[t],
                                       b.smem_t[t], b.keep_t[t], s));
    }
    for (BPlan &p : b.P) { // final dose D (A y) in FP32 and F (apertures not placed have cps = -1)
        VMAT_TRY(aperture_fluence(&p.mlc, std::max(p.n_ap, 0), p.cps, p.leaves_seq, p.y, p.x, s));
        VMAT_TRY(dose_forward_impl(*p.h, p.x, p.dose, false, s));
        VMAT_TRY(objective_impl_ws(p.V, p.dose, nullptr, &p.vox, nullptr, nullptr, p.F_dev, 0.0, p.obj_ws, s, nullptr));
    }
    return VMAT_OK;
}

static vmat_status make_batch(Batch &b, int32_t n_plans, const vmat_plan_desc *plans, const vmat_bb_opts *opts,
                              cudaStream_t s) {
    if (n_plans < 1 || n_plans > VMAT_MAX_BATCH || !plans)
        return set_error(VMAT_EINVAL, "vmat_batch_create: need 1 .. %d plans", VMAT_MAX_BATCH);
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    b.n = n_plans;
    if (opts) b.opts = *opts;
    if (b.opts.max_iter < 1) return set_error(VMAT_EINVAL, "vmat_batch_create: max_iter must be >= 1");
    b.P.resize(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        const vmat_plan_desc &d = plans[i];
        if (!d.ddc || !d.mlc || !d.vox) return set_error(VMAT_EINVAL, "vmat_batch_create: plan %d has a NULL field", i);
        VMAT_TRY(validate_mlc(d.mlc));
        VMAT_TRY(validate_voxels(d.vox));
        Ddc *h = as_ddc(d.ddc);
        if (!h->built_D || !h->built_Dt)
            return set_error(VMAT_ESTATE, "vmat_batch_create: plan %d needs both CSR(D) and CSR(D^T)", i);
        if ((int64_t)d.mlc->K * d.mlc->n_rows * d.mlc->n_cols != h->J)
            return set_error(VMAT_EINVAL, "vmat_batch_create: plan %d: K*n_rows*n_cols != J", i);
        if (d.n_apertures < 0 || d.n_apertures > std::min(d.mlc->K, 96))
            return set_error(VMAT_EINVAL, "vmat_batch_create: plan %d: n_apertures must be in [0, min(K, 96)]", i);
        if (i == 0) b.dt = h->dtype;
        else if (h->dtype != b.dt)
            return set_error(VMAT_EINVAL, "vmat_batch_create: every plan must store its values in the same type");
        BPlan &p = b.P[i];
        p.h = h;
        p.mlc = *d.mlc;
        p.arcs.assign(d.mlc->arc_first_cp, d.mlc->arc_first_cp + d.mlc->n_arcs);
        p.mlc.arc_first_cp = p.arcs.data();
        if (d.mlc->machine) {
            p.machine = *d.mlc->machine;
            p.mlc.machine = &p.machine;
        }
        p.vox = *d.vox;
        p.n_ap = d.n_apertures;
        p.V = h->V;
        p.J = h->J;
        p.K = d.mlc->K;
        p.NR = d.mlc->n_rows;
        p.bpc = d.mlc->n_rows * d.mlc->n_cols;
        p.NA = h->n_active;
        b.any_interdig = b.any_interdig || d.mlc->interdigitation;
        b.T = std::max(b.T, p.n_ap);
        b.max_cols = std::max(b.max_cols, d.mlc->n_cols);
        b.max_K = std::max(b.max_K, d.mlc->K);
        if (std::find(b.cols.begin(), b.cols.end(), d.mlc->n_cols) == b.cols.end()) b.cols.push_back(d.mlc->n_cols);
    }
    if (b.max_cols > 1024) return set_error(VMAT_EUNSUPPORTED, "vmat_batch_create: more than 1024 MLC columns");
    VMAT_CUDA(cudaMallocHost(&b.h_ctl, (size_t)n_plans * CTL_N * sizeof(int32_t)));
    VMAT_CUDA(cudaStreamCreateWithFlags(&b.cs, cudaStreamNonBlocking));
    VMAT_TRY(b.get(&b.d_ctl, (size_t)n_plans * CTL_N));
    VMAT_TRY(b.get(&b.d_targets, n_plans));
    VMAT_TRY(b.get(&b.d_one, 1));
    batch_fill_i32<<<1, 32, 0, s>>>(b.d_one, 1, 1);
    VMAT_LAUNCH_CHECK();

    // ---- per-plan device state and set-up
    std::vector<int64_t *> cpo_dev(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        BPlan &p = b.P[i];
        const int nap = std::max(p.n_ap, 1);
        p.n_wtiles = ((int64_t)std::max(p.NA, 1) + 31) / 32;
        p.wstride = mp_wtile_stride(nap);
        VMAT_TRY(b.get(&p.z_c, std::max(p.NA, 1)));
        VMAT_TRY(b.get(&p.g_full, g_positions(*p.h))); // in CSR(D^T)'s column order
        VMAT_TRY(b.get(&p.pi, p.J));
        VMAT_TRY(b.get(&p.DA, (size_t)p.n_wtiles * p.wstride));
        VMAT_TRY(b.get(&p.y, nap));
        if (p.mlc.machine) {
            VMAT_TRY(b.get(&p.lo, nap));
            VMAT_TRY(b.get(&p.hi, nap));
        }
        VMAT_TRY(b.get(&p.x, p.J));
        VMAT_TRY(b.get(&p.dose, p.V));
        VMAT_TRY(b.get(&p.occupied, p.K));
        VMAT_TRY(b.get(&p.active, p.K));
        VMAT_TRY(b.get(&p.sid_c, std::max(p.NA, 1)));
        VMAT_TRY(b.get(&p.leaves_all, (size_t)p.K * p.NR * 2));
        VMAT_TRY(b.get(&p.best_leaves, (size_t)p.NR * 2));
        VMAT_TRY(b.get(&p.leaves_seq, (size_t)nap * p.NR * 2));
        VMAT_TRY(b.get(&p.best_cp, 2));
        VMAT_TRY(b.get(&p.cps, nap));
        VMAT_TRY(b.get(&p.best_price, 2));
        VMAT_TRY(b.get(&p.F_dev, 2));
        VMAT_TRY(b.get(&p.F0, 2));
        VMAT_TRY(b.get((char **)&p.obj_ws, objective_scratch_bytes(ctx->n_sm)));
        VMAT_TRY(b.get((char **)&p.pr_ws, pricing_scratch_bytes(&p.mlc)));
        VMAT_TRY(b.get((char **)&p.mp_ws, mp_workspace_bytes(std::min(nap, 96))));
        VMAT_TRY(b.get(&cpo_dev[i], (size_t)p.K + 1));
        VMAT_TRY(b.get(&p.win, (size_t)p.K * p.NR));
        VMAT_TRY(b.get(&p.live_flag, (size_t)p.n_wtiles));
        VMAT_TRY(b.get(&p.c_tile, (size_t)p.n_wtiles));
        VMAT_TRY(b.get(&p.live_tiles, (size_t)p.n_wtiles));
        VMAT_TRY(b.get(&p.n_live, 1));
        VMAT_TRY(b.get(&p.F_off, 1));
        VMAT_TRY(b.get(&p.live_bcnt, (size_t)mp_live_blocks(p.n_wtiles)));
        VMAT_TRY(b.get(&p.live_bpart, (size_t)mp_live_blocks(p.n_wtiles)));
        b.max_wtiles = std::max(b.max_wtiles, p.n_wtiles);
        VMAT_TRY(b.get(&p.wcount, (size_t)3 * std::max(b.T, 1)));
        p.ctl = b.d_ctl + (size_t)i * CTL_N;
        // columns not yet generated must read as 0 (later runs overwrite only columns they generate)
        VMAT_CUDA(cudaMemsetAsync(p.DA, 0, (size_t)p.n_wtiles * p.wstride * 4, s));
        VMAT_CUDA(cudaMemsetAsync(p.g_full, 0, (size_t)g_positions(*p.h) * 4, s));
        VMAT_CUDA(cudaMemsetAsync(p.obj_ws, 0, 64, s));
        batch_fill_u8<<<std::max(1, (p.K + 255) / 256), 256, 0, s>>>(p.active, p.K, 1);
        VMAT_LAUNCH_CHECK();
        if (p.NA > 0) {
            batch_gather_u8<<<std::max(1, std::min(ctx->n_sm * 4, (p.NA + 255) / 256)), 256, 0, s>>>(
                p.vox.struct_id, p.h->act_vox, p.NA, p.sid_c);
            VMAT_LAUNCH_CHECK();
            VMAT_TRY(mp_write_labels(p.sid_c, p.NA, p.wstride, p.DA, s));
        }
        VMAT_TRY(mp_tile_consts(p.sid_c, p.NA, &p.vox, p.n_wtiles, p.c_tile, s));
        p.vox_c = p.vox;
        p.vox_c.struct_id = p.sid_c;
        VMAT_TRY(inactive_objective(*p.h, &p.vox, p.F0, s));
        VMAT_TRY(ddc_cp_table(*p.h, p.K, p.bpc, s));
        batch_cp_offsets<<<std::max(1, (p.K + 256) / 256), 256, 0, s>>>(p.h->Dt.rowptr, p.K, p.bpc, cpo_dev[i]);
        VMAT_LAUNCH_CHECK();
    }
    VMAT_CUDA(cudaMemsetAsync(b.d_ctl, 0, (size_t)n_plans * CTL_N * sizeof(int32_t), s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n_plans; ++i) {
        BPlan &p = b.P[i];
        VMAT_CUDA(cudaMemcpy(&p.F_offset, p.F0, sizeof(double), cudaMemcpyDeviceToHost));
        p.cpo.resize(p.K + 1);
        VMAT_CUDA(cudaMemcpy(p.cpo.data(), cpo_dev[i], (size_t)(p.K + 1) * 8, cudaMemcpyDeviceToHost));
    }

    // ---- descriptor tables
    std::vector<SpmvPlan> spmv(n_plans);
    std::vector<PricePlan> price(n_plans);
    std::vector<WinPlan> wins(n_plans);
    std::vector<MpLive> lives(n_plans);
    std::vector<DaPlan> da(n_plans);
    std::vector<ObjPlan> obj(n_plans);
    std::vector<CommitPlan> com(n_plans);
    std::vector<int64_t> rows_off(n_plans + 1, 0), price_off(n_plans + 1, 0), na_off(n_plans + 1, 0);
    std::vector<int32_t> targets(n_plans);
    const size_t argb = mp_args_bytes();
    std::vector<unsigned char> mpargs((size_t)n_plans * argb);
    for (int i = 0; i < n_plans; ++i) {
        BPlan &p = b.P[i];
        const Ddc &h = *p.h;
        const bool fp8 = h.dtype == VMAT_FP8E4M3;
        spmv[i] = SpmvPlan{h.Dt.rowptr, h.Dt.col, h.Dt.val, p.g_full, p.pi, fp8 ? h.scale : nullptr, nullptr,
                           RowMask{nullptr, p.win, p.bpc, p.mlc.n_cols}, p.ctl, h.Dt.n_rows};
        PricePlan &q = price[i];
        VMAT_TRY(pricing_geom(&p.mlc, &q.g));
        wins[i] = WinPlan{q.g, p.occupied, p.leaves_all, p.win, h.Dt.rowptr, p.wcount, p.ctl};
        const bool interdig = p.mlc.interdigitation != 0; // no rows in the shared launch, skipped by its CP kernel
        const int64_t prow = interdig ? 0 : (int64_t)p.K * p.NR;
        q.pi = p.pi;
        q.occupied = p.occupied;
        q.leaves = p.leaves_all;
        q.rb_v = static_cast<double *>(p.pr_ws);
        q.rb_lr = reinterpret_cast<int16_t *>(q.rb_v + prow);
        q.rb_ok = reinterpret_cast<uint8_t *>(q.rb_lr + 2 * prow);
        q.best_cp = p.best_cp;
        q.best_leaves = p.best_leaves;
        q.best_price = p.best_price;
        q.skip = interdig ? b.d_one : p.ctl;
        const bool tab_ok = h.cp_tab && h.cp_tab_K == p.K && h.cp_tab_bpc == p.bpc;
        da[i] = DaPlan{h.D.rowptr, h.D.col, h.D.val, fp8 ? h.scale : nullptr, tab_ok ? h.cp_tab : nullptr, p.K, p.NR,
                       p.mlc.n_cols, p.cps,
                       p.best_leaves, p.DA, p.wstride, p.ctl};
        obj[i] = ObjPlan{p.z_c, h.act_vox, p.vox.struct_id, p.vox.T, p.vox.w_over, p.vox.w_under, p.g_full, p.ctl,
                         h.act_gpos};
        com[i] = CommitPlan{p.NR, p.best_cp, p.best_price, p.best_leaves, p.occupied, p.active, p.leaves_all,
                            p.leaves_seq, p.cps, p.y, p.ctl};
        rows_off[i + 1] = rows_off[i] + h.Dt.n_rows;
        price_off[i + 1] = price_off[i] + prow;
        na_off[i + 1] = na_off[i] + p.NA;
        targets[i] = p.n_ap;
        lives[i] = MpLive{p.DA, p.wstride, p.n_wtiles, p.live_flag, p.c_tile, p.live_tiles, p.n_live, p.F_off, p.F0,
                          p.ctl, p.live_bcnt, p.live_bpart};
        // over the live tiles; F_off holds F0 and the constant of the other tiles
        VMAT_TRY(mp_fill_plan_args(mpargs.data() + (size_t)i * argb, p.mp_ws, std::min(std::max(p.n_ap, 1), 96), p.DA,
                                   p.wstride, p.NA, p.sid_c, &p.vox_c, p.lo, p.hi, p.y, p.z_c, &b.opts, 0.0, p.ctl,
                                   p.ctl + CTL_BBITERS, &lives[i]));
    }
    b.tot_rows = rows_off[n_plans];
    b.tot_price = price_off[n_plans];
    b.tot_na = na_off[n_plans];
    VMAT_TRY(b.get(&b.d_spmv, n_plans));
    VMAT_TRY(b.get(&b.d_price, n_plans));
    VMAT_TRY(b.get(&b.d_win, n_plans));
    VMAT_TRY(b.get(&b.d_live, n_plans));
    VMAT_TRY(b.get(&b.d_da, n_plans));
    VMAT_TRY(b.get(&b.d_obj, n_plans));
    VMAT_TRY(b.get(&b.d_commit, n_plans));
    VMAT_TRY(b.get(&b.d_rows_off, n_plans + 1));
    VMAT_TRY(b.get(&b.d_price_off, n_plans + 1));
    VMAT_TRY(b.get(&b.d_na_off, n_plans + 1));
    VMAT_TRY(b.get((char **)&b.d_mpargs, (size_t)n_plans * argb));
    VMAT_CUDA(cudaMemcpy(b.d_spmv, spmv.data(), n_plans * sizeof(SpmvPlan), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_price, price.data(), n_plans * sizeof(PricePlan), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_win, wins.data(), n_plans * sizeof(WinPlan), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_live, lives.data(), n_plans * sizeof(MpLive), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_da, da.data(), n_plans * sizeof(DaPlan), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_obj, obj.data(), n_plans * sizeof(ObjPlan), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_commit, com.data(), n_plans * sizeof(CommitPlan), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_rows_off, rows_off.data(), (n_plans + 1) * 8, cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_price_off, price_off.data(), (n_plans + 1) * 8, cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_na_off, na_off.data(), (n_plans + 1) * 8, cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_mpargs, mpargs.data(), (size_t)n_plans * argb, cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemcpy(b.d_targets, targets.data(), n_plans * 4, cudaMemcpyHostToDevice));
    bool any_machine = false;
    std::vector<BoundsPlan> bounds(n_plans);
    for (int i = 0; i < n_plans; ++i) {
        BPlan &p = b.P[i];
        bounds[i] = BoundsPlan{};
        if (!p.mlc.machine) continue; // lo == NULL: the kernel skips this plan
        VMAT_TRY(bounds_geom(&p.mlc, &bounds[i].g));
        bounds[i].cps = p.cps;
        bounds[i].leaves = p.leaves_seq;
        bounds[i].lo = p.lo;
        bounds[i].hi = p.hi;
        bounds[i].skip = p.ctl;
        any_machine = true;
    }
    if (any_machine) {
        VMAT_TRY(b.get(&b.d_bounds, n_plans));
        VMAT_CUDA(cudaMemcpy(b.d_bounds, bounds.data(), n_plans * sizeof(BoundsPlan), cudaMemcpyHostToDevice));
    }

    // ---- master-problem launch shapes for every aperture count (the kernel splits the CTAs)
    b.grid_t.assign(std::max(b.T, 1), 1);
    b.stages_t.assign(std::max(b.T, 1), 2);
    b.smem_t.assign(std::max(b.T, 1), 0);
    b.keep_t.assign(std::max(b.T, 1), 0);
    std::vector<int64_t> weight(n_plans);
    for (int i = 0; i < n_plans; ++i) weight[i] = b.P[i].n_wtiles;
    for (int t = 0; t < b.T; ++t) {
        int32_t g = 0, st = 0;
        size_t sm = 0;
        VMAT_TRY(mp_batched_grid(t + 1, n_plans, &g, &st, &sm));
        b.grid_t[t] = g;
        b.stages_t[t] = st;
        b.smem_t[t] = sm;
        double da_bytes = 0.0; // DA read by one pass over every plan: keep it in L2 when it fits there
        for (int i = 0; i < n_plans; ++i)
            da_bytes += (double)b.P[i].n_wtiles * (128.0 + 512.0 * ((t + 1 + 3) / 4));
        b.keep_t[t] = da_bytes <= 64.0 * 1024 * 1024 ? 1 : 0;
    }
    VMAT_TRY(b.get(&b.d_weight, n_plans));
    VMAT_TRY(b.get(&b.d_gctl, 8));
    VMAT_CUDA(cudaMemcpy(b.d_weight, weight.data(), n_plans * sizeof(int64_t), cudaMemcpyHostToDevice));
    VMAT_CUDA(cudaMemset(b.d_gctl, 0, 32));

    // ---- autotune the batched D^T g over every warp-row configuration (all CPs active:
    // the windows of the empty state cover every row)
    for (BPlan &p : b.P) {
        VMAT_CUDA(cudaMemsetAsync(p.occupied, 0, p.K, s));
        VMAT_CUDA(cudaMemsetAsync(p.ctl, 0, CTL_N * sizeof(int32_t), s));
    }
    VMAT_TRY(price_windows_batched(b.d_win, n_plans, b.max_K, 0, s));
    {
        cudaEvent_t e0, e1;
        VMAT_CUDA(cudaEventCreate(&e0));
        VMAT_CUDA(cudaEventCreate(&e1));
        float best = 1e30f;
        for (int cfg = 0; cfg < spmv_n_configs() && cfg < 32; ++cfg) {  // warp-row families only
            if (!spmv_batched_config(cfg)) continue;
            VMAT_TRY(spmv_rows_batched(b.dt, cfg, b.d_spmv, b.d_rows_off, n_plans, b.tot_rows, s, b.cols.data(),
                                       (int)b.cols.size())); // warm-up
            VMAT_CUDA(cudaEventRecord(e0, s));
            VMAT_TRY(spmv_rows_batched(b.dt, cfg, b.d_spmv, b.d_rows_off, n_plans, b.tot_rows, s, b.cols.data(),
                                       (int)b.cols.size()));
            VMAT_CUDA(cudaEventRecord(e1, s));
            VMAT_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            VMAT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            b.autotune_ms[cfg] = ms;
            if (ms < best) {
                best = ms;
                b.spmv_cfg = cfg;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }

    // ---- record the run as a CUDA graph (on a private stream); without it, runs enqueue directly
    {
        cudaGraph_t g = nullptr;
        VMAT_TRY(pricing_attributes()); // function attributes are set outside the capture
        VMAT_CUDA(cudaStreamBeginCapture(b.cs, cudaStreamCaptureModeThreadLocal));
        const vmat_status st = enqueue_run(b, b.cs);
        const cudaError_t ec = cudaStreamEndCapture(b.cs, &g);
        if (st == VMAT_OK && ec == cudaSuccess && g) {
            cudaGraphExec_t ex = nullptr;
            if (cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                b.graph = g;
                b.exec = ex;
                size_t nn = 0;
                cudaGraphGetNodes(g, nullptr, &nn);
                b.graph_nodes = (int64_t)nn;
            } else {
                cudaGraphDestroy(g);
            }
        } else if (g) {
            cudaGraphDestroy(g);
        }
        cudaGetLastError(); // a failed capture leaves no device fault; the eager path is used instead
        clear_error();
    }
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" {

vmat_status vmat_batch_create(int32_t n_plans, const vmat_plan_desc *plans, const vmat_bb_opts *opts, void *stream,
                              vmat_batch *out) {
    clear_error();
    if (!out) return set_error(VMAT_EINVAL, "vmat_batch_create: out is NULL");
    *out = nullptr;
    Batch *b = new Batch();
    const vmat_status st = make_batch(*b, n_plans, plans, opts, as_stream(stream));
    if (st != VMAT_OK) {
        delete b;
        return st;
    }
    *out = reinterpret_cast<vmat_batch>(b);
    return VMAT_OK;
}

vmat_status vmat_batch_run(vmat_batch hb, double *F_out, vmat_plan_stats *stats, void *stream) {
    clear_error();
    if (!hb) return set_error(VMAT_EINVAL, "vmat_batch_run: batch is NULL");
    Batch &b = *reinterpret_cast<Batch *>(hb);
    cudaStream_t s = as_stream(stream);
    const long long launches0 = g_launches.load();
    cudaEvent_t t0, t1;
    VMAT_CUDA(cudaEventCreate(&t0));
    VMAT_CUDA(cudaEventCreate(&t1));
    VMAT_CUDA(cudaEventRecord(t0, s));
    if (b.exec) {
        VMAT_CUDA(cudaGraphLaunch(b.exec, s));
    } else {
        VMAT_TRY(enqueue_run(b, s));
    }
    VMAT_CUDA(cudaEventRecord(t1, s));
    VMAT_CUDA(cudaMemcpyAsync(b.h_ctl, b.d_ctl, (size_t)b.n * CTL_N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    b.last_ms = ms;
    b.ran = true;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    int32_t dev_status = 0;
    VMAT_CUDA(cudaMemcpy(&dev_status, ctx->status, 4, cudaMemcpyDeviceToHost));
    if (dev_status & DEV_TIMEOUT) return set_error(VMAT_ETIMEOUT, "vmat_batch_run: a device-side wait ran out");
    const long long launches = g_launches.load() - launches0;
    for (int i = 0; i < b.n; ++i) {
        BPlan &p = b.P[i];
        const int32_t *c = b.h_ctl + (size_t)i * CTL_N;
        if (F_out) VMAT_CUDA(cudaMemcpy(F_out + i, p.F_dev, 8, cudaMemcpyDeviceToHost));
        if (!stats) continue;
        vmat_plan_stats &st = stats[i];
        memset(&st, 0, sizeof(st));
        const int n_ap = c[CTL_NAP];
        const int stop = c[CTL_REASON] ? c[CTL_REASON] : VMAT_STOP_COUNT;
        std::vector<int32_t> cps(std::max(n_ap, 1));
        if (n_ap > 0) VMAT_CUDA(cudaMemcpy(cps.data(), p.cps, (size_t)n_ap * 4, cudaMemcpyDeviceToHost));
        const Ddc &h = *p.h;
        const int vb = value_bytes(h.dtype);
        const bool fp8 = h.dtype == VMAT_FP8E4M3;
        std::vector<unsigned long long> wc((size_t)3 * std::max(p.n_ap, 1));
        VMAT_CUDA(cudaMemcpy(wc.data(), p.wcount, wc.size() * 8, cudaMemcpyDeviceToHost));
        std::vector<char> occ(p.K, 0);
        const int n_pp1 = n_ap + (stop == VMAT_STOP_PRICE ? 1 : 0);
        double pp1 = 0.0, pp1_full = 0.0;
        for (int t = 0; t < n_pp1; ++t) {
            double bb = 4.0 * p.V;
            for (int k = 0; k < p.K; ++k)
                if (!occ[k])
                    bb += (double)(p.cpo[k + 1] - p.cpo[k]) * (vb + 4) + p.bpc * (8.0 + 4.0) + (fp8 ? 4.0 * p.bpc : 0.0);
            pp1_full += bb;
            if (t < std::max(p.n_ap, 1)) {
                const double rows = (double)wc[3 * t], nnz = (double)wc[3 * t + 1];
                pp1 += 4.0 * p.V + 4.0 * p.K * p.NR + nnz * (vb + 4) + rows * (8.0 + 4.0) + (fp8 ? 4.0 * rows : 0.0);
            }
            if (t < n_ap) occ[cps[t]] = 1;
        }
        st.t_total_ms = ms;
        st.pp1_spmv_launches = n_pp1;
        st.pp1_spmv_bytes = pp1;
        st.pp1_full_bytes = pp1_full;
        st.other_spmv_bytes = csr_pass_bytes(h.D.cfg, vb, (double)h.D.nnz, h.D.n_rows + 1.0, (double)h.D.n_chunks) +
                              4.0 * p.J + 4.0 * p.V + (fp8 ? 4.0 * p.J : 0.0);
        st.n_apertures = n_ap;
        st.bb_iters_total = c[CTL_BBITERS];
        st.stop_reason = stop;
        st.kernel_launches = launches;
    }
    return VMAT_OK;
}

vmat_status vmat_batch_result(vmat_batch hb, int32_t i, int32_t *cps_out, int16_t *leaves_out, float *y_out,
                              float *dose_out, void *stream) {
    clear_error();
    if (!hb) return set_error(VMAT_EINVAL, "vmat_batch_result: batch is NULL");
    Batch &b = *reinterpret_cast<Batch *>(hb);
    if (i < 0 || i >= b.n) return set_error(VMAT_EINVAL, "vmat_batch_result: plan %d out of range", i);
    if (!b.ran) return set_error(VMAT_ESTATE, "vmat_batch_result: the batch has not run");
    cudaStream_t s = as_stream(stream);
    BPlan &p = b.P[i];
    const int n_ap = b.h_ctl[(size_t)i * CTL_N + CTL_NAP];
    const int N = p.n_ap;
    if (cps_out && N > 0) VMAT_CUDA(cudaMemcpyAsync(cps_out, p.cps, (size_t)N * 4, cudaMemcpyDefault, s));
    if (leaves_out && N > 0) {
        VMAT_CUDA(cudaMemsetAsync(p.leaves_seq + (size_t)n_ap * p.NR * 2, 0, (size_t)(N - n_ap) * p.NR * 4, s));
        VMAT_CUDA(cudaMemcpyAsync(leaves_out, p.leaves_seq, (size_t)N * p.NR * 4, cudaMemcpyDefault, s));
    }
    if (y_out && N > 0) {
        VMAT_CUDA(cudaMemsetAsync(p.y + n_ap, 0, (size_t)(N - n_ap) * 4, s));
        VMAT_CUDA(cudaMemcpyAsync(y_out, p.y, (size_t)N * 4, cudaMemcpyDefault, s));
    }
    if (dose_out) VMAT_CUDA(cudaMemcpyAsync(dose_out, p.dose, (size_t)p.V * 4, cudaMemcpyDefault, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    return VMAT_OK;
}

vmat_status vmat_batch_info_get(vmat_batch hb, vmat_batch_info *info) {
    clear_error();
    if (!hb || !info) return set_error(VMAT_EINVAL, "vmat_batch_info_get: NULL argument");
    const Batch &b = *reinterpret_cast<const Batch *>(hb);
    memset(info, 0, sizeof(*info));
    info->n_plans = b.n;
    info->max_apertures = b.T;
    info->spmv_cfg = b.spmv_cfg;
    info->graph = b.exec ? 1 : 0;
    info->graph_nodes = b.graph_nodes;
    info->device_bytes = b.device_bytes;
    for (int i = 0; i < 32; ++i) info->autotune_ms[i] = b.autotune_ms[i];
    return VMAT_OK;
}

vmat_status vmat_batch_free(vmat_batch hb) {
    clear_error();
    delete reinterpret_cast<Batch *>(hb);
    return VMAT_OK;
}

} // extern "C"
