// Column generation (Section 2.1, Fig. 1a): starting from z = 0 and no
// apertures, repeat
//   PP1  g = -grad F(z) (Eq. 4) and pi = D^T g over the unoccupied CPs (Eq. 3)
//   PP2  best opening per MLC row, best CP (Section 2.2.2)
//   DA   the new aperture's dose vector (Eq. 5)
//   MP   BB solve over all apertures (Eq. 6-10), warm start, new y = 0
// until n_apertures exist or no CP has a positive price.  Then the final dose
// D (A y) is recomputed in FP32 from the stored matrix and F is evaluated.
//
// Everything stays on the device and the loop is device-driven: a one-thread
// kernel commits each priced aperture (or sets the stop flag when no CP has a
// positive price), the aperture dose kernel reads the chosen CP from device
// memory, and every later kernel returns at once when the stop flag is set.
// The host enqueues the whole plan without waiting on the GPU (up to 96
// apertures; beyond that the host-driven master-problem solver polls).  The
// master problem runs in the compact space of voxels that have at least one
// nonzero (the rows of CSR(D)); the other voxels always receive zero dose, so
// their penalty is a constant added to F.
#include <string.h>

#include <algorithm>
#include <vector>

#include <mutex>

#include "internal.cuh"

namespace vmat {


__global__ void gather_u8(const uint8_t *src, const int32_t *idx, int32_t n, uint8_t *dst) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

__global__ void fill_u8(uint8_t *p, int32_t n, uint8_t v) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

__global__ void fill_i32(int32_t *p, int32_t n, int32_t v) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// Commits the aperture priced at iteration t, or stops the plan when no CP has a
// positive price (Section 2.1).  One block.
__global__ void commit_aperture(int32_t t, int32_t NR, const int32_t *best_cp, const double *best_price,
                                const int16_t *best_leaves, uint8_t *occupied, uint8_t *active, int16_t *leaves_all,
                                int16_t *leaves_seq, int32_t *cps, float *y, int32_t *ctl) {
    commit_aperture_block(t, NR, best_cp, best_price, best_leaves, occupied, active, leaves_all, leaves_seq, cps, y,
                          ctl);
}

// rowptr of CSR(D^T) at the first beamlet of every CP (K + 1 values).
__global__ void cp_offsets(const int64_t *rowptr, int32_t K, int32_t bpc, int64_t *out) {
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x)
        out[k] = rowptr[(int64_t)k * bpc];
}

namespace {

// Device scratch of one cg_plan call.  Blocks come from the handle's cache of earlier calls'
// blocks (same size) when it holds one, else from cudaMalloc; at the end of the call the
// stream is synchronised and the blocks go back to the cache (at most PLAN_CACHE_BYTES in
// all; the rest are freed), so a plan repeated on a handle allocates nothing.
constexpr size_t PLAN_CACHE_BYTES = (size_t)8 << 30;
std::mutex g_plan_cache_mu;

struct DevArena {
    Ddc &h;
    cudaStream_t s;
    std::vector<std::pair<size_t, void *>> got;
    DevArena(Ddc &h_, cudaStream_t s_) : h(h_), s(s_) {}
    ~DevArena() {
        if (got.empty()) return;
        cudaStreamSynchronize(s); // nothing of this call still runs on its blocks
        std::lock_guard<std::mutex> lk(g_plan_cache_mu);
        size_t held = 0;
        for (auto &b : h.plan_blocks) held += b.first;
        for (auto &b : got) {
            if (held + b.first <= PLAN_CACHE_BYTES) {
                h.plan_blocks.push_back(b);
                held += b.first;
            } else {
                cudaFree(b.second);
            }
        }
    }
    template <typename T> vmat_status get(T **out, size_t n) {
        const size_t bytes = std::max<size_t>(n * sizeof(T), 16);
        void *p = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_plan_cache_mu);
            for (size_t i = 0; i < h.plan_blocks.size(); ++i)
                if (h.plan_blocks[i].first == bytes) {
                    p = h.plan_blocks[i].second;
                    h.plan_blocks.erase(h.plan_blocks.begin() + (std::ptrdiff_t)i);
                    break;
                }
        }
        if (!p) {
            cudaError_t e = cudaMalloc(&p, bytes);
            if (e != cudaSuccess)
                return set_error(e == cudaErrorMemoryAllocation ? VMAT_ENOMEM : VMAT_ECUDA, "cg_plan: %s",
                                 cudaGetErrorString(e));
        }
        got.emplace_back(bytes, p);
        *out = static_cast<T *>(p);
        return VMAT_OK;
    }
};

// The handle's pinned control block when no other call holds it, else one of this call's own.
struct HostCtl {
    Ddc &h;
    int32_t *p = nullptr;
    bool own = false;
    explicit HostCtl(Ddc &h_) : h(h_) {}
    vmat_status get() {
        {
            std::lock_guard<std::mutex> lk(g_plan_cache_mu);
            p = h.plan_hctl;
            h.plan_hctl = nullptr;
        }
        if (!p) VMAT_CUDA(cudaMallocHost(&p, CTL_N * sizeof(int32_t)));
        return VMAT_OK;
    }
    ~HostCtl() {
        if (!p) return;
        std::lock_guard<std::mutex> lk(g_plan_cache_mu);
        if (!h.plan_hctl) h.plan_hctl = p;
        else cudaFreeHost(p);
    }
};

struct PhaseTimer {
    bool on;
    cudaStream_t s;
    std::vector<cudaEvent_t> ev;
    std::vector<int> which; // phase index of each (start, end) pair
    explicit PhaseTimer(bool on_, cudaStream_t s_) : on(on_), s(s_) {}
    ~PhaseTimer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
    void mark(int phase) { // start of a phase
        if (!on) return;
        cudaEvent_t a;
        cudaEventCreate(&a);
        cudaEventRecord(a, s);
        ev.push_back(a);
        which.push_back(phase);
    }
    void end() { mark(-1); }
    void accumulate(double *acc) { // acc[phase] += ms between a phase mark and the next mark
        for (size_t i = 0; i + 1 < ev.size(); ++i) {
            if (which[i] < 0) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
            acc[which[i]] += ms;
        }
    }
};

enum { PH_PP1 = 0, PH_SPMV, PH_PP2, PH_DA, PH_MP, PH_FINAL, PH_REFINE, PH_N };

} // namespace

} // namespace vmat

using namespace vmat;

extern "C" vmat_status cg_plan(vmat_ddc hd, const vmat_mlc *mlc, const vmat_voxels *vox, int32_t n_apertures,
                               const vmat_bb_opts *opts, int32_t *cps_out, int16_t *leaves_out, float *y_out,
                               float *dose_out, double *F_out, vmat_plan_stats *stats, void *stream) {
    clear_error();
    if (!hd) return set_error(VMAT_EINVAL, "cg_plan: handle is NULL");
    VMAT_TRY(validate_mlc(mlc));
    VMAT_TRY(validate_voxels(vox));
    Ddc &h = *as_ddc(hd);
    if (!h.built_D || !h.built_Dt) return set_error(VMAT_ESTATE, "cg_plan: needs both CSR(D) and CSR(D^T)");
    if ((int64_t)mlc->K * mlc->n_rows * mlc->n_cols != h.J)
        return set_error(VMAT_EINVAL, "cg_plan: K*n_rows*n_cols != J");
    if (n_apertures < 0 || n_apertures > mlc->K)
        return set_error(VMAT_EINVAL, "cg_plan: n_apertures must be in [0, K] (each CP holds one aperture)");
    if (mlc->machine && n_apertures > BOUNDS_MAX_AP)
        return set_error(VMAT_EINVAL, "cg_plan: at most %d apertures with a machine", BOUNDS_MAX_AP);
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    cudaStream_t s = as_stream(stream);
    const int32_t V = h.V, J = h.J, K = mlc->K, NR = mlc->n_rows, NA = h.n_active;
    const int32_t bpc = NR * mlc->n_cols;
    // DA in the master problem's warp-tile layout (32-voxel tiles: a label head, then
    // the apertures in groups of four interleaved per voxel)
    const int64_t n_wtiles = ((int64_t)std::max(NA, 1) + 31) / 32;
    const int64_t ld = n_wtiles * 32;                                  // voxel slots
    const int64_t wstride = mp_wtile_stride(std::max(n_apertures, 1)); // floats per warp tile
    const int nap_max = std::max(n_apertures, 1);
    const int g256 = std::max(1, ctx->n_sm * 4);

    DevArena ar(h, s);
    float *z_c, *g_full, *pi, *DA, *y, *x, *dose;
    uint8_t *occupied, *active, *sid_c;
    int16_t *leaves_all, *best_leaves, *leaves_seq;
    int32_t *best_cp, *cps_dev;
    double *best_price, *F_dev, *F0;
    void *obj_ws, *pr_ws;
    VMAT_TRY(ar.get(&z_c, std::max(NA, 1)));
    VMAT_TRY(ar.get(&g_full, g_positions(h))); // in CSR(D^T)'s column order
    VMAT_TRY(ar.get(&pi, J));
    VMAT_TRY(ar.get(&DA, (size_t)n_wtiles * wstride));
    VMAT_TRY(ar.get(&y, nap_max));
    VMAT_TRY(ar.get(&x, J));
    VMAT_TRY(ar.get(&dose, V));
    VMAT_TRY(ar.get(&occupied, K));
    VMAT_TRY(ar.get(&active, K));
    VMAT_TRY(ar.get(&sid_c, std::max(NA, 1)));
    VMAT_TRY(ar.get(&leaves_all, (size_t)K * NR * 2));
    VMAT_TRY(ar.get(&best_leaves, (size_t)NR * 2));
    VMAT_TRY(ar.get(&leaves_seq, (size_t)nap_max * NR * 2));
    VMAT_TRY(ar.get(&best_cp, 2));
    VMAT_TRY(ar.get(&cps_dev, nap_max));
    VMAT_TRY(ar.get(&best_price, 2));
    VMAT_TRY(ar.get(&F_dev, 2));
    VMAT_TRY(ar.get(&F0, 2));
    VMAT_TRY(ar.get((char **)&obj_ws, objective_scratch_bytes(ctx->n_sm)));
    VMAT_TRY(ar.get((char **)&pr_ws, pricing_scratch_bytes_prefix(mlc)));
    // leaf-travel windows of every (CP, MLC row) before each D^T g, and the rows,
    // nonzeros and 16-bit-index chunks inside them per pass
    PricingGeom pg;
    VMAT_TRY(pricing_geom(mlc, &pg));
    short2 *win;
    int32_t *woff; // the rows inside the windows as one list (window_offsets)
    unsigned long long *wcount;
    VMAT_TRY(ar.get(&win, (size_t)K * NR));
    VMAT_TRY(ar.get(&woff, (size_t)K * NR + 1));
    VMAT_TRY(ar.get(&wcount, (size_t)3 * nap_max));
    // live tiles of the master problem (the 32-voxel tiles some placed aperture reaches)
    MpLive live;
    uint8_t *live_flag;
    double *c_tile, *F_off;
    int32_t *live_tiles, *n_live;
    VMAT_TRY(ar.get(&live_flag, (size_t)n_wtiles));
    VMAT_TRY(ar.get(&c_tile, (size_t)n_wtiles));
    VMAT_TRY(ar.get(&live_tiles, (size_t)n_wtiles));
    VMAT_TRY(ar.get(&n_live, 1));
    VMAT_TRY(ar.get(&F_off, 1));
    VMAT_TRY(ar.get(&live.bcnt, (size_t)mp_live_blocks(n_wtiles)));
    VMAT_TRY(ar.get(&live.bpart, (size_t)mp_live_blocks(n_wtiles)));
    // the live tiles packed (heads and the four-aperture groups that hold a nonzero)
    VMAT_TRY(ar.get(&live.gmask, (size_t)n_wtiles));
    VMAT_TRY(ar.get(&live.packed, (size_t)n_wtiles * wstride));
    VMAT_TRY(ar.get(&live.poff, (size_t)n_wtiles + 1));
    VMAT_TRY(ar.get(&live.bsize, (size_t)mp_live_blocks(n_wtiles)));
    live.DA = DA;
    live.wstride = wstride;
    live.n_wtiles = n_wtiles;
    live.flag = live_flag;
    live.c_tile = c_tile;
    live.tiles = live_tiles;
    live.n_live = n_live;
    live.F_off = F_off;
    live.F0 = F0;
    live.skip = nullptr;
    const long long launches0 = g_launches.load();
    PhaseTimer tm(stats != nullptr, s);
    cudaEvent_t t0, t1;
    VMAT_CUDA(cudaEventCreate(&t0));
    VMAT_CUDA(cudaEventCreate(&t1));
    VMAT_CUDA(cudaEventRecord(t0, s));

    VMAT_CUDA(cudaMemsetAsync(z_c, 0, (size_t)std::max(NA, 1) * 4, s));
    // columns not yet generated (and voxel slots past the last one) must read as 0
    VMAT_CUDA(cudaMemsetAsync(DA, 0, (size_t)n_wtiles * wstride * 4, s));
    VMAT_CUDA(cudaMemsetAsync(g_full, 0, (size_t)g_positions(h) * 4, s));
    VMAT_CUDA(cudaMemsetAsync(occupied, 0, K, s));
    VMAT_CUDA(cudaMemsetAsync(leaves_all, 0, (size_t)K * NR * 4, s));
    VMAT_CUDA(cudaMemsetAsync(obj_ws, 0, 64, s));
    VMAT_CUDA(cudaMemsetAsync(wcount, 0, (size_t)3 * nap_max * 8, s));
    fill_u8<<<std::max(1, (K + 255) / 256), 256, 0, s>>>(active, K, 1);
    VMAT_LAUNCH_CHECK();
    fill_i32<<<1, 256, 0, s>>>(cps_dev, nap_max, -1);
    VMAT_LAUNCH_CHECK();
    if (NA > 0) {
        gather_u8<<<std::max(1, std::min(g256, (NA + 255) / 256)), 256, 0, s>>>(vox->struct_id, h.act_vox, NA, sid_c);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(mp_write_labels(sid_c, NA, wstride, DA, s));
        VMAT_TRY(mp_tile_consts(sid_c, NA, vox, n_wtiles, c_tile, s));
    }
    VMAT_CUDA(cudaMemsetAsync(live_flag, 0, (size_t)n_wtiles, s));
    VMAT_CUDA(cudaMemsetAsync(live.gmask, 0, (size_t)n_wtiles * sizeof(uint32_t), s));
    VMAT_TRY(inactive_objective(h, vox, F0, s));
    VMAT_TRY(ddc_cp_table(h, K, bpc, s)); // CP offsets of CSR(D) rows for the aperture dose
    double F_offset = 0.0;
    VMAT_CUDA(cudaMemcpyAsync(&F_offset, F0, sizeof(double), cudaMemcpyDeviceToHost, s));
    // nonzeros per CP in CSR(D^T): algorithmic bytes of each pricing pass
    int64_t *cpo_dev;
    VMAT_TRY(ar.get(&cpo_dev, (size_t)K + 1));
    cp_offsets<<<std::max(1, (K + 256) / 256), 256, 0, s>>>(h.Dt.rowptr, K, bpc, cpo_dev);
    VMAT_LAUNCH_CHECK();
    std::vector<int64_t> cpo(K + 1), cco(K + 1, 0); // nonzeros and 16-bit-index chunks before each CP
    VMAT_CUDA(cudaMemcpyAsync(cpo.data(), cpo_dev, (size_t)(K + 1) * 8, cudaMemcpyDeviceToHost, s));
    // the windowed passes' SpMV configuration (autotuned handles: timed once per MLC shape)
    int dt_cfg = h.Dt.cfg;
    VMAT_TRY(ddc_window_config(h, mlc->n_cols, K * NR, s, &dt_cfg));
    CsrMat Dt_win = h.Dt;
    Dt_win.cfg = dt_cfg;
    const bool z_dt = spmv_config_index16(dt_cfg);
    if (z_dt) {
        VMAT_CUDA(cudaStreamSynchronize(s)); // cpo_dev is reused
        cp_offsets<<<std::max(1, (K + 256) / 256), 256, 0, s>>>(h.Dt.cptr, K, bpc, cpo_dev);
        VMAT_LAUNCH_CHECK();
        VMAT_CUDA(cudaMemcpyAsync(cco.data(), cpo_dev, (size_t)(K + 1) * 8, cudaMemcpyDeviceToHost, s));
    }
    VMAT_CUDA(cudaStreamSynchronize(s));
    vmat_voxels vox_c = *vox;
    vox_c.struct_id = sid_c;
    int bb_extra = 0;

    // fluence-rate bounds of the apertures placed so far (Eq. 2, 6), with a machine
    BoundsGeom bg;
    VMAT_TRY(bounds_geom(mlc, &bg));
    float *lo = nullptr, *hi = nullptr;
    if (bg.has_machine) {
        VMAT_TRY(ar.get(&lo, nap_max));
        VMAT_TRY(ar.get(&hi, nap_max));
    }
    int32_t *ctl;
    VMAT_TRY(ar.get(&ctl, CTL_N));
    live.skip = ctl;
    VMAT_CUDA(cudaMemsetAsync(ctl, 0, CTL_N * sizeof(int32_t), s));
    const int n_cap = std::min(std::max(n_apertures, 1), 96);
    void *mp_ws;
    VMAT_TRY(ar.get((char **)&mp_ws, mp_workspace_bytes(n_cap)));
    double *mp_bytes_dev; // bytes the persistent master-problem passes moved
    VMAT_TRY(ar.get(&mp_bytes_dev, 1));
    VMAT_CUDA(cudaMemsetAsync(mp_bytes_dev, 0, sizeof(double), s));
    double mp_bytes_host = 0.0; // the same for host-driven solves (column-major DA, every active voxel)
    int64_t spmv_launches = 0;
    const int vb = value_bytes(h.dtype);
    const double bytes_D_full = csr_pass_bytes(h.D.cfg, vb, (double)h.D.nnz, h.D.n_rows + 1.0, (double)h.D.n_chunks) +
                                4.0 * J + 4.0 * V + (h.dtype == VMAT_FP8E4M3 ? 4.0 * J : 0.0);
    HostCtl hc(h);
    VMAT_TRY(hc.get());
    int32_t *const hctl = hc.p;

    for (int t = 0; t < n_apertures; ++t) {
        if (t + 1 > n_cap) { // past the persistent solver's limit: the host decides whether to go on
            VMAT_CUDA(cudaMemcpyAsync(hctl, ctl, CTL_N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            VMAT_CUDA(cudaStreamSynchronize(s));
            if (hctl[CTL_STOPPED]) break;
        }
        // ---- PP1
        tm.mark(PH_PP1);
        if (NA > 0)
            VMAT_TRY(objective_impl_ws(NA, z_c, h.act_vox, vox, nullptr, g_full, nullptr, 0.0, obj_ws, s, ctl,
                                       h.act_gpos));
        // prices only where pricing reads them: the columns of each row's window
        VMAT_TRY(price_windows(pg, occupied, leaves_all, win, h.Dt.rowptr, z_dt ? h.Dt.cptr : nullptr,
                               t < nap_max ? wcount + 3 * t : nullptr, ctl, s));
        VMAT_TRY(window_offsets(win, K * NR, woff, ctl, s));
        tm.mark(PH_SPMV);
        VMAT_TRY(spmv_run(h, Dt_win, g_full, pi, h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr,
                          RowMask{nullptr, win, bpc, mlc->n_cols, woff, K * NR}, s, ctl));
        ++spmv_launches;
        // ---- PP2, and the commit (or the stop) on the device
        tm.mark(PH_PP2);
        VMAT_TRY(price_apertures_impl(mlc, pi, occupied, leaves_all, best_cp, best_leaves, best_price, pr_ws, s, ctl,
                                      true));
        commit_aperture<<<1, 128, 0, s>>>(t, NR, best_cp, best_price, best_leaves, occupied, active, leaves_all,
                                         leaves_seq, cps_dev, y, ctl);
        VMAT_LAUNCH_CHECK();
        // ---- DA (Eq. 5)
        tm.mark(PH_DA);
        VMAT_TRY(aperture_dose_dev(h, mlc, cps_dev + t, best_leaves, DA + 32 + (size_t)(t >> 2) * 128 + (t & 3),
                                   wstride, ctl, s));
        if (NA > 0) {
            VMAT_TRY(mp_live_update(live, t, s));
            VMAT_TRY(mp_pack(live, t + 1, s));
        }
        // ---- MP (Eq. 6-10)
        tm.mark(PH_MP);
        if (lo) VMAT_TRY(fluence_bounds_enqueue(bg, t + 1, cps_dev, leaves_seq, lo, hi, ctl, s));
        if (NA > 0) {
            if (t + 1 <= n_cap) {
                // over the live tiles; F_off holds F0 and the constant of the other tiles
                VMAT_TRY(mp_bb_enqueue(DA, NA, t + 1, n_cap, wstride, sid_c, &vox_c, lo, hi, y, z_c, opts, 0.0, mp_ws,
                                       ctl, ctl + CTL_BBITERS, s, &live, mp_bytes_dev));
            } else {
                VMAT_CUDA(cudaMemcpyAsync(hctl, ctl, CTL_N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                VMAT_CUDA(cudaStreamSynchronize(s));
                if (!hctl[CTL_STOPPED]) {
                    vmat_bb_report rep;
                    VMAT_TRY(mp_bb_impl(DA, NA, t + 1, ld, sid_c, wstride, &vox_c, lo, hi, y, z_c, opts, F_offset,
                                        &rep, s));
                    bb_extra += rep.iters;
                    mp_bytes_host += (double)rep.iters * (double)NA * (4.0 * (t + 1) + 9.0);
                }
            }
        }
        tm.end();
    }
    // ---- FP32 refinement of a BF16 / FP8 plan: every placed aperture's DA column from the
    // FP32 values of CSR(D), the master problem again from the plan's y, then the final dose
    // from the same values.  hf reads the handle's CSR(D) through those values.
    const bool refine = h.D_val_f32 != nullptr && h.dtype != VMAT_F32 && NA > 0;
    Ddc hf = h;
    if (refine) {
        hf.dtype = VMAT_F32;
        hf.D.val = h.D_val_f32;
        hf.scale = nullptr;
        hf.cpm_loc = nullptr; // the CP-major copy holds the stored values
        hf.cpm_val = nullptr;
        hf.cpm_base = nullptr;
    }
    int refine_extra = 0;
    int32_t *refine_iters = nullptr;
    if (refine) {
        VMAT_TRY(ar.get(&refine_iters, 1));
        VMAT_CUDA(cudaMemsetAsync(refine_iters, 0, sizeof(int32_t), s));
        VMAT_CUDA(cudaMemcpyAsync(hctl, ctl, CTL_N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VMAT_CUDA(cudaStreamSynchronize(s));
        const int n_placed = hctl[CTL_NAP];
        MpLive live_r = live; // runs whether or not the plan stopped on its prices
        live_r.skip = nullptr;
        tm.mark(PH_REFINE);
        // the objective the low-precision master problem reached (its compact dose, plus
        // the constant penalty of the voxels without entries)
        VMAT_TRY(objective_impl(NA, z_c, h.act_vox, vox, nullptr, nullptr, F_dev + 1, F_offset, s));
        for (int t = 0; t < n_placed; ++t) {
            VMAT_TRY(aperture_dose_dev(hf, mlc, cps_dev + t, leaves_seq + (size_t)t * NR * 2,
                                       DA + 32 + (size_t)(t >> 2) * 128 + (t & 3), wstride, nullptr, s));
            VMAT_TRY(mp_live_mark(live_r, t, s)); // FP32 columns can reach tiles an FP8 column rounded to 0
        }
        if (n_placed > 0) {
            VMAT_TRY(mp_live_rebuild(live_r, s));
            VMAT_TRY(mp_pack(live_r, n_placed, s));
            if (n_placed <= n_cap) {
                VMAT_TRY(mp_bb_enqueue(DA, NA, n_placed, n_cap, wstride, sid_c, &vox_c, lo, hi, y, z_c, opts, 0.0,
                                       mp_ws, nullptr, refine_iters, s, &live_r));
            } else {
                vmat_bb_report rep;
                VMAT_TRY(mp_bb_impl(DA, NA, n_placed, ld, sid_c, wstride, &vox_c, lo, hi, y, z_c, opts, F_offset,
                                    &rep, s));
                refine_extra = rep.iters;
            }
        }
        tm.end();
    }
    // ---- final dose D (A y) in FP32 and its objective (apertures not placed have cps = -1)
    tm.mark(PH_FINAL);
    VMAT_TRY(aperture_fluence(mlc, n_apertures, cps_dev, leaves_seq, y, x, s));
    VMAT_TRY(dose_forward_impl(refine ? hf : h, x, dose, false, s));
    VMAT_TRY(objective_impl(V, dose, nullptr, vox, nullptr, nullptr, F_dev, 0.0, s));
    tm.end();
    VMAT_CUDA(cudaEventRecord(t1, s));
    VMAT_CUDA(cudaMemcpyAsync(hctl, ctl, CTL_N * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    const int n_ap = hctl[CTL_NAP];
    const int stop = hctl[CTL_STOPPED] ? hctl[CTL_REASON] : VMAT_STOP_COUNT;
    const int bb_total = hctl[CTL_BBITERS] + bb_extra;
    std::vector<int32_t> cps_host(std::max(n_ap, 1));
    if (n_ap > 0) VMAT_CUDA(cudaMemcpy(cps_host.data(), cps_dev, (size_t)n_ap * 4, cudaMemcpyDeviceToHost));
    // the format's own bytes of each pricing pass (the rows inside the windows, the
    // window table, g once) and of the final D x; pp1_full_bytes: the same passes over
    // every row of the CPs unoccupied at that pass
    double pp1_bytes = 0.0, pp1_full = 0.0, other_bytes = bytes_D_full;
    {
        std::vector<unsigned long long> wc((size_t)3 * nap_max);
        VMAT_CUDA(cudaMemcpy(wc.data(), wcount, wc.size() * 8, cudaMemcpyDeviceToHost));
        const double fp8_row = h.dtype == VMAT_FP8E4M3 ? 4.0 : 0.0;
        std::vector<char> occ(K, 0);
        const int n_pp1 = n_ap + (stop == VMAT_STOP_PRICE ? 1 : 0);
        for (int t = 0; t < n_pp1; ++t) {
            double b = 4.0 * V;
            for (int kk = 0; kk < K; ++kk)
                if (!occ[kk])
                    b += csr_pass_bytes(dt_cfg, vb, (double)(cpo[kk + 1] - cpo[kk]), (double)bpc,
                                        (double)(cco[kk + 1] - cco[kk])) +
                         (4.0 + fp8_row) * bpc;
            pp1_full += b;
            if (t < nap_max) {
                const double rows = (double)wc[3 * t], nnz = (double)wc[3 * t + 1], ch = (double)wc[3 * t + 2];
                pp1_bytes += 4.0 * V + 4.0 * K * NR + csr_pass_bytes(dt_cfg, vb, nnz, rows, ch) +
                             (4.0 + fp8_row) * rows;
            }
            if (t < n_ap) occ[cps_host[t]] = 1;
        }
        spmv_launches = n_pp1;
    }

    if (cps_out) {
        VMAT_CUDA(cudaMemcpyAsync(cps_out, cps_dev, (size_t)std::max(n_apertures, 0) * 4, cudaMemcpyDefault, s));
    }
    if (leaves_out && n_apertures > 0) {
        VMAT_CUDA(cudaMemsetAsync(leaves_seq + (size_t)n_ap * NR * 2, 0, (size_t)(n_apertures - n_ap) * NR * 4, s));
        VMAT_CUDA(cudaMemcpyAsync(leaves_out, leaves_seq, (size_t)n_apertures * NR * 4, cudaMemcpyDefault, s));
    }
    if (y_out && n_apertures > 0) {
        VMAT_CUDA(cudaMemsetAsync(y + n_ap, 0, (size_t)(n_apertures - n_ap) * 4, s));
        VMAT_CUDA(cudaMemcpyAsync(y_out, y, (size_t)n_apertures * 4, cudaMemcpyDefault, s));
    }
    if (dose_out) VMAT_CUDA(cudaMemcpyAsync(dose_out, dose, (size_t)V * 4, cudaMemcpyDefault, s));
    double Fh[2] = {0.0, 0.0}, mp_bytes = 0.0;
    int32_t refine_it = 0;
    VMAT_CUDA(cudaMemcpyAsync(Fh, F_dev, 16, cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaMemcpyAsync(&mp_bytes, mp_bytes_dev, 8, cudaMemcpyDeviceToHost, s));
    if (refine_iters) VMAT_CUDA(cudaMemcpyAsync(&refine_it, refine_iters, 4, cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    if (F_out) *F_out = Fh[0];
    if (stats) {
        double acc[PH_N] = {0};
        tm.accumulate(acc);
        memset(stats, 0, sizeof(*stats));
        float tot = 0.f;
        cudaEventElapsedTime(&tot, t0, t1);
        stats->t_total_ms = tot;
        stats->pp1_spmv_ms = acc[PH_SPMV];
        stats->t_pp1_ms = acc[PH_PP1] + acc[PH_SPMV];
        stats->t_pp2_ms = acc[PH_PP2];
        stats->t_da_ms = acc[PH_DA];
        stats->t_mp_ms = acc[PH_MP];
        stats->t_final_ms = acc[PH_FINAL];
        stats->pp1_spmv_launches = spmv_launches;
        stats->pp1_spmv_bytes = pp1_bytes;
        stats->pp1_full_bytes = pp1_full;
        stats->other_spmv_bytes = other_bytes;
        stats->n_apertures = n_ap;
        stats->bb_iters_total = bb_total;
        stats->stop_reason = stop;
        stats->kernel_launches = g_launches.load() - launches0;
        stats->refined = refine ? 1 : 0;
        stats->refine_bb_iters = refine_it + refine_extra;
        stats->t_refine_ms = acc[PH_REFINE];
        stats->F_before_refine = refine ? Fh[1] : Fh[0];
        stats->mp_bytes = mp_bytes + mp_bytes_host;
        stats->pp1_spmv_cfg = dt_cfg;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    int32_t dev_status = 0;
    VMAT_CUDA(cudaMemcpy(&dev_status, ctx->status, 4, cudaMemcpyDeviceToHost));
    if (dev_status & DEV_TIMEOUT) return set_error(VMAT_ETIMEOUT, "cg_plan: a device-side wait ran out");
    return VMAT_OK;
}
