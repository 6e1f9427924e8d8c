// Error state, per-device context, scratch, prefix scan, validation and the
// handle-level C entry points (ddc_load_coo, ddc_free, ddc_info, diagnostics).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace vmat {

static thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};

vmat_status set_error(vmat_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

void clear_error() { g_last_error.clear(); }

static std::mutex g_ctx_mu;
static std::vector<DeviceCtx *> g_ctx;

vmat_status device_ctx(DeviceCtx **out) {
    int dev = -1;
    VMAT_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_ctx_mu);
    if ((int)g_ctx.size() <= dev) g_ctx.resize(dev + 1, nullptr);
    if (!g_ctx[dev]) {
        auto *c = new DeviceCtx();
        c->device = dev;
        VMAT_CUDA(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev));
        VMAT_CUDA(cudaMalloc(&c->status, sizeof(int32_t)));
        VMAT_CUDA(cudaMemset(c->status, 0, sizeof(int32_t)));
        VMAT_CUDA(cudaDeviceSynchronize());
        g_ctx[dev] = c;
    }
    *out = g_ctx[dev];
    return VMAT_OK;
}

vmat_status Scratch::alloc(size_t bytes, cudaStream_t s) {
    stream = s;
    if (bytes == 0) bytes = 16;
    VMAT_CUDA(cudaMallocAsync(&ptr, bytes, s));
    return VMAT_OK;
}

int value_bytes(vmat_dtype t) { return t == VMAT_F32 ? 4 : (t == VMAT_BF16 ? 2 : 1); }

void Ddc::free_all() {
    auto f = [](void *p) {
        if (p) cudaFree(p);
    };
    f(coo_vox);
    f(coo_blt);
    f(coo_val);
    coo_vox = coo_blt = nullptr;
    coo_val = nullptr;
    for (CsrMat *m : {&D, &Dt}) {
        f(m->rowptr);
        f(m->col);
        f(m->val);
        f(m->tile_row);
        f(m->carry_val);
        f(m->tile_flag);
        f(m->tile_list);
        f(m->n_list);
        f(m->col16);
        f(m->cbase);
        f(m->cptr);
        *m = CsrMat();
    }
    f(act_vox);
    f(vox2act);
    f(act_gpos);
    act_gpos = nullptr;
    brick = BrickGrid();
    tuned = false;
    win_cfg = -1;
    win_ncols = win_nseg = 0;
    for (auto &b : plan_blocks) cudaFree(b.second);
    plan_blocks.clear();
    if (plan_hctl) cudaFreeHost(plan_hctl);
    plan_hctl = nullptr;
    f(D_val_f32);
    D_val_f32 = nullptr;
    f(scale);
    f(xs);
    f(cp_tab);
    cp_tab = nullptr;
    f(cpm_loc);
    f(cpm_val);
    f(cpm_base);
    cpm_loc = nullptr;
    cpm_val = nullptr;
    cpm_base = nullptr;
    cp_tab_K = cp_tab_bpc = 0;
    act_vox = vox2act = nullptr;
    scale = xs = nullptr;
}

// ---------------------------------------------------------------------------
// Exclusive scan: int32 counts -> int64 offsets, out[n] = total.
// Three passes: per-block totals, one-block scan of the totals, block-local scan.
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int64_t off = 0, all = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        if (w < wid) off += warp_tot[w];
        all += warp_tot[w];
    }
    __syncthreads();
    *total = all;
    return off + x - v;
}

__global__ void scan_block_totals(const int32_t *in, int64_t n, int64_t *block_tot) {
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK;
    int64_t s = 0;
    for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) s += in[k];
    }
    int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) block_tot[blockIdx.x] = tot;
}

__global__ void scan_totals(int64_t *block_tot, int64_t nb) {
    // one block: exclusive scan of nb totals in place
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += SCAN_THREADS) {
        int64_t k = base + threadIdx.x;
        int64_t v = k < nb ? block_tot[k] : 0;
        int64_t tot;
        int64_t ex = block_excl_scan(v, &tot);
        if (k < nb) block_tot[k] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void scan_local(const int32_t *in, int64_t n, const int64_t *block_off, int64_t *out) {
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t k = base + i;
        v[i] = k < n ? in[k] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t ex = block_excl_scan(s, &tot) + block_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t k = base + i;
        if (k < n) out[k] = ex;
        ex += v[i];
    }
    if (base <= n - 1 && n - 1 < base + SCAN_ITEMS) out[n] = ex; // thread holding the last item
}

__global__ void scan_write_zero_total(int64_t *out) { out[0] = 0; }

vmat_status scan_counts(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
    if (n == 0) {
        scan_write_zero_total<<<1, 1, 0, s>>>(out);
        VMAT_LAUNCH_CHECK();
        return VMAT_OK;
    }
    int64_t nb = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
    Scratch tot;
    VMAT_TRY(tot.alloc(nb * sizeof(int64_t), s));
    int64_t *bt = (int64_t *)tot.ptr;
    scan_block_totals<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bt);
    VMAT_LAUNCH_CHECK();
    scan_totals<<<1, SCAN_THREADS, 0, s>>>(bt, nb);
    VMAT_LAUNCH_CHECK();
    scan_local<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, bt, out);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status validate_mlc(const vmat_mlc *mlc) {
    if (!mlc) return set_error(VMAT_EINVAL, "mlc is NULL");
    if (mlc->K <= 0 || mlc->n_rows <= 0 || mlc->n_cols <= 0 || mlc->n_cols > 1024 || mlc->travel_cols < 0)
        return set_error(VMAT_EINVAL, "mlc sizes invalid (K=%d n_rows=%d n_cols=%d travel=%d; need n_cols <= 1024)",
                         mlc->K, mlc->n_rows, mlc->n_cols, mlc->travel_cols);
    if ((int64_t)mlc->K * mlc->n_rows * mlc->n_cols > INT32_MAX)
        return set_error(VMAT_EINVAL, "mlc has more than 2^31-1 beamlets");
    if (mlc->interdigitation && mlc->n_cols > INTERDIG_MAX_COLS)
        return set_error(VMAT_EUNSUPPORTED, "mlc: interdigitation needs n_cols <= %d", INTERDIG_MAX_COLS);
    if (mlc->n_arcs <= 0 || !mlc->arc_first_cp || mlc->arc_first_cp[0] != 0)
        return set_error(VMAT_EINVAL, "mlc arcs invalid: need n_arcs >= 1 and arc_first_cp[0] == 0");
    for (int a = 1; a < mlc->n_arcs; ++a)
        if (mlc->arc_first_cp[a] <= mlc->arc_first_cp[a - 1] || mlc->arc_first_cp[a] >= mlc->K)
            return set_error(VMAT_EINVAL, "mlc arc_first_cp must be strictly increasing and < K");
    if (const vmat_machine *m = mlc->machine) {
        const double v[7] = {m->cp_step_deg, m->speed_min, m->speed_max, m->speed_step_max,
                             m->rate_min, m->rate_max, m->leaf_speed_cols};
        for (double x : v)
            if (!std::isfinite(x)) return set_error(VMAT_EINVAL, "machine: every limit must be finite");
        if (!(m->cp_step_deg > 0.0) || !(m->speed_max > 0.0) || !(m->leaf_speed_cols > 0.0))
            return set_error(VMAT_EINVAL, "machine: cp_step_deg, speed_max and leaf_speed_cols must be > 0");
        if (!(m->speed_min >= 0.0 && m->speed_min <= m->speed_max) || !(m->speed_step_max >= 0.0) ||
            !(m->rate_min >= 0.0 && m->rate_min <= m->rate_max))
            return set_error(VMAT_EINVAL, "machine: need 0 <= speed_min <= speed_max, speed_step_max >= 0 and "
                                          "0 <= rate_min <= rate_max");
        // the travel window must be reachable at the slowest gantry speed, so every
        // interval cap is >= speed_min and the bounds stay ordered
        if ((double)mlc->travel_cols * m->speed_min > m->cp_step_deg * m->leaf_speed_cols)
            return set_error(VMAT_EINVAL, "machine: travel_cols * speed_min (%g) exceeds cp_step_deg * "
                                          "leaf_speed_cols (%g)",
                             (double)mlc->travel_cols * m->speed_min, m->cp_step_deg * m->leaf_speed_cols);
    }
    return VMAT_OK;
}

vmat_status validate_voxels(const vmat_voxels *vox) {
    if (!vox || !vox->struct_id || !vox->T || !vox->w_over || !vox->w_under)
        return set_error(VMAT_EINVAL, "voxels: NULL pointer");
    if (vox->n_struct <= 0 || vox->n_struct > 256)
        return set_error(VMAT_EINVAL, "voxels: n_struct must be in [1, 256] (got %d)", vox->n_struct);
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" {

const char *vmat_last_error(void) { return g_last_error.c_str(); }

const char *vmat_version(void) { return "libvmat 0.1 (sm_103a)"; }

int64_t vmat_launch_count(void) { return g_launches.load(); }

int32_t vmat_spmv_config_count(void) { return spmv_n_configs(); }

int32_t vmat_device_status(int32_t reset) {
    DeviceCtx *c = nullptr;
    if (device_ctx(&c) != VMAT_OK) return -1;
    int32_t v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    if (cudaMemcpy(&v, c->status, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    if (reset && cudaMemset(c->status, 0, sizeof(int32_t)) != cudaSuccess) return -1;
    if (reset && cudaDeviceSynchronize() != cudaSuccess) return -1;
    return v;
}

vmat_status ddc_load_coo(int32_t V, int32_t J, int64_t nnz, const int32_t *vox, const int32_t *blt,
                         const float *val, int32_t on_device, void *stream, vmat_ddc *out) {
    clear_error();
    if (!out) return set_error(VMAT_EINVAL, "ddc_load_coo: out is NULL");
    *out = nullptr;
    if (V <= 0 || J <= 0 || nnz < 0)
        return set_error(VMAT_EINVAL, "ddc_load_coo: need V > 0, J > 0, nnz >= 0 (V=%d J=%d nnz=%lld)", V, J,
                         (long long)nnz);
    if (nnz > (int64_t)INT32_MAX * 4)
        return set_error(VMAT_EUNSUPPORTED, "ddc_load_coo: nnz %lld too large", (long long)nnz);
    if (nnz > 0 && (!vox || !blt || !val)) return set_error(VMAT_EINVAL, "ddc_load_coo: NULL array");
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    cudaStream_t s = as_stream(stream);
    Ddc *h = new Ddc();
    h->V = V;
    h->J = J;
    h->nnz = nnz;
    h->device = ctx->device;
    size_t n = (size_t)(nnz > 0 ? nnz : 1);
    cudaError_t e = cudaMalloc(&h->coo_vox, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&h->coo_blt, n * 4);
    if (e == cudaSuccess) e = cudaMalloc(&h->coo_val, n * 4);
    if (e == cudaSuccess && nnz > 0) {
        cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        e = cudaMemcpyAsync(h->coo_vox, vox, nnz * 4, k, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->coo_blt, blt, nnz * 4, k, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->coo_val, val, nnz * 4, k, s);
    }
    if (e != cudaSuccess) {
        h->free_all();
        delete h;
        return set_error(e == cudaErrorMemoryAllocation ? VMAT_ENOMEM : VMAT_ECUDA, "ddc_load_coo: %s",
                         cudaGetErrorString(e));
    }
    *out = reinterpret_cast<vmat_ddc>(h);
    return VMAT_OK;
}

vmat_status ddc_free(vmat_ddc hd) {
    clear_error();
    if (!hd) return VMAT_OK;
    Ddc *h = as_ddc(hd);
    cudaDeviceSynchronize();
    h->free_all();
    delete h;
    return VMAT_OK;
}

vmat_status ddc_info(vmat_ddc hd, vmat_ddc_info *out) {
    clear_error();
    if (!hd || !out) return set_error(VMAT_EINVAL, "ddc_info: NULL argument");
    Ddc *h = as_ddc(hd);
    memset(out, 0, sizeof(*out));
    out->V = h->V;
    out->J = h->J;
    out->nnz = h->nnz;
    out->n_active_vox = h->n_active;
    out->dtype = h->dtype;
    out->built_D = h->built_D;
    out->built_Dt = h->built_Dt;
    out->tile_nnz_D = h->D.tile;
    out->tile_nnz_Dt = h->Dt.tile;
    int vb = value_bytes(h->dtype);
    if (h->built_D) out->bytes_D = h->D.nnz * (int64_t)(vb + 4) + (int64_t)(h->D.n_rows + 1) * 8;
    if (h->built_Dt) out->bytes_Dt = h->Dt.nnz * (int64_t)(vb + 4) + (int64_t)(h->Dt.n_rows + 1) * 8;
    out->build_ms = h->build_ms;
    out->cfg_D = h->D.cfg;
    out->cfg_Dt = h->Dt.cfg;
    out->index16_D = h->D.col16 ? 1 : 0;
    out->index16_Dt = h->Dt.col16 ? 1 : 0;
    for (const CsrMat *m : {&h->D, &h->Dt}) {
        const int64_t b = m->col16 ? m->nnz * 2 + m->n_chunks * 4 + (int64_t)(m->n_rows + 1) * 8 : 0;
        (m == &h->D ? out->bytes16_D : out->bytes16_Dt) = b;
    }
    out->refine_f32 = h->D_val_f32 ? 1 : 0;
    out->vox_brick = h->brick.on() ? 1 : 0;
    return VMAT_OK;
}

} // extern "C"
