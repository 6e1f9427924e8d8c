// Apertures <-> beamlets.
//
// aperture_dose (Eq. 5): DA_i(A) = sum of D_ij over the beamlets j of the
// aperture.  The paper sums COO columns on the CPU (Section 2.2.2) because its
// GPUs only hold D^T.  Here the rows of CSR(D) are sorted by beamlet and the
// beamlets of one CP are a contiguous index range, so one warp per voxel row
// finds the CP's slice (a guessed window, else a binary search) and adds the
// entries whose column lies between the row's leaves (deterministic, no atomics).
//
// aperture_fluence: x = A y (beamlet fluence of a set of weighted apertures).
// aperture_grad:    A^T pi (summed price of each aperture's beamlets).
#include <algorithm>

#include "internal.cuh"

namespace vmat {

template <typename VT> struct StoredVal;
template <> struct StoredVal<float> {
    static __device__ __forceinline__ float get(const void *v, int64_t e) { return static_cast<const float *>(v)[e]; }
};
template <> struct StoredVal<__nv_bfloat16> {
    static __device__ __forceinline__ float get(const void *v, int64_t e) {
        return __uint_as_float((uint32_t) static_cast<const uint16_t *>(v)[e] << 16);
    }
};
template <> struct StoredVal<__nv_fp8_e4m3> {
    static __device__ __forceinline__ float get(const void *v, int64_t e) {
        __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t) static_cast<const uint8_t *>(v)[e], __NV_E4M3);
        return __half2float(*reinterpret_cast<__half *>(&hr));
    }
};

// Start of CP cp's run in row `row` (the row's entries are sorted by beamlet):
// from the offset table when there is one, else a binary search.
__device__ __forceinline__ int64_t cp_run_start(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                const uint16_t *__restrict__ tab, int32_t n_rows, int32_t row,
                                                int32_t cp, int32_t j0) {
    const int64_t s = rowptr[row];
    if (tab) return s + tab[(int64_t)cp * n_rows + row];
    int64_t lo = s, hi = rowptr[row + 1];
    while (lo < hi) { // first entry with column >= j0
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j0) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Sum of D_ij over the beamlets j in [j0, j1) between the leaves of their MLC
// row, in entry order (one thread per voxel row).
template <typename VT>
__device__ __forceinline__ float aperture_row(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                              const void *__restrict__ val, const float *__restrict__ scale,
                                              const uint16_t *__restrict__ tab, int32_t n_rows, int32_t row,
                                              int32_t cp, int32_t n_cols, int32_t j0, int32_t j1,
                                              const int16_t *__restrict__ leaves) {
    float acc = 0.f;
    const int64_t end = rowptr[row + 1];
    for (int64_t e = cp_run_start(rowptr, col, tab, n_rows, row, cp, j0); e < end; ++e) {
        const int32_t j = col[e];
        if (j >= j1) break;
        const int32_t loc = j - j0, r = loc / n_cols, c = loc - r * n_cols;
        if (c >= leaves[2 * r] && c < leaves[2 * r + 1]) {
            float v = StoredVal<VT>::get(val, e);
            if (scale) v *= scale[j];
            acc += v;
        }
    }
    return acc;
}

// Offsets of each CP's first entry in each row (one thread per row, entries in order).
__global__ void build_cp_table(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int32_t n_rows,
                               int32_t K, int32_t bpc, uint16_t *__restrict__ tab) {
    for (int32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < n_rows; row += gridDim.x * blockDim.x) {
        const int64_t s = rowptr[row], e = rowptr[row + 1];
        int32_t k = 0;
        for (int64_t q = s; q < e; ++q) {
            const int32_t cpq = col[q] / bpc;
            for (; k <= cpq && k <= K; ++k) tab[(int64_t)k * n_rows + row] = (uint16_t)(q - s);
        }
        for (; k <= K; ++k) tab[(int64_t)k * n_rows + row] = (uint16_t)(e - s);
    }
}

// Entries of CP k in the 32 rows of group g (a warp per (k, g); lane = row).
__global__ void cpm_group_sizes(const uint16_t *__restrict__ tab, int32_t n_rows, int32_t K, int32_t n_grp,
                                int32_t *__restrict__ gsum) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)K * n_grp) return; // warp-uniform
    const int lane = threadIdx.x & 31;
    const int32_t k = (int32_t)(w / n_grp), g = (int32_t)(w - (int64_t)k * n_grp), row = g * 32 + lane;
    int32_t len = row < n_rows ? (int32_t)tab[(int64_t)(k + 1) * n_rows + row] - (int32_t)tab[(int64_t)k * n_rows + row]
                               : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) len += __shfl_xor_sync(0xffffffffu, len, d);
    if (lane == 0) gsum[w] = len;
}

// Copies CP k's run of each row of group g to the group's place in the CP-major block
// (a warp per (k, g)): the runs of the 32 rows follow each other there; lane l writes
// destination entries l, l + 32, ... (coalesced) and finds each one's row among the
// 32 inclusive run-length prefixes by a 5-step search over the lanes' values.
template <typename VT>
__global__ void cpm_fill(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                         const VT *__restrict__ val, const uint16_t *__restrict__ tab, int32_t n_rows, int32_t K,
                         int32_t bpc, int32_t n_grp, const int64_t *__restrict__ base, uint16_t *__restrict__ loc,
                         VT *__restrict__ cval) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)K * n_grp) return; // warp-uniform
    const int lane = threadIdx.x & 31;
    const int32_t k = (int32_t)(w / n_grp), g = (int32_t)(w - (int64_t)k * n_grp), row = g * 32 + lane;
    int32_t len = 0;
    int64_t src = 0; // where this lane's run starts in CSR(D)
    if (row < n_rows) {
        const int32_t a = tab[(int64_t)k * n_rows + row];
        len = (int32_t)tab[(int64_t)(k + 1) * n_rows + row] - a;
        src = rowptr[row] + a;
    }
    int32_t incl = len; // inclusive scan of the run lengths over the lanes
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
    }
    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const int64_t dst0 = base[w];
    for (int32_t e0 = 0; e0 < total; e0 += 32) { // warp-uniform trip count
        const int32_t e = e0 + lane;
        int r = 0; // the first lane whose inclusive prefix exceeds e
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const int32_t v = __shfl_sync(0xffffffffu, incl, r + st - 1);
            if (v <= e) r += st;
        }
        const int32_t start = __shfl_sync(0xffffffffu, incl - len, r);
        const int64_t s0 = __shfl_sync(0xffffffffu, src, r);
        if (e < total) {
            const int64_t i = s0 + (e - start);
            loc[dst0 + e] = (uint16_t)(col[i] - k * bpc);
            cval[dst0 + e] = val[i];
        }
    }
}

// Builds the CP-major copy (VMAT_OK without one when memory is short).
static vmat_status ddc_cpm_build(Ddc &h, int32_t K, int32_t bpc, cudaStream_t s) {
    if (bpc > 65536) return VMAT_OK; // a beamlet's index within its CP must fit 16 bits
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int32_t n = h.D.n_rows, n_grp = (n + 31) / 32;
    const int64_t n_w = (int64_t)K * n_grp;
    const int vb = value_bytes(h.dtype);
    uint16_t *loc = nullptr;
    void *cval = nullptr;
    int64_t *base = nullptr;
    int32_t *gsum = nullptr;
    auto fail = [&]() {
        cudaGetLastError();
        cudaFree(loc);
        cudaFree(cval);
        cudaFree(base);
        cudaFree(gsum);
        return VMAT_OK; // no room: the aperture dose reads CSR(D) itself
    };
    if (cudaMalloc(&loc, (size_t)std::max<int64_t>(h.D.nnz, 1) * 2) != cudaSuccess) return fail();
    if (cudaMalloc(&cval, (size_t)std::max<int64_t>(h.D.nnz, 1) * vb) != cudaSuccess) return fail();
    if (cudaMalloc(&base, (size_t)(n_w + 1) * 8) != cudaSuccess) return fail();
    if (cudaMalloc(&gsum, (size_t)std::max<int64_t>(n_w, 1) * 4) != cudaSuccess) return fail();
    const unsigned blocks = (unsigned)((n_w * 32 + 255) / 256);
    cpm_group_sizes<<<blocks, 256, 0, s>>>(h.cp_tab, n, K, n_grp, gsum);
    VMAT_LAUNCH_CHECK();
    VMAT_TRY(scan_counts(gsum, base, n_w, s));
    if (h.dtype == VMAT_F32)
        cpm_fill<float><<<blocks, 256, 0, s>>>(h.D.rowptr, h.D.col, static_cast<const float *>(h.D.val), h.cp_tab, n,
                                               K, bpc, n_grp, base, loc, static_cast<float *>(cval));
    else if (h.dtype == VMAT_BF16)
        cpm_fill<uint16_t><<<blocks, 256, 0, s>>>(h.D.rowptr, h.D.col, static_cast<const uint16_t *>(h.D.val),
                                                  h.cp_tab, n, K, bpc, n_grp, base, loc,
                                                  static_cast<uint16_t *>(cval));
    else
        cpm_fill<uint8_t><<<blocks, 256, 0, s>>>(h.D.rowptr, h.D.col, static_cast<const uint8_t *>(h.D.val), h.cp_tab,
                                                 n, K, bpc, n_grp, base, loc, static_cast<uint8_t *>(cval));
    VMAT_LAUNCH_CHECK();
    VMAT_CUDA(cudaStreamSynchronize(s));
    cudaFree(gsum);
    h.cpm_loc = loc;
    h.cpm_val = cval;
    h.cpm_base = base;
    return VMAT_OK;
}

vmat_status ddc_cp_table(Ddc &h, int32_t K, int32_t bpc, cudaStream_t s) {
    if (!h.built_D || h.D.n_rows == 0) return VMAT_OK;
    if (h.cp_tab && h.cp_tab_K == K && h.cp_tab_bpc == bpc) return VMAT_OK;
    if (h.cp_tab) {
        VMAT_CUDA(cudaStreamSynchronize(s));
        cudaFree(h.cp_tab);
        h.cp_tab = nullptr;
        h.cp_tab_K = h.cp_tab_bpc = 0;
        cudaFree(h.cpm_loc);
        cudaFree(h.cpm_val);
        cudaFree(h.cpm_base);
        h.cpm_loc = nullptr;
        h.cpm_val = nullptr;
        h.cpm_base = nullptr;
    }
    if (h.D.max_row > 65535) return VMAT_OK; // offsets would not fit 16 bits: search instead
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    uint16_t *tab = nullptr;
    const cudaError_t e = cudaMalloc(&tab, (size_t)(K + 1) * h.D.n_rows * sizeof(uint16_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VMAT_OK; // no room for the table: the aperture dose searches
    }
    const int grid = std::max(1, std::min(ctx->n_sm * 8, (h.D.n_rows + 255) / 256));
    build_cp_table<<<grid, 256, 0, s>>>(h.D.rowptr, h.D.col, h.D.n_rows, K, bpc, tab);
    VMAT_LAUNCH_CHECK();
    h.cp_tab = tab;
    h.cp_tab_K = K;
    h.cp_tab_bpc = bpc;
    return ddc_cpm_build(h, K, bpc, s);
}

template <typename VT>
__global__ void aperture_dose_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                     const void *__restrict__ val, const float *__restrict__ scale,
                                     const uint16_t *__restrict__ tab, int32_t n_rows,
                                     const int32_t *__restrict__ row_ids, int32_t cp_arg, const int32_t *cp_dev,
                                     const int32_t *skip, int32_t n_rrows, int32_t n_cols,
                                     const int16_t *__restrict__ leaves, float *__restrict__ da, int64_t wstride) {
    if (skip && *skip) return;
    const int32_t cp = cp_dev ? *cp_dev : cp_arg;
    extern __shared__ int16_t sl[]; // [n_rrows][2]
    for (int i = threadIdx.x; i < 2 * n_rrows; i += blockDim.x) sl[i] = leaves[i];
    __syncthreads();
    const int32_t bpc = n_rrows * n_cols;
    const int32_t j0 = cp * bpc, j1 = j0 + bpc;
    for (int32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < n_rows; row += gridDim.x * blockDim.x) {
        const float acc = aperture_row<VT>(rowptr, col, val, scale, tab, n_rows, row, cp, n_cols, j0, j1, sl);
        // output: voxel space, compact row space, or the master problem's warp-tile
        // layout (row r at (r / 32) * wstride + (r % 32) * 4 from da, the column's base)
        const int64_t o =
            row_ids ? row_ids[row] : (wstride ? (int64_t)(row >> 5) * wstride + ((row & 31) << 2) : row);
        da[o] = acc;
    }
}

// The same sums from the CP-major copy: a warp per group of 32 rows, lane = row; the
// group's runs of CP cp are one contiguous block (cpm_base), each lane reads its own run
// (the warp's entries share a few cache lines).  Entries in beamlet order, as above: the
// same bits as aperture_dose_kernel.
template <typename VT>
__global__ void aperture_dose_cpm_kernel(const uint16_t *__restrict__ loc, const void *__restrict__ val,
                                         const int64_t *__restrict__ base, const float *__restrict__ scale,
                                         const uint16_t *__restrict__ tab, int32_t n_rows, int32_t n_grp,
                                         const int32_t *__restrict__ row_ids, int32_t cp_arg, const int32_t *cp_dev,
                                         const int32_t *skip, int32_t n_rrows, int32_t n_cols,
                                         const int16_t *__restrict__ leaves, float *__restrict__ da, int64_t wstride) {
    if (skip && *skip) return;
    const int32_t cp = cp_dev ? *cp_dev : cp_arg;
    extern __shared__ int16_t sl[]; // [n_rrows][2]
    for (int i = threadIdx.x; i < 2 * n_rrows; i += blockDim.x) sl[i] = leaves[i];
    __syncthreads();
    const int32_t bpc = n_rrows * n_cols;
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < n_grp; g += n_warps) {
        const int32_t row = (int32_t)g * 32 + lane;
        int32_t len = 0;
        if (row < n_rows) len = (int32_t)tab[(int64_t)(cp + 1) * n_rows + row] - (int32_t)tab[(int64_t)cp * n_rows + row];
        int32_t incl = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        const int64_t start = base[(int64_t)cp * n_grp + g] + (incl - len);
        float acc = 0.f;
        for (int32_t e = 0; e < len; ++e) {
            const int32_t lc = loc[start + e];
            const int32_t r = lc / n_cols, c = lc - r * n_cols;
            if (c >= sl[2 * r] && c < sl[2 * r + 1]) {
                float v = StoredVal<VT>::get(val, start + e);
                if (scale) v *= scale[(int64_t)cp * bpc + lc];
                acc += v;
            }
        }
        if (row < n_rows) {
            const int64_t o =
                row_ids ? row_ids[row] : (wstride ? (int64_t)(row >> 5) * wstride + ((row & 31) << 2) : row);
            da[o] = acc;
        }
    }
}

using DaFn = void (*)(const int64_t *, const int32_t *, const void *, const float *, const uint16_t *, int32_t,
                      const int32_t *, int32_t, const int32_t *, const int32_t *, int32_t, int32_t, const int16_t *,
                      float *, int64_t);
static DaFn da_kernel_for(vmat_dtype dt) {
    return dt == VMAT_F32 ? aperture_dose_kernel<float>
           : dt == VMAT_BF16 ? aperture_dose_kernel<__nv_bfloat16>
                             : aperture_dose_kernel<__nv_fp8_e4m3>;
}

static vmat_status launch_da(const Ddc &h, const vmat_mlc *mlc, int32_t cp, const int32_t *cp_dev, const int32_t *skip,
                             const int16_t *leaves, float *da, const int32_t *row_ids, int64_t wstride, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int32_t n = h.D.n_rows;
    if (n == 0) return VMAT_OK;
    const int32_t bpc = mlc->n_rows * mlc->n_cols;
    const uint16_t *tab = h.cp_tab && h.cp_tab_K == mlc->K && h.cp_tab_bpc == bpc ? h.cp_tab : nullptr;
    const size_t sl_bytes = (size_t)mlc->n_rows * 2 * sizeof(int16_t);
    if (tab && h.cpm_val) { // the CP-major copy, built with this table
        const int32_t n_grp = (n + 31) / 32;
        const int g = std::max(1, std::min(ctx->n_sm * 16, (n_grp * 32 + 255) / 256));
        const float *sc = h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr;
        if (h.dtype == VMAT_F32)
            aperture_dose_cpm_kernel<float><<<g, 256, sl_bytes, s>>>(h.cpm_loc, h.cpm_val, h.cpm_base, sc, tab, n,
                                                                     n_grp, row_ids, cp, cp_dev, skip, mlc->n_rows,
                                                                     mlc->n_cols, leaves, da, wstride);
        else if (h.dtype == VMAT_BF16)
            aperture_dose_cpm_kernel<__nv_bfloat16><<<g, 256, sl_bytes, s>>>(
                h.cpm_loc, h.cpm_val, h.cpm_base, sc, tab, n, n_grp, row_ids, cp, cp_dev, skip, mlc->n_rows,
                mlc->n_cols, leaves, da, wstride);
        else
            aperture_dose_cpm_kernel<__nv_fp8_e4m3><<<g, 256, sl_bytes, s>>>(
                h.cpm_loc, h.cpm_val, h.cpm_base, sc, tab, n, n_grp, row_ids, cp, cp_dev, skip, mlc->n_rows,
                mlc->n_cols, leaves, da, wstride);
        VMAT_LAUNCH_CHECK();
        return VMAT_OK;
    }
    const int grid = std::max(1, std::min(ctx->n_sm * 8, (n + 255) / 256));
    da_kernel_for(h.dtype)<<<grid, 256, sl_bytes, s>>>(
        h.D.rowptr, h.D.col, h.D.val, h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr, tab, n, row_ids, cp, cp_dev, skip,
        mlc->n_rows, mlc->n_cols, leaves, da, wstride);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

// Batched Eq. 5 for aperture t of every plan: global row g is compact row g - off[p]
// of plan p; the CP is cps[t] and the leaves best_leaves (device), the column goes
// to the plan's warp-tile DA.  One thread per row, plan looked up by binary search.
template <typename VT>
__global__ void aperture_dose_batched_kernel(const DaPlan *__restrict__ plans, const int64_t *__restrict__ off,
                                             int32_t n_plans, int64_t total, int32_t t) {
    __shared__ int64_t soff[VMAT_MAX_BATCH + 1];
    for (int i = threadIdx.x; i <= n_plans; i += blockDim.x) soff[i] = off[i];
    __syncthreads();
    for (int64_t gr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gr < total;
         gr += (int64_t)gridDim.x * blockDim.x) {
        int a = 0, b = n_plans;
        while (b - a > 1) {
            const int m = (a + b) >> 1;
            if (soff[m] <= gr) a = m;
            else b = m;
        }
        const DaPlan &P = plans[a];
        if (P.skip && *P.skip) continue;
        const int32_t row = (int32_t)(gr - soff[a]);
        const int32_t n_rows = (int32_t)(soff[a + 1] - soff[a]);
        const int32_t bpc = P.n_rrows * P.n_cols;
        const int32_t cp = P.cps[t];
        const int32_t j0 = cp * bpc;
        const float acc = aperture_row<VT>(P.rowptr, P.col, P.val, P.scale, P.cp_tab, n_rows, row, cp, P.n_cols, j0,
                                           j0 + bpc, P.leaves);
        P.DA[32 + (int64_t)(t >> 2) * 128 + (t & 3) + (int64_t)(row >> 5) * P.wstride + ((row & 31) << 2)] = acc;
    }
}

vmat_status aperture_dose_batched(vmat_dtype dt, const DaPlan *plans, const int64_t *off, int32_t n_plans,
                                  int64_t total, int32_t t, cudaStream_t s) {
    if (total <= 0) return VMAT_OK;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)ctx->n_sm * 8));
    if (dt == VMAT_F32) aperture_dose_batched_kernel<float><<<grid, 256, 0, s>>>(plans, off, n_plans, total, t);
    else if (dt == VMAT_BF16)
        aperture_dose_batched_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(plans, off, n_plans, total, t);
    else aperture_dose_batched_kernel<__nv_fp8_e4m3><<<grid, 256, 0, s>>>(plans, off, n_plans, total, t);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status aperture_dose_impl(const Ddc &h, const vmat_mlc *mlc, int32_t cp, const int16_t *leaves, float *da,
                               bool compact, cudaStream_t s, int64_t wstride) {
    if (!compact) VMAT_CUDA(cudaMemsetAsync(da, 0, (size_t)h.V * 4, s));
    return launch_da(h, mlc, cp, nullptr, nullptr, leaves, da, compact ? nullptr : h.D.row_ids, compact ? wstride : 0, s);
}

vmat_status aperture_dose_dev(const Ddc &h, const vmat_mlc *mlc, const int32_t *cp_dev, const int16_t *leaves,
                              float *da, int64_t wstride, const int32_t *skip, cudaStream_t s) {
    return launch_da(h, mlc, 0, cp_dev, skip, leaves, da, nullptr, wstride, s);
}

// x_j = sum over apertures n (in order) containing beamlet j of y_n.
__global__ void aperture_fluence_kernel(int32_t J, int32_t n_rrows, int32_t n_cols, int32_t n_ap,
                                        const int32_t *__restrict__ cps, const int16_t *__restrict__ leaves,
                                        const float *__restrict__ y, float *__restrict__ x) {
    const int32_t bpc = n_rrows * n_cols;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
        const int32_t k = j / bpc, loc = j - k * bpc, r = loc / n_cols, c = loc - r * n_cols;
        float acc = 0.f;
        for (int32_t n = 0; n < n_ap; ++n) {
            if (cps[n] != k) continue;
            const int64_t o = ((int64_t)n * n_rrows + r) * 2;
            if (c >= leaves[o] && c < leaves[o + 1]) acc += y[n];
        }
        x[j] = acc;
    }
}

// gy_n = sum of pi over aperture n's beamlets; rows summed in column order, then
// a fixed-order FP64 tree over rows.
__global__ void aperture_grad_kernel(int32_t K, int32_t n_rrows, int32_t n_cols, const int32_t *__restrict__ cps,
                                     const int16_t *__restrict__ leaves, const float *__restrict__ pi,
                                     float *__restrict__ gy, int32_t *status) {
    __shared__ double sh[256];
    const int32_t n = blockIdx.x;
    const int32_t k = cps[n];
    if (k < 0 || k >= K) { // index check: record it and give this aperture 0
        if (threadIdx.x == 0) {
            atomicOr(status, DEV_INDEX);
            gy[n] = 0.f;
        }
        return;
    }
    double acc = 0.0;
    for (int r = threadIdx.x; r < n_rrows; r += blockDim.x) {
        const int64_t o = ((int64_t)n * n_rrows + r) * 2;
        const float *row = pi + ((int64_t)k * n_rrows + r) * n_cols;
        double s = 0.0;
        const int c0 = max(0, (int)leaves[o]), c1 = min(n_cols, (int)leaves[o + 1]);
        for (int c = c0; c < c1; ++c) s += (double)row[c];
        acc += s;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int d = blockDim.x / 2; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) gy[n] = (float)sh[0];
}

} // namespace vmat

using namespace vmat;

extern "C" {

vmat_status aperture_dose(vmat_ddc hd, const vmat_mlc *mlc, int32_t cp, const int16_t *leaves, float *da,
                          void *stream) {
    clear_error();
    if (!hd || !leaves || !da) return set_error(VMAT_EINVAL, "aperture_dose: NULL argument");
    VMAT_TRY(validate_mlc(mlc));
    Ddc *h = as_ddc(hd);
    if (!h->built_D) return set_error(VMAT_ESTATE, "aperture_dose: CSR(D) not built");
    if ((int64_t)mlc->K * mlc->n_rows * mlc->n_cols != h->J)
        return set_error(VMAT_EINVAL, "aperture_dose: K*n_rows*n_cols (%lld) != J (%d)",
                         (long long)mlc->K * mlc->n_rows * mlc->n_cols, h->J);
    if (cp < 0 || cp >= mlc->K) return set_error(VMAT_EINVAL, "aperture_dose: cp %d out of range", cp);
    VMAT_TRY(ddc_cp_table(*h, mlc->K, mlc->n_rows * mlc->n_cols, as_stream(stream)));
    return aperture_dose_impl(*h, mlc, cp, leaves, da, false, as_stream(stream));
}

vmat_status aperture_fluence(const vmat_mlc *mlc, int32_t n_ap, const int32_t *cps, const int16_t *leaves,
                             const float *y, float *x, void *stream) {
    clear_error();
    VMAT_TRY(validate_mlc(mlc));
    if (n_ap < 0 || !x || (n_ap > 0 && (!cps || !leaves || !y)))
        return set_error(VMAT_EINVAL, "aperture_fluence: bad arguments");
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int32_t J = mlc->K * mlc->n_rows * mlc->n_cols;
    const int grid = std::max(1, std::min(ctx->n_sm * 8, (J + 255) / 256));
    aperture_fluence_kernel<<<grid, 256, 0, as_stream(stream)>>>(J, mlc->n_rows, mlc->n_cols, n_ap, cps, leaves, y,
                                                                 x);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status aperture_grad(const vmat_mlc *mlc, int32_t n_ap, const int32_t *cps, const int16_t *leaves,
                          const float *pi, float *gy, void *stream) {
    clear_error();
    VMAT_TRY(validate_mlc(mlc));
    if (n_ap < 0 || (n_ap > 0 && (!cps || !leaves || !pi || !gy)))
        return set_error(VMAT_EINVAL, "aperture_grad: bad arguments");
    if (n_ap == 0) return VMAT_OK;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    aperture_grad_kernel<<<n_ap, 256, 0, as_stream(stream)>>>(mlc->K, mlc->n_rows, mlc->n_cols, cps, leaves, pi, gy,
                                                              ctx->status);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

} // extern "C"
