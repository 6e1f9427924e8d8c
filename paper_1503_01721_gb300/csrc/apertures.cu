// Apertures <-> beamlets.
//
// aperture_dose (Eq. 5): DA_i(A) = sum of D_ij over the beamlets j of the
// aperture.  The paper sums COO columns on the CPU (Section 2.2.2) because its
// GPUs only hold D^T.  Here the rows of CSR(D) are sorted by beamlet and the
// beamlets of one CP are a contiguous index range, so each voxel row finds the
// CP's slice with a binary search and adds the entries whose column lies
// between the row's leaves, in beamlet order (deterministic, no atomics).
//
// aperture_fluence: x = A y (beamlet fluence of a set of weighted apertures).
// aperture_grad:    A^T pi (summed price of each aperture's beamlets).
#include <algorithm>

#include "internal.cuh"

namespace vmat {

__device__ __forceinline__ float load_val(const void *val, int64_t e, vmat_dtype dt) {
    if (dt == VMAT_F32) return static_cast<const float *>(val)[e];
    if (dt == VMAT_BF16) {
        const uint16_t b = static_cast<const uint16_t *>(val)[e];
        return __uint_as_float((uint32_t)b << 16);
    }
    const uint8_t q = static_cast<const uint8_t *>(val)[e];
    __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3);
    return __half2float(*reinterpret_cast<__half *>(&hr));
}

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

__global__ void aperture_dose_kernel(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                     const void *__restrict__ val, vmat_dtype dt, const float *__restrict__ scale,
                                     int32_t n_rows, const int32_t *__restrict__ row_ids, int32_t cp_arg,
                                     const int32_t *cp_dev, const int32_t *skip, int32_t n_rrows, int32_t n_cols,
                                     const int16_t *__restrict__ leaves, float *__restrict__ da, int64_t wstride) {
    if (skip && *skip) return;
    const int32_t cp = cp_dev ? *cp_dev : cp_arg;
    extern __shared__ int16_t sl[]; // [n_rrows][2]
    for (int i = threadIdx.x; i < 2 * n_rrows; i += blockDim.x) sl[i] = leaves[i];
    __syncthreads();
    const int32_t bpc = n_rrows * n_cols;
    const int32_t j0 = cp * bpc, j1 = j0 + bpc;
    for (int32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < n_rows; row += gridDim.x * blockDim.x) {
        int64_t lo = rowptr[row], hi = rowptr[row + 1];
        while (lo < hi) { // first entry with column >= j0
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] < j0) lo = mid + 1;
            else hi = mid;
        }
        float acc = 0.f;
        const int64_t end = rowptr[row + 1];
        for (int64_t e = lo; e < end; ++e) {
            const int32_t j = col[e];
            if (j >= j1) break;
            const int32_t loc = j - j0, r = loc / n_cols, c = loc - r * n_cols;
            if (c >= sl[2 * r] && c < sl[2 * r + 1]) {
                float v = load_val(val, e, dt);
                if (scale) v *= scale[j];
                acc += v;
            }
        }
        // output: voxel space, compact row space, or the master problem's warp-tile
        // layout (row r at (r / 32) * wstride + (r % 32) * 4 from da, the column's base)
        const int64_t o =
            row_ids ? row_ids[row] : (wstride ? (int64_t)(row >> 5) * wstride + ((row & 31) << 2) : row);
        da[o] = acc;
    }
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
        const int32_t bpc = P.n_rrows * P.n_cols;
        const int32_t cp = P.cps[t];
        const int32_t j0 = cp * bpc, j1 = j0 + bpc;
        int64_t lo = P.rowptr[row], hi = P.rowptr[row + 1];
        while (lo < hi) { // first entry with column >= j0
            const int64_t mid = (lo + hi) >> 1;
            if (P.col[mid] < j0) lo = mid + 1;
            else hi = mid;
        }
        float acc = 0.f;
        const int64_t end = P.rowptr[row + 1];
        for (int64_t e = lo; e < end; ++e) {
            const int32_t j = P.col[e];
            if (j >= j1) break;
            const int32_t loc = j - j0, r = loc / P.n_cols, c = loc - r * P.n_cols;
            if (c >= P.leaves[2 * r] && c < P.leaves[2 * r + 1]) {
                float v = StoredVal<VT>::get(P.val, e);
                if (P.scale) v *= P.scale[j];
                acc += v;
            }
        }
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
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    if (!compact) VMAT_CUDA(cudaMemsetAsync(da, 0, (size_t)h.V * 4, s));
    const int32_t n = h.D.n_rows;
    if (n == 0) return VMAT_OK;
    const int grid = std::max(1, std::min(ctx->n_sm * 8, (n + 255) / 256));
    aperture_dose_kernel<<<grid, 256, (size_t)mlc->n_rows * 2 * sizeof(int16_t), s>>>(
        h.D.rowptr, h.D.col, h.D.val, h.dtype, h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr, n,
        compact ? nullptr : h.D.row_ids, cp, nullptr, nullptr, mlc->n_rows, mlc->n_cols, leaves, da,
        compact ? wstride : 0);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status aperture_dose_dev(const Ddc &h, const vmat_mlc *mlc, const int32_t *cp_dev, const int16_t *leaves,
                              float *da, int64_t wstride, const int32_t *skip, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int32_t n = h.D.n_rows;
    if (n == 0) return VMAT_OK;
    const int grid = std::max(1, std::min(ctx->n_sm * 8, (n + 255) / 256));
    aperture_dose_kernel<<<grid, 256, (size_t)mlc->n_rows * 2 * sizeof(int16_t), s>>>(
        h.D.rowptr, h.D.col, h.D.val, h.dtype, h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr, n, nullptr, 0, cp_dev,
        skip, mlc->n_rows, mlc->n_cols, leaves, da, wstride);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
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
