// Voxel objective (Eq. 1) and its negative gradient g = -grad F (Eq. 4).
//
// One pass over the voxels: g in FP32, F summed in FP64.  The per-block FP64
// partials are combined by the last block to finish (a counter in scratch), in
// block order, so F is reproducible bit for bit.
#include <algorithm>

#include "internal.cuh"

namespace vmat {

constexpr int OBJ_THREADS = 256;

__device__ __forceinline__ double block_sum_f64(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t; // valid in thread 0
}

// z[i] is the dose of voxel v = idx ? idx[i] : i.  Writes g[i] (or g_scatter[v], or
// g_scatter[gpos[i]] when gpos is given: g in brick order).
__global__ void __launch_bounds__(OBJ_THREADS)
    objective_kernel(int32_t n, const float *__restrict__ z, const int32_t *__restrict__ idx,
                     const uint8_t *__restrict__ sid, const float *T, const float *wo, const float *wu,
                     int32_t n_struct, float *g, float *g_scatter, double *partial, unsigned *counter, double *F,
                     double F_offset, const int32_t *skip, const int32_t *__restrict__ gpos) {
    if (skip && *skip) return;
    __shared__ float sT[256], sO[256], sU[256];
    __shared__ double sh[OBJ_THREADS / 32];
    __shared__ bool last;
    for (int k = threadIdx.x; k < n_struct; k += blockDim.x) {
        sT[k] = T[k];
        sO[k] = wo[k];
        sU[k] = wu[k];
    }
    __syncthreads();
    double acc = 0.0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t v = idx ? idx[i] : i;
        const int k = sid[v];
        const float zi = z[i], t = sT[k];
        if (g || g_scatter) {
            const float gi = -2.f * sO[k] * fmaxf(0.f, zi - t) + 2.f * sU[k] * fmaxf(0.f, t - zi);
            if (g_scatter) g_scatter[gpos ? gpos[i] : v] = gi;
            else g[i] = gi;
        }
        if (F) { // the FP64 objective only when asked for (FP64 is slow on this GPU)
            const double dz = (double)zi - (double)t;
            const double dd = dz > 0.0 ? (double)sO[k] : (double)sU[k];
            acc = fma(dd * dz, dz, acc);
        }
    }
    if (!F) return;
    const double bs = block_sum_f64(acc, sh);
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = bs;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile double *)partial)[b];
    const double tot = block_sum_f64(s, sh);
    if (threadIdx.x == 0) {
        *F = tot + F_offset;
        *counter = 0u;
    }
}

// Batched g = -grad F (no F): global voxel g is compact voxel i = g - off[p] of plan p,
// whose voxel index is idx[i]; g is written at g_scatter[idx[i]].
__global__ void __launch_bounds__(OBJ_THREADS)
    objective_grad_batched_kernel(const ObjPlan *__restrict__ plans, const int64_t *__restrict__ off, int32_t n_plans,
                                  int64_t total) {
    __shared__ int64_t soff[VMAT_MAX_BATCH + 1];
    for (int i = threadIdx.x; i <= n_plans; i += blockDim.x) soff[i] = off[i];
    __syncthreads();
    for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gi < total;
         gi += (int64_t)gridDim.x * blockDim.x) {
        int a = 0, b = n_plans;
        while (b - a > 1) {
            const int m = (a + b) >> 1;
            if (soff[m] <= gi) a = m;
            else b = m;
        }
        const ObjPlan &P = plans[a];
        if (P.skip && *P.skip) continue;
        const int64_t i = gi - soff[a];
        const int32_t v = P.idx[i];
        const int k = P.sid[v];
        const float zi = P.z[i], t = P.T[k];
        P.g_scatter[P.gpos ? P.gpos[i] : v] = -2.f * P.wo[k] * fmaxf(0.f, zi - t) + 2.f * P.wu[k] * fmaxf(0.f, t - zi);
    }
}

vmat_status objective_grad_batched(const ObjPlan *plans, const int64_t *off, int32_t n_plans, int64_t total,
                                   cudaStream_t s) {
    if (total <= 0) return VMAT_OK;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + OBJ_THREADS - 1) / OBJ_THREADS,
                                                                  (int64_t)ctx->n_sm * 8));
    objective_grad_batched_kernel<<<grid, OBJ_THREADS, 0, s>>>(plans, off, n_plans, total);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

// F_i(0) summed over voxels outside every row of CSR(D) (their dose is always 0).
__global__ void __launch_bounds__(OBJ_THREADS)
    inactive_objective_kernel(int32_t V, const int32_t *vox2act, const uint8_t *sid, const float *T, const float *wo,
                              const float *wu, double *partial) {
    __shared__ double sh[OBJ_THREADS / 32];
    double acc = 0.0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        if (vox2act[v] >= 0) continue;
        const int k = sid[v];
        const double t = T[k];
        const double over = -t > 0.0 ? -t : 0.0, under = t > 0.0 ? t : 0.0;
        acc += (double)wo[k] * over * over + (double)wu[k] * under * under;
    }
    const double bs = block_sum_f64(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

__global__ void sum_partials(const double *partial, int n, double *out) {
    __shared__ double sh[OBJ_THREADS / 32];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) s += partial[b];
    const double t = block_sum_f64(s, sh);
    if (threadIdx.x == 0) *out = t;
}

static int obj_grid(int64_t n, int n_sm) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + OBJ_THREADS - 1) / OBJ_THREADS, (int64_t)n_sm * 4));
}

size_t objective_scratch_bytes(int n_sm) { return 64 + (size_t)n_sm * 4 * sizeof(double); }

vmat_status objective_impl_ws(int32_t n, const float *z, const int32_t *idx, const vmat_voxels *vox, float *g,
                              float *g_scatter, double *F, double F_offset, void *ws, cudaStream_t s,
                              const int32_t *skip, const int32_t *gpos) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int grid = obj_grid(n, ctx->n_sm);
    unsigned *counter = reinterpret_cast<unsigned *>(ws);
    double *partial = reinterpret_cast<double *>(static_cast<char *>(ws) + 64);
    objective_kernel<<<grid, OBJ_THREADS, 0, s>>>(n, z, idx, vox->struct_id, vox->T, vox->w_over, vox->w_under,
                                                  vox->n_struct, g, g_scatter, partial, counter, F, F_offset, skip,
                                                  gpos);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status objective_impl(int32_t n, const float *z, const int32_t *idx, const vmat_voxels *vox, float *g,
                           float *g_scatter, double *F, double F_offset, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    Scratch ws;
    VMAT_TRY(ws.alloc(objective_scratch_bytes(ctx->n_sm), s));
    VMAT_CUDA(cudaMemsetAsync(ws.ptr, 0, 64, s));
    return objective_impl_ws(n, z, idx, vox, g, g_scatter, F, F_offset, ws.ptr, s, nullptr);
}

vmat_status inactive_objective(const Ddc &h, const vmat_voxels *vox, double *F0, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int grid = obj_grid(h.V, ctx->n_sm);
    Scratch ws;
    VMAT_TRY(ws.alloc((size_t)grid * sizeof(double), s));
    inactive_objective_kernel<<<grid, OBJ_THREADS, 0, s>>>(h.V, h.vox2act, vox->struct_id, vox->T, vox->w_over,
                                                           vox->w_under, (double *)ws.ptr);
    VMAT_LAUNCH_CHECK();
    sum_partials<<<1, OBJ_THREADS, 0, s>>>((double *)ws.ptr, grid, F0);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" vmat_status objective_grad(int32_t V, const float *z, const vmat_voxels *vox, float *g, double *F,
                                      void *stream) {
    clear_error();
    if (V < 0 || (V > 0 && !z)) return set_error(VMAT_EINVAL, "objective_grad: bad V or z");
    VMAT_TRY(validate_voxels(vox));
    if (V == 0) {
        if (F) VMAT_CUDA(cudaMemsetAsync(F, 0, sizeof(double), as_stream(stream)));
        return VMAT_OK;
    }
    return objective_impl(V, z, nullptr, vox, g, nullptr, F, 0.0, as_stream(stream));
}
