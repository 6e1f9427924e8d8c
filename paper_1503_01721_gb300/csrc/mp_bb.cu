// Master problem (Eq. 6): min F(DA y) subject to lo <= y <= hi, by
// Barzilai-Borwein steps (Eq. 7-8, used alternately) with the subspace scheme
// of Eq. 9-10 and the stopping rules of Section 2.1.
//
// The paper runs four steps per iteration on one GPU (aperture gradient, step
// length with cuBLAS dot products, subspace update, dose update).  Here each
// iteration is two kernels:
//   mp_pass  (all SMs): z = DA y, the objective terms and g = -grad F per voxel,
//            and per-block partials of G = grad_y F = -DA^T g, reading DA once
//            from HBM (the second read of each column chunk hits L1/L2);
//   mp_step  (one block): FP64 reduction of the partials in block order, the
//            Eq. 9-10 freeze, the stopping tests, the BB step and the projected
//            update of y.
// The first iteration takes a Cauchy step, which needs DA G: two more kernels.
// Readings (where the paper is silent): G is the gradient of F, so both BB
// step lengths are positive and Eq. 9-10 freeze at lo when G > 0 and at hi when
// G < 0; y is projected onto the box after each step; BB1 on even and BB2 on
// odd iterations; s.r <= 0 takes the largest step; steps are clamped to
// [delta_min, delta_max] times the Cauchy step.
#include <math.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace vmat {

constexpr int MP_THREADS = 256;
constexpr int MP_NW = MP_THREADS / 32;
constexpr int MP_CHUNK = 8; // iterations launched between host polls

struct BBState {
    double F_hist[6];
    double F;
    double delta0;
    double gg;
    int32_t t;
    int32_t done;
    int32_t stop;
    int32_t iters;
    int32_t need_cauchy;
    int32_t pad;
};

struct MPArgs {
    const float *DA;
    int64_t ld;
    int32_t V, n;
    const uint8_t *sid;
    const float *T, *wo, *wu;
    int32_t n_struct;
    float *y;
    float *z;
    const float *lo, *hi; // may be null
    double *G, *Gprev;
    float *yprev;
    double *part;  // [P][n + 1]
    double *cpart; // [P]
    int32_t P;
    BBState *st;
    vmat_bb_opts opts;
    double F_offset;
};

__device__ __forceinline__ float lo_of(const MPArgs &a, int k) { return a.lo ? a.lo[k] : 0.f; }
__device__ __forceinline__ float hi_of(const MPArgs &a, int k) { return a.hi ? a.hi[k] : INFINITY; }

__global__ void mp_init_kernel(MPArgs a) {
    for (int k = threadIdx.x; k < a.n; k += blockDim.x) a.y[k] = fminf(fmaxf(a.y[k], lo_of(a, k)), hi_of(a, k));
    if (threadIdx.x == 0) {
        BBState s = {};
        *a.st = s;
    }
}

__global__ void __launch_bounds__(MP_THREADS) mp_pass_kernel(MPArgs a) {
    if (a.st->done || a.st->need_cauchy) return;
    extern __shared__ __align__(16) unsigned char sm[];
    float *sy = reinterpret_cast<float *>(sm);                  // [n]
    double *accG = reinterpret_cast<double *>(sy + ((a.n + 3) & ~3)); // [n]
    float *gs = reinterpret_cast<float *>(accG + a.n);           // [MP_THREADS]
    float *sT = gs + MP_THREADS, *sO = sT + 256, *sU = sO + 256;
    __shared__ double sh[MP_NW];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = tid; k < a.n; k += MP_THREADS) {
        sy[k] = a.y[k];
        accG[k] = 0.0;
    }
    for (int k = tid; k < a.n_struct; k += MP_THREADS) {
        sT[k] = a.T[k];
        sO[k] = a.wo[k];
        sU[k] = a.wu[k];
    }
    __syncthreads();
    double facc = 0.0;
    for (int64_t base = (int64_t)blockIdx.x * MP_THREADS; base < a.V; base += (int64_t)gridDim.x * MP_THREADS) {
        const int64_t i = base + tid;
        float gi = 0.f;
        if (i < a.V) {
            float zi = 0.f;
            for (int k = 0; k < a.n; ++k) zi = fmaf(a.DA[(int64_t)k * a.ld + i], sy[k], zi);
            a.z[i] = zi;
            const int s = a.sid[i];
            const float t = sT[s];
            gi = -2.f * sO[s] * fmaxf(0.f, zi - t) + 2.f * sU[s] * fmaxf(0.f, t - zi);
            const double dz = (double)zi - (double)t;
            const double ov = dz > 0.0 ? dz : 0.0, un = dz < 0.0 ? -dz : 0.0;
            facc += (double)sO[s] * ov * ov + (double)sU[s] * un * un;
        }
        gs[tid] = gi;
        __syncthreads();
        for (int k = wid; k < a.n; k += MP_NW) {
            const float *col = a.DA + (int64_t)k * a.ld + base;
            float sum = 0.f;
#pragma unroll
            for (int m = lane; m < MP_THREADS; m += 32)
                if (base + m < a.V) sum = fmaf(col[m], gs[m], sum);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, d);
            if (lane == 0) accG[k] += (double)sum;
        }
        __syncthreads();
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) facc += __shfl_down_sync(0xffffffffu, facc, d);
    if (lane == 0) sh[wid] = facc;
    __syncthreads();
    double *out = a.part + (int64_t)blockIdx.x * (a.n + 1);
    for (int k = tid; k < a.n; k += MP_THREADS) out[k] = accG[k];
    if (tid == 0) {
        double f = 0.0;
        for (int w = 0; w < MP_NW; ++w) f += sh[w];
        out[a.n] = f;
    }
}

// Fixed-order block reduction of a double (result valid in every thread).
__device__ double block_reduce_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < MP_NW; ++w) t += sh[w];
    return t;
}

__device__ double block_reduce_max(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, d));
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = sh[0];
    for (int w = 1; w < MP_NW; ++w) t = fmax(t, sh[w]);
    return t;
}

__device__ void finish(BBState *st, int reason, int t) {
    st->done = 1;
    st->stop = reason;
    st->iters = t + 1;
}

// Projected update y <- clamp(y - delta G) after saving (y, G) as the previous iterate.
__device__ void take_step(const MPArgs &a, double delta) {
    for (int k = threadIdx.x; k < a.n; k += MP_THREADS) {
        const float yk = a.y[k];
        a.yprev[k] = yk;
        a.Gprev[k] = a.G[k];
        const double yn = (double)yk - delta * a.G[k];
        a.y[k] = fminf(fmaxf((float)yn, lo_of(a, k)), hi_of(a, k));
    }
}

__global__ void __launch_bounds__(MP_THREADS) mp_step_kernel(MPArgs a) {
    BBState *st = a.st;
    if (st->done || st->need_cauchy) return;
    __shared__ double sh[MP_NW];
    const int t = st->t;
    const int n = a.n;
    // G_k = -sum_b part[b][k]; F = sum_b part[b][n] + offset (block order)
    for (int k = threadIdx.x; k <= n; k += MP_THREADS) {
        double s = 0.0;
        for (int b = 0; b < a.P; ++b) s += a.part[(int64_t)b * (n + 1) + k];
        if (k < n) a.G[k] = -s;
        else st->F = s + a.F_offset;
    }
    __syncthreads();
    // Eq. 9-10: freeze components at a bound whose gradient points out of the box
    for (int k = threadIdx.x; k < n; k += MP_THREADS) {
        const float yk = a.y[k], l = lo_of(a, k), h = hi_of(a, k);
        const double g = a.G[k];
        if (yk <= l && g > 0.0) {
            a.y[k] = l;
            a.G[k] = 0.0;
        } else if (yk >= h && g < 0.0) {
            a.y[k] = h;
            a.G[k] = 0.0;
        }
    }
    __syncthreads();
    const double F = st->F;
    // stopping tests (Section 2.1)
    double dy = 0.0, ymax = 0.0, gg = 0.0, ss = 0.0, sr = 0.0, rr = 0.0;
    for (int k = threadIdx.x; k < n; k += MP_THREADS) {
        const double yk = a.y[k], g = a.G[k];
        ymax = fmax(ymax, fabs(yk));
        gg += g * g;
        if (t > 0) {
            const double s = yk - (double)a.yprev[k], r = g - a.Gprev[k];
            dy = fmax(dy, fabs(s));
            ss += s * s;
            sr += s * r;
            rr += r * r;
        }
    }
    dy = block_reduce_max(dy, sh);
    ymax = block_reduce_max(ymax, sh);
    gg = block_reduce_sum(gg, sh);
    ss = block_reduce_sum(ss, sh);
    sr = block_reduce_sum(sr, sh);
    rr = block_reduce_sum(rr, sh);
    __shared__ int decided;
    __shared__ double delta_s;
    if (threadIdx.x == 0) {
        decided = 1;
        st->F_hist[t % 6] = F;
        if (t >= 5 && fabs(st->F_hist[(t - 5) % 6] - F) <= a.opts.rel_tol5 * F) finish(st, VMAT_STOP_REL, t);
        else if (t >= 1 && dy <= a.opts.step_tol * fmax(1.0, ymax)) finish(st, VMAT_STOP_STEP, t);
        else if (t == a.opts.max_iter - 1) finish(st, VMAT_STOP_MAXIT, t);
        else if (t == 0) {
            if (gg == 0.0) finish(st, VMAT_STOP_GRAD0, t);
            else {
                st->gg = gg;
                st->need_cauchy = 1; // the step length needs DA G
            }
        } else {
            double delta;
            if (sr <= 0.0) delta = a.opts.delta_max * st->delta0;
            else if (t & 1) delta = sr / rr;
            else delta = ss / sr;
            delta = fmin(fmax(delta, a.opts.delta_min * st->delta0), a.opts.delta_max * st->delta0);
            delta_s = delta;
            decided = 0;
        }
    }
    __syncthreads();
    if (!decided) {
        take_step(a, delta_s);
        if (threadIdx.x == 0) st->t = t + 1;
    }
}

// Cauchy step, part 1: curvature 2 sum_i w_i (DA G)_i^2 with w the active penalty weight.
__global__ void __launch_bounds__(MP_THREADS) mp_cauchy_pass_kernel(MPArgs a) {
    if (a.st->done || !a.st->need_cauchy) return;
    extern __shared__ __align__(16) unsigned char sm[];
    float *sg = reinterpret_cast<float *>(sm); // [n]
    float *sT = sg + ((a.n + 3) & ~3), *sO = sT + 256, *sU = sO + 256;
    __shared__ double sh[MP_NW];
    const int tid = threadIdx.x;
    for (int k = tid; k < a.n; k += MP_THREADS) sg[k] = (float)a.G[k];
    for (int k = tid; k < a.n_struct; k += MP_THREADS) {
        sT[k] = a.T[k];
        sO[k] = a.wo[k];
        sU[k] = a.wu[k];
    }
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * MP_THREADS + tid; i < a.V; i += (int64_t)gridDim.x * MP_THREADS) {
        float q = 0.f;
        for (int k = 0; k < a.n; ++k) q = fmaf(a.DA[(int64_t)k * a.ld + i], sg[k], q);
        const int s = a.sid[i];
        const float zi = a.z[i], t = sT[s];
        const float w = zi > t ? sO[s] : (zi < t ? sU[s] : 0.f);
        acc += (double)w * (double)q * (double)q;
    }
    const double b = block_reduce_sum(acc, sh);
    if (tid == 0) a.cpart[blockIdx.x] = b;
}

// Cauchy step, part 2: delta0 = G.G / curvature, then the first projected step.
__global__ void __launch_bounds__(MP_THREADS) mp_cauchy_step_kernel(MPArgs a) {
    BBState *st = a.st;
    if (st->done || !st->need_cauchy) return;
    __shared__ double curv_s;
    if (threadIdx.x == 0) {
        double c = 0.0;
        for (int b = 0; b < a.P; ++b) c += a.cpart[b];
        curv_s = 2.0 * c;
        st->need_cauchy = 0;
        if (curv_s == 0.0) finish(st, VMAT_STOP_FLAT, 0);
        else st->delta0 = st->gg / curv_s;
    }
    __syncthreads();
    if (curv_s == 0.0) return;
    take_step(a, st->delta0);
    if (threadIdx.x == 0) st->t = 1;
}

size_t mp_scratch_bytes(int32_t n, int P) {
    return 256 + (size_t)n * (2 * sizeof(double) + sizeof(float)) + (size_t)P * (n + 2) * sizeof(double) + 256;
}

vmat_status mp_bb_impl(const float *DA, int32_t V, int32_t n_ap, int64_t ld, const uint8_t *struct_id,
                       const int32_t *struct_idx, const vmat_voxels *vox, const float *lo, const float *hi, float *y,
                       float *z, const vmat_bb_opts *opts_in, double F_offset, vmat_bb_report *rep, cudaStream_t s) {
    (void)struct_idx;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    vmat_bb_opts opts = {500, 1e-6, 1e-9, 1e-12, 1e12};
    if (opts_in) opts = *opts_in;
    if (opts.max_iter < 1) return set_error(VMAT_EINVAL, "mp_bb_solve: max_iter must be >= 1");
    const int P = std::max(1, std::min<int>((int)((V + MP_THREADS - 1) / MP_THREADS), ctx->n_sm * 4));
    Scratch ws;
    VMAT_TRY(ws.alloc(mp_scratch_bytes(n_ap, P), s));
    char *p = static_cast<char *>(ws.ptr);
    MPArgs a;
    a.st = reinterpret_cast<BBState *>(p);
    p += 256;
    a.G = reinterpret_cast<double *>(p);
    a.Gprev = a.G + n_ap;
    a.part = a.Gprev + n_ap;
    a.cpart = a.part + (size_t)P * (n_ap + 1);
    a.yprev = reinterpret_cast<float *>(a.cpart + P);
    a.DA = DA;
    a.ld = ld;
    a.V = V;
    a.n = n_ap;
    a.sid = struct_id;
    a.T = vox->T;
    a.wo = vox->w_over;
    a.wu = vox->w_under;
    a.n_struct = vox->n_struct;
    a.y = y;
    a.z = z;
    a.lo = lo;
    a.hi = hi;
    a.P = P;
    a.opts = opts;
    a.F_offset = F_offset;

    const size_t smem_pass = (size_t)((n_ap + 3) & ~3) * 4 + (size_t)n_ap * 8 + MP_THREADS * 4 + 3 * 256 * 4;
    const size_t smem_cauchy = (size_t)((n_ap + 3) & ~3) * 4 + 3 * 256 * 4;
    if (smem_pass > 200 * 1024) return set_error(VMAT_EUNSUPPORTED, "mp_bb_solve: too many apertures (%d)", n_ap);
    static bool attr = false;
    if (!attr) {
        VMAT_CUDA(cudaFuncSetAttribute(mp_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        VMAT_CUDA(cudaFuncSetAttribute(mp_cauchy_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    static thread_local BBState *host_st = nullptr;
    if (!host_st) VMAT_CUDA(cudaMallocHost(&host_st, sizeof(BBState)));

    mp_init_kernel<<<1, MP_THREADS, 0, s>>>(a);
    VMAT_LAUNCH_CHECK();
    int launched = 0;
    while (launched < opts.max_iter) {
        const int chunk = launched == 0 ? 1 : std::min(MP_CHUNK, opts.max_iter - launched);
        for (int c = 0; c < chunk; ++c) {
            mp_pass_kernel<<<P, MP_THREADS, smem_pass, s>>>(a);
            mp_step_kernel<<<1, MP_THREADS, 0, s>>>(a);
            g_launches.fetch_add(2, std::memory_order_relaxed);
            if (launched + c == 0) {
                mp_cauchy_pass_kernel<<<P, MP_THREADS, smem_cauchy, s>>>(a);
                mp_cauchy_step_kernel<<<1, MP_THREADS, 0, s>>>(a);
                g_launches.fetch_add(2, std::memory_order_relaxed);
            }
        }
        VMAT_CUDA(cudaGetLastError());
        launched += chunk;
        VMAT_CUDA(cudaMemcpyAsync(host_st, a.st, sizeof(BBState), cudaMemcpyDeviceToHost, s));
        VMAT_CUDA(cudaStreamSynchronize(s));
        if (host_st->done) break;
    }
    if (!host_st->done) return set_error(VMAT_ECUDA, "mp_bb_solve: solver did not reach a stopping rule");
    if (rep) {
        rep->iters = host_st->iters;
        rep->stop_reason = host_st->stop;
        rep->F = host_st->F;
    }
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" vmat_status mp_bb_solve(const float *DA, int32_t V, int32_t n_ap, int64_t ld, const vmat_voxels *vox,
                                   const float *lo, const float *hi, float *y, float *z, const vmat_bb_opts *opts,
                                   vmat_bb_report *rep, void *stream) {
    clear_error();
    VMAT_TRY(validate_voxels(vox));
    if (V <= 0 || n_ap <= 0 || ld < V || !DA || !y || !z)
        return set_error(VMAT_EINVAL, "mp_bb_solve: need V > 0, n_ap > 0, ld >= V and non-NULL DA, y, z");
    return mp_bb_impl(DA, V, n_ap, ld, vox->struct_id, nullptr, vox, lo, hi, y, z, opts, 0.0, rep, as_stream(stream));
}
