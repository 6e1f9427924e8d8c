// Master problem (Eq. 6): min F(DA y) subject to lo <= y <= hi, by
// Barzilai-Borwein steps (Eq. 7-8, used alternately) with the subspace scheme
// of Eq. 9-10 and the stopping rules of Section 2.1.
//
// The paper runs four steps per iteration on one GPU (aperture gradient, step
// length with cuBLAS dot products, subspace update, dose update).  Here one
// kernel does a whole iteration.  DA is kept in a grouped tile layout:
// 256-voxel tiles, and inside a tile the apertures in groups of four with the
// four values of a voxel side by side,
//     DA(i, k) = DA[(i / 256) * tstride + (k / 4) * 1024 + (i % 256) * 4 + k % 4],
// so the first n columns of a tile are one contiguous block.  Every CTA streams
// tiles into shared memory with one bulk copy each (several in flight on an
// mbarrier ring); each thread owns a voxel, reads its four-aperture groups
// with 128-bit shared loads, forms z = DA y with four independent chains, the
// objective terms and g = -grad F, and adds DA_ik g_i to its register-resident
// shares of G = grad_y F = -DA^T g.  DA is read from HBM once per iteration.
// The last CTA to finish (a ticket counter) reduces the partials in a fixed
// order (FP64) and takes the step: the Eq. 9-10 freeze, the stopping tests, the
// BB step length and the projected update.  The first iteration's Cauchy step
// needs DA G and takes two more kernels.
//
// Readings (where the paper is silent): G is the gradient of F, so both BB
// step lengths are positive and Eq. 9-10 freeze at lo when G > 0 and at hi when
// G < 0; y is projected onto the box after each step; BB1 on even and BB2 on
// odd iterations; s.r <= 0 takes the largest step; steps are clamped to
// [delta_min, delta_max] times the Cauchy step.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace vmat {

constexpr int MP_THREADS = 256; // = voxels per DA tile
constexpr int MP_NW = MP_THREADS / 32;
constexpr int MP_STAGES = 2;
constexpr int MP_CHUNK = 8; // iterations launched between host polls
constexpr size_t MP_SMEM_LIMIT = 200 * 1024;
constexpr int MP_NMAX = 96; // register-resident gradient shares: up to 96 apertures

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
    uint32_t ticket; // CTAs of the current pass that have written their partials
};

struct MPArgs {
    const float *DA; // grouped tile layout (see above)
    int64_t tstride; // floats per 256-voxel tile (a multiple of 1024)
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
    int32_t n_tiles;
    BBState *st;
    int32_t *status;
    vmat_bb_opts opts;
    double F_offset;
};

__device__ __forceinline__ int64_t min64(int64_t x, int64_t y) { return x < y ? x : y; }

// Offset of DA(voxel i, aperture k) in the grouped tile layout.
__device__ __forceinline__ int64_t da_at(const MPArgs &a, int64_t i, int k) {
    return (i >> 8) * a.tstride + (int64_t)(k >> 2) * 1024 + ((i & 255) << 2) + (k & 3);
}

__device__ __forceinline__ float lo_of(const MPArgs &a, int k) { return a.lo ? a.lo[k] : 0.f; }
__device__ __forceinline__ float hi_of(const MPArgs &a, int k) { return a.hi ? a.hi[k] : INFINITY; }

__global__ void mp_init_kernel(MPArgs a) {
    for (int k = threadIdx.x; k < a.n; k += blockDim.x) a.y[k] = fminf(fmaxf(a.y[k], lo_of(a, k)), hi_of(a, k));
    if (threadIdx.x == 0) {
        BBState s = {};
        *a.st = s;
    }
}

// Fixed-order block reductions (result valid in every thread).
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

// G_k = -sum_b part[b][k] and F = sum_b part[b][n] + offset.  One warp per column;
// lane l sums blocks l, l + 32, ... in order, then a fixed butterfly.
__device__ void reduce_partials(const MPArgs &a, int P) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n = a.n;
    for (int k = wid; k <= n; k += MP_NW) {
        double s = 0.0;
        // other CTAs' writes: bypass L1; 8 loads in flight per lane
#pragma unroll 8
        for (int b = lane; b < P; b += 32) s += __ldcg(a.part + (int64_t)b * (n + 1) + k);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
        if (lane == 0) {
            if (k < n) a.G[k] = -s;
            else a.st->F = s + a.F_offset;
        }
    }
    __syncthreads();
}

// Eq. 9-10 freeze, stopping tests, BB step length and projected update (one block).
__device__ void bb_step(const MPArgs &a) {
    BBState *st = a.st;
    __shared__ double sh[MP_NW];
    __shared__ int decided;
    __shared__ double delta_s;
    const int t = st->t;
    const int n = a.n;
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
    { // one combined block reduction of the six quantities (two maxima, four sums)
        __shared__ double red[MP_NW][6];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            dy = fmax(dy, __shfl_down_sync(0xffffffffu, dy, d));
            ymax = fmax(ymax, __shfl_down_sync(0xffffffffu, ymax, d));
            gg += __shfl_down_sync(0xffffffffu, gg, d);
            ss += __shfl_down_sync(0xffffffffu, ss, d);
            sr += __shfl_down_sync(0xffffffffu, sr, d);
            rr += __shfl_down_sync(0xffffffffu, rr, d);
        }
        if (lane == 0) {
            red[wid][0] = dy;
            red[wid][1] = ymax;
            red[wid][2] = gg;
            red[wid][3] = ss;
            red[wid][4] = sr;
            red[wid][5] = rr;
        }
        __syncthreads();
        dy = red[0][0];
        ymax = red[0][1];
        gg = red[0][2];
        ss = red[0][3];
        sr = red[0][4];
        rr = red[0][5];
        for (int w = 1; w < MP_NW; ++w) {
            dy = fmax(dy, red[w][0]);
            ymax = fmax(ymax, red[w][1]);
            gg += red[w][2];
            ss += red[w][3];
            sr += red[w][4];
            rr += red[w][5];
        }
    }
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

// Per-voxel part of an iteration for voxel i with dose zi: returns g_i, adds F_i to facc.
// The deviation d = z - T and the active weight are formed in FP32 (FP64 is a
// small fraction of the FP32 rate on this GPU); the term w d^2 is then formed and
// accumulated in FP64 from those FP32 values: one multiply and one FMA per voxel.
__device__ __forceinline__ float voxel_terms(const float *sT, const float *sO, const float *sU, int s, float zi,
                                             double &facc) {
    const float d = zi - sT[s];
    const float w = d > 0.f ? sO[s] : sU[s];
    const double dd = (double)d;
    facc = fma((double)w * dd, dd, facc);
    return -2.f * w * d; // g = -grad F: -2 w+ (z - T) above, +2 w- (T - z) below
}

// Ends a pass: write this CTA's partials; the last CTA reduces them and steps.
__device__ void pass_epilogue(const MPArgs &a, const double *accG, double facc) {
    __shared__ double sh[MP_NW];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const double fb = block_reduce_sum(facc, sh);
    double *out = a.part + (int64_t)blockIdx.x * (a.n + 1);
    for (int k = tid; k < a.n; k += MP_THREADS) out[k] = accG[k];
    if (tid == 0) out[a.n] = fb;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&a.st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    reduce_partials(a, gridDim.x);
    bb_step(a);
    if (tid == 0) a.st->ticket = 0u;
}

// One BB iteration with DA tiles staged in shared memory by 2-D tensor copies
// (one [n x 256] box per tile, `stages` tiles in flight, zero fill past V).
// Each thread owns one voxel of every tile and keeps its share of
// G = -DA^T g for all columns in registers (NMAX >= n) across the tiles of its
// CTA; one block reduction per pass.  Needs DA 16-byte aligned and ld a
// multiple of 4 (the tensor map's row pitch).

// One BB iteration: tiles of DA (the first n columns of 256 voxels, one block of
// ceil(n/4) * 4 KB) are bulk-copied into shared memory, `stages` in flight.
// Each thread owns one voxel of every tile and keeps its share of G for all
// columns in registers (NMAX >= n) across the tiles of its CTA; one block
// reduction per pass.  Slots of columns >= n inside the last group hold 0.
template <int NMAX>
__global__ void __launch_bounds__(MP_THREADS) mp_iter_tma_kernel(MPArgs a, int stages, int keep_in_l2) {
    if (a.st->done || a.st->need_cauchy) return;
    extern __shared__ __align__(128) unsigned char sm_raw[];
    // align the staging area explicitly: this kernel's static shared memory may
    // shift the dynamic region
    unsigned char *sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
    constexpr int GMAX = NMAX / 4;
    const int n = a.n, G = (n + 3) >> 2;
    float *DAs = reinterpret_cast<float *>(sm);                              // [stages][G][256][4]
    float4 *sy4 = reinterpret_cast<float4 *>(DAs + (size_t)stages * G * 1024); // [GMAX]
    double *accG = reinterpret_cast<double *>(sy4 + GMAX);                     // [NMAX]
    float *wred = reinterpret_cast<float *>(accG + NMAX);                      // [MP_NW][NMAX]
    float *sT = wred + MP_NW * NMAX, *sO = sT + 256, *sU = sO + 256;           // [256] each
    uint64_t *bars = reinterpret_cast<uint64_t *>(sU + 256);                   // [stages]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = tid; k < 4 * GMAX; k += MP_THREADS) reinterpret_cast<float *>(sy4)[k] = k < n ? a.y[k] : 0.f;
    for (int k = tid; k < a.n_struct; k += MP_THREADS) {
        sT[k] = a.T[k];
        sO[k] = a.wo[k];
        sU[k] = a.wu[k];
    }
    if (tid == 0) {
        for (int s = 0; s < stages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // DA is read again by the next iteration: keep it in L2 when it fits there
    const uint64_t pol = keep_in_l2 ? l2_evict_last_policy() : l2_evict_first_policy();
    const uint32_t bytes = (uint32_t)G * 4096u;
    auto issue = [&](int32_t tile, int s) {
        mbar_arrive_expect_tx(&bars[s], bytes);
        bulk_g2s(DAs + (size_t)s * G * 1024, a.DA + (int64_t)tile * a.tstride, bytes, &bars[s], pol);
    };
    if (tid == 0)
        for (int s = 0; s < stages; ++s) {
            const int32_t tile = blockIdx.x + s * gridDim.x;
            if (tile < a.n_tiles) issue(tile, s);
        }
    float gacc[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) gacc[k] = 0.f;
    double facc = 0.0;
    int it = 0;
    bool timed_out = false;
    for (int32_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
        const int s = it % stages;
        const bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((it / stages) & 1), WAIT_LIMIT_CYCLES);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const float4 *T4 = reinterpret_cast<const float4 *>(DAs + (size_t)s * G * 1024) + tid; // group g at [g * 256]
        const int64_t i = (int64_t)tile * MP_THREADS + tid;
        if (i < a.V) {
            float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
            for (int g = 0; g < GMAX; ++g)
                if (g < G) {
                    const float4 v = T4[g * 256], w = sy4[g];
                    z0 = fmaf(v.x, w.x, z0);
                    z1 = fmaf(v.y, w.y, z1);
                    z2 = fmaf(v.z, w.z, z2);
                    z3 = fmaf(v.w, w.w, z3);
                }
            const float zi = (z0 + z1) + (z2 + z3);
            a.z[i] = zi;
            const float gi = voxel_terms(sT, sO, sU, a.sid[i], zi, facc);
#pragma unroll
            for (int g = 0; g < GMAX; ++g)
                if (g < G) {
                    const float4 v = T4[g * 256];
                    gacc[4 * g + 0] = fmaf(v.x, gi, gacc[4 * g + 0]);
                    gacc[4 * g + 1] = fmaf(v.y, gi, gacc[4 * g + 1]);
                    gacc[4 * g + 2] = fmaf(v.z, gi, gacc[4 * g + 2]);
                    gacc[4 * g + 3] = fmaf(v.w, gi, gacc[4 * g + 3]);
                }
        }
        __syncthreads(); // every read of stage s is done before its next copy
        if (tid == 0) {
            const int32_t nt = tile + stages * gridDim.x;
            if (nt < a.n_tiles) issue(nt, s);
        }
    }
    if (timed_out) {
        // a copy that never landed: record it, let issued copies finish, stop the solve
        if (tid == 0) {
            atomicOr(a.status, DEV_TIMEOUT);
            a.st->done = 1;
            a.st->stop = VMAT_STOP_MAXIT;
            for (int k = 0; k < stages; ++k) {
                const int it2 = it + k;
                if (blockIdx.x + it2 * gridDim.x < a.n_tiles)
                    mbar_wait_bounded(&bars[it2 % stages], (uint32_t)((it2 / stages) & 1), WAIT_LIMIT_CYCLES);
            }
        }
        return;
    }
    // block reduction of the per-thread shares: butterfly per warp, warps in order
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        if (k < n) {
            float x = gacc[k];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
            if (lane == 0) wred[wid * NMAX + k] = x;
        }
    }
    __syncthreads();
    for (int k = tid; k < n; k += MP_THREADS) {
        double sum = 0.0;
        for (int w = 0; w < MP_NW; ++w) sum += (double)wred[w * NMAX + k];
        accG[k] = sum;
    }
    __syncthreads();
    pass_epilogue(a, accG, facc);
}

// The same iteration reading DA from global memory with per-tile reductions
// (more apertures than the register-resident shares hold).
__global__ void __launch_bounds__(MP_THREADS) mp_iter_ldg_kernel(MPArgs a) {
    if (a.st->done || a.st->need_cauchy) return;
    extern __shared__ __align__(16) unsigned char sm[];
    const int n = a.n;
    float *sy = reinterpret_cast<float *>(sm);                          // [n]
    double *accG = reinterpret_cast<double *>(sy + ((n + 3) & ~3));     // [n]
    float *gs = reinterpret_cast<float *>(accG + n);                    // [256]
    float *sT = gs + MP_THREADS, *sO = sT + 256, *sU = sO + 256;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = tid; k < n; k += MP_THREADS) {
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
    for (int32_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
        const int64_t i0 = (int64_t)tile * MP_THREADS, i = i0 + tid;
        float gi = 0.f;
        if (i < a.V) {
            float zi = 0.f;
            for (int k = 0; k < n; ++k) zi = fmaf(a.DA[da_at(a, i, k)], sy[k], zi);
            a.z[i] = zi;
            gi = voxel_terms(sT, sO, sU, a.sid[i], zi, facc);
        }
        gs[tid] = gi;
        __syncthreads();
        const int nvalid = (int)min64(MP_THREADS, a.V - i0);
        for (int k = wid; k < n; k += MP_NW) {
            float sum = 0.f;
#pragma unroll
            for (int m = lane; m < MP_THREADS; m += 32)
                if (m < nvalid) sum = fmaf(a.DA[da_at(a, i0 + m, k)], gs[m], sum);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, d);
            if (lane == 0) accG[k] += (double)sum;
        }
        __syncthreads();
    }
    pass_epilogue(a, accG, facc);
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
        for (int k = 0; k < a.n; ++k) q = fmaf(a.DA[da_at(a, i, k)], sg[k], q);
        const int s = a.sid[i];
        const float zi = a.z[i], t = sT[s];
        const float w = zi > t ? sO[s] : (zi < t ? sU[s] : 0.f);
        acc += (double)w * (double)q * (double)q;
    }
    const double b = block_reduce_sum(acc, sh);
    if (tid == 0) a.cpart[blockIdx.x] = b;
}

// Cauchy step, part 2: delta0 = G.G / curvature, then the first projected step.
__global__ void __launch_bounds__(MP_THREADS) mp_cauchy_step_kernel(MPArgs a, int P) {
    BBState *st = a.st;
    if (st->done || !st->need_cauchy) return;
    __shared__ double curv_s;
    if (threadIdx.x == 0) {
        double c = 0.0;
        for (int b = 0; b < P; ++b) c += a.cpart[b];
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


// Grouped tile layout from a column-major matrix (DA[k * ld + i]); padding 0.
__global__ void to_grouped_tiles(const float *src, int64_t ld, int32_t V, int32_t n, int64_t tstride,
                                 int32_t n_tiles, float *dst) {
    const int64_t total = (int64_t)n_tiles * tstride;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t tile = o / tstride, r = o % tstride;
        const int k = (int)((r >> 10) << 2) + (int)(r & 3);
        const int64_t i = tile * 256 + ((r & 1023) >> 2);
        dst[o] = (k < n && i < V) ? src[(int64_t)k * ld + i] : 0.f;
    }
}

static int tma_nmax(int n) { return ((n + 7) / 8) * 8; }
// Tiles in flight per CTA (~n KB each): ~100 KB so that two CTAs share an SM while
// that still allows 3 stages, else ~190 KB for one CTA; at least double-buffered.
static int tma_stages(int n) {
    const int kb = 4 * ((std::max(n, 1) + 3) / 4);
    const int budget = 3 * kb <= 100 ? 100 : 190;
    return std::max(MP_STAGES, std::min(6, budget / kb));
}
static size_t tma_smem(int n, int stages) {
    const int nmax = tma_nmax(n), G = (n + 3) / 4;
    return 128 /* alignment slack */ + (size_t)stages * G * 4096 + (size_t)(nmax / 4) * 16 + (size_t)nmax * 8 +
           (size_t)MP_NW * nmax * 4 + 3 * 256 * 4 + (size_t)stages * 8;
}

using TmaIterFn = void (*)(MPArgs, int, int);
static TmaIterFn tma_kernel_for(int n) {
    switch ((n + 7) / 8) {
    case 1: return mp_iter_tma_kernel<8>;
    case 2: return mp_iter_tma_kernel<16>;
    case 3: return mp_iter_tma_kernel<24>;
    case 4: return mp_iter_tma_kernel<32>;
    case 5: return mp_iter_tma_kernel<40>;
    case 6: return mp_iter_tma_kernel<48>;
    case 7: return mp_iter_tma_kernel<56>;
    case 8: return mp_iter_tma_kernel<64>;
    case 9: return mp_iter_tma_kernel<72>;
    case 10: return mp_iter_tma_kernel<80>;
    case 11: return mp_iter_tma_kernel<88>;
    case 12: return mp_iter_tma_kernel<96>;
    default: return nullptr;
    }
}
static size_t ldg_smem(int n) { return (size_t)((n + 3) & ~3) * 4 + (size_t)n * 8 + MP_THREADS * 4 + 3 * 256 * 4; }

int64_t mp_tile_stride(int32_t n_cap) { return (int64_t)((n_cap + 3) / 4) * 1024; }

vmat_status mp_bb_impl(const float *DA, int32_t V, int32_t n_ap, int64_t ld, const uint8_t *struct_id,
                       int64_t tstride, const vmat_voxels *vox, const float *lo, const float *hi, float *y,
                       float *z, const vmat_bb_opts *opts_in, double F_offset, vmat_bb_report *rep, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    vmat_bb_opts opts = {500, 1e-6, 1e-9, 1e-12, 1e12};
    if (opts_in) opts = *opts_in;
    if (opts.max_iter < 1) return set_error(VMAT_EINVAL, "mp_bb_solve: max_iter must be >= 1");
    if (ldg_smem(n_ap) > MP_SMEM_LIMIT) return set_error(VMAT_EUNSUPPORTED, "mp_bb_solve: too many apertures (%d)", n_ap);
    const int32_t n_tiles = (int32_t)((V + MP_THREADS - 1) / MP_THREADS);

    // a column-major input is copied once into the grouped tile layout
    Scratch conv;
    if (tstride == 0) {
        tstride = mp_tile_stride(n_ap);
        VMAT_TRY(conv.alloc((size_t)n_tiles * tstride * sizeof(float), s));
        const int64_t total = (int64_t)n_tiles * tstride;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)ctx->n_sm * 16));
        to_grouped_tiles<<<g, 256, 0, s>>>(DA, ld, V, n_ap, tstride, n_tiles, static_cast<float *>(conv.ptr));
        VMAT_LAUNCH_CHECK();
        DA = static_cast<const float *>(conv.ptr);
    }

    const int stages = tma_stages(n_ap);
    const bool tma = n_ap <= MP_NMAX && tma_smem(n_ap, stages) <= MP_SMEM_LIMIT && tstride % 1024 == 0;
    TmaIterFn tma_fn = tma ? tma_kernel_for(n_ap) : nullptr;
    const size_t smem_pass = tma ? tma_smem(n_ap, stages) : ldg_smem(n_ap);
    const int keep_in_l2 = (double)n_ap * (double)V * 4.0 <= 64.0 * 1024 * 1024 ? 1 : 0;
    static bool attr = false;
    if (!attr) {
        for (int q = 1; q <= MP_NMAX / 8; ++q)
            VMAT_CUDA(cudaFuncSetAttribute(tma_kernel_for(8 * q), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           MP_SMEM_LIMIT));
        VMAT_CUDA(cudaFuncSetAttribute(mp_iter_ldg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_SMEM_LIMIT));
        VMAT_CUDA(cudaFuncSetAttribute(mp_cauchy_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       MP_SMEM_LIMIT));
        attr = true;
    }
    int bps = 1;
    if (tma) VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tma_fn, MP_THREADS, smem_pass));
    else VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, mp_iter_ldg_kernel, MP_THREADS, smem_pass));
    bps = std::max(bps, 1);
    const int P = std::max(1, std::min<int>(n_tiles, ctx->n_sm * bps));
    const int Pc = std::max(1, std::min<int>(n_tiles, ctx->n_sm * 4));

    Scratch ws;
    const size_t bytes = 256 + (size_t)n_ap * (2 * sizeof(double) + sizeof(float)) +
                         (size_t)P * (n_ap + 1) * sizeof(double) + (size_t)Pc * sizeof(double) + 256;
    VMAT_TRY(ws.alloc(bytes, s));
    char *p = static_cast<char *>(ws.ptr);
    MPArgs a;
    a.st = reinterpret_cast<BBState *>(p);
    p += 256;
    a.G = reinterpret_cast<double *>(p);
    a.Gprev = a.G + n_ap;
    a.part = a.Gprev + n_ap;
    a.cpart = a.part + (size_t)P * (n_ap + 1);
    a.yprev = reinterpret_cast<float *>(a.cpart + Pc);
    a.DA = DA;
    a.tstride = tstride;
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
    a.n_tiles = n_tiles;
    a.status = ctx->status;
    a.opts = opts;
    a.F_offset = F_offset;
    const size_t smem_cauchy = (size_t)((n_ap + 3) & ~3) * 4 + 3 * 256 * 4;

    static thread_local BBState *host_st = nullptr;
    if (!host_st) VMAT_CUDA(cudaMallocHost(&host_st, sizeof(BBState)));

    mp_init_kernel<<<1, MP_THREADS, 0, s>>>(a);
    VMAT_LAUNCH_CHECK();
    int launched = 0;
    while (launched < opts.max_iter) {
        const int chunk = launched == 0 ? 1 : std::min(MP_CHUNK, opts.max_iter - launched);
        for (int c = 0; c < chunk; ++c) {
            if (tma) tma_fn<<<P, MP_THREADS, smem_pass, s>>>(a, stages, keep_in_l2);
            else mp_iter_ldg_kernel<<<P, MP_THREADS, smem_pass, s>>>(a);
            g_launches.fetch_add(1, std::memory_order_relaxed);
            if (launched + c == 0) {
                mp_cauchy_pass_kernel<<<Pc, MP_THREADS, smem_cauchy, s>>>(a);
                mp_cauchy_step_kernel<<<1, MP_THREADS, 0, s>>>(a, Pc);
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
    int32_t dev_status = 0;
    VMAT_CUDA(cudaMemcpy(&dev_status, ctx->status, 4, cudaMemcpyDeviceToHost));
    if (dev_status & DEV_TIMEOUT) return set_error(VMAT_ETIMEOUT, "mp_bb_solve: a device-side wait ran out");
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
    return mp_bb_impl(DA, V, n_ap, ld, vox->struct_id, 0, vox, lo, hi, y, z, opts, 0.0, rep, as_stream(stream));
}
