// Master problem (Eq. 6): min F(DA y) subject to lo <= y <= hi, by
// Barzilai-Borwein steps (Eq. 7-8, used alternately) with the subspace scheme
// of Eq. 9-10 and the stopping rules of Section 2.1.
//
// The paper runs four steps per iteration on one GPU (aperture gradient, step
// length with cuBLAS dot products, subspace update, dose update).  Here one
// persistent cooperative kernel runs a whole solve.  DA is kept in a warp-tile
// layout: blocks of 32 voxels, each block a 128-byte head holding the 32 voxels'
// structure labels, then the apertures in groups of four with the four values
// of a voxel side by side,
//     DA(i, k) = DA[(i / 32) * wstride + 32 + (k / 4) * 128 + (i % 32) * 4 + k % 4],
// so the labels and the first n columns of a block are one contiguous run of
// 128 + 512 ceil(n / 4) bytes.  Every warp streams its own blocks into shared
// memory with one bulk copy each (several in flight on the warp's own mbarrier
// ring, continuing across iterations; no CTA-wide barrier in the loop); each
// lane owns a voxel, reads its four-aperture groups with 128-bit shared loads,
// forms z = DA y with four independent chains, the objective term and
// g = -grad F, and adds DA_ik g_i to its register-resident shares of
// G = grad_y F = -DA^T g.  DA is read from HBM (or L2, when it fits there) once
// per iteration.  Objective terms w d^2 are formed in FP32 and summed per lane
// with compensation (Kahan), then as float pairs across lanes and CTAs: the
// voxel loop runs no FP64 instruction (FP64 issues at a small fraction of the
// FP32 rate on this GPU).  After a grid barrier one warp per column reduces the
// CTA partials in a fixed order; after a second barrier every CTA takes the
// same step in shared memory: the Eq. 9-10 freeze, the stopping tests, the BB
// step length (FP64) and the projected update.  The first iteration's Cauchy
// step needs DA G and one more pass.
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

constexpr int MP_THREADS = 256; // voxels per tile of the fallback and Cauchy kernels
constexpr int MP_NW = MP_THREADS / 32;
constexpr int MP_WT = 32;       // voxels per warp tile
constexpr int MP_HEAD = 32;     // floats of a warp tile's label head (128 bytes)
constexpr int MP_CHUNK = 8;     // iterations launched between host polls
constexpr size_t MP_SMEM_LIMIT = 220 * 1024;
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
    uint32_t ticket;  // CTAs of the current pass that have written their partials
    int32_t started;  // elastic batched solver: the state below t was saved by a previous epoch
};

struct MPArgs {
    const float *DA; // warp-tile layout (see above)
    int64_t wstride; // floats per 32-voxel warp tile (32 + 128 * groups)
    int32_t V, n;
    const uint8_t *sid;
    const float *T, *wo, *wu;
    int32_t n_struct;
    float *y;
    float *z;
    const float *lo, *hi; // may be null
    double *G, *Gprev;
    float *yprev;
    double *part;  // fallback solver: [P][n + 1] doubles; persistent solver: two buffers (by iteration
                   // parity) of float pairs, [2][n + 1][pstride] (column k of CTA c at k * pstride + c)
    double *cpart; // [P]
    int32_t P;
    int32_t pstride; // CTAs a persistent partial buffer has room for
    int32_t n_tiles;  // 256-voxel tiles (fallback and Cauchy kernels)
    int64_t n_wtiles; // 32-voxel warp tiles
    BBState *st;
    unsigned *bar_count, *bar_gen; // grid barrier of the persistent solver
    unsigned *epoch_snap;          // elastic batched solver: the batch epoch seen at this problem's last barrier
    const int32_t *skip;           // when non-null and set, the solve is skipped (device-driven plans)
    int32_t *iters_acc;            // when non-null, the persistent solver adds its iteration count
    double *bytes_acc;             // when non-null, the persistent solver adds the bytes its passes moved
    int32_t *status;
    vmat_bb_opts opts;
    double F_offset;
    // Live-tile solves (tiles may be null: every tile): only the warp tiles
    // tiles[0 .. *n_live) of DA are in the problem (the tiles some placed aperture
    // reaches), and *F_off_dev, the constant penalty of the others, is added to F.
    const int32_t *tiles;
    const int32_t *n_live;
    const double *F_off_dev;
    // Packed live tiles (null: read DA's tiles whole): list entry i at 128-byte unit poff[i] of
    // packed, its head (labels, group mask at byte 32) then its marked groups.
    const float *packed;
    const int32_t *poff;
};

__device__ __forceinline__ int64_t min64(int64_t x, int64_t y) { return x < y ? x : y; }

// Offset of DA(voxel i, aperture k) in the warp-tile layout.
__device__ __forceinline__ int64_t da_at(const MPArgs &a, int64_t i, int k) {
    return (i >> 5) * a.wstride + MP_HEAD + (int64_t)(k >> 2) * 128 + ((i & 31) << 2) + (k & 3);
}

__device__ __forceinline__ float lo_of(const MPArgs &a, int k) { return a.lo ? a.lo[k] : 0.f; }
__device__ __forceinline__ float hi_of(const MPArgs &a, int k) { return a.hi ? a.hi[k] : INFINITY; }

__global__ void mp_init_kernel(MPArgs a) {
    if (a.skip && *a.skip) return;
    for (int k = threadIdx.x; k < a.n; k += blockDim.x) a.y[k] = fminf(fmaxf(a.y[k], lo_of(a, k)), hi_of(a, k));
    if (threadIdx.x == 0) {
        BBState s = {};
        *a.st = s;
        if (a.bar_count) {
            *a.bar_count = 0u;
            *a.bar_gen = 0u;
        }
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
            else a.st->F = s + a.F_offset + (a.F_off_dev ? __ldcg(a.F_off_dev) : 0.0);
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

// Per-voxel part of an iteration for voxel i with dose zi (fallback kernel):
// returns g_i, adds F_i to facc.
__device__ __forceinline__ float voxel_terms(const float *sT, const float *sO, const float *sU, int s, float zi,
                                             double &facc) {
    const float d = zi - sT[s];
    const float w = d > 0.f ? sO[s] : sU[s];
    facc += (double)((w * d) * d);
    return -2.f * w * d; // g = -grad F: -2 w+ (z - T) above, +2 w- (T - z) below
}

// Ends a pass: write this CTA's partials; the last of the n_cta CTAs reduces them and steps.
__device__ void pass_epilogue(const MPArgs &a, const double *accG, double facc, int cta, int n_cta) {
    __shared__ double sh[MP_NW];
    __shared__ bool last;
    const int tid = threadIdx.x;
    const double fb = block_reduce_sum(facc, sh);
    double *out = a.part + (int64_t)cta * (a.n + 1);
    for (int k = tid; k < a.n; k += MP_THREADS) out[k] = accG[k];
    if (tid == 0) out[a.n] = fb;
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&a.st->ticket, 1u) == (unsigned)n_cta - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    reduce_partials(a, n_cta);
    bb_step(a);
    if (tid == 0) a.st->ticket = 0u;
}

// Bytes one bulk copy brings for n apertures: a warp tile's label head and its first ceil(n/4) groups.
__host__ __device__ constexpr size_t wt_copy_bytes(int n) { return 128 + (size_t)((n + 3) / 4) * 512; }

// ---------------------------------------------------------------------------
// Persistent solver: one cooperative launch runs the whole BB loop.  Every
// iteration is a pass over DA (each warp streams its own tiles), a grid
// barrier, a column reduction of the CTA partials (one warp per column), a
// second grid barrier, and the step, which every CTA computes identically in
// its own shared memory from the same reduced values.  Cross-thread sums of
// FP32 values are formed as unevaluated float pairs (hi + lo, Knuth's TwoSum),
// in a fixed order; the BB dot products, F and the step stay FP64.
// ---------------------------------------------------------------------------
struct FF {
    float hi, lo;
};

// (a.hi + a.lo) + (b.hi + b.lo) as a float pair: TwoSum of the high parts, then
// the low parts, renormalised.  No multiply, so no FMA contraction applies.
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    const float e = (a.hi - (s - bv)) + (b.hi - bv);
    const float t = e + (a.lo + b.lo);
    const float h = s + t;
    return FF{h, t - (h - s)};
}

__device__ __forceinline__ FF ff_shfl_xor(FF v, int d) {
    return FF{__shfl_xor_sync(0xffffffffu, v.hi, d), __shfl_xor_sync(0xffffffffu, v.lo, d)};
}

__device__ __forceinline__ double ff_to_double(FF v) { return (double)v.hi + (double)v.lo; }

// Grid barrier over n_cta co-resident CTAs (cooperative launch): arrival counter
// plus a generation word.  Gives up after WAIT_LIMIT_CYCLES; returns false then.
// When snap_dst is given, the last CTA to arrive copies *snap_src there before it
// releases the others, so every CTA of the barrier reads the same value after it.
__device__ bool grid_sync(unsigned *count, unsigned *gen, unsigned n_cta, unsigned *snap_dst = nullptr,
                          const unsigned *snap_src = nullptr) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vg = gen;
        const unsigned g0 = *vg;
        __threadfence();
        int ok = 1;
        if (atomicAdd(count, 1u) == n_cta - 1) {
            if (snap_dst) *(volatile unsigned *)snap_dst = *(const volatile unsigned *)snap_src;
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g0) {
                if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Grid barrier of a solve whose CTAs stay with it from start to end: one arrival
// counter that only grows (zeroed by the init kernel before the launch); the e-th
// barrier (e = 1, 2, ...) ends when the counter reaches e n_cta.  No CTA reads a word
// before it arrives and no CTA resets one after the last arrival, so the barrier ends
// one round trip after the last arrival.  Gives up after WAIT_LIMIT_CYCLES; returns
// false then.
__device__ bool grid_sync_count(unsigned *count, unsigned target) {
    __shared__ int ok_c;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        const long long t0 = clock64();
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if ((int)(v - target) >= 0) break;
            if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        ok_c = ok;
    }
    __syncthreads();
    return ok_c != 0;
}

// Barrier of the whole batched grid.  The last CTA to arrive records the batch
// epoch (gctl[3]) and the set of problems still iterating (gctl[4..5]) before it
// releases the others: the CTA split that follows reads only these words, which
// no CTA changes until every CTA has arrived at the next batch barrier.
struct MPArgs;
__device__ bool batch_sync(unsigned *gctl, unsigned n_cta, const MPArgs *args, int n_plans);

// Solver state every CTA keeps in shared memory (identical in all CTAs).
struct PState {
    double F_hist[6];
    double F, delta0, gg, delta;
    int t, done, stop, decided;
    int passes; // passes over DA (iterations and the Cauchy pass)
    int stop_rel, stop_step; // the step's stopping tests, formed in parallel
    double delta_c;          // the step's BB step size, formed in parallel
};

struct SolveSmem {
    unsigned char *stage0; // [MP_NW][stages][cbytes]
    float4 *sy4;           // [GMAX]   y, zero-padded
    float4 *sg4;           // [GMAX]   G as float (Cauchy pass), zero-padded
    double *sG, *sGp;      // [NMAX]   G_t, G_{t-1}
    double *sS, *sR;       // [NMAX]   s = y_t - y_{t-1}, r = G_t - G_{t-1} (the step's inputs)
    double *sRed;          // [8]      the step's sums and maxima
    FF *sGff;              // [NMAX + 1] the reduced sums as float pairs: -G, then F (converted in the step)
    float *sYp;            // [NMAX]   y_{t-1}
    float *wred;           // [MP_NW][NMAX]
    float *sT, *sO, *sU;   // [256]
    uint64_t *bars;        // [MP_NW][PQ]
    uint32_t *ring_meta;   // [MP_NW][PQ][2] packed tiles: ring offset, bytes held
    int32_t *wlist;        // [MP_NW][WL_CAP][3] the warp's first tiles: tile, packed unit offset, units
};

// Resident CTAs per SM the persistent solvers are compiled for (a register budget): more
// CTAs for fewer apertures, whose tiles are small and whose warps wait on copies.
__host__ __device__ constexpr int mp_min_ctas(int nmax) { return nmax <= 8 ? 4 : (nmax <= 24 ? 3 : (nmax <= 48 ? 2 : 1)); }

// Copies in flight per warp at most (mbarriers per warp): the tile stages of whole tiles, or
// the packed tiles that fit in the warp's byte ring.
constexpr int PQ = 8;
// Tiles of a warp whose index and packed place are kept in shared memory (loaded once per
// solve, so that issuing a copy and placing a tile's voxels wait on no global load); a
// warp's tiles past the first WL_CAP are looked up in global memory.
constexpr int WL_CAP = 64;

template <int NMAX> __host__ __device__ constexpr size_t solve_fixed_smem() {
    return 128 /* alignment slack */ + 2 * (NMAX / 4) * 16 + 4 * (size_t)NMAX * 8 + 8 * 8 + 8 * (size_t)(NMAX + 1) +
           (size_t)NMAX * 4 +
           (size_t)MP_NW * NMAX * 4 + 3 * 256 * 4 + (size_t)MP_NW * PQ * (8 + 8) + (size_t)MP_NW * WL_CAP * 12;
}

// Bulk copy of the warp's pipeline slot `it` (global tile-use index across passes).
struct WarpPipe {
    unsigned char *my;
    uint64_t *mb;
    const unsigned char *src;
    int64_t tile_bytes, w0, W, n_my;
    const int32_t *tiles; // warp tile of list entry q (null: tile q)
    int64_t it_base; // pipeline slot of this tile set's first tile
    uint32_t cbytes;
    int stages;
    uint64_t pol;
    // Packed tiles (poff non-null): each is copied whole into the warp's byte ring (stages *
    // cbytes bytes, the tiles in issue order, a tile that would cross the end starting again
    // at 0), up to PQ copies in flight, as many as the ring holds.  Lane 0 is the producer.
    const unsigned char *packed; // packed live tiles
    const int32_t *poff;         // list entry q at 128-byte unit poff[q] of packed
    uint32_t *moff, *mspan;      // [PQ] per slot: ring offset of its tile, ring bytes it holds
    int32_t *wl;                 // [WL_CAP][3] this warp's tile j: tile, packed unit offset, units
    uint32_t ring_bytes;
    int64_t iss;                 // lane 0: the next tile to issue
    int64_t jiss;                // lane 0: its place in the warp's tile cycle, (iss - it_base) mod n_my
    uint32_t pos, span;          // lane 0: ring write position, ring bytes held by tiles in flight
    __device__ __forceinline__ int64_t tile_of(int64_t q) const { return tiles ? (int64_t)__ldg(tiles + q) : q; }
    // the warp's tile j (0 <= j < n_my): tile index, from the shared list when it holds it
    __device__ __forceinline__ int64_t my_tile(int64_t j) const {
        return j < WL_CAP ? (int64_t)wl[3 * j] : tile_of(w0 + j * W);
    }
    __device__ __forceinline__ void issue(int64_t it) const {
        const int s = (int)((uint32_t)it % (uint32_t)stages);
        const int64_t wt = my_tile((uint32_t)(it - it_base) % (uint32_t)n_my);
        mbar_arrive_expect_tx(&mb[s], cbytes);
        bulk_g2s(my + (size_t)s * cbytes, src + wt * tile_bytes, cbytes, &mb[s], pol);
    }
    __device__ __forceinline__ bool wait(int64_t it) const {
        return mbar_wait_bounded(&mb[(uint32_t)it % (uint32_t)stages], ((uint32_t)it / (uint32_t)stages) & 1u,
                                 WAIT_LIMIT_CYCLES);
    }
    // packed: issue tiles iss, iss + 1, ... while fewer than PQ are in flight past tile `it`
    // (the next to be consumed) and the ring has room (lane 0)
    __device__ __forceinline__ void fill(int64_t it) {
        if (span == 0) pos = 0; // an empty ring: any tile fits from its start
        while (iss - it < PQ) {
            const int64_t j = jiss;
            int64_t u0;
            uint32_t units;
            if (j < WL_CAP) {
                u0 = wl[3 * j + 1];
                units = (uint32_t)wl[3 * j + 2];
            } else {
                const int64_t q = w0 + j * W;
                u0 = __ldg(poff + q);
                units = (uint32_t)(__ldg(poff + q + 1) - u0);
            }
            const uint32_t bytes = units * 128u; // at most cbytes <= ring_bytes
            uint32_t start = pos, gap = 0;
            if (pos + bytes > ring_bytes) { // the ring's end: skip the rest, start at 0
                gap = ring_bytes - pos;
                start = 0;
            }
            if (span + gap + bytes > ring_bytes) break;
            const int s = (int)(iss % PQ);
            moff[s] = start;
            mspan[s] = gap + bytes;
            mbar_arrive_expect_tx(&mb[s], bytes);
            bulk_g2s(my + start, packed + u0 * 128, bytes, &mb[s], pol);
            pos = start + bytes;
            span += gap + bytes;
            ++iss;
            if (++jiss == n_my) jiss = 0;
        }
    }
    // after consuming tile `it` (lane 0): packed, release its ring bytes and top the ring up;
    // whole tiles, reuse its slot for the tile `stages` ahead
    __device__ __forceinline__ void refill(int64_t it, bool packed_mode) {
        if (packed_mode) {
            span -= mspan[it % PQ];
            fill(it + 1);
        } else {
            issue(it + stages);
        }
    }
    __device__ __forceinline__ bool wait_packed(int64_t it) const {
        return mbar_wait_bounded(&mb[it % PQ], (uint32_t)((it / PQ) & 1), WAIT_LIMIT_CYCLES);
    }
};

enum { PASS_ITER = 0, PASS_CAUCHY = 1 };

// One sweep over this warp's tiles.  PASS_ITER: z = DA y, objective terms, G
// shares; PASS_CAUCHY: q = DA G and the curvature terms w q^2.  Consumes
// pipeline slots it .. it + n_my - 1 (advancing it) and issues slot + stages
// after each.  Returns false (it at the slot) if a copy never landed.
template <int NMAX, int MODE, bool PACKED>
__device__ __forceinline__ bool solve_pass(const MPArgs &a, const SolveSmem &S, WarpPipe &P, int64_t &it,
                                           float *gacc, float &fs, float &fc) {
    constexpr int GMAX = NMAX / 4;
    // From 56 to 72 apertures (one CTA per SM, registers to spare) a tile's groups stay in
    // registers between the dose and the G shares, so its slot is refilled before the
    // objective; the Cauchy pass reads the slot once and refills at the same point.
    constexpr bool KEEP = NMAX >= 56 && NMAX <= 72 && MODE == PASS_ITER;
    constexpr bool EARLY = KEEP || MODE == PASS_CAUCHY;
    const int G = (a.n + 3) >> 2;
    const int lane = threadIdx.x & 31;
    for (int64_t j = 0; j < P.n_my; ++j, ++it) {
        const bool ok = PACKED ? P.wait_packed(it) : P.wait(it);
        if (!__all_sync(0xffffffffu, ok)) return false;
        const unsigned char *blk =
            PACKED ? P.my + P.moff[it % PQ] : P.my + (size_t)((uint32_t)it % (uint32_t)P.stages) * P.cbytes;
        const float4 *D4 = reinterpret_cast<const float4 *>(blk + 128) + lane; // group g at D4[32 g]
        const float4 *w4 = MODE == PASS_ITER ? S.sy4 : S.sg4;
        // packed: the marked groups only, in order (a group left out holds zeros, which add nothing)
        const uint32_t gm = PACKED ? reinterpret_cast<const uint32_t *>(blk)[8] : 0u;
        float4 vk[KEEP ? GMAX : 1];
        float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
        int slot = 0;
#pragma unroll
        for (int g = 0; g < GMAX; ++g)
            if (g < G && (!PACKED || ((gm >> g) & 1u))) {
                const float4 v = D4[32 * (PACKED ? slot++ : g)], w = w4[g];
                if (KEEP) vk[KEEP ? g : 0] = v;
                z0 = fmaf(v.x, w.x, z0);
                z1 = fmaf(v.y, w.y, z1);
                z2 = fmaf(v.z, w.z, z2);
                z3 = fmaf(v.w, w.w, z3);
            }
        const int sid = blk[lane];
        if (EARLY) {
            __syncwarp(); // every lane's reads of this slot are done before its next copy
            if (lane == 0) P.refill(it, PACKED);
        }
        const float zi = (z0 + z1) + (z2 + z3);
        const int64_t i = P.my_tile(j) * MP_WT + lane;
        float gi = 0.f;
        if (i < a.V) {
            if (MODE == PASS_ITER) {
                a.z[i] = zi;
                const float d = zi - S.sT[sid];
                const float w = d > 0.f ? S.sO[sid] : S.sU[sid];
                const float yk = (w * d) * d - fc; // Kahan step
                const float tk = fs + yk;
                fc = (tk - fs) - yk;
                fs = tk;
                gi = -2.f * w * d; // g = -grad F: -2 w+ (z - T) above, +2 w- (T - z) below
            } else {
                // curvature of F along DA G: the active weight (0 exactly at the threshold)
                const float zc = a.z[i], T = S.sT[sid];
                const float w = zc > T ? S.sO[sid] : (zc < T ? S.sU[sid] : 0.f);
                const float yk = (w * zi) * zi - fc;
                const float tk = fs + yk;
                fc = (tk - fs) - yk;
                fs = tk;
            }
        }
        if (MODE == PASS_ITER) {
            slot = 0;
#pragma unroll
            for (int g = 0; g < GMAX; ++g)
                if (g < G && (!PACKED || ((gm >> g) & 1u))) {
                    const float4 v = KEEP ? vk[KEEP ? g : 0] : D4[32 * (PACKED ? slot++ : g)];
                    gacc[4 * g + 0] = fmaf(v.x, gi, gacc[4 * g + 0]);
                    gacc[4 * g + 1] = fmaf(v.y, gi, gacc[4 * g + 1]);
                    gacc[4 * g + 2] = fmaf(v.z, gi, gacc[4 * g + 2]);
                    gacc[4 * g + 3] = fmaf(v.w, gi, gacc[4 * g + 3]);
                }
        }
        if (!EARLY) {
            __syncwarp(); // every lane's reads of this slot are done before its next copy
            if (lane == 0) P.refill(it, PACKED);
        }
    }
    return true;
}

// The warp's sums over its 32 lanes of the G shares gacc[0 .. n), written to out[0 .. n).
// From 16 apertures on, by halving exchanges over 32-column chunks: at the exchange of
// width w each lane keeps half of its remaining columns (the upper half when its lane bit
// w is set), sends the other half to lane ^ w and adds what it receives; after five
// exchanges lane l holds column l of the chunk.  31 shuffles per chunk instead of 5 per
// column.  Columns at or past n hold zero (their DA groups are zero padding).  A fixed
// order: every warp of every CTA adds the same way.
template <int NMAX>
__device__ __forceinline__ void warp_share_sums(const float *gacc, int n, float *out, int lane) {
    if (NMAX < 16) {
#pragma unroll
        for (int k = 0; k < NMAX; ++k) {
            if (k < n) {
                float x = gacc[k];
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
                if (lane == 0) out[k] = x;
            }
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < (NMAX + 31) / 32; ++c) {
        if (32 * c < n) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = 32 * c + i < NMAX ? gacc[32 * c + i] : 0.f;
#pragma unroll
            for (int w = 16; w >= 1; w >>= 1) {
                const bool up = (lane & w) != 0;
#pragma unroll
                for (int i = 0; i < w; ++i) {
                    const float send = up ? v[i] : v[i + w];
                    const float keep = up ? v[i + w] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
                }
            }
            if (32 * c + lane < n) out[32 * c + lane] = v[0];
        }
    }
}

// CTA sum of one float pair per thread (result in thread 0): warp butterflies, warps in order.
__device__ FF block_ff(FF v, FF *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v = ff_add(v, ff_shfl_xor(v, d));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    FF t = sh[0];
    if (threadIdx.x == 0)
        for (int w = 1; w < MP_NW; ++w) t = ff_add(t, sh[w]);
    __syncthreads();
    return t;
}

// Eq. 9-10 freeze, stopping tests, BB step length (FP64) and projected update, on the
// shared-memory copy of the state, run by the whole CTA.  FP64 issues at a small
// fraction of the FP32 rate on this GPU and one warp's chain of FP64 operations was
// the step's cost, so the work is spread: one aperture per thread (freeze, s, r),
// then one warp per sum or maximum (each lane over apertures l, l + 32, ... in
// order, then a fixed butterfly), then thread 0 decides.  Every CTA runs it on
// identical inputs.  Ends synchronised.
template <int NMAX>
__device__ void solve_step_cta(const MPArgs &a, const SolveSmem &S, PState &ps) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int n = a.n, t = ps.t;
    float *y = reinterpret_cast<float *>(S.sy4);
    // FP64 issues at a small fraction of the FP32 rate on this GPU: the reduced float pairs
    // are converted here, one column per thread, not one column per warp instruction
    if (tid == MP_THREADS - 1) ps.F = ff_to_double(S.sGff[n]) + a.F_offset + (a.F_off_dev ? __ldcg(a.F_off_dev) : 0.0);
    for (int k = tid; k < n; k += MP_THREADS) {
        float yk = y[k];
        const float l = lo_of(a, k), h = hi_of(a, k);
        const FF gf = S.sGff[k]; // g = -(hi + lo): its sign from a float compare (the pair's sum is not rounded to 0)
        double g = -ff_to_double(gf);
        if (yk <= l && gf.hi < -gf.lo) {
            yk = l;
            g = 0.0;
        } else if (yk >= h && gf.hi > -gf.lo) {
            yk = h;
            g = 0.0;
        }
        y[k] = yk;
        S.sG[k] = g;
        if (t > 0) {
            S.sS[k] = (double)yk - (double)S.sYp[k];
            S.sR[k] = g - S.sGp[k];
        }
    }
    __syncthreads();
    // Warp 0: the four sums, eight lanes each (lanes 8q .. 8q + 7: 0 G.G, 1 s.s, 2 s.r,
    // 3 r.r), lane j of a group over apertures j, j + 8, ... in order, then a fixed
    // butterfly of the group: one warp's FP64 instructions serve all four.  Warp 1: the
    // maxima |s| (lanes 0-15) and |y| (lanes 16-31) as integer maxima of the bit
    // patterns of non-negative values (the order of their values), off the FP64 pipe.
    // (the group's operands come through selected pointers, so that the warp does not
    // diverge; at t = 0 the groups other than G.G read stale values, never used)
    if (wid == 0) {
        const int q = lane >> 3, j = lane & 7;
        const double *xa = q == 0 ? S.sG : (q == 3 ? S.sR : S.sS);
        const double *za = q == 2 ? S.sR : xa;
        double v = 0.0;
        for (int k = j; k < n; k += 8) v += xa[k] * za[k];
#pragma unroll
        for (int d = 4; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        if (j == 0) S.sRed[q] = v;
    } else if (wid == 1) {
        const bool ys = lane >= 16;
        const int j = lane & 15;
        unsigned long long m = 0;
        if (ys) {
            for (int k = j; k < n; k += 16) m = max(m, (unsigned long long)(__float_as_uint(y[k]) & 0x7fffffffu));
        } else if (t > 0) {
            for (int k = j; k < n; k += 16)
                m = max(m, (unsigned long long)__double_as_longlong(S.sS[k]) & 0x7fffffffffffffffull);
        }
#pragma unroll
        for (int d = 8; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
        if (j == 0) S.sRed[ys ? 5 : 4] = ys ? (double)__uint_as_float((unsigned)m) : __longlong_as_double((long long)m);
    }
    __syncthreads();
    // the two stopping tests and the BB step size, each by lane 0 of its own warp (their
    // FP64 chains run side by side); thread 0 then decides in the sequential order
    if (lane == 0 && wid < 3) {
        const double ss = S.sRed[1], sr = S.sRed[2], rr = S.sRed[3], dy = S.sRed[4], ymax = S.sRed[5];
        if (wid == 0) {
            const double F = ps.F;
            ps.stop_rel = t >= 5 && fabs(ps.F_hist[(t - 5) % 6] - F) <= a.opts.rel_tol5 * F;
        } else if (wid == 1) {
            ps.stop_step = t >= 1 && dy <= a.opts.step_tol * fmax(1.0, ymax);
        } else if (t > 0) {
            double delta;
            if (sr <= 0.0) delta = a.opts.delta_max * ps.delta0;
            else if (t & 1) delta = sr / rr;
            else delta = ss / sr;
            ps.delta_c = fmin(fmax(delta, a.opts.delta_min * ps.delta0), a.opts.delta_max * ps.delta0);
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double gg = S.sRed[0];
        ps.decided = 1;
        ps.F_hist[t % 6] = ps.F;
        if (ps.stop_rel) {
            ps.done = 1;
            ps.stop = VMAT_STOP_REL;
        } else if (ps.stop_step) {
            ps.done = 1;
            ps.stop = VMAT_STOP_STEP;
        } else if (t == a.opts.max_iter - 1) {
            ps.done = 1;
            ps.stop = VMAT_STOP_MAXIT;
        } else if (t == 0) {
            if (gg == 0.0) {
                ps.done = 1;
                ps.stop = VMAT_STOP_GRAD0;
            } else {
                ps.gg = gg;
                ps.decided = 2; // the first step is the Cauchy step (needs DA G)
            }
        } else {
            ps.delta = ps.delta_c;
            ps.decided = 0;
        }
    }
    __syncthreads();
}

// y <- clamp(y - delta G) after saving (y, G) as the previous iterate, one aperture
// per thread (the whole CTA).  Ends synchronised.
__device__ void solve_take_step_cta(const MPArgs &a, const SolveSmem &S, double delta) {
    float *y = reinterpret_cast<float *>(S.sy4);
    for (int k = threadIdx.x; k < a.n; k += MP_THREADS) {
        const float yk = y[k];
        S.sYp[k] = yk;
        S.sGp[k] = S.sG[k];
        const double yn = (double)yk - delta * S.sG[k];
        y[k] = fminf(fmaxf((float)yn, lo_of(a, k)), hi_of(a, k));
    }
    __syncthreads();
}

// Shared-memory layout of the solver for NMAX apertures and `stages` tiles per warp.
template <int NMAX> __device__ __forceinline__ SolveSmem solve_layout(unsigned char *sm, int stages, uint32_t cbytes) {
    constexpr int GMAX = NMAX / 4;
    SolveSmem S;
    S.stage0 = sm;
    S.sy4 = reinterpret_cast<float4 *>(sm + (size_t)MP_NW * stages * cbytes);
    S.sg4 = S.sy4 + GMAX;
    S.sG = reinterpret_cast<double *>(S.sg4 + GMAX);
    S.sGp = S.sG + NMAX;
    S.sS = S.sGp + NMAX;
    S.sR = S.sS + NMAX;
    S.sRed = S.sR + NMAX;
    S.sGff = reinterpret_cast<FF *>(S.sRed + 8);
    S.sYp = reinterpret_cast<float *>(S.sGff + NMAX + 1);
    S.wred = S.sYp + NMAX;
    S.sT = S.wred + MP_NW * NMAX;
    S.sO = S.sT + 256;
    S.sU = S.sO + 256;
    S.bars = reinterpret_cast<uint64_t *>(S.sU + 256);
    S.ring_meta = reinterpret_cast<uint32_t *>(S.bars + MP_NW * PQ);
    S.wlist = reinterpret_cast<int32_t *>(S.ring_meta + MP_NW * PQ * 2);
    return S;
}

// Loads one problem's tables and state into shared memory: a fresh start (y from
// a.y, clamped by the init kernel) or, for the elastic solver, the state a
// previous epoch saved (t, F history, step scale, y, y_prev, G_prev).
template <int NMAX> __device__ void solve_load(const MPArgs &a, const SolveSmem &S, PState &ps, bool resume) {
    constexpr int GMAX = NMAX / 4;
    const int n = a.n, tid = threadIdx.x;
    for (int k = tid; k < 4 * GMAX; k += MP_THREADS) {
        reinterpret_cast<float *>(S.sy4)[k] = k < n ? a.y[k] : 0.f;
        reinterpret_cast<float *>(S.sg4)[k] = 0.f;
    }
    for (int k = tid; k < a.n_struct; k += MP_THREADS) {
        S.sT[k] = a.T[k];
        S.sO[k] = a.wo[k];
        S.sU[k] = a.wu[k];
    }
    if (resume)
        for (int k = tid; k < n; k += MP_THREADS) {
            S.sYp[k] = a.yprev[k];
            S.sGp[k] = a.Gprev[k];
        }
    if (tid == 0) {
        PState z = {};
        ps = z;
        if (resume) {
            for (int i = 0; i < 6; ++i) ps.F_hist[i] = a.st->F_hist[i];
            ps.F = a.st->F;
            ps.delta0 = a.st->delta0;
            ps.gg = a.st->gg;
            ps.t = a.st->t;
        }
    }
    __syncthreads();
}

// The state a later epoch resumes from (one CTA writes it).
template <int NMAX> __device__ void solve_save(const MPArgs &a, const SolveSmem &S, const PState &ps) {
    const float *y = reinterpret_cast<const float *>(S.sy4);
    for (int k = threadIdx.x; k < a.n; k += MP_THREADS) {
        a.y[k] = y[k];
        a.yprev[k] = S.sYp[k];
        a.Gprev[k] = S.sGp[k];
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 6; ++i) a.st->F_hist[i] = ps.F_hist[i];
        a.st->F = ps.F;
        a.st->delta0 = ps.delta0;
        a.st->gg = ps.gg;
        a.st->t = ps.t;
        a.st->started = 1;
    }
    __threadfence();
}

// The end of a solve (one CTA): y, the report and the iteration count.
template <int NMAX> __device__ void solve_finish(const MPArgs &a, const SolveSmem &S, const PState &ps, bool ok) {
    const float *y = reinterpret_cast<const float *>(S.sy4);
    if (ok)
        for (int k = threadIdx.x; k < a.n; k += MP_THREADS) a.y[k] = y[k];
    if (threadIdx.x == 0) {
        a.st->F = ps.F;
        a.st->t = ps.t;
        a.st->done = 1;
        a.st->stop = ok ? ps.stop : VMAT_STOP_MAXIT;
        a.st->iters = ps.t + 1;
        a.st->delta0 = ps.delta0;
        if (ok && a.iters_acc) *a.iters_acc += ps.t + 1;
        if (ok && a.bytes_acc) { // each pass reads the tiles' labels and columns and writes (or reads) their dose
            const int64_t tiles = a.tiles ? min64((int64_t)max(__ldcg(a.n_live), 0), a.n_wtiles) : a.n_wtiles;
            const double per_tile_read = a.poff ? 0.0 : (double)wt_copy_bytes(a.n);
            const double packed_read = a.poff ? 128.0 * (double)__ldcg(a.poff + tiles) : 0.0;
            *a.bytes_acc += (double)ps.passes * ((double)tiles * (per_tile_read + 4.0 * MP_WT) + packed_read);
        }
    }
    __threadfence();
}

enum { LOOP_DONE = 0, LOOP_ABORT = 1, LOOP_REBALANCE = 2 };

// BB iterations of one problem as CTA `cta` of n_cta, until a stopping rule
// (LOOP_DONE), a wait that ran out (LOOP_ABORT) or, for the elastic solver
// (epoch_src non-null), a change of the batch epoch seen at the second barrier of
// an iteration (LOOP_REBALANCE, after this CTA has saved the state if cta == 0).
template <int NMAX>
__device__ int solve_loop(const MPArgs &a, const SolveSmem &S, WarpPipe &P, PState &ps, int64_t &it,
                          const unsigned cta, const unsigned n_cta, const unsigned *epoch_src, unsigned epoch_local) {
    constexpr int GMAX = NMAX / 4;
    __shared__ FF shff[MP_NW];
    __shared__ int abort_s;
    const int n = a.n;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) abort_s = 0;
    __syncthreads();
    // the single-problem solve (no epochs) keeps its CTAs: its barriers count arrivals
    // on one growing counter; the elastic solver's use the counter and generation pair
    unsigned bar_e = 0;
    auto sync_grid = [&](bool snap) -> bool {
        if (!epoch_src) return grid_sync_count(a.bar_count, ++bar_e * n_cta);
        return snap ? grid_sync(a.bar_count, a.bar_gen, n_cta, a.epoch_snap, epoch_src)
                    : grid_sync(a.bar_count, a.bar_gen, n_cta);
    };
    float gacc[NMAX];
    FF *part = reinterpret_cast<FF *>(a.part);
    FF *cpart = reinterpret_cast<FF *>(a.cpart);
    while (true) {
        // ---- pass: z = DA y, g, F and this CTA's shares of G = -DA^T g
#pragma unroll
        for (int k = 0; k < NMAX; ++k) gacc[k] = 0.f;
        float fs = 0.f, fc = 0.f;
        const bool pass_ok = P.n_my == 0 || (P.poff ? solve_pass<NMAX, PASS_ITER, true>(a, S, P, it, gacc, fs, fc)
                                                    : solve_pass<NMAX, PASS_ITER, false>(a, S, P, it, gacc, fs, fc));
        if (tid == 0) ++ps.passes;
        if (!pass_ok && lane == 0) atomicOr(&abort_s, 1);
        warp_share_sums<NMAX>(gacc, n, S.wred + wid * NMAX, lane);
        const FF fb = block_ff(FF{fs, -fc}, shff); // includes a __syncthreads after wred
        // this CTA's partials, column-major by CTA, in the buffer of this iteration's parity: a CTA
        // writes buffer b again two iterations later, after the barrier that every CTA reaches only
        // once it has read buffer b
        FF *pb = part + (size_t)(ps.t & 1) * (n + 1) * a.pstride;
        for (int k = tid; k < n; k += MP_THREADS) {
            FF sum{S.wred[k], 0.f};
            for (int w = 1; w < MP_NW; ++w) sum = ff_add(sum, FF{S.wred[w * NMAX + k], 0.f});
            pb[(size_t)k * a.pstride + cta] = sum;
        }
        if (tid == 0) pb[(size_t)n * a.pstride + cta] = fb;
        if (abort_s || !sync_grid(true)) return LOOP_ABORT;
        // ---- every CTA reduces every column itself: warp w takes columns w, w + MP_NW, ...,
        // CB at a time with eight loads per column in flight per lane (every load of the group
        // issued before the first add; CB grows with NMAX, whose kernels have fewer CTAs per SM
        // and more columns per warp, and stays 1 where registers set the CTAs per SM); lane l
        // sums CTAs l, l + 32, ... in order, then a fixed butterfly: the same G and F in every
        // CTA, with no second barrier
        constexpr int CB = NMAX >= 56 ? 4 : (NMAX >= 32 ? 2 : 1);
        for (int k0 = wid; k0 <= n; k0 += MP_NW * CB) {
            FF v[CB];
#pragma unroll
            for (int j = 0; j < CB; ++j) v[j] = FF{0.f, 0.f};
            for (unsigned b0 = lane; b0 < n_cta; b0 += 32 * 8) {
                float2 q[CB][8];
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    const int k = k0 + MP_NW * j;
                    const float2 *col = reinterpret_cast<const float2 *>(pb + (size_t)min(k, n) * a.pstride);
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const unsigned b = b0 + 32u * u;
                        q[j][u] = k <= n && b < n_cta ? __ldcg(col + b) : make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int j = 0; j < CB; ++j)
#pragma unroll
                    for (int u = 0; u < 8; ++u) v[j] = ff_add(v[j], FF{q[j][u].x, q[j][u].y});
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1)
#pragma unroll
                for (int j = 0; j < CB; ++j) v[j] = ff_add(v[j], ff_shfl_xor(v[j], d));
            if (lane == 0) { // float pairs: the step converts them a column per thread
#pragma unroll
                for (int j = 0; j < CB; ++j) {
                    const int k = k0 + MP_NW * j;
                    if (k <= n) S.sGff[k] = v[j];
                }
            }
        }
        __syncthreads();
        solve_step_cta<NMAX>(a, S, ps);
        if (ps.decided == 0) solve_take_step_cta(a, S, ps.delta);
        if (ps.decided == 2) {
            // ---- Cauchy step: delta0 = G.G / (2 sum_i w_i (DA G)_i^2)
            for (int k = tid; k < 4 * GMAX; k += MP_THREADS)
                reinterpret_cast<float *>(S.sg4)[k] = k < n ? (float)S.sG[k] : 0.f;
            __syncthreads();
            float cs = 0.f, cc = 0.f;
            const bool c_ok = P.n_my == 0 || (P.poff ? solve_pass<NMAX, PASS_CAUCHY, true>(a, S, P, it, gacc, cs, cc)
                                                      : solve_pass<NMAX, PASS_CAUCHY, false>(a, S, P, it, gacc, cs, cc));
            if (tid == 0) ++ps.passes;
            if (!c_ok && lane == 0) atomicOr(&abort_s, 1);
            const FF cb = block_ff(FF{cs, -cc}, shff);
            if (tid == 0) cpart[cta] = cb;
            if (abort_s || !sync_grid(false)) return LOOP_ABORT;
            if (wid == 0) {
                FF v{0.f, 0.f};
                for (unsigned b0 = lane; b0 < n_cta; b0 += 32 * 8) {
                    float2 q[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const unsigned b = b0 + 32u * u;
                        q[u] = b < n_cta ? __ldcg(reinterpret_cast<const float2 *>(cpart) + b) : make_float2(0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) v = ff_add(v, FF{q[u].x, q[u].y});
                }
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) v = ff_add(v, ff_shfl_xor(v, d));
                const double curv = 2.0 * ff_to_double(v);
                if (lane == 0) {
                    if (curv == 0.0) {
                        ps.done = 1;
                        ps.stop = VMAT_STOP_FLAT;
                    } else {
                        ps.delta0 = ps.gg / curv;
                    }
                }
            }
            __syncthreads();
            if (!ps.done) solve_take_step_cta(a, S, ps.delta0);
        }
        if (ps.done) return LOOP_DONE;
        if (tid == 0) ++ps.t;
        __syncthreads();
        if (epoch_src && __ldcg(a.epoch_snap) != epoch_local) { // the same word for every CTA of the problem
            if (cta == 0) solve_save<NMAX>(a, S, ps);
            return LOOP_REBALANCE;
        }
    }
}

// Sets up a warp's pipeline for tiles w0, w0 + W, ... of problem a, starting at slot it.
__device__ __forceinline__ void pipe_start(WarpPipe &P, const MPArgs &a, unsigned cta, unsigned n_cta, int64_t it) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P.src = reinterpret_cast<const unsigned char *>(a.DA);
    P.tile_bytes = a.wstride * 4;
    P.W = (int64_t)n_cta * MP_NW;
    P.w0 = (int64_t)cta * MP_NW + wid;
    P.tiles = a.tiles;
    P.packed = reinterpret_cast<const unsigned char *>(a.packed);
    P.poff = a.packed ? a.poff : nullptr;
    P.iss = it;
    P.jiss = 0;
    P.pos = 0;
    P.span = 0;
    int64_t n_wt = a.n_wtiles;
    if (a.tiles) // the live list: written by earlier kernels of the stream, fixed during the solve
        n_wt = min64((int64_t)max(__ldcg(a.n_live), 0), a.n_wtiles);
    P.n_my = P.w0 < n_wt ? (n_wt - 1 - P.w0) / P.W + 1 : 0;
    P.it_base = it;
    // the warp's first WL_CAP tiles: index, and the packed place when packed (lane per tile)
    for (int64_t j = lane; j < min64(P.n_my, (int64_t)WL_CAP); j += 32) {
        const int64_t q = P.w0 + j * P.W;
        P.wl[3 * j] = (int32_t)P.tile_of(q);
        if (P.poff) {
            const int32_t u0 = __ldg(P.poff + q);
            P.wl[3 * j + 1] = u0;
            P.wl[3 * j + 2] = __ldg(P.poff + q + 1) - u0;
        }
    }
    __syncwarp();
    if (lane == 0 && P.n_my > 0) {
        if (P.poff) P.fill(it);
        else
            for (int s = 0; s < P.stages; ++s) P.issue(it + s);
    }
}

// Copies issued ahead for a pass that will not run: let them land (this warp's slots it ..).
__device__ __forceinline__ void pipe_drain(const WarpPipe &P, int64_t it) {
    if ((threadIdx.x & 31) == 0 && P.n_my > 0) {
        if (P.poff)
            for (int64_t k = it; k < P.iss; ++k) P.wait_packed(k);
        else
            for (int s = 0; s < P.stages; ++s) P.wait(it + s);
    }
    __syncwarp();
}

__device__ __forceinline__ void pipe_init(WarpPipe &P, const SolveSmem &S, int stages, uint32_t cbytes,
                                          int keep_in_l2) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    P.my = S.stage0 + (size_t)wid * stages * cbytes;
    P.mb = S.bars + wid * PQ;
    P.ring_bytes = (uint32_t)stages * cbytes;
    P.moff = S.ring_meta + wid * PQ * 2;
    P.mspan = P.moff + PQ;
    P.wl = S.wlist + wid * WL_CAP * 3;
    P.cbytes = cbytes;
    P.stages = stages;
    // DA is read again by every iteration: keep it in L2 when it fits there
    P.pol = keep_in_l2 ? l2_evict_last_policy() : l2_evict_first_policy();
    P.n_my = 0;
    if (lane == 0) {
        for (int s = 0; s < PQ; ++s) mbar_init(&P.mb[s], 1);
        fence_mbar_init();
    }
}

template <int NMAX>
__global__ void __launch_bounds__(MP_THREADS, mp_min_ctas(NMAX)) mp_solve_kernel(MPArgs a, int stages, int keep_in_l2) {
    if (a.skip && *a.skip) return; // the same flag for every CTA: all return together
    extern __shared__ __align__(128) unsigned char sm_raw[];
    __shared__ PState ps;
    // align the staging area explicitly: static shared memory may shift the dynamic region
    unsigned char *sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
    const uint32_t cbytes = (uint32_t)wt_copy_bytes(a.n);
    const SolveSmem S = solve_layout<NMAX>(sm, stages, cbytes);
    WarpPipe P;
    pipe_init(P, S, stages, cbytes, keep_in_l2);
    solve_load<NMAX>(a, S, ps, false); // ends with a __syncthreads (barriers initialised)
    int64_t it = 0;
    pipe_start(P, a, blockIdx.x, gridDim.x, it);
    const int r = solve_loop<NMAX>(a, S, P, ps, it, blockIdx.x, gridDim.x, nullptr, 0u);
    if (r == LOOP_ABORT && threadIdx.x == 0) atomicOr(a.status, DEV_TIMEOUT);
    pipe_drain(P, it);
    if (blockIdx.x == 0) solve_finish<NMAX>(a, S, ps, r != LOOP_ABORT);
}

__device__ bool batch_sync(unsigned *gctl, unsigned n_cta, const MPArgs *args, int n_plans) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vg = gctl + 1;
        const unsigned g0 = *vg;
        __threadfence();
        int ok = 1;
        if (atomicAdd(gctl, 1u) == n_cta - 1) {
            unsigned long long mask = 0ull;
            for (int p = 0; p < n_plans; ++p) {
                const MPArgs &q = args[p];
                const bool act = !(q.skip && *(volatile const int32_t *)q.skip) && !*(volatile int32_t *)&q.st->done;
                if (act) mask |= 1ull << p;
            }
            gctl[4] = (unsigned)(mask & 0xffffffffu);
            gctl[5] = (unsigned)(mask >> 32);
            gctl[3] = *(volatile unsigned *)(gctl + 2);
            atomicExch(gctl, 0u);
            __threadfence();
            atomicAdd(gctl + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g0) {
                if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Several independent problems in one persistent launch.  All CTAs are split
// among the problems still iterating, in proportion to their warp tiles (the same
// computation in every CTA); each problem has its own grid barrier.  When a
// problem stops it bumps the batch epoch (gctl[2]); every other problem sees the
// change at its next second barrier, saves its state and joins a barrier of the
// whole grid (gctl[0..1]), after which the CTAs are split again among the
// problems left.  Every problem has n apertures.
template <int NMAX>
__global__ void __launch_bounds__(MP_THREADS, mp_min_ctas(NMAX))
    mp_solve_batched_kernel(const MPArgs *__restrict__ args, const int64_t *__restrict__ weight, int32_t n_plans,
                            int32_t n, unsigned *gctl, int stages, int keep_in_l2) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    __shared__ MPArgs sa;
    __shared__ PState ps;
    __shared__ int sp, sc, sn, resume_s;
    __shared__ unsigned epoch_s;
    unsigned char *sm = sm_raw + ((128u - (smem_u32(sm_raw) & 127u)) & 127u);
    const uint32_t cbytes = (uint32_t)wt_copy_bytes(n);
    const SolveSmem S = solve_layout<NMAX>(sm, stages, cbytes);
    WarpPipe P;
    pipe_init(P, S, stages, cbytes, keep_in_l2);
    __syncthreads();
    int64_t it = 0;
    unsigned epoch_local = 0;
    bool ok = true;
    while (true) {
        if (threadIdx.x == 0) { // CTA split among the problems still iterating (identical in every CTA)
            const unsigned long long mask =
                (unsigned long long)__ldcg(gctl + 4) | ((unsigned long long)__ldcg(gctl + 5) << 32);
            double wsum = 0.0;
            int n_act = 0;
            for (int q = 0; q < n_plans; ++q)
                if ((mask >> q) & 1ull) {
                    wsum += (double)weight[q];
                    ++n_act;
                }
            sp = -1;
            if (n_act > 0) {
                const int G = (int)gridDim.x;
                int start = 0, seen = 0;
                for (int q = 0; q < n_plans && sp < 0; ++q) {
                    if (!((mask >> q) & 1ull)) continue;
                    ++seen;
                    int cnt = seen == n_act ? G - start
                                            : 1 + (int)((double)(G - n_act) * (double)weight[q] / wsum);
                    cnt = max(1, min(cnt, G - start - (n_act - seen)));
                    if ((int)blockIdx.x < start + cnt) {
                        sp = q;
                        sc = (int)blockIdx.x - start;
                        sn = cnt;
                    }
                    start += cnt;
                }
            }
            epoch_s = __ldcg(gctl + 3); // the epoch at the last batch barrier
        }
        __syncthreads();
        const int p = sp;
        if (p < 0) break;
        epoch_local = epoch_s;
        for (int i = threadIdx.x; i < (int)(sizeof(MPArgs) / 4); i += MP_THREADS)
            reinterpret_cast<int32_t *>(&sa)[i] = reinterpret_cast<const int32_t *>(args + p)[i];
        __syncthreads();
        if (threadIdx.x == 0) {
            sa.n = n;
            resume_s = *(volatile int32_t *)&args[p].st->started;
        }
        __syncthreads();
        const unsigned c = (unsigned)sc, nc = (unsigned)sn;
        solve_load<NMAX>(sa, S, ps, resume_s != 0);
        pipe_start(P, sa, c, nc, it);
        const int r = solve_loop<NMAX>(sa, S, P, ps, it, c, nc, gctl + 2, epoch_local);
        pipe_drain(P, it);
        if (P.n_my > 0) it += stages; // the drained slots were issued (a warp without tiles issued none)
        if (r == LOOP_ABORT) {
            ok = false;
            if (threadIdx.x == 0) atomicOr(sa.status, DEV_TIMEOUT);
            if (c == 0) solve_finish<NMAX>(sa, S, ps, false);
            break;
        }
        if (r == LOOP_DONE && c == 0) {
            solve_finish<NMAX>(sa, S, ps, true);
            if (threadIdx.x == 0) atomicAdd(gctl + 2, 1u);
        }
        if (!batch_sync(gctl, gridDim.x, args, n_plans)) {
            ok = false;
            if (threadIdx.x == 0) atomicOr(sa.status, DEV_TIMEOUT);
            break;
        }
    }
    (void)ok;
}

// Per-problem set-up of the batched solver (one block per problem).
// gctl words: [0] arrivals, [1] generation of the batch barrier, [2] the batch
// epoch (bumped when a problem stops), [3] the epoch seen at the last batch
// barrier, [4..5] the problems still iterating then (a 64-bit mask).
__global__ void mp_init_batched_kernel(const MPArgs *__restrict__ args, int32_t n_plans, int32_t n, unsigned *gctl) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long mask = 0ull;
        for (int p = 0; p < n_plans; ++p)
            if (!(args[p].skip && *args[p].skip)) mask |= 1ull << p;
        gctl[0] = gctl[1] = gctl[2] = gctl[3] = 0u;
        gctl[4] = (unsigned)(mask & 0xffffffffu);
        gctl[5] = (unsigned)(mask >> 32);
    }
    MPArgs a = args[blockIdx.x];
    a.n = n;
    if (a.skip && *a.skip) return;
    for (int k = threadIdx.x; k < n; k += blockDim.x) a.y[k] = fminf(fmaxf(a.y[k], lo_of(a, k)), hi_of(a, k));
    if (threadIdx.x == 0) {
        BBState st = {};
        *a.st = st;
        *a.bar_count = 0u;
        *a.bar_gen = 0u;
        *a.epoch_snap = 0u;
    }
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
    pass_epilogue(a, accG, facc, blockIdx.x, gridDim.x);
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


// Warp-tile layout from a column-major matrix (DA[k * ld + i]) and the labels; padding 0.
__global__ void to_warp_tiles(const float *src, int64_t ld, int32_t V, int32_t n, const uint8_t *sid,
                              int64_t wstride, int64_t n_wtiles, float *dst) {
    const int64_t total = n_wtiles * wstride;
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t wt = o / wstride, r = o % wstride;
        if (r < MP_HEAD) { // labels of voxels 4r .. 4r + 3 of the tile (words 8 .. 31 stay 0)
            uint32_t packed = 0u;
            if (r < MP_WT / 4)
                for (int j = 0; j < 4; ++j) {
                    const int64_t i = wt * MP_WT + 4 * r + j;
                    if (i < V) packed |= (uint32_t)sid[i] << (8 * j);
                }
            reinterpret_cast<uint32_t *>(dst)[o] = packed;
        } else {
            const int64_t q = r - MP_HEAD;
            const int k = (int)((q >> 7) << 2) + (int)(q & 3);
            const int64_t i = wt * MP_WT + ((q & 127) >> 2);
            dst[o] = (k < n && i < V) ? src[(int64_t)k * ld + i] : 0.f;
        }
    }
}

// Label heads of every warp tile (the DA columns are written by the caller).
__global__ void write_label_heads(const uint8_t *sid, int32_t V, int64_t wstride, int64_t n_wtiles,
                                  uint32_t *dst) {
    for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < n_wtiles * (MP_WT / 4);
         o += (int64_t)gridDim.x * blockDim.x) {
        const int64_t wt = o / (MP_WT / 4), r = o % (MP_WT / 4);
        uint32_t packed = 0u;
        for (int j = 0; j < 4; ++j) {
            const int64_t i = wt * MP_WT + 4 * r + j;
            if (i < V) packed |= (uint32_t)sid[i] << (8 * j);
        }
        dst[wt * wstride + r] = packed;
    }
}

// ---------------------------------------------------------------------------
// Live tiles (MpLive): the 32-voxel tiles that some placed aperture reaches.
// ---------------------------------------------------------------------------

// Penalty at zero dose of each tile's voxels (a warp per tile, fixed butterfly).
__global__ void mp_tile_const_kernel(const uint8_t *sid, int32_t NA, const float *T, const float *wo,
                                     const float *wu, int64_t n_wtiles, double *c_tile) {
    const int64_t wt = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wt >= n_wtiles) return; // warp-uniform
    const int lane = threadIdx.x & 31;
    const int64_t i = wt * MP_WT + lane;
    double f = 0.0;
    if (i < NA) {
        const int k = sid[i];
        const double d = -(double)T[k]; // z - T at z = 0
        const double w = d > 0.0 ? (double)wo[k] : (double)wu[k];
        f = w * d * d;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) f += __shfl_xor_sync(0xffffffffu, f, d);
    if (lane == 0) c_tile[wt] = f;
}

// Marks the tiles that column t of DA reaches (a warp per tile; the flag stays set).
__device__ __forceinline__ void live_mark(const MpLive &L, int32_t t, int64_t wt) {
    const int lane = threadIdx.x & 31;
    const float v = L.DA[wt * L.wstride + MP_HEAD + (int64_t)(t >> 2) * 128 + (lane << 2) + (t & 3)];
    if (__any_sync(0xffffffffu, v != 0.f) && lane == 0) {
        L.flag[wt] = 1;
        if (L.gmask) L.gmask[wt] |= 1u << (t >> 2); // one writer per tile and launch
    }
}

__global__ void mp_live_mark_kernel(MpLive L, int32_t t) {
    if (L.skip && *L.skip) return;
    const int64_t wt = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wt < L.n_wtiles) live_mark(L, t, wt); // warp-uniform
}

__global__ void mp_live_mark_batched_kernel(const MpLive *plans, int32_t t) {
    const MpLive &L = plans[blockIdx.y];
    if (L.skip && *L.skip) return;
    const int64_t wt = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (wt < L.n_wtiles) live_mark(L, t, wt);
}

constexpr int LV_THREADS = MP_LIVE_BLOCK; // a thread per tile

// Block b of the list: the live count of tiles b * 1024 .. and the sum of the
// others' constants (a fixed tree).
__device__ void live_count(const MpLive &L) {
    __shared__ double sums[LV_THREADS];
    const int tid = threadIdx.x;
    const int64_t q = (int64_t)blockIdx.x * LV_THREADS + tid;
    const bool in = q < L.n_wtiles;
    const int f = in && L.flag[q];
    sums[tid] = in && !f ? L.c_tile[q] : 0.0;
    const int c = __syncthreads_count(f);
    for (int st = LV_THREADS / 2; st > 0; st >>= 1) {
        if (tid < st) sums[tid] += sums[tid + st];
        __syncthreads();
    }
    if (L.gmask) { // packed units of the block's live tiles: a head and 4 per marked group
        int32_t u = f ? 1 + 4 * __popc(L.gmask[q]) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) u += __shfl_xor_sync(0xffffffffu, u, d);
        __shared__ int32_t wu[LV_THREADS / 32];
        if ((tid & 31) == 0) wu[tid >> 5] = u;
        __syncthreads();
        if (tid == 0) {
            int32_t tot = 0;
            for (int w = 0; w < LV_THREADS / 32; ++w) tot += wu[w];
            L.bsize[blockIdx.x] = tot;
        }
    }
    if (tid == 0) {
        L.bcnt[blockIdx.x] = c;
        L.bpart[blockIdx.x] = sums[0];
    }
}

// Block b writes its live tiles after those of blocks 0 .. b-1 (ballot ranks within
// a warp, warp offsets by a scan of the 32 warp counts); block 0 also forms the
// count and F_off = F0 + the block sums in block order.
__device__ void live_write(const MpLive &L, int64_t n_blocks) {
    __shared__ int32_t woff[32];
    __shared__ int32_t base_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t q = (int64_t)blockIdx.x * LV_THREADS + tid;
    const bool f = q < L.n_wtiles && L.flag[q];
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) woff[wid] = __popc(m);
    if (tid == 0) {
        int32_t b = 0;
        for (int64_t k = 0; k < blockIdx.x; ++k) b += L.bcnt[k];
        base_s = b;
    }
    __syncthreads();
    if (wid == 0) { // exclusive scan of the warp counts
        const int32_t v = woff[lane];
        int32_t x = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        woff[lane] = x - v;
    }
    __syncthreads();
    const int32_t li = base_s + woff[wid] + __popc(m & ((1u << lane) - 1u)); // list index of a live tile
    if (f) L.tiles[li] = (int32_t)q;
    if (L.gmask) { // packed offsets in list order: earlier blocks' units, then a block scan
        __shared__ int32_t su[32];
        __shared__ int32_t ubase_s;
        const int32_t u = f ? 1 + 4 * __popc(L.gmask[q]) : 0;
        int32_t x = u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) su[wid] = x;
        if (tid == 0) {
            int32_t b = 0;
            for (int64_t k = 0; k < blockIdx.x; ++k) b += L.bsize[k];
            ubase_s = b;
        }
        __syncthreads();
        if (wid == 0) {
            const int32_t v = su[lane];
            int32_t y = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t o = __shfl_up_sync(0xffffffffu, y, d);
                if (lane >= d) y += o;
            }
            su[lane] = y - v;
        }
        __syncthreads();
        if (f) L.poff[li] = ubase_s + su[wid] + x - u;
    }
    if (blockIdx.x == 0 && tid == 0) {
        int32_t n = 0, units = 0;
        double acc = 0.0;
        for (int64_t k = 0; k < n_blocks; ++k) {
            n += L.bcnt[k];
            acc += L.bpart[k];
            if (L.gmask) units += L.bsize[k];
        }
        *L.n_live = n;
        *L.F_off = *L.F0 + acc;
        if (L.gmask) L.poff[n] = units;
    }
}

__global__ void __launch_bounds__(LV_THREADS) mp_live_count_kernel(MpLive L) {
    if (L.skip && *L.skip) return;
    if ((int64_t)blockIdx.x < mp_live_blocks(L.n_wtiles)) live_count(L);
}

__global__ void __launch_bounds__(LV_THREADS) mp_live_write_kernel(MpLive L) {
    if (L.skip && *L.skip) return;
    const int64_t nb = mp_live_blocks(L.n_wtiles);
    if ((int64_t)blockIdx.x < nb) live_write(L, nb);
}

__global__ void __launch_bounds__(LV_THREADS) mp_live_count_batched_kernel(const MpLive *plans) {
    const MpLive &L = plans[blockIdx.y];
    if (L.skip && *L.skip) return;
    if ((int64_t)blockIdx.x < mp_live_blocks(L.n_wtiles)) live_count(L);
}

__global__ void __launch_bounds__(LV_THREADS) mp_live_write_batched_kernel(const MpLive *plans) {
    const MpLive &L = plans[blockIdx.y];
    if (L.skip && *L.skip) return;
    const int64_t nb = mp_live_blocks(L.n_wtiles);
    if ((int64_t)blockIdx.x < nb) live_write(L, nb);
}

vmat_status mp_tile_consts(const uint8_t *sid_c, int32_t NA, const vmat_voxels *vox, int64_t n_wtiles, double *c_tile,
                           cudaStream_t s) {
    if (n_wtiles < 1) return VMAT_OK;
    const int64_t blocks = (n_wtiles * 32 + 255) / 256;
    mp_tile_const_kernel<<<(unsigned)blocks, 256, 0, s>>>(sid_c, NA, vox->T, vox->w_over, vox->w_under, n_wtiles,
                                                          c_tile);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

// A warp per live list entry: the tile's labels and group mask, then its marked groups
// of the first G groups, ascending (float4 per lane; the group's 512 bytes per warp).
__global__ void mp_pack_kernel(MpLive L, int32_t G) {
    if (L.skip && *L.skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t n_live = min64((int64_t)max(__ldcg(L.n_live), 0), L.n_wtiles);
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n_live;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t q = __ldcg(L.tiles + i);
        const float *src = L.DA + q * L.wstride;
        float *dst = L.packed + (int64_t)__ldcg(L.poff + i) * 32;
        const uint32_t mask = __ldcg(L.gmask + q);
        if (lane < 8) dst[lane] = src[lane]; // the 32 labels
        if (lane == 8) dst[8] = __uint_as_float(mask);
        int slot = 0;
        for (int g = 0; g < G; ++g) {
            if (!((mask >> g) & 1u)) continue; // warp-uniform
            const float4 v = reinterpret_cast<const float4 *>(src + MP_HEAD + g * 128)[lane];
            reinterpret_cast<float4 *>(dst + MP_HEAD + slot * 128)[lane] = v;
            ++slot;
        }
    }
}

vmat_status mp_pack(const MpLive &L, int32_t n, cudaStream_t s) {
    if (L.n_wtiles < 1 || !L.packed) return VMAT_OK;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int64_t want = (L.n_wtiles * 32 + 255) / 256;
    mp_pack_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->n_sm * 8)), 256, 0, s>>>(
        L, (n + 3) / 4);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status mp_live_mark(const MpLive &L, int32_t t, cudaStream_t s) {
    if (L.n_wtiles < 1) return VMAT_OK;
    mp_live_mark_kernel<<<(unsigned)((L.n_wtiles * 32 + 255) / 256), 256, 0, s>>>(L, t);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status mp_live_rebuild(const MpLive &L, cudaStream_t s) {
    if (L.n_wtiles < 1) return VMAT_OK;
    const unsigned nb = (unsigned)mp_live_blocks(L.n_wtiles);
    mp_live_count_kernel<<<nb, LV_THREADS, 0, s>>>(L);
    VMAT_LAUNCH_CHECK();
    mp_live_write_kernel<<<nb, LV_THREADS, 0, s>>>(L);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status mp_live_update(const MpLive &L, int32_t t, cudaStream_t s) {
    if (L.n_wtiles < 1) return VMAT_OK;
    mp_live_mark_kernel<<<(unsigned)((L.n_wtiles * 32 + 255) / 256), 256, 0, s>>>(L, t);
    VMAT_LAUNCH_CHECK();
    const unsigned nb = (unsigned)mp_live_blocks(L.n_wtiles);
    mp_live_count_kernel<<<nb, LV_THREADS, 0, s>>>(L);
    VMAT_LAUNCH_CHECK();
    mp_live_write_kernel<<<nb, LV_THREADS, 0, s>>>(L);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status mp_live_update_batched(const MpLive *plans, int32_t n_plans, int64_t max_wtiles, int32_t t,
                                   cudaStream_t s) {
    if (n_plans < 1 || max_wtiles < 1) return VMAT_OK;
    mp_live_mark_batched_kernel<<<dim3((unsigned)((max_wtiles * 32 + 255) / 256), n_plans), 256, 0, s>>>(plans, t);
    VMAT_LAUNCH_CHECK();
    const dim3 g((unsigned)mp_live_blocks(max_wtiles), (unsigned)n_plans);
    mp_live_count_batched_kernel<<<g, LV_THREADS, 0, s>>>(plans);
    VMAT_LAUNCH_CHECK();
    mp_live_write_batched_kernel<<<g, LV_THREADS, 0, s>>>(plans);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status mp_write_labels(const uint8_t *sid, int32_t V, int64_t wstride, float *DA, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const int64_t n_wt = ((int64_t)V + MP_WT - 1) / MP_WT;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>((n_wt * 8 + 255) / 256, (int64_t)ctx->n_sm * 8));
    write_label_heads<<<g, 256, 0, s>>>(sid, V, wstride, n_wt, reinterpret_cast<uint32_t *>(DA));
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

static int solve_nmax(int n) { return ((n + 7) / 8) * 8; }
static size_t solve_fixed(int n) {
    const int nmax = solve_nmax(n);
    return 128 /* alignment slack */ + 2 * (size_t)(nmax / 4) * 16 + 4 * (size_t)nmax * 8 + 8 * 8 +
           8 * (size_t)(nmax + 1) + (size_t)nmax * 4 + (size_t)MP_NW * nmax * 4 + 3 * 256 * 4 + (size_t)MP_NW * PQ * (8 + 8) +
           (size_t)MP_NW * WL_CAP * 12;
}
static size_t solve_smem(int n, int stages) { return solve_fixed(n) + (size_t)stages * MP_NW * wt_copy_bytes(n); }
// Tiles in flight per warp: as many as fit (up to 8) in ~110 KB, so that two CTAs
// share an SM; where not even two fit there, up to the per-CTA limit (one CTA per SM).
static int solve_stages(int n) {
    const size_t per = MP_NW * wt_copy_bytes(n);
    const size_t small = 110 * 1024;
    const size_t st = solve_fixed(n) + 2 * per <= small ? (small - solve_fixed(n)) / per
                                                        : (MP_SMEM_LIMIT - solve_fixed(n)) / per;
    return (int)std::min<size_t>(8, st);
}

using SolveFn = void (*)(MPArgs, int, int);
static SolveFn solve_kernel_for(int n) {
    switch ((n + 7) / 8) {
    case 1: return mp_solve_kernel<8>;
    case 2: return mp_solve_kernel<16>;
    case 3: return mp_solve_kernel<24>;
    case 4: return mp_solve_kernel<32>;
    case 5: return mp_solve_kernel<40>;
    case 6: return mp_solve_kernel<48>;
    case 7: return mp_solve_kernel<56>;
    case 8: return mp_solve_kernel<64>;
    case 9: return mp_solve_kernel<72>;
    case 10: return mp_solve_kernel<80>;
    case 11: return mp_solve_kernel<88>;
    case 12: return mp_solve_kernel<96>;
    default: return nullptr;
    }
}
using SolveBatchFn = void (*)(const MPArgs *, const int64_t *, int32_t, int32_t, unsigned *, int, int);
static SolveBatchFn solve_batched_kernel_for(int n) {
    switch ((n + 7) / 8) {
    case 1: return mp_solve_batched_kernel<8>;
    case 2: return mp_solve_batched_kernel<16>;
    case 3: return mp_solve_batched_kernel<24>;
    case 4: return mp_solve_batched_kernel<32>;
    case 5: return mp_solve_batched_kernel<40>;
    case 6: return mp_solve_batched_kernel<48>;
    case 7: return mp_solve_batched_kernel<56>;
    case 8: return mp_solve_batched_kernel<64>;
    case 9: return mp_solve_batched_kernel<72>;
    case 10: return mp_solve_batched_kernel<80>;
    case 11: return mp_solve_batched_kernel<88>;
    case 12: return mp_solve_batched_kernel<96>;
    default: return nullptr;
    }
}
static size_t ldg_smem(int n) { return (size_t)((n + 3) & ~3) * 4 + (size_t)n * 8 + MP_THREADS * 4 + 3 * 256 * 4; }

int64_t mp_wtile_stride(int32_t n_cap) { return MP_HEAD + (int64_t)((n_cap + 3) / 4) * 128; }

// Launch configuration of one solve with n apertures over V voxels.
struct MPLaunch {
    bool persistent;
    SolveFn fn;
    int stages, keep_in_l2, P, Pc;
    size_t smem;
};

static vmat_status mp_set_attributes() {
    static bool attr = false;
    if (attr) return VMAT_OK;
    for (int q = 1; q <= MP_NMAX / 8; ++q) {
        VMAT_CUDA(cudaFuncSetAttribute(solve_kernel_for(8 * q), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       MP_SMEM_LIMIT));
        VMAT_CUDA(cudaFuncSetAttribute(solve_batched_kernel_for(8 * q), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       MP_SMEM_LIMIT));
    }
    VMAT_CUDA(cudaFuncSetAttribute(mp_iter_ldg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_SMEM_LIMIT));
    VMAT_CUDA(cudaFuncSetAttribute(mp_cauchy_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_SMEM_LIMIT));
    attr = true;
    return VMAT_OK;
}

// Persistent solver (one cooperative launch) up to MP_NMAX apertures, else one
// launch per iteration reading DA from global memory.
static vmat_status mp_configure(int32_t V, int32_t n_ap, const DeviceCtx *ctx, MPLaunch *L) {
    VMAT_TRY(mp_set_attributes());
    const int64_t n_wtiles = ((int64_t)V + MP_WT - 1) / MP_WT;
    const int32_t n_tiles = (int32_t)((V + MP_THREADS - 1) / MP_THREADS);
    L->stages = solve_stages(n_ap);
    L->persistent = n_ap <= MP_NMAX && L->stages >= 2 && solve_smem(n_ap, L->stages) <= MP_SMEM_LIMIT;
    L->fn = L->persistent ? solve_kernel_for(n_ap) : nullptr;
    L->smem = L->persistent ? solve_smem(n_ap, L->stages) : ldg_smem(n_ap);
    L->keep_in_l2 = (double)n_wtiles * (double)wt_copy_bytes(n_ap) <= 64.0 * 1024 * 1024 ? 1 : 0;
    int bps = 1;
    if (L->persistent) VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, L->fn, MP_THREADS, L->smem));
    else VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, mp_iter_ldg_kernel, MP_THREADS, L->smem));
    if (bps < 1) return set_error(VMAT_ECUDA, "mp_bb_solve: the solver kernel does not fit on an SM");
    // every CTA of the persistent grid must be resident at once (grid barriers)
    L->P = (int)std::max<int64_t>(1, std::min<int64_t>(L->persistent ? (n_wtiles + MP_NW - 1) / MP_NW : n_tiles,
                                                        (int64_t)ctx->n_sm * bps));
    L->Pc = std::max(1, std::min<int>(n_tiles, ctx->n_sm * 4));
    return VMAT_OK;
}

// Upper bound on co-resident CTAs of MP_THREADS threads (2048 threads per SM).
static int mp_p_max(const DeviceCtx *ctx) { return ctx->n_sm * (2048 / MP_THREADS); }

static size_t mp_ws_bytes(int n_cap, int p_max) {
    return 256 + (size_t)(n_cap + 1) * sizeof(double) + (size_t)n_cap * (sizeof(double) + sizeof(float)) +
           2 * (size_t)p_max * (n_cap + 1) * sizeof(double) + (size_t)p_max * sizeof(double) + 256;
}

size_t mp_workspace_bytes(int32_t n_cap) {
    DeviceCtx *ctx;
    if (device_ctx(&ctx) != VMAT_OK) return 0;
    return mp_ws_bytes(n_cap, mp_p_max(ctx));
}

static void mp_fill_args(MPArgs &a, void *ws, int n_cap, int p_max, const float *DA, int64_t wstride, int32_t V,
                         int32_t n_ap, const uint8_t *struct_id, const vmat_voxels *vox, const float *lo,
                         const float *hi, float *y, float *z, const vmat_bb_opts &opts, double F_offset,
                         const MPLaunch &L, const DeviceCtx *ctx) {
    char *p = static_cast<char *>(ws);
    a.st = reinterpret_cast<BBState *>(p);
    a.bar_count = reinterpret_cast<unsigned *>(p + 192);
    a.bar_gen = reinterpret_cast<unsigned *>(p + 224);
    a.epoch_snap = reinterpret_cast<unsigned *>(p + 240);
    p += 256;
    a.G = reinterpret_cast<double *>(p); // [n + 1]: G, then F in the persistent solver
    a.Gprev = a.G + n_cap + 1;
    a.part = a.Gprev + n_cap;
    a.cpart = a.part + 2 * (size_t)p_max * (n_cap + 1);
    a.yprev = reinterpret_cast<float *>(a.cpart + p_max);
    a.DA = DA;
    a.wstride = wstride;
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
    a.P = L.P;
    a.pstride = p_max;
    a.n_tiles = (int32_t)((V + MP_THREADS - 1) / MP_THREADS);
    a.n_wtiles = ((int64_t)V + MP_WT - 1) / MP_WT;
    a.status = ctx->status;
    a.opts = opts;
    a.F_offset = F_offset;
    a.skip = nullptr;
    a.iters_acc = nullptr;
    a.bytes_acc = nullptr;
    a.tiles = nullptr;
    a.n_live = nullptr;
    a.F_off_dev = nullptr;
    a.packed = nullptr;
    a.poff = nullptr;
}

static vmat_status mp_launch_persistent(MPArgs &a, const MPLaunch &L, cudaStream_t s) {
    mp_init_kernel<<<1, MP_THREADS, 0, s>>>(a);
    VMAT_LAUNCH_CHECK();
    int st_arg = L.stages, l2_arg = L.keep_in_l2;
    void *args[] = {&a, &st_arg, &l2_arg};
    VMAT_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(L.fn), dim3(L.P), dim3(MP_THREADS), args,
                                          L.smem, s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return VMAT_OK;
}

vmat_status mp_bb_enqueue(const float *DA, int32_t V, int32_t n_ap, int32_t n_cap, int64_t wstride,
                          const uint8_t *struct_id, const vmat_voxels *vox, const float *lo, const float *hi, float *y,
                          float *z, const vmat_bb_opts *opts_in, double F_offset, void *ws, const int32_t *skip,
                          int32_t *iters_acc, cudaStream_t s, const MpLive *live, double *bytes_acc) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    vmat_bb_opts opts = {500, 1e-6, 1e-9, 1e-12, 1e12};
    if (opts_in) opts = *opts_in;
    if (opts.max_iter < 1) return set_error(VMAT_EINVAL, "mp_bb_solve: max_iter must be >= 1");
    if (n_ap > n_cap) return set_error(VMAT_EINVAL, "mp_bb_enqueue: n_ap > n_cap");
    MPLaunch L;
    VMAT_TRY(mp_configure(V, n_ap, ctx, &L));
    if (!L.persistent)
        return set_error(VMAT_EUNSUPPORTED, "mp_bb_enqueue: %d apertures need the host-driven solver", n_ap);
    MPArgs a;
    mp_fill_args(a, ws, n_cap, mp_p_max(ctx), DA, wstride, V, n_ap, struct_id, vox, lo, hi, y, z, opts, F_offset, L,
                 ctx);
    a.skip = skip;
    a.iters_acc = iters_acc;
    a.bytes_acc = bytes_acc;
    if (live) {
        a.tiles = live->tiles;
        a.n_live = live->n_live;
        a.F_off_dev = live->F_off;
        a.packed = live->packed;
        a.poff = live->poff;
    }
    return mp_launch_persistent(a, L, s);
}

size_t mp_args_bytes() { return sizeof(MPArgs); }

vmat_status mp_fill_plan_args(void *out, void *ws, int32_t n_cap, const float *DA, int64_t wstride, int32_t V,
                              const uint8_t *struct_id, const vmat_voxels *vox, const float *lo, const float *hi,
                              float *y, float *z, const vmat_bb_opts *opts_in, double F_offset, const int32_t *skip,
                              int32_t *iters_acc, const MpLive *live) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    vmat_bb_opts opts = {500, 1e-6, 1e-9, 1e-12, 1e12};
    if (opts_in) opts = *opts_in;
    if (opts.max_iter < 1) return set_error(VMAT_EINVAL, "mp_bb_solve: max_iter must be >= 1");
    MPLaunch L = {};
    L.P = 1;
    MPArgs a;
    mp_fill_args(a, ws, n_cap, mp_p_max(ctx), DA, wstride, V, n_cap, struct_id, vox, lo, hi, y, z, opts, F_offset, L,
                 ctx);
    a.skip = skip;
    a.iters_acc = iters_acc;
    if (live) {
        a.tiles = live->tiles;
        a.n_live = live->n_live;
        a.F_off_dev = live->F_off;
    }
    memcpy(out, &a, sizeof(MPArgs));
    return VMAT_OK;
}

vmat_status mp_batched_grid(int32_t n, int32_t n_plans, int32_t *grid, int32_t *stages, size_t *smem) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    VMAT_TRY(mp_set_attributes());
    if (n < 1 || n > MP_NMAX) return set_error(VMAT_EUNSUPPORTED, "batched master problem: %d apertures (max %d)", n, MP_NMAX);
    const int st = solve_stages(n);
    const size_t sm = solve_smem(n, st);
    if (st < 2 || sm > MP_SMEM_LIMIT) return set_error(VMAT_EUNSUPPORTED, "batched master problem: no fit for %d", n);
    int bps = 0;
    VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, solve_batched_kernel_for(n), MP_THREADS, sm));
    if (bps < 1) return set_error(VMAT_ECUDA, "batched master problem: kernel does not fit on an SM");
    const int64_t P = (int64_t)ctx->n_sm * bps; // every CTA resident at once (grid barriers)
    if (P < n_plans) return set_error(VMAT_EUNSUPPORTED, "batched master problem: more plans than resident CTAs");
    *grid = (int32_t)P;
    *stages = st;
    *smem = sm;
    return VMAT_OK;
}

vmat_status mp_bb_enqueue_batched(const void *args, const int64_t *weight, unsigned *gctl, int32_t n_plans, int32_t n,
                                  int32_t grid, int32_t stages, size_t smem, int keep_in_l2, cudaStream_t s) {
    mp_init_batched_kernel<<<n_plans, 128, 0, s>>>(static_cast<const MPArgs *>(args), n_plans, n, gctl);
    VMAT_LAUNCH_CHECK();
    SolveBatchFn fn = solve_batched_kernel_for(n);
    if (!fn) return set_error(VMAT_EUNSUPPORTED, "batched master problem: %d apertures", n);
    const MPArgs *a = static_cast<const MPArgs *>(args);
    int32_t np = n_plans, nn = n;
    int st = stages, l2 = keep_in_l2;
    void *kargs[] = {&a, &weight, &np, &nn, &gctl, &st, &l2};
    VMAT_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(fn), dim3(grid), dim3(MP_THREADS), kargs, smem,
                                          s));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return VMAT_OK;
}

vmat_status mp_bb_impl(const float *DA, int32_t V, int32_t n_ap, int64_t ld, const uint8_t *struct_id,
                       int64_t wstride, const vmat_voxels *vox, const float *lo, const float *hi, float *y,
                       float *z, const vmat_bb_opts *opts_in, double F_offset, vmat_bb_report *rep, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    vmat_bb_opts opts = {500, 1e-6, 1e-9, 1e-12, 1e12};
    if (opts_in) opts = *opts_in;
    if (opts.max_iter < 1) return set_error(VMAT_EINVAL, "mp_bb_solve: max_iter must be >= 1");
    if (ldg_smem(n_ap) > MP_SMEM_LIMIT) return set_error(VMAT_EUNSUPPORTED, "mp_bb_solve: too many apertures (%d)", n_ap);
    const int64_t n_wtiles = ((int64_t)V + MP_WT - 1) / MP_WT;

    // a column-major input is copied once into the warp-tile layout (with the labels)
    Scratch conv;
    if (wstride == 0) {
        wstride = mp_wtile_stride(n_ap);
        VMAT_TRY(conv.alloc((size_t)n_wtiles * wstride * sizeof(float), s));
        const int64_t total = n_wtiles * wstride;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)ctx->n_sm * 16));
        to_warp_tiles<<<g, 256, 0, s>>>(DA, ld, V, n_ap, struct_id, wstride, n_wtiles, static_cast<float *>(conv.ptr));
        VMAT_LAUNCH_CHECK();
        DA = static_cast<const float *>(conv.ptr);
    }
    MPLaunch L;
    VMAT_TRY(mp_configure(V, n_ap, ctx, &L));
    const int p_max = std::max(mp_p_max(ctx), std::max(L.P, L.Pc));
    Scratch ws;
    VMAT_TRY(ws.alloc(mp_ws_bytes(n_ap, p_max), s));
    MPArgs a;
    mp_fill_args(a, ws.ptr, n_ap, p_max, DA, wstride, V, n_ap, struct_id, vox, lo, hi, y, z, opts, F_offset, L, ctx);
    const size_t smem_cauchy = (size_t)((n_ap + 3) & ~3) * 4 + 3 * 256 * 4;

    static thread_local BBState *host_st = nullptr;
    if (!host_st) VMAT_CUDA(cudaMallocHost(&host_st, sizeof(BBState)));

    if (L.persistent) {
        VMAT_TRY(mp_launch_persistent(a, L, s));
        VMAT_CUDA(cudaMemcpyAsync(host_st, a.st, sizeof(BBState), cudaMemcpyDeviceToHost, s));
        VMAT_CUDA(cudaStreamSynchronize(s));
    } else {
        mp_init_kernel<<<1, MP_THREADS, 0, s>>>(a);
        VMAT_LAUNCH_CHECK();
        int launched = 0;
        while (launched < opts.max_iter) {
            const int chunk = launched == 0 ? 1 : std::min(MP_CHUNK, opts.max_iter - launched);
            for (int c = 0; c < chunk; ++c) {
                mp_iter_ldg_kernel<<<L.P, MP_THREADS, L.smem, s>>>(a);
                g_launches.fetch_add(1, std::memory_order_relaxed);
                if (launched + c == 0) {
                    mp_cauchy_pass_kernel<<<L.Pc, MP_THREADS, smem_cauchy, s>>>(a);
                    mp_cauchy_step_kernel<<<1, MP_THREADS, 0, s>>>(a, L.Pc);
                    g_launches.fetch_add(2, std::memory_order_relaxed);
                }
            }
            VMAT_CUDA(cudaGetLastError());
            launched += chunk;
            VMAT_CUDA(cudaMemcpyAsync(host_st, a.st, sizeof(BBState), cudaMemcpyDeviceToHost, s));
            VMAT_CUDA(cudaStreamSynchronize(s));
            if (host_st->done) break;
        }
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
