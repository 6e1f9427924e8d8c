// Pricing problem, second step (Section 2.2.2): the best opening [L, R) of every
// MLC row of every unoccupied control point, then the CP whose aperture (the
// sum of its row bests) has the largest price.
//
// The paper uses one thread per row for the first kernel and one thread per CP
// for the second.  Here one warp handles a row: lane 0 builds the float64
// prefix sums P_c sequentially in column order over the row's leaf-travel
// window [Lmin, Rmax) (no price outside it is read, so the beamlet price pass
// may skip those beamlets), the lanes evaluate every feasible pair
// (P_R - P_L) and the warp reduces with the full tie-break key
// (value desc, width asc, |L + R - n_cols| asc, L asc).  Every compared value is
// produced by the same float64 operations in the same order as the sequential
// definition, and the key is a total order, so the choice is bit-exact.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace vmat {

constexpr int PR_WARPS = 8;

// A candidate opening: v = P_R - P_L as a double, also as an order-preserving
// unsigned key (v is never -0: the prefix sums start at +0 and x - x = +0).
struct RowBest {
    uint64_t key;
    int32_t w, cd, L;
    bool has;
};

__device__ __forceinline__ uint64_t order_key(double v) {
    const uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(uint64_t k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

// The exact tie-break order (value desc, width asc, |L + R - n_cols| asc, L asc)
// with integer compares only.
__device__ __forceinline__ bool better(const RowBest &a, const RowBest &b) {
    if (!a.has) return false;
    if (!b.has) return true;
    if (a.key != b.key) return a.key > b.key;
    if (a.w != b.w) return a.w < b.w;
    if (a.cd != b.cd) return a.cd < b.cd;
    return a.L < b.L;
}

// Nearest occupied CP on one side of k within its arc (search direction dir).
__device__ int nearest_occupied(const PricingGeom &g, const uint8_t *occupied, int k, int dir, int lane) {
    int a = 0;
    while (a + 1 < g.n_arcs && g.arc_first[a + 1] <= k) ++a;
    const int lo = g.arc_first[a], hi = g.arc_first[a + 1]; // [lo, hi)
    for (int base = k + dir; base >= lo && base < hi; base += 32 * dir) {
        const int kk = base + lane * dir;
        const bool hit = kk >= lo && kk < hi && occupied[kk];
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) return base + (__ffs(m) - 1) * dir;
    }
    return -1;
}

// The same search by one thread.
__device__ int nearest_occupied_seq(const PricingGeom &g, const uint8_t *occupied, int k, int dir) {
    int a = 0;
    while (a + 1 < g.n_arcs && g.arc_first[a + 1] <= k) ++a;
    const int lo = g.arc_first[a], hi = g.arc_first[a + 1];
    for (int kk = k + dir; kk >= lo && kk < hi; kk += dir)
        if (occupied[kk]) return kk;
    return -1;
}

// Leaf-travel window of MLC row r at CP k (reading R7): each leaf moves at most
// travel columns per CP step from its position at the nearest occupied CP on each
// side (kl, kr; -1: none).
struct RowWindow {
    int Lmin, Lmax, Rmin, Rmax;
};
// The window narrowed by the leaves (Ln, Rn) of the occupied CP kk.
__device__ __forceinline__ void window_clip(RowWindow &w, int k, int kk, int travel, int Ln, int Rn) {
    const int reach = abs(k - kk) * travel;
    w.Lmin = max(w.Lmin, Ln - reach);
    w.Lmax = min(w.Lmax, Ln + reach);
    w.Rmin = max(w.Rmin, Rn - reach);
    w.Rmax = min(w.Rmax, Rn + reach);
}
__device__ __forceinline__ RowWindow row_window(const PricingGeom &g, const int16_t *__restrict__ leaves, int k,
                                                int r, int kl, int kr) {
    RowWindow w{0, g.n_cols, 0, g.n_cols};
    for (int side = 0; side < 2; ++side) {
        const int kk = side ? kr : kl;
        if (kk < 0) continue;
        window_clip(w, k, kk, g.travel, leaves[((int64_t)kk * g.n_rows + r) * 2],
                    leaves[((int64_t)kk * g.n_rows + r) * 2 + 1]);
    }
    return w;
}

// Float64 prefix sums of one MLC row's prices over its window (reading R8): P_c = 0
// for c <= Lmin, P_{c+1} = P_c + pi_c for Lmin <= c < Rmax, constant after Rmax, in
// column order.  Prices outside [Lmin, Rmax) are never read.
__device__ __forceinline__ void window_prefix(const float *__restrict__ row, int N, int Lmin, int Rmax, double *P) {
    double acc = 0.0;
    P[0] = 0.0;
    for (int c = 0; c < N; ++c) {
        if (c >= Lmin && c < Rmax) acc = acc + (double)row[c];
        P[c + 1] = acc;
    }
}

// Shared memory per warp of the row kernel: the float64 prefix sums and their
// float32 roundings, n_cols + 1 of each.
__host__ __device__ constexpr size_t row_smem_stride(int n_cols) { return (((size_t)(n_cols + 1) * 12) + 15) & ~15; }

// Best opening of MLC row r of CP k (one warp; ws: row_smem_stride(n_cols) bytes of
// shared memory for this warp).  Writes the row's entry gw of rb_*.
//
// The float64 prefix sums P_c are formed sequentially in column order (lane 0),
// exactly as the definition.  Every feasible pair is first valued in float32 from
// the rounded prefix sums; only the pairs whose float32 value lies within 3E of
// the float32 maximum are valued in float64 (E = 2^-20 max|P| bounds the
// difference between a pair's float32 value and its float64 value P_R - P_L:
// two roundings of P to float32, one float32 and one float64 subtraction, each at
// most 2^-24 or 2^-53 relative, with a factor 4 to spare).  The pairs that attain
// the float64 maximum are always among them, so the choice, ties included, is the
// one the exhaustive float64 search makes.
__device__ __forceinline__ void price_row_warp(const PricingGeom &g, const float *__restrict__ pi,
                                               const uint8_t *__restrict__ occupied, const int16_t *__restrict__ leaves,
                                               int64_t gw, unsigned char *ws, double *rb_v, int16_t *rb_lr,
                                               uint8_t *rb_ok, const double *__restrict__ Pall = nullptr) {
    const int lane = threadIdx.x & 31;
    const int k = (int)(gw / g.n_rows), r = (int)(gw % g.n_rows);
    if (occupied[k]) return;
    const int N = g.n_cols;
    double *P = reinterpret_cast<double *>(ws);
    float *P32 = reinterpret_cast<float *>(ws + (size_t)(N + 1) * 8);
    const int kl = nearest_occupied(g, occupied, k, -1, lane), kr = nearest_occupied(g, occupied, k, 1, lane);
    const RowWindow win = row_window(g, leaves, k, r, kl, kr);
    const int Lmin = win.Lmin, Lmax = win.Lmax, Rmin = win.Rmin, Rmax = win.Rmax;
    if (Pall) { // the same prefix sums, formed by window_prefix_kernel a thread per row
        for (int c = lane; c <= N; c += 32) P[c] = Pall[gw * (N + 1) + c];
    } else if (lane == 0) {
        window_prefix(pi + ((int64_t)k * g.n_rows + r) * N, N, Lmin, Rmax, P);
    }
    __syncwarp();
    float pmax = 0.f;
    for (int c = lane; c <= N; c += 32) {
        const float q = (float)P[c];
        P32[c] = q;
        pmax = fmaxf(pmax, fabsf(q));
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, d));
    __syncwarp();
    // float32 maximum over the feasible pairs
    float m32 = -INFINITY;
    for (int L = Lmin + lane; L <= Lmax; L += 32) {
        const float pl = P32[L];
        for (int R = max(L, Rmin); R <= Rmax; ++R) m32 = fmaxf(m32, P32[R] - pl);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m32 = fmaxf(m32, __shfl_xor_sync(0xffffffffu, m32, d));
    const float E = pmax * 0x1p-20f + 0x1p-140f;
    // (prefix sums beyond the float32 range: every pair is a candidate)
    const float thr = isfinite(pmax) ? m32 - 3.f * E : -INFINITY;
    // float64 values of the candidates, exact key order
    RowBest best;
    best.has = false;
    best.key = 0;
    best.w = best.cd = best.L = 0;
    for (int L = Lmin + lane; L <= Lmax; L += 32) {
        const float pl = P32[L];
        const long long bl = __double_as_longlong(P[L]);
        for (int R = max(L, Rmin); R <= Rmax; ++R) {
            if (P32[R] - pl < thr) continue;
            const long long br = __double_as_longlong(P[R]);
            const double v = br == bl ? 0.0 : P[R] - P[L];
            RowBest c;
            c.has = true;
            c.key = order_key(v);
            c.w = R - L;
            c.cd = abs(L + R - N);
            c.L = L;
            if (better(c, best)) best = c;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        RowBest o;
        o.key = __shfl_down_sync(0xffffffffu, best.key, d);
        o.w = __shfl_down_sync(0xffffffffu, best.w, d);
        o.cd = __shfl_down_sync(0xffffffffu, best.cd, d);
        o.L = __shfl_down_sync(0xffffffffu, best.L, d);
        o.has = __shfl_down_sync(0xffffffffu, (int)best.has, d) != 0;
        if (lane + d < 32 && better(o, best)) best = o;
    }
    if (lane == 0) {
        rb_v[gw] = best.has ? key_value(best.key) : 0.0;
        rb_lr[2 * gw] = (int16_t)best.L;
        rb_lr[2 * gw + 1] = (int16_t)(best.L + best.w);
        rb_ok[gw] = best.has ? 1 : 0;
    }
}

__global__ void __launch_bounds__(PR_WARPS * 32)
    price_rows_kernel(PricingGeom g, const float *__restrict__ pi, const uint8_t *__restrict__ occupied,
                      const int16_t *__restrict__ leaves, double *rb_v, int16_t *rb_lr, uint8_t *rb_ok,
                      const int32_t *skip, const double *__restrict__ Pall) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sP[]; // PR_WARPS x row_smem_stride(n_cols)
    const int wid = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * PR_WARPS + wid;
    if (gw >= (int64_t)g.K * g.n_rows) return;
    price_row_warp(g, pi, occupied, leaves, gw, sP + wid * row_smem_stride(g.n_cols), rb_v, rb_lr, rb_ok, Pall);
}

constexpr int CP_THREADS = 1024;

// The CP with the largest price (sum of its row bests, in row order), smallest k
// on ties, and its leaves (one block).
__device__ __forceinline__ void price_cps_block(const PricingGeom &g, const uint8_t *__restrict__ occupied,
                                                const double *__restrict__ rb_v, const int16_t *__restrict__ rb_lr,
                                                const uint8_t *__restrict__ rb_ok, int32_t *best_cp,
                                                int16_t *best_leaves, double *best_price) {
    __shared__ double sv[CP_THREADS / 32];
    __shared__ int sk[CP_THREADS / 32];
    __shared__ int kwin;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double bv = -INFINITY;
    int bk = -1;
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) { // k ascending: a strict > keeps the smallest k
        if (occupied[k]) continue;
        double price = 0.0;
        bool ok = true;
        for (int r = 0; r < g.n_rows; ++r) {
            const int64_t i = (int64_t)k * g.n_rows + r;
            ok = ok && rb_ok[i];
            price = price + rb_v[i];
        }
        if (ok && (bk < 0 || price > bv)) {
            bv = price;
            bk = k;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, bv, d);
        const int ok = __shfl_down_sync(0xffffffffu, bk, d);
        if (lane + d < 32 && ok >= 0 && (bk < 0 || ov > bv || (ov == bv && ok < bk))) {
            bv = ov;
            bk = ok;
        }
    }
    if (lane == 0) {
        sv[wid] = bv;
        sk[wid] = bk;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = -INFINITY;
        int kb = -1;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w)
            if (sk[w] >= 0 && (kb < 0 || sv[w] > v || (sv[w] == v && sk[w] < kb))) {
                v = sv[w];
                kb = sk[w];
            }
        *best_cp = kb;
        *best_price = kb >= 0 ? v : -INFINITY;
        kwin = kb;
    }
    __syncthreads();
    if (kwin >= 0)
        for (int r = threadIdx.x; r < g.n_rows; r += blockDim.x) {
            const int64_t i = (int64_t)kwin * g.n_rows + r;
            best_leaves[2 * r] = rb_lr[2 * i];
            best_leaves[2 * r + 1] = rb_lr[2 * i + 1];
        }
}

__global__ void __launch_bounds__(CP_THREADS)
    price_cps_kernel(PricingGeom g, const uint8_t *__restrict__ occupied, const double *__restrict__ rb_v,
                     const int16_t *__restrict__ rb_lr, const uint8_t *__restrict__ rb_ok, int32_t *best_cp,
                     int16_t *best_leaves, double *best_price, const int32_t *skip) {
    if (skip && *skip) return;
    price_cps_block(g, occupied, rb_v, rb_lr, rb_ok, best_cp, best_leaves, best_price);
}

// Batched pricing: global row g of plan p is (CP, MLC row) pair g - off[p].
__global__ void __launch_bounds__(PR_WARPS * 32)
    price_rows_batched_kernel(const PricePlan *__restrict__ plans, const int64_t *__restrict__ off, int32_t n_plans,
                              int64_t total, int32_t max_cols) {
    extern __shared__ __align__(16) unsigned char sP[]; // PR_WARPS x row_smem_stride(max_cols)
    __shared__ int64_t soff[VMAT_MAX_BATCH + 1];
    for (int i = threadIdx.x; i <= n_plans; i += blockDim.x) soff[i] = off[i];
    __syncthreads();
    const int wid = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * PR_WARPS + wid;
    if (gw >= total) return;
    int a = 0, b = n_plans;
    while (b - a > 1) {
        const int m = (a + b) >> 1;
        if (soff[m] <= gw) a = m;
        else b = m;
    }
    const PricePlan &P = plans[a];
    if (P.skip && *P.skip) return;
    price_row_warp(P.g, P.pi, P.occupied, P.leaves, gw - soff[a], sP + wid * row_smem_stride(max_cols), P.rb_v,
                   P.rb_lr, P.rb_ok);
}

__global__ void __launch_bounds__(CP_THREADS) price_cps_batched_kernel(const PricePlan *__restrict__ plans) {
    const PricePlan &P = plans[blockIdx.x];
    if (P.skip && *P.skip) return;
    price_cps_block(P.g, P.occupied, P.rb_v, P.rb_lr, P.rb_ok, P.best_cp, P.best_leaves, P.best_price);
}

// ---------------------------------------------------------------------------
// Interdigitation (Section 2.2.2, second variant): L_r <= min(R_{r-1}, R_{r+1}).
// The best aperture of a CP is a chain over the rows: S_r(L, R) = S_{r-1}(pred) +
// (P_R - P_L) in float64 (S_0 = P_R - P_L), where pred is the compatible state of
// row r - 1 (L <= R' and L' <= R) with the largest S_{r-1}, ties by the row key
// (width asc, |L + R - n_cols| asc, L asc).  The dominance maximum over
// {L <= a, R >= b} is formed by a suffix pass over R and a prefix pass over L, both
// restricted to the window rectangle of the previous row (the only states with a
// chain).  One block per CP; every compare is an integer compare of order keys,
// every value the float64 of the sequential definition.
// ---------------------------------------------------------------------------
constexpr int ID_THREADS = 1024;

// A state's tie key (width, |L + R - n_cols|, L, each below 1024) in one word:
// smaller is better among equal values.
__device__ __forceinline__ uint32_t state_sec(int L, int R, int N) {
    return ((uint32_t)(R - L) << 20) | ((uint32_t)abs(L + R - N) << 10) | (uint32_t)L;
}
// a strictly better than b: larger value key, then smaller tie key.
__device__ __forceinline__ bool key_better(uint64_t ka, uint32_t sa, uint64_t kb, uint32_t sb) {
    return ka > kb || (ka == kb && sa < sb);
}

constexpr int INTERDIG_PSTRIDE = 96; // doubles per row of prefix sums in shared memory (>= INTERDIG_MAX_COLS + 1)
static_assert(INTERDIG_PSTRIDE >= INTERDIG_MAX_COLS + 1 && INTERDIG_PSTRIDE % 2 == 0, "prefix-sum rows");
__host__ __device__ constexpr size_t interdig_smem(int N) {
    // S_{r-1} and S_r as order keys, two rows of prefix sums, the scans' tie keys
    return (size_t)(N + 1) * (N + 1) * (8 + 8 + 4) + 2 * INTERDIG_PSTRIDE * 8 + 64;
}

// Window prefix sums of every MLC row of every unoccupied CP (a thread per row,
// float64 in column order, as the definition), for the chain kernels and the row
// kernel.  FP64 issues at a small fraction of the FP32 rate on this GPU: a row per
// lane keeps 32 rows' sequential sums in one instruction stream, where a row per
// warp spends a warp-wide FP64 instruction on every add of one row.
__global__ void window_prefix_kernel(PricingGeom g, const float *__restrict__ pi,
                                       const uint8_t *__restrict__ occupied, const int16_t *__restrict__ leaves,
                                       double *__restrict__ Pall, const int32_t *skip) {
    if (skip && *skip) return;
    const int N = g.n_cols;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < (int64_t)g.K * g.n_rows;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(row / g.n_rows), r = (int)(row % g.n_rows);
        if (occupied[k]) continue;
        const RowWindow w = row_window(g, leaves, k, r, nearest_occupied_seq(g, occupied, k, -1),
                                       nearest_occupied_seq(g, occupied, k, 1));
        window_prefix(pi + row * N, N, w.Lmin, w.Rmax, Pall + row * (N + 1));
    }
}

// Windows of one CP (a warp): [Lmin, max(Lmin, Rmax)) per MLC row, empty when the CP
// is occupied; the rows, nonzeros and chunks inside them added to counts.
__device__ __forceinline__ void cp_windows_warp(const PricingGeom &g, const uint8_t *__restrict__ occupied,
                                                const int16_t *__restrict__ leaves, int k, short2 *win,
                                                const int64_t *__restrict__ rowptr, const int64_t *__restrict__ cptr,
                                                unsigned long long *counts) {
    const int lane = threadIdx.x & 31;
    const bool occ = occupied[k] != 0;
    int kl = -1, kr = -1;
    if (!occ) {
        kl = nearest_occupied(g, occupied, k, -1, lane);
        kr = nearest_occupied(g, occupied, k, 1, lane);
    }
    unsigned long long rows = 0, nnz = 0, chunks = 0;
    for (int r = lane; r < g.n_rows; r += 32) {
        int lo = 0, hi = 0;
        if (!occ) {
            const RowWindow w = row_window(g, leaves, k, r, kl, kr);
            lo = w.Lmin;
            hi = max(w.Lmin, w.Rmax);
        }
        const int64_t q = (int64_t)k * g.n_rows + r;
        win[q] = make_short2((short)lo, (short)hi);
        if (counts && hi > lo) {
            const int64_t b = q * g.n_cols;
            rows += (unsigned long long)(hi - lo);
            nnz += (unsigned long long)(rowptr[b + hi] - rowptr[b + lo]);
            if (cptr) chunks += (unsigned long long)(cptr[b + hi] - cptr[b + lo]);
        }
    }
    if (!counts) return;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        rows += __shfl_xor_sync(0xffffffffu, rows, d);
        nnz += __shfl_xor_sync(0xffffffffu, nnz, d);
        chunks += __shfl_xor_sync(0xffffffffu, chunks, d);
    }
    if (lane == 0 && rows > 0) {
        atomicAdd(counts, rows);
        atomicAdd(counts + 1, nnz);
        atomicAdd(counts + 2, chunks);
    }
}

constexpr int WIN_WARPS = 4;

__global__ void __launch_bounds__(WIN_WARPS * 32)
    price_windows_kernel(PricingGeom g, const uint8_t *__restrict__ occupied, const int16_t *__restrict__ leaves,
                         short2 *win, const int64_t *__restrict__ rowptr, const int64_t *__restrict__ cptr,
                         unsigned long long *counts, const int32_t *skip) {
    if (skip && *skip) return;
    const int k = blockIdx.x * WIN_WARPS + (threadIdx.x >> 5);
    if (k >= g.K) return; // warp-uniform
    cp_windows_warp(g, occupied, leaves, k, win, rowptr, cptr, counts);
}

__global__ void __launch_bounds__(WIN_WARPS * 32)
    price_windows_batched_kernel(const WinPlan *__restrict__ plans, int32_t t) {
    const WinPlan &P = plans[blockIdx.y];
    if (P.skip && *P.skip) return;
    const int k = blockIdx.x * WIN_WARPS + (threadIdx.x >> 5);
    if (k >= P.g.K) return; // warp-uniform
    cp_windows_warp(P.g, P.occupied, P.leaves, k, P.win, P.rowptr, nullptr, P.counts ? P.counts + 3 * (int64_t)t : nullptr);
}

// Inclusive "best so far" scans over the previous row's window rectangle
// [pL0, pL1] x [pR0, pR1], G threads per line (the largest power of two up to 32 that
// fits every line into the block): each thread takes the best of a contiguous segment
// of its line in scan order, the segment bests are scanned across the line's G lanes
// by shuffles, and each thread rescans its segment from the carry of the segments
// before it, writing every element's best so far as its two keys (order key of
// S_{r-1}, tie key) to CK and CM.
//   SUFFIX: line L, elements R = pR1 down to max(L, pR0) (the states of the line);
//           C[L][R] = the best state (L, R'), R' >= R.  The columns R < L of the
//           rectangle get the line's best state (every state of the line has R' >= L
//           > R), or no state (key 0, tie key SEC_NONE, below every state) if the
//           line has none.
//   else:   line b, elements a = pL0 up to pL1, rewritten in place with M[a][b], the
//           best state with L <= a, R >= b.
constexpr uint32_t SEC_NONE = 0xffffffffu;
constexpr uint64_t KEY_NEG_INF = 0x000fffffffffffffull; // order_key(-inf)
constexpr uint64_t KEY_POS_INF = 0xfff0000000000000ull; // order_key(+inf)

template <bool SUFFIX>
__device__ __forceinline__ void rect_line_scans(const uint64_t *__restrict__ Kp, uint64_t *CK, uint32_t *CM, int N,
                                                int pL0, int pL1, int pR0, int pR1) {
    const int n1 = N + 1, tid = threadIdx.x;
    const int n_lines = SUFFIX ? pL1 - pL0 + 1 : pR1 - pR0 + 1;
    int lg = 5;
    while (lg > 0 && (n_lines << lg) > ID_THREADS) --lg;
    const int G = 1 << lg;
    const int line = tid >> lg, sg = tid & (G - 1);
    const bool act = line < n_lines;
    const int L = pL0 + line;                      // SUFFIX: the line's L
    const int lo = SUFFIX ? max(L, pR0) : 0;       // SUFFIX: its first state's R
    const int len = !act ? 0 : SUFFIX ? max(0, pR1 - lo + 1) : pL1 - pL0 + 1;
    const int seg = (len + G - 1) >> lg;
    const int e0 = min(sg * seg, len), e1 = min(e0 + seg, len);
    auto pos_of = [&](int e) { return SUFFIX ? L * n1 + (pR1 - e) : (pL0 + e) * n1 + pR0 + line; };
    uint64_t bk = 0;
    uint32_t bs = SEC_NONE;
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
        const int pos = pos_of(e);
        const uint64_t kk = SUFFIX ? Kp[pos] : CK[pos];
        const uint32_t ss = SUFFIX ? state_sec(L, pR1 - e, N) : CM[pos];
        if (key_better(kk, ss, bk, bs)) {
            bk = kk;
            bs = ss;
        }
    }
    for (int d = 1; d < G; d <<= 1) { // inclusive scan of the segment bests along the line
        const uint64_t ok = __shfl_up_sync(0xffffffffu, bk, d, G);
        const uint32_t os = __shfl_up_sync(0xffffffffu, bs, d, G);
        if (sg >= d && key_better(ok, os, bk, bs)) {
            bk = ok;
            bs = os;
        }
    }
    uint64_t ck = __shfl_up_sync(0xffffffffu, bk, 1, G); // carry: the segments before this one
    uint32_t cs = __shfl_up_sync(0xffffffffu, bs, 1, G);
    if (sg == 0) {
        ck = 0;
        cs = SEC_NONE;
    }
    if (SUFFIX) { // the line's best, for the columns left of its states
        const uint64_t tk = __shfl_sync(0xffffffffu, bk, G - 1, G);
        const uint32_t ts = __shfl_sync(0xffffffffu, bs, G - 1, G);
        if (act)
            for (int b = pR0 + sg; b < min(lo, pR1 + 1); b += G) {
                CK[L * n1 + b] = tk;
                CM[L * n1 + b] = ts;
            }
    }
#pragma unroll 4
    for (int e = e0; e < e1; ++e) {
        const int pos = pos_of(e);
        const uint64_t kk = SUFFIX ? Kp[pos] : CK[pos];
        const uint32_t ss = SUFFIX ? state_sec(L, pR1 - e, N) : CM[pos];
        if (key_better(kk, ss, ck, cs)) {
            ck = kk;
            cs = ss;
        }
        CK[pos] = ck;
        CM[pos] = cs;
    }
}

// The states L <= R of the window rectangle [L0, L1] x [R0, R1], numbered without
// gaps: first the lines L <= R0 (every R of the rectangle), wR states each, then the
// lines R0 < L <= min(L1, R1), whose states run from R = L to R1 (one fewer each).
struct RectStates {
    int L0, R0, R1, wR, nA, cellsA, Lb0, m, total;
    float inv_wR;
    __device__ __forceinline__ void init(int l0, int l1, int r0, int r1) {
        L0 = l0;
        R0 = r0;
        R1 = r1;
        wR = r1 - r0 + 1;
        total = 0;
        if (l1 < l0 || r1 < r0) return;
        nA = max(0, min(l1, r0) - l0 + 1);
        cellsA = nA * wR;
        Lb0 = max(l0, r0 + 1);
        const int nB = max(0, min(l1, r1) - Lb0 + 1);
        m = r1 - Lb0 + 1;
        total = cellsA + nB * m - nB * (nB - 1) / 2;
        inv_wR = 1.0f / (float)wR;
    }
    // state u -> (L, R).  In the first part (u + 0.5) / wR is at least 0.5 / wR away
    // from an integer and the float quotient is within 2^-22 of it (u < 8192, wR <= 89),
    // so its floor is exact; in the second the line j solves j (2m + 1 - j) / 2 <= u'
    // (float root, then at most a step either way to the exact integer answer).
    __device__ __forceinline__ void at(int u, int &L, int &R) const {
        if (u < cellsA) {
            const int q = (int)(((float)u + 0.5f) * inv_wR);
            L = L0 + q;
            R = R0 + (u - q * wR);
            return;
        }
        const int v = u - cellsA, b = 2 * m + 1;
        int j = (int)(0.5f * ((float)b - sqrtf((float)(b * b - 8 * v))));
        j = max(j, 0);
        while (j > 0 && j * (b - j) > 2 * v) --j;
        while ((j + 1) * (b - j - 1) <= 2 * v) ++j;
        L = Lb0 + j;
        R = L + (v - j * (b - j) / 2);
    }
};

// One CP's chain: its best price (cp_val/cp_ok) and its predecessor table (the
// feasible states' predecessors per row, then the best final state) for the backtrack.
// Shared memory: S as order keys (S_{r-1} until the scans have read it, then S_r, in
// place), the scans' key and tie-key columns CK and CM, and the prefix sums of the
// current and the next row.  The next row's prefix sums and leaf-travel window are
// loaded while the current row is processed.
__device__ void interdig_chain(const PricingGeom &g, const double *__restrict__ Pall,
                               const uint8_t *__restrict__ occupied, const int16_t *__restrict__ leaves, int k,
                               unsigned char *sm, int16_t *pred_tab, double *out_val, uint8_t *out_ok) {
    const int N = g.n_cols, n1 = N + 1, NS = n1 * n1;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    uint64_t *Ks = reinterpret_cast<uint64_t *>(sm);
    uint64_t *CK = Ks + NS;
    double *Pb = reinterpret_cast<double *>(CK + NS); // [2][INTERDIG_PSTRIDE]
    uint32_t *CM = reinterpret_cast<uint32_t *>(Pb + 2 * INTERDIG_PSTRIDE);
    __shared__ int kk_s[2];
    __shared__ int4 win_s[2];
    __shared__ uint64_t wk[ID_THREADS / 32];
    __shared__ uint32_t wsec[ID_THREADS / 32];
    const double *Pk = Pall + (int64_t)k * g.n_rows * n1;
    if (wid == 0) {
        const int left = nearest_occupied(g, occupied, k, -1, lane);
        const int right = nearest_occupied(g, occupied, k, 1, lane);
        if (lane == 0) {
            kk_s[0] = left;
            kk_s[1] = right;
            const RowWindow w = row_window(g, leaves, k, 0, left, right);
            win_s[0] = make_int4(w.Lmin, w.Lmax, w.Rmin, w.Rmax);
        }
    }
    for (int c = tid; c < n1; c += ID_THREADS) Pb[c] = Pk[c];
    __syncthreads();
    int pL0 = 0, pL1 = -1, pR0 = 0, pR1 = -1; // the previous row's rectangle (none yet)
    for (int r = 0; r < g.n_rows; ++r) {
        const int4 w = win_s[r & 1];
        const double *P = Pb + (r & 1) * INTERDIG_PSTRIDE;
        // the next row's prefix sums and window, in flight during this row
        const bool more = r + 1 < g.n_rows;
        const double pn = more && tid < n1 ? Pk[(int64_t)(r + 1) * n1 + tid] : 0.0;
        // (the leaves are loaded here and used at the end of the row, so that no warp
        // waits for them before the scans)
        int nb[4] = {0, 0, 0, 0};
        if (more && tid == ID_THREADS - 1)
            for (int side = 0; side < 2; ++side)
                if (kk_s[side] >= 0) {
                    const int16_t *q = leaves + ((int64_t)kk_s[side] * g.n_rows + r + 1) * 2;
                    nb[2 * side] = q[0];
                    nb[2 * side + 1] = q[1];
                }
        const bool prev = pL0 <= pL1 && pR0 <= pR1;
        if (r > 0 && prev) {
            rect_line_scans<true>(Ks, CK, CM, N, pL0, pL1, pR0, pR1);
            __syncthreads();
            rect_line_scans<false>(Ks, CK, CM, N, pL0, pL1, pR0, pR1);
            __syncthreads();
        }
        // S_r over the rectangle's states L <= R (the states with L > R are never read),
        // from the best compatible state of row r - 1, M[R'][L'] clamped to its rectangle
        RectStates rs;
        rs.init(w.x, w.y, w.z, w.w);
        int16_t *pt = pred_tab + (int64_t)r * NS;
        for (int u = tid; u < rs.total; u += ID_THREADS) {
            int L, R;
            rs.at(u, L, R);
            const int idx = L * n1 + R;
            const double v = P[R] - P[L];
            double sv = v;
            if (r > 0) {
                sv = -INFINITY;
                if (prev && R >= pL0 && L <= pR1) {
                    const int q = min(R, pL1) * n1 + max(L, pR0);
                    const uint32_t s = CM[q];
                    const uint64_t pk = CK[q];
                    if (s != SEC_NONE) {
                        const int pl = (int)(s & 1023u);
                        if (pk > KEY_NEG_INF && pk <= KEY_POS_INF) sv = key_value(pk) + v; // S_{r-1} > -inf
                        pt[idx] = (int16_t)(pl * n1 + pl + (int)(s >> 20));
                    }
                }
            }
            Ks[idx] = order_key(sv);
        }
        if (more && tid < n1) Pb[((r + 1) & 1) * INTERDIG_PSTRIDE + tid] = pn;
        if (more && tid == ID_THREADS - 1) {
            RowWindow x{0, N, 0, N};
            for (int side = 0; side < 2; ++side)
                if (kk_s[side] >= 0) window_clip(x, k, kk_s[side], g.travel, nb[2 * side], nb[2 * side + 1]);
            win_s[(r + 1) & 1] = make_int4(x.Lmin, x.Lmax, x.Rmin, x.Rmax);
        }
        __syncthreads();
        pL0 = w.x;
        pL1 = rs.total ? w.y : -1;
        pR0 = w.z;
        pR1 = w.w;
    }
    // best final state (value > -inf; value desc, then tie key)
    uint64_t bk = 0;
    uint32_t bs = SEC_NONE;
    {
        RectStates rs;
        rs.init(pL0, pL1, pR0, pR1);
        for (int u = tid; u < rs.total; u += ID_THREADS) {
            int L, R;
            rs.at(u, L, R);
            const uint64_t kv = Ks[L * n1 + R];
            if (!(kv > KEY_NEG_INF && kv <= KEY_POS_INF)) continue;
            const uint32_t sv = state_sec(L, R, N);
            if (key_better(kv, sv, bk, bs)) {
                bk = kv;
                bs = sv;
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const uint64_t ok = __shfl_down_sync(0xffffffffu, bk, d);
        const uint32_t os = __shfl_down_sync(0xffffffffu, bs, d);
        if (lane + d < 32 && key_better(ok, os, bk, bs)) {
            bk = ok;
            bs = os;
        }
    }
    if (lane == 0) {
        wk[wid] = bk;
        wsec[wid] = bs;
    }
    __syncthreads();
    if (tid == 0) {
        uint64_t kb = 0;
        uint32_t sb = SEC_NONE;
        for (int x = 0; x < ID_THREADS / 32; ++x)
            if (key_better(wk[x], wsec[x], kb, sb)) {
                kb = wk[x];
                sb = wsec[x];
            }
        const bool found = sb != SEC_NONE;
        const int L = (int)(sb & 1023u), id = found ? L * n1 + L + (int)(sb >> 20) : 0;
        out_val[k] = found ? key_value(kb) : -INFINITY;
        out_ok[k] = found ? 1 : 0;
        pred_tab[(int64_t)g.n_rows * NS] = (int16_t)id; // the final state, for the backtrack
    }
}

// CTA i runs the chain of CP cand[i], i < *n_cand.
__global__ void __launch_bounds__(ID_THREADS, 1)
    price_cps_interdig_kernel(PricingGeom g, const double *__restrict__ Pall, const uint8_t *__restrict__ occupied,
                              const int16_t *__restrict__ leaves, double *cp_val, uint8_t *cp_ok, int16_t *pred_all,
                              const int32_t *skip, const int32_t *__restrict__ cand, const int32_t *n_cand) {
    if (skip && *skip) return;
    if ((int)blockIdx.x >= *n_cand) return;
    const int k = cand[blockIdx.x];
    extern __shared__ __align__(16) unsigned char smi[];
    const int64_t NS = (int64_t)(g.n_cols + 1) * (g.n_cols + 1);
    interdig_chain(g, Pall, occupied, leaves, k, smi, pred_all + (int64_t)k * (g.n_rows * NS + 1), cp_val, cp_ok);
}

// Which CPs run the chain.  The chain's price of a CP is at most its price without
// the interdigitation constraint, the sum over rows (in row order, float64) of each
// row's best opening in its window: every chain term P_R - P_L is at most its row's
// best, and a float64 sum rounded at each step is monotone in each term.  So the
// chains run in two rounds: first the CPs with the B largest unconstrained prices
// (B = the CTAs that run at once; all unoccupied CPs when they are no more than B),
// then every other CP whose unconstrained price could still reach the best chain
// price of the first round (above it, or equal with a smaller k).  The CP the pick
// chooses over the CPs that ran is the one it chooses over all CPs.
enum { IDC_SKIP_ROWS = 0, IDC_N1 = 1, IDC_N2 = 2, IDC_UNOCC = 3, IDC_PRUNE = 4, IDC_WORDS = 8 };
constexpr int ID_SEL_THREADS = 1024;
constexpr int ID_PRUNE_MAX_K = 2048; // above this the ranking is skipped: every CP runs in the first round

// Counts the unoccupied CPs, clears every cp_ok and decides whether the row bests
// (the bounds) are needed: ctl[IDC_SKIP_ROWS] also skips the row kernel when the
// plan is done.
__global__ void __launch_bounds__(ID_SEL_THREADS)
    interdig_setup_kernel(PricingGeom g, const uint8_t *__restrict__ occupied, uint8_t *cp_ok, int32_t *ctl,
                          int32_t B, const int32_t *skip) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const bool sk = skip && *skip;
    int c = 0;
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
        cp_ok[k] = 0;
        c += occupied[k] ? 0 : 1;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool prune = cnt > B && g.K <= ID_PRUNE_MAX_K;
        ctl[IDC_SKIP_ROWS] = (sk || !prune) ? 1 : 0;
        ctl[IDC_UNOCC] = cnt;
        ctl[IDC_PRUNE] = prune ? 1 : 0;
        ctl[IDC_N1] = 0;
        ctl[IDC_N2] = 0;
    }
}

// The first round: every unoccupied CP (no pruning), or the B best by unconstrained
// price (order key desc, k asc; a CP with a row without any opening has no chain and
// runs in neither round).  bound[k] keeps the unconstrained price, feasible or -inf.
__global__ void __launch_bounds__(ID_SEL_THREADS)
    interdig_select_kernel(PricingGeom g, const uint8_t *__restrict__ occupied, const double *__restrict__ rb_v,
                           const uint8_t *__restrict__ rb_ok, double *bound, uint64_t *bkey, uint8_t *in1,
                           int32_t *cand1, int32_t *ctl, int32_t B, const int32_t *skip) {
    if (skip && *skip) return;
    __shared__ int n1;
    if (threadIdx.x == 0) n1 = 0;
    __syncthreads();
    const bool prune = ctl[IDC_PRUNE] != 0;
    if (!prune) {
        for (int k = threadIdx.x; k < g.K; k += blockDim.x)
            if (!occupied[k]) cand1[atomicAdd(&n1, 1)] = k;
        __syncthreads();
        if (threadIdx.x == 0) ctl[IDC_N1] = n1;
        return;
    }
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
        uint64_t key = 0; // 0: no chain (occupied, or a row without any opening)
        double b = -INFINITY;
        if (!occupied[k]) {
            double price = 0.0;
            bool ok = true;
            for (int r = 0; r < g.n_rows; ++r) {
                const int64_t i = (int64_t)k * g.n_rows + r;
                ok = ok && rb_ok[i];
                price = price + rb_v[i];
            }
            if (ok) {
                b = price;
                // nonzero (the low bit only orders the first round, which any order keeps exact)
                key = order_key(price) | 1ull;
            }
        }
        bound[k] = b;
        bkey[k] = key;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
        const uint64_t kk = bkey[k];
        int rank = B;
        if (kk) {
            rank = 0;
            for (int j = 0; j < g.K; ++j) {
                const uint64_t kj = bkey[j];
                rank += (kj > kk || (kj == kk && j < k)) ? 1 : 0;
            }
        }
        in1[k] = rank < B ? 1 : 0;
        if (rank < B) {
            cand1[rank] = k;
            atomicAdd(&n1, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl[IDC_N1] = n1;
}

// The second round: the CPs outside the first whose bound can still reach the first
// round's best chain price v* (at CP k*): bound > v*, or bound == v* and k < k*; every
// one of them when v* or the bound is not finite, or when no first-round chain exists.
__global__ void __launch_bounds__(ID_SEL_THREADS)
    interdig_threshold_kernel(PricingGeom g, const double *__restrict__ bound, const uint64_t *__restrict__ bkey,
                              const uint8_t *__restrict__ in1, const double *__restrict__ cp_val,
                              const uint8_t *__restrict__ cp_ok, const int32_t *__restrict__ cand1, int32_t *cand2,
                              int32_t *ctl, const int32_t *skip) {
    if (skip && *skip) return;
    if (!ctl[IDC_PRUNE]) return;
    __shared__ double sv[ID_SEL_THREADS / 32];
    __shared__ int sk[ID_SEL_THREADS / 32];
    __shared__ int n2;
    __shared__ double vs;
    __shared__ int ks;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int n1 = ctl[IDC_N1];
    double v = -INFINITY;
    int kb = -1;
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const int k = cand1[i];
        if (cp_ok[k] && (kb < 0 || cp_val[k] > v || (cp_val[k] == v && k < kb))) {
            v = cp_val[k];
            kb = k;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, d);
        const int ok = __shfl_down_sync(0xffffffffu, kb, d);
        if (lane + d < 32 && ok >= 0 && (kb < 0 || ov > v || (ov == v && ok < kb))) {
            v = ov;
            kb = ok;
        }
    }
    if (lane == 0) {
        sv[wid] = v;
        sk[wid] = kb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = -INFINITY;
        int bk = -1;
        for (int w = 0; w < ID_SEL_THREADS / 32; ++w)
            if (sk[w] >= 0 && (bk < 0 || sv[w] > bv || (sv[w] == bv && sk[w] < bk))) {
                bv = sv[w];
                bk = sk[w];
            }
        vs = bv;
        ks = bk;
        n2 = 0;
    }
    __syncthreads();
    const double vstar = vs;
    const int kstar = ks;
    const bool vfin = kstar >= 0 && isfinite(vstar);
    for (int k = threadIdx.x; k < g.K; k += blockDim.x) {
        if (!bkey[k] || in1[k]) continue; // no chain, or ran in the first round
        const double b = bound[k];
        const bool prune = vfin && isfinite(b) && (b < vstar || (b == vstar && k > kstar));
        if (!prune) cand2[atomicAdd(&n2, 1)] = k;
    }
    __syncthreads();
    if (threadIdx.x == 0) ctl[IDC_N2] = n2;
}

// The best CP (price desc, smallest k on ties, in k order as the sequential
// definition: the warp loads 32 CPs at a time and every lane applies the same
// comparisons in k order) and its leaves, backtracked through the predecessor table
// its chain stored.
__global__ void price_pick_interdig_kernel(PricingGeom g, const uint8_t *__restrict__ occupied,
                                           const double *cp_val, const uint8_t *cp_ok, const int16_t *pred_all,
                                           int32_t *best_cp, int16_t *best_leaves, double *best_price,
                                           const int32_t *skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x;
    int kb = -1;
    double v = -INFINITY;
    for (int base = 0; base < g.K; base += 32) {
        const int k = base + lane;
        const bool cand = k < g.K && !occupied[k] && cp_ok[k];
        const double x = cand ? cp_val[k] : 0.0;
        const unsigned m = __ballot_sync(0xffffffffu, cand);
        for (int j = 0; j < 32; ++j) {
            const double xj = __shfl_sync(0xffffffffu, x, j);
            if (((m >> j) & 1u) && (kb < 0 || xj > v)) { // a strict > keeps the smallest k
                v = xj;
                kb = base + j;
            }
        }
    }
    if (lane != 0) return;
    *best_cp = kb;
    *best_price = kb >= 0 ? v : -INFINITY;
    if (kb < 0) return;
    const int N = g.n_cols;
    const int64_t NS = (int64_t)(N + 1) * (N + 1);
    const int16_t *pt = pred_all + (int64_t)kb * (g.n_rows * NS + 1);
    int cur = pt[g.n_rows * NS];
    for (int r = g.n_rows - 1; r >= 0; --r) {
        best_leaves[2 * r] = (int16_t)(cur / (N + 1));
        best_leaves[2 * r + 1] = (int16_t)(cur % (N + 1));
        if (r > 0) cur = pt[(int64_t)r * NS + cur];
    }
}

vmat_status pricing_geom(const vmat_mlc *mlc, PricingGeom *g) {
    if (mlc->n_arcs > MAX_ARCS) return set_error(VMAT_EUNSUPPORTED, "price_apertures: more than %d arcs", MAX_ARCS);
    g->K = mlc->K;
    g->n_rows = mlc->n_rows;
    g->n_cols = mlc->n_cols;
    g->travel = mlc->travel_cols;
    g->interdig = mlc->interdigitation ? 1 : 0;
    g->n_arcs = mlc->n_arcs;
    for (int a = 0; a < mlc->n_arcs; ++a) g->arc_first[a] = mlc->arc_first_cp[a];
    g->arc_first[mlc->n_arcs] = mlc->K;
    return VMAT_OK;
}

vmat_status price_windows(const PricingGeom &g, const uint8_t *occupied, const int16_t *leaves, short2 *win,
                          const int64_t *rowptr, const int64_t *cptr, unsigned long long *counts,
                          const int32_t *skip, cudaStream_t s) {
    if (g.K < 1) return VMAT_OK;
    price_windows_kernel<<<(g.K + WIN_WARPS - 1) / WIN_WARPS, WIN_WARPS * 32, 0, s>>>(g, occupied, leaves, win, rowptr,
                                                                                   cptr, counts, skip);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

// Exclusive scan of the window lengths (one block of WO_THREADS): warp w takes the
// contiguous block of segments [w per, (w + 1) per), 32 consecutive ones per step (one
// coalesced load), first to total its block, then, after a scan of the warp totals, to
// write each segment's offset (warp scan per step, the running sum carried in lane 31).
constexpr int WO_THREADS = 1024, WO_WARPS = WO_THREADS / 32;
__global__ void __launch_bounds__(WO_THREADS)
    window_offsets_kernel(const short2 *__restrict__ win, int32_t nseg, int32_t *__restrict__ woff,
                          const int32_t *skip) {
    if (skip && *skip) return;
    __shared__ int32_t wsum[WO_WARPS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = (nseg + WO_WARPS - 1) / WO_WARPS;
    const int q0 = min(wid * per, nseg), q1 = min(q0 + per, nseg);
    auto len = [&](int q) -> int32_t {
        if (q >= q1) return 0;
        const short2 w = win[q];
        return max(0, (int)w.y - (int)w.x);
    };
    int32_t tot = 0;
    for (int q = q0 + lane; q < q1; q += 32) tot += len(q);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, d);
    if (lane == 0) wsum[wid] = tot;
    __syncthreads();
    int32_t base = 0;
    for (int w = 0; w < wid; ++w) base += wsum[w];
    for (int q = q0; q < q1; q += 32) {
        const int32_t v = len(q + lane);
        int32_t incl = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        if (q + lane < q1) woff[q + lane] = base + incl - v;
        base += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (wid == WO_WARPS - 1 && lane == 0) { // every segment counted: the total
        int32_t all = 0;
        for (int w = 0; w < WO_WARPS; ++w) all += wsum[w];
        woff[nseg] = all;
    }
}

vmat_status window_offsets(const short2 *win, int32_t nseg, int32_t *woff, const int32_t *skip, cudaStream_t s) {
    if (nseg < 1) return VMAT_OK;
    window_offsets_kernel<<<1, WO_THREADS, 0, s>>>(win, nseg, woff, skip);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status price_windows_batched(const WinPlan *plans, int32_t n_plans, int32_t max_K, int32_t t, cudaStream_t s) {
    if (n_plans < 1 || n_plans > VMAT_MAX_BATCH || max_K < 1)
        return set_error(VMAT_EINVAL, "price_windows_batched: bad plan count or K");
    price_windows_batched_kernel<<<dim3((max_K + WIN_WARPS - 1) / WIN_WARPS, n_plans), WIN_WARPS * 32, 0, s>>>(plans,
                                                                                                            t);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

// Dynamic shared-memory limits of the pricing kernels, raised once per process for
// their largest MLC (1024 columns; the interdigitation kernel's own column limit).
// Not a stream operation: callers that record a CUDA graph call it before capture.
vmat_status pricing_attributes() {
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        err = cudaFuncSetAttribute(price_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(PR_WARPS * row_smem_stride(1024)));
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(price_rows_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(PR_WARPS * row_smem_stride(1024)));
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(price_cps_interdig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)interdig_smem(INTERDIG_MAX_COLS));

    });
    if (err != cudaSuccess)
        return set_error(VMAT_ECUDA, "pricing: cudaFuncSetAttribute failed: %s", cudaGetErrorString(err));
    return VMAT_OK;
}

vmat_status price_apertures_batched(const PricePlan *plans, const int64_t *off, int32_t n_plans, int64_t total,
                                    int32_t max_cols, cudaStream_t s) {
    if (n_plans < 1 || n_plans > VMAT_MAX_BATCH) return set_error(VMAT_EINVAL, "price_apertures_batched: bad plan count");
    VMAT_TRY(pricing_attributes());
    if (total > 0) {
        const int64_t blocks = (total + PR_WARPS - 1) / PR_WARPS;
        price_rows_batched_kernel<<<(unsigned)blocks, PR_WARPS * 32, PR_WARPS * row_smem_stride(max_cols), s>>>(
            plans, off, n_plans, total, max_cols);
        VMAT_LAUNCH_CHECK();
    }
    price_cps_batched_kernel<<<n_plans, CP_THREADS, 0, s>>>(plans);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

// Bytes of the per-row bests (value, leaves, flag) of `rows` rows, rounded up to 16.
static size_t row_best_bytes(int64_t rows) {
    return ((size_t)rows * (sizeof(double) + 2 * sizeof(int16_t) + 1) + 15) & ~(size_t)15;
}

// Scratch of the interdigitation pricing, carved from one array (8-byte arrays first,
// then 4-, 2- and 1-byte ones): per-CP chain prices, bounds and their keys, the row
// bests, every row's prefix sums, the control words and the two rounds' CP lists,
// the row bests' leaves, every CP's predecessor table (16-bit), the flags.
struct InterdigScratch {
    double *cp_val, *bound, *rb_v, *Pall;
    uint64_t *bkey;
    int32_t *ctl, *cand1, *cand2;
    int16_t *rb_lr, *pred_all;
    uint8_t *cp_ok, *rb_ok, *in1;
    size_t bytes;
};
static InterdigScratch interdig_scratch(void *ws, const PricingGeom &g) {
    InterdigScratch x{};
    const int64_t K = g.K, rows = K * g.n_rows, NS = (int64_t)(g.n_cols + 1) * (g.n_cols + 1);
    char *p = static_cast<char *>(ws);
    size_t off = 0;
    auto take = [&](size_t n) {
        char *q = p ? p + off : nullptr;
        off += n;
        return q;
    };
    x.cp_val = reinterpret_cast<double *>(take(K * 8));
    x.bound = reinterpret_cast<double *>(take(K * 8));
    x.rb_v = reinterpret_cast<double *>(take(rows * 8));
    x.Pall = reinterpret_cast<double *>(take(rows * (g.n_cols + 1) * 8));
    x.bkey = reinterpret_cast<uint64_t *>(take(K * 8));
    x.ctl = reinterpret_cast<int32_t *>(take(IDC_WORDS * 4));
    x.cand1 = reinterpret_cast<int32_t *>(take(K * 4));
    x.cand2 = reinterpret_cast<int32_t *>(take(K * 4));
    x.rb_lr = reinterpret_cast<int16_t *>(take(rows * 4));
    x.pred_all = reinterpret_cast<int16_t *>(take(K * (g.n_rows * NS + 1) * 2));
    x.cp_ok = reinterpret_cast<uint8_t *>(take(K));
    x.rb_ok = reinterpret_cast<uint8_t *>(take(rows));
    x.in1 = reinterpret_cast<uint8_t *>(take(K));
    x.bytes = off + 64;
    return x;
}

// CTAs of the chain kernel that run at once on the current device (one round),
// queried once per device and shared-memory size.
static vmat_status interdig_wave(size_t smem, int *B) {
    static std::mutex mu;
    static std::vector<std::pair<std::pair<int, size_t>, int>> known;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(VMAT_ECUDA, "interdigitation pricing: cudaGetDevice failed: %s",
                                           cudaGetErrorString(e));
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &x : known)
        if (x.first.first == dev && x.first.second == smem) {
            *B = x.second;
            return VMAT_OK;
        }
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, price_cps_interdig_kernel, ID_THREADS, smem);
    if (e != cudaSuccess) return set_error(VMAT_ECUDA, "interdigitation pricing: occupancy query failed: %s",
                                           cudaGetErrorString(e));
    *B = std::max(1, sms * std::max(per, 1));
    known.push_back({{dev, smem}, *B});
    return VMAT_OK;
}

vmat_status price_apertures_impl(const vmat_mlc *mlc, const float *pi, const uint8_t *occupied, const int16_t *leaves,
                                 int32_t *best_cp, int16_t *best_leaves, double *best_price, void *ws,
                                 cudaStream_t s, const int32_t *skip, bool ws_has_prefix) {
    PricingGeom g;
    VMAT_TRY(pricing_geom(mlc, &g));
    const int64_t rows = (int64_t)g.K * g.n_rows;
    double *rb_v = static_cast<double *>(ws);
    int16_t *rb_lr = reinterpret_cast<int16_t *>(rb_v + rows);
    uint8_t *rb_ok = reinterpret_cast<uint8_t *>(rb_lr + 2 * rows);
    if (g.interdig) {
        const InterdigScratch x = interdig_scratch(ws, g);
        const size_t sm = interdig_smem(g.n_cols);
        VMAT_TRY(pricing_attributes());
        int B = 0;
        VMAT_TRY(interdig_wave(sm, &B));
        window_prefix_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 127) / 128, 4096)), 128, 0,
                                 s>>>(g, pi, occupied, leaves, x.Pall, skip);
        VMAT_LAUNCH_CHECK();
        interdig_setup_kernel<<<1, ID_SEL_THREADS, 0, s>>>(g, occupied, x.cp_ok, x.ctl, B, skip);
        VMAT_LAUNCH_CHECK();
        // the unconstrained row bests (the bounds), only when the CPs exceed one round
        price_rows_kernel<<<(unsigned)((rows + PR_WARPS - 1) / PR_WARPS), PR_WARPS * 32,
                            PR_WARPS * row_smem_stride(g.n_cols), s>>>(g, pi, occupied, leaves, x.rb_v, x.rb_lr,
                                                                       x.rb_ok, x.ctl + IDC_SKIP_ROWS, x.Pall);
        VMAT_LAUNCH_CHECK();
        interdig_select_kernel<<<1, ID_SEL_THREADS, 0, s>>>(g, occupied, x.rb_v, x.rb_ok, x.bound, x.bkey, x.in1,
                                                            x.cand1, x.ctl, B, skip);
        VMAT_LAUNCH_CHECK();
        const int grid1 = g.K > ID_PRUNE_MAX_K ? g.K : std::min(g.K, B);
        price_cps_interdig_kernel<<<grid1, ID_THREADS, sm, s>>>(g, x.Pall, occupied, leaves, x.cp_val, x.cp_ok,
                                                                 x.pred_all, skip, x.cand1, x.ctl + IDC_N1);
        VMAT_LAUNCH_CHECK();
        if (g.K > grid1) {
            interdig_threshold_kernel<<<1, ID_SEL_THREADS, 0, s>>>(g, x.bound, x.bkey, x.in1, x.cp_val, x.cp_ok,
                                                                   x.cand1, x.cand2, x.ctl, skip);
            VMAT_LAUNCH_CHECK();
            price_cps_interdig_kernel<<<g.K - grid1, ID_THREADS, sm, s>>>(
                g, x.Pall, occupied, leaves, x.cp_val, x.cp_ok, x.pred_all, skip, x.cand2, x.ctl + IDC_N2);
            VMAT_LAUNCH_CHECK();
        }
        price_pick_interdig_kernel<<<1, 32, 0, s>>>(g, occupied, x.cp_val, x.cp_ok, x.pred_all, best_cp, best_leaves,
                                                    best_price, skip);
        VMAT_LAUNCH_CHECK();
        return VMAT_OK;
    }
    const size_t smem = PR_WARPS * row_smem_stride(g.n_cols);
    VMAT_TRY(pricing_attributes());
    const int64_t blocks = (rows + PR_WARPS - 1) / PR_WARPS;
    double *Pall = nullptr;
    if (ws_has_prefix) { // after the row bests (pricing_scratch_bytes_prefix)
        Pall = reinterpret_cast<double *>(static_cast<char *>(ws) + row_best_bytes(rows));
        window_prefix_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((rows + 127) / 128, 4096)), 128, 0,
                               s>>>(g, pi, occupied, leaves, Pall, skip);
        VMAT_LAUNCH_CHECK();
    }
    price_rows_kernel<<<(unsigned)blocks, PR_WARPS * 32, smem, s>>>(g, pi, occupied, leaves, rb_v, rb_lr, rb_ok, skip,
                                                                     Pall);
    VMAT_LAUNCH_CHECK();
    price_cps_kernel<<<1, CP_THREADS, 0, s>>>(g, occupied, rb_v, rb_lr, rb_ok, best_cp, best_leaves, best_price, skip);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

size_t pricing_scratch_bytes_prefix(const vmat_mlc *mlc) {
    const size_t rows = (size_t)mlc->K * mlc->n_rows;
    if (mlc->interdigitation) return pricing_scratch_bytes(mlc);
    return std::max(pricing_scratch_bytes(mlc), row_best_bytes((int64_t)rows) + rows * (mlc->n_cols + 1) * 8 + 64);
}

size_t pricing_scratch_bytes(const vmat_mlc *mlc) {
    const size_t rows = (size_t)mlc->K * mlc->n_rows;
    size_t b = rows * (sizeof(double) + 2 * sizeof(int16_t) + 1) + 64;
    if (mlc->interdigitation) {
        PricingGeom g{};
        g.K = mlc->K;
        g.n_rows = mlc->n_rows;
        g.n_cols = mlc->n_cols;
        b = std::max(b, interdig_scratch(nullptr, g).bytes);
    }
    return b;
}

// Scratch of price_apertures_noalloc: one fixed device array that every GPU loading
// the library keeps until the process exits.  Host code must not use the symbol as a
// pointer: its device address on the current device comes from cudaGetSymbolAddress.
constexpr size_t NOALLOC_BYTES = VMAT_NOALLOC_SCRATCH_BYTES;
static_assert(NOALLOC_BYTES == (size_t)VMAT_NOALLOC_MAX_ROWS * (sizeof(double) + 2 * sizeof(int16_t) + 1) + 64,
              "the fixed scratch holds the per-row bests of VMAT_NOALLOC_MAX_ROWS rows");
static __device__ __align__(256) unsigned char g_noalloc_price_scratch[NOALLOC_BYTES];

// Looked up on every call rather than cached: a cached address would outlive a
// cudaDeviceReset or a re-created primary context.
static vmat_status noalloc_scratch(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_price_scratch);
    if (e != cudaSuccess || !p)
        return set_error(VMAT_ECUDA, "price_apertures_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    *out = p;
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" vmat_status price_apertures(const vmat_mlc *mlc, const float *pi, const uint8_t *occupied,
                                       const int16_t *leaves, int32_t *best_cp, int16_t *best_leaves,
                                       double *best_price, void *stream) {
    clear_error();
    VMAT_TRY(validate_mlc(mlc));
    if (!pi || !occupied || !leaves || !best_cp || !best_leaves || !best_price)
        return set_error(VMAT_EINVAL, "price_apertures: NULL argument");
    cudaStream_t s = as_stream(stream);
    Scratch ws;
    VMAT_TRY(ws.alloc(pricing_scratch_bytes_prefix(mlc), s));
    return price_apertures_impl(mlc, pi, occupied, leaves, best_cp, best_leaves, best_price, ws.ptr, s, nullptr, true);
}

// Same computation as price_apertures with the fixed device scratch above: no
// device allocation in the call.  Nothing in the scratch has to start at zero:
// every per-row entry the CP kernel reads (unoccupied CPs) is written first by
// the row kernel of the same call.
extern "C" vmat_status price_apertures_noalloc(const vmat_mlc *mlc, const float *pi, const uint8_t *occupied,
                                               const int16_t *leaves, int32_t *best_cp, int16_t *best_leaves,
                                               double *best_price, void *stream) {
    clear_error();
    VMAT_TRY(validate_mlc(mlc));
    if (!pi || !occupied || !leaves || !best_cp || !best_leaves || !best_price)
        return set_error(VMAT_EINVAL, "price_apertures_noalloc: NULL argument");
    if ((int64_t)mlc->K * mlc->n_rows <= VMAT_NOALLOC_MAX_ROWS && pricing_scratch_bytes(mlc) > NOALLOC_BYTES)
        return set_error(VMAT_EINVAL, "price_apertures_noalloc: this MLC needs %zu bytes of scratch, over the fixed "
                         "scratch limit of %zu bytes; use price_apertures", pricing_scratch_bytes(mlc), NOALLOC_BYTES);
    if ((int64_t)mlc->K * mlc->n_rows > VMAT_NOALLOC_MAX_ROWS)
        return set_error(VMAT_EINVAL,
                         "price_apertures_noalloc: K * n_rows = %lld exceeds the fixed scratch limit of %d "
                         "(CP, MLC row) pairs; use price_apertures",
                         (long long)mlc->K * mlc->n_rows, VMAT_NOALLOC_MAX_ROWS);
    void *ws = nullptr;
    VMAT_TRY(noalloc_scratch(&ws));
    return price_apertures_impl(mlc, pi, occupied, leaves, best_cp, best_leaves, best_price, ws,
                                as_stream(stream), nullptr);
}
