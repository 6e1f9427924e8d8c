// Tile-streamed CSR SpMV for the two hot products of the paper:
//   beamlet price   pi = D^T g   (Eq. 3; CSR(D^T), one row per beamlet)
//   forward dose    d  = D x     (Section 2.1, Eq. 5; CSR(D), one row per non-empty voxel)
//
// The paper assigns one warp per beamlet row on Fermi (Section 2.2.2).  Here the
// nonzeros are cut into fixed tiles of THREADS*E entries independent of row
// boundaries, so every CTA streams the same number of bytes whatever the row
// lengths.  Per tile:
//   1. one elected thread moves the tile's values and column indices into shared
//      memory with cp.async.bulk (TMA bulk copies, L2 evict-first), STAGES tiles
//      ahead, completion counted on an mbarrier;
//   2. every thread takes 4-entry chunks in lane order (consecutive lanes hold
//      consecutive nonzeros, so the gathers x[col] of a warp touch few L2
//      sectors), multiplies, and stores the products to shared memory in an
//      XOR-swizzled layout;
//   3. every thread reads back E consecutive products (conflict-free), walks its
//      row boundaries, writes rows that start and end inside its run, and takes
//      part in a keyed (segmented) scan over the CTA for rows that span threads;
//   4. the partial sum of the row open at the tile's end is stored as a carry and
//      a second small kernel adds carries to their rows in tile order.
// All orders of addition are fixed, so results are bitwise reproducible.
#include <algorithm>

#include "internal.cuh"

namespace vmat {

struct SpmvParams {
    const int64_t *rowptr;
    const int32_t *col;
    const void *val;
    const float *x;
    float *y;
    const float *row_scale;  // multiply row r's sum by row_scale[r] (FP8 CSR(D^T)), or null
    const int32_t *row_ids;  // write row r to y[row_ids[r]], or null for y[r]
    const int32_t *tile_row; // [n_tiles + 1]
    const int32_t *tile_list; // tiles to process, or null for all
    const int32_t *n_list;   // device count of tile_list
    int32_t n_tiles;
    int32_t n_rows;
    int64_t nnz;
    float *carry_val;
    int32_t *status;
    const int32_t *skip; // when non-null and set, the kernel does nothing
};

template <typename VT> struct Vals;
template <> struct Vals<float> {
    static __device__ __forceinline__ void load4(const unsigned char *base, int e0, float v[4]) {
        float4 t = *reinterpret_cast<const float4 *>(base + (size_t)e0 * 4);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
};
template <> struct Vals<__nv_bfloat16> {
    static __device__ __forceinline__ void load4(const unsigned char *base, int e0, float v[4]) {
        uint2 t = *reinterpret_cast<const uint2 *>(base + (size_t)e0 * 2);
        v[0] = __uint_as_float(t.x << 16);
        v[1] = __uint_as_float(t.x & 0xffff0000u);
        v[2] = __uint_as_float(t.y << 16);
        v[3] = __uint_as_float(t.y & 0xffff0000u);
    }
};
template <> struct Vals<__nv_fp8_e4m3> {
    static __device__ __forceinline__ void load4(const unsigned char *base, int e0, float v[4]) {
        uint32_t t = *reinterpret_cast<const uint32_t *>(base + e0);
        __half2_raw a = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(t & 0xffffu), __NV_E4M3);
        __half2_raw b = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(t >> 16), __NV_E4M3);
        float2 fa = __half22float2(*reinterpret_cast<__half2 *>(&a));
        float2 fb = __half22float2(*reinterpret_cast<__half2 *>(&b));
        v[0] = fa.x;
        v[1] = fa.y;
        v[2] = fb.x;
        v[3] = fb.y;
    }
};

constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v / 2); }

template <int THREADS, int E, int STAGES, typename VT> struct TileShape {
    static constexpr int TILE = THREADS * E;
    static constexpr int NW = THREADS / 32;
    static constexpr int Q = E / 4;                      // float4 chunks per thread run
    static constexpr int SWZ_SHIFT = ilog2c(8 / (Q < 8 ? Q : 8)); // keeps 8 readers on distinct 16B slots
    static constexpr int VBYTES = TILE * (int)sizeof(VT);
    static constexpr int CBYTES = TILE * 4;
    static constexpr int OFF_COL = STAGES * VBYTES;
    static constexpr int OFF_PROD = OFF_COL + STAGES * CBYTES;
    static constexpr int OFF_BAR = OFF_PROD + TILE * 4;
    static constexpr int OFF_W = OFF_BAR + STAGES * 8;
    static constexpr int SMEM = OFF_W + NW * 12;
    static_assert(E % 4 == 0 && (Q & (Q - 1)) == 0, "E must be 4 * power of two");
    static_assert(VBYTES % 16 == 0 && CBYTES % 16 == 0, "bulk copies need 16-byte multiples");
};

__device__ __forceinline__ void store_row(const SpmvParams &p, int32_t r, float v) {
    if (p.row_scale) v *= p.row_scale[r];
    p.y[p.row_ids ? p.row_ids[r] : r] = v;
}

template <int THREADS, int E, int STAGES, typename VT>
__global__ void __launch_bounds__(THREADS) spmv_tile_kernel(SpmvParams p) {
    if (p.skip && *p.skip) return;
    using S = TileShape<THREADS, E, STAGES, VT>;
    constexpr int TILE = S::TILE, Q = S::Q, NW = S::NW;
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *sval = smem;
    unsigned char *scol = smem + S::OFF_COL;
    float *prod = reinterpret_cast<float *>(smem + S::OFF_PROD);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + S::OFF_BAR);
    int32_t *wkey = reinterpret_cast<int32_t *>(smem + S::OFF_W);
    int32_t *wfirst = wkey + NW;
    float *wval = reinterpret_cast<float *>(wfirst + NW);

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t n_work = p.tile_list ? *p.n_list : p.n_tiles;
    const int32_t n_rows = p.n_rows;
    const uint64_t pol = l2_evict_first_policy();

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int32_t w, int s) {
        const int32_t b = p.tile_list ? p.tile_list[w] : w;
        mbar_arrive_expect_tx(&bars[s], S::VBYTES + S::CBYTES);
        bulk_g2s(sval + s * S::VBYTES, static_cast<const unsigned char *>(p.val) + (size_t)b * S::VBYTES, S::VBYTES,
                 &bars[s], pol);
        bulk_g2s(scol + s * S::CBYTES, p.col + (size_t)b * TILE, S::CBYTES, &bars[s], pol);
    };
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            int32_t w = blockIdx.x + s * gridDim.x;
            if (w < n_work) issue(w, s);
        }
    }

    int it = 0;
    bool timed_out = false;
    for (int32_t w = blockIdx.x; w < n_work; w += gridDim.x, ++it) {
        const int s = it % STAGES;
        const uint32_t parity = (uint32_t)((it / STAGES) & 1);
        bool ok = mbar_wait_bounded(&bars[s], parity, WAIT_LIMIT_CYCLES);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(p.status, DEV_TIMEOUT);
            timed_out = true;
            break;
        }
        const int32_t b = p.tile_list ? p.tile_list[w] : w;
        const int64_t tstart = (int64_t)b * TILE;

        // ---- phase A: products in lane order, stored swizzled
        const unsigned char *sv = sval + s * S::VBYTES;
        const int32_t *sc = reinterpret_cast<const int32_t *>(scol + s * S::CBYTES);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int c = q * THREADS + tid; // chunk of 4 entries
            const int e0 = c * 4;
            int4 cc = *reinterpret_cast<const int4 *>(sc + e0);
            float v[4];
            Vals<VT>::load4(sv, e0, v);
            const int64_t g0 = tstart + e0;
            float4 pr;
            pr.x = g0 + 0 < p.nnz ? v[0] * __ldg(p.x + cc.x) : 0.f;
            pr.y = g0 + 1 < p.nnz ? v[1] * __ldg(p.x + cc.y) : 0.f;
            pr.z = g0 + 2 < p.nnz ? v[2] * __ldg(p.x + cc.z) : 0.f;
            pr.w = g0 + 3 < p.nnz ? v[3] * __ldg(p.x + cc.w) : 0.f;
            const int tr = c / Q, qq = c % Q;
            const int phys = tr * Q + (qq ^ ((tr >> S::SWZ_SHIFT) & (Q - 1)));
            reinterpret_cast<float4 *>(prod)[phys] = pr;
        }
        __syncthreads(); // stage s fully consumed, products visible
        if (tid == 0) { // the barrier orders all reads of stage s before its next copy
            const int32_t wn = w + STAGES * gridDim.x;
            if (wn < n_work) issue(wn, s);
        }

        // ---- phase B: each thread owns entries [a, a + E) of the tile
        float pv[E];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int phys = tid * Q + (q ^ ((tid >> S::SWZ_SHIFT) & (Q - 1)));
            float4 t = reinterpret_cast<const float4 *>(prod)[phys];
            pv[4 * q + 0] = t.x;
            pv[4 * q + 1] = t.y;
            pv[4 * q + 2] = t.z;
            pv[4 * q + 3] = t.w;
        }
        const int64_t a = tstart + (int64_t)tid * E;
        // row containing entry a: largest r with rowptr[r] <= a (n_rows once past the end)
        int32_t lo = p.tile_row[b], hi = p.tile_row[b + 1];
        while (lo < hi) {
            int32_t mid = (int32_t)(((int64_t)lo + hi + 1) >> 1);
            if (__ldg(p.rowptr + mid) <= a) lo = mid;
            else hi = mid - 1;
        }
        int32_t r = lo;
        if (b == 0 && tid == 0)
            for (int32_t rr = 0; rr < r; ++rr) store_row(p, rr, 0.f); // leading empty rows
        int64_t nxt = r < n_rows ? __ldg(p.rowptr + r + 1) : INT64_MAX;
        float run = 0.f;
        int32_t head_row = -1;
        float head_val = 0.f;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            run += pv[e];
            const int64_t i1 = a + e + 1;
            while (i1 == nxt) { // row r ends after entry a + e (empty rows end here too)
                if (head_row < 0 && r == lo) {
                    head_row = r;
                    head_val = run;
                } else {
                    store_row(p, r, run);
                }
                run = 0.f;
                ++r;
                nxt = r < n_rows ? __ldg(p.rowptr + r + 1) : INT64_MAX;
            }
        }
        // ---- keyed inclusive scan of the open-row partials over the CTA
        int32_t key = r;
        float val = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t k2 = __shfl_up_sync(0xffffffffu, key, d);
            float v2 = __shfl_up_sync(0xffffffffu, val, d);
            if (lane >= d && k2 == key) val += v2;
        }
        const int32_t kfirst = __shfl_sync(0xffffffffu, key, 0);
        if (lane == 31) {
            wkey[wid] = key;
            wval[wid] = val;
        }
        if (lane == 0) wfirst[wid] = key;
        __syncthreads();
        float tprev = 0.f;
        int32_t kprev = -2;
        if (wid > 0) {
            float t = 0.f;
            for (int ww = 0; ww < wid; ++ww) {
                const bool cont = ww > 0 && wfirst[ww] == wkey[ww] && wkey[ww - 1] == wkey[ww];
                t = wval[ww] + (cont ? t : 0.f);
            }
            tprev = t;
            kprev = wkey[wid - 1];
            if (key == kfirst && kprev == key) val += tprev;
        }
        float pval = __shfl_up_sync(0xffffffffu, val, 1);
        int32_t pkey = __shfl_up_sync(0xffffffffu, key, 1);
        if (lane == 0) {
            pval = tprev;
            pkey = kprev;
        }
        if (head_row >= 0) store_row(p, head_row, head_val + (pkey == head_row ? pval : 0.f));
        // The row open at the tile's end is tile_row[b + 1] (the row holding entry
        // (b + 1) * TILE, or n_rows): the last thread's key.  Its partial is the carry.
        if (tid == THREADS - 1) p.carry_val[b] = val;
        __syncthreads(); // products and warp totals are reused by the next tile
    }
    if (timed_out && tid == 0) {
        // let copies already issued land before the CTA exits (bounded)
        for (int k = 0; k < STAGES; ++k) {
            const int it2 = it + k;
            const int32_t w2 = blockIdx.x + it2 * gridDim.x;
            if (w2 < n_work) mbar_wait_bounded(&bars[it2 % STAGES], (uint32_t)((it2 / STAGES) & 1), WAIT_LIMIT_CYCLES);
        }
    }
}

// ---------------------------------------------------------------------------
// Warp-per-row variant (the paper's mapping, Section 2.2.2), vectorised: each
// lane streams 4-entry chunks with 128-bit loads that bypass L1 and are marked
// evict-first in L2 (the matrix is read once), keeps one accumulator per chunk
// position, and the warp reduces with a fixed butterfly.  Row heads and tails
// that are not 4-aligned are taken one entry per lane.  No shared memory, so
// occupancy is set by registers; rows of inactive CPs are skipped outright.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ldg_stream_f4(const void *p, uint64_t pol) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ int4 ldg_stream_i4(const void *p, uint64_t pol) {
    int4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint2 ldg_stream_u2(const void *p, uint64_t pol) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
        : "=r"(r.x), "=r"(r.y)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ldg_stream_u1(const void *p, uint64_t pol) {
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ uint32_t ldg_stream_b16(const void *p, uint64_t pol) {
    unsigned short r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ldg_stream_b8(const void *p, uint64_t pol) {
    unsigned short r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u8 %0, [%1], %2;" : "=h"(r) : "l"(p), "l"(pol));
    return r;
}

// One stored value, streamed (consecutive-lane kernel).
template <typename VT> struct StreamVal1;
template <> struct StreamVal1<float> {
    static __device__ __forceinline__ float load(const void *val, int64_t e, uint64_t pol) {
        return __uint_as_float(ldg_stream_u1(static_cast<const float *>(val) + e, pol));
    }
};
template <> struct StreamVal1<__nv_bfloat16> {
    static __device__ __forceinline__ float load(const void *val, int64_t e, uint64_t pol) {
        return __uint_as_float(ldg_stream_b16(static_cast<const uint16_t *>(val) + e, pol) << 16);
    }
};
template <> struct StreamVal1<__nv_fp8_e4m3> {
    static __device__ __forceinline__ float load(const void *val, int64_t e, uint64_t pol) {
        __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)ldg_stream_b8(static_cast<const uint8_t *>(val) + e, pol),
                                               __NV_E4M3);
        return __half2float(*reinterpret_cast<__half *>(&h));
    }
};

template <typename VT> struct StreamVals;
template <> struct StreamVals<float> {
    static __device__ __forceinline__ void load4(const void *val, int64_t e0, uint64_t pol, float v[4]) {
        float4 t = ldg_stream_f4(static_cast<const float *>(val) + e0, pol);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    }
    static __device__ __forceinline__ float load1(const void *val, int64_t e) {
        return __ldg(static_cast<const float *>(val) + e);
    }
};
template <> struct StreamVals<__nv_bfloat16> {
    static __device__ __forceinline__ void load4(const void *val, int64_t e0, uint64_t pol, float v[4]) {
        uint2 t = ldg_stream_u2(static_cast<const uint16_t *>(val) + e0, pol);
        v[0] = __uint_as_float(t.x << 16);
        v[1] = __uint_as_float(t.x & 0xffff0000u);
        v[2] = __uint_as_float(t.y << 16);
        v[3] = __uint_as_float(t.y & 0xffff0000u);
    }
    static __device__ __forceinline__ float load1(const void *val, int64_t e) {
        return __uint_as_float((uint32_t)__ldg(static_cast<const unsigned short *>(val) + e) << 16);
    }
};
template <> struct StreamVals<__nv_fp8_e4m3> {
    static __device__ __forceinline__ void load4(const void *val, int64_t e0, uint64_t pol, float v[4]) {
        uint32_t t = ldg_stream_u1(static_cast<const uint8_t *>(val) + e0, pol);
        __half2_raw a = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(t & 0xffffu), __NV_E4M3);
        __half2_raw b = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(t >> 16), __NV_E4M3);
        float2 fa = __half22float2(*reinterpret_cast<__half2 *>(&a));
        float2 fb = __half22float2(*reinterpret_cast<__half2 *>(&b));
        v[0] = fa.x;
        v[1] = fa.y;
        v[2] = fb.x;
        v[3] = fb.y;
    }
    static __device__ __forceinline__ float load1(const void *val, int64_t e) {
        __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)__ldg(static_cast<const unsigned char *>(val) + e),
                                               __NV_E4M3);
        return __half2float(*reinterpret_cast<__half *>(&h));
    }
};

struct RowParams {
    const int64_t *rowptr;
    const int32_t *col;
    const void *val;
    const float *x;
    float *y;
    const float *row_scale;
    const int32_t *row_ids;
    RowMask mask; // the rows to compute
    int32_t n_rows;
    int64_t stride; // rows between a warp's consecutive rows (<= the launch's warps; warps past it idle)
    const int32_t *skip; // when non-null and set, the kernel does nothing
    const uint16_t *col16; // 16-bit column index (configurations that read it)
    const int32_t *cbase;
    const int64_t *cptr;
};

// Sum of row r (all lanes of a warp; the result is valid in every lane): 4-entry
// chunks per lane with 128-bit streaming loads, 4 accumulators per lane, a fixed
// butterfly.  The head (< 4 entries before the first 4-aligned one) and the tail
// take one entry per lane.
template <int UNROLL, typename VT>
__device__ __forceinline__ float warp_row_sum(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                              const void *__restrict__ val, const float *__restrict__ x, int64_t r,
                                              int lane, uint64_t pol) {
    const int64_t s = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
    const int64_t a = min((s + 3) & ~(int64_t)3, e); // first 4-aligned entry
    const int64_t b = max(a, e & ~(int64_t)3);        // end of the aligned body
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if (lane < a - s) {
        const int64_t i = s + lane;
        acc[0] = StreamVals<VT>::load1(val, i) * __ldg(x + __ldg(col + i));
    }
    if (lane < e - b) {
        const int64_t i = b + lane;
        acc[1] = StreamVals<VT>::load1(val, i) * __ldg(x + __ldg(col + i));
    }
    const int64_t nch = (b - a) >> 2;
    for (int64_t c = lane; c < nch; c += 32 * UNROLL) {
        float v[UNROLL][4];
        int4 cc[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t cu = c + 32 * u;
            if (cu < nch) {
                const int64_t e0 = a + 4 * cu;
                StreamVals<VT>::load4(val, e0, pol, v[u]);
                cc[u] = ldg_stream_i4(col + e0, pol);
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (c + 32 * u < nch) {
                acc[0] = fmaf(v[u][0], __ldg(x + cc[u].x), acc[0]);
                acc[1] = fmaf(v[u][1], __ldg(x + cc[u].y), acc[1]);
                acc[2] = fmaf(v[u][2], __ldg(x + cc[u].z), acc[2]);
                acc[3] = fmaf(v[u][3], __ldg(x + cc[u].w), acc[3]);
            }
        }
    }
    float sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    return sum;
}

// The same row sum with consecutive entries across the lanes: chunk m of 32 U
// entries gives lane l the entries base + 32 u + l (u < U), so each gather of x
// by the warp covers 32 consecutive (sorted) column indices and touches fewer
// cache lines.  Scalar streaming loads of the values and columns; entry
// base + 32 u + l goes to accumulator u % 4 of lane l, in a fixed order.
template <int UNROLL, typename VT>
__device__ __forceinline__ float warp_row_sum_c(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                const void *__restrict__ val, const float *__restrict__ x, int64_t r,
                                                int lane, uint64_t pol) {
    const int64_t s = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t b = s; b < e; b += 32 * UNROLL) {
        float v[UNROLL];
        int32_t c[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t i = b + 32 * u + lane;
            if (i < e) {
                v[u] = StreamVal1<VT>::load(val, i, pol);
                c[u] = (int32_t)ldg_stream_u1(col + i, pol);
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (b + 32 * u + lane < e) acc[u & 3] = fmaf(v[u], __ldg(x + c[u]), acc[u & 3]);
    }
    float sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    return sum;
}

// The consecutive-lane row sum reading the 16-bit column index: entry i of chunk
// t (i - s in [t ZCHUNK, (t + 1) ZCHUNK)) has column cbase[cptr[r] + t] + col16[i].
// The chunk base is the same for all lanes of a load (one broadcast load, one per
// iteration); the products and their order are those of warp_row_sum_c, so the
// sums are identical.
template <int UNROLL, typename VT>
__device__ __forceinline__ float warp_row_sum_z(const int64_t *__restrict__ rowptr, const int64_t *__restrict__ cptr,
                                                const int32_t *__restrict__ cbase, const uint16_t *__restrict__ col16,
                                                const void *__restrict__ val, const float *__restrict__ x, int64_t r,
                                                int lane, uint64_t pol) {
    static_assert((32 * UNROLL) % ZCHUNK == 0, "an iteration covers whole chunks");
    const int64_t s = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
    const int32_t *cb = cbase + __ldg(cptr + r);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int64_t b = s; b < e; b += 32 * UNROLL, cb += 32 * UNROLL / ZCHUNK) {
        float v[UNROLL];
        int32_t c[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const int64_t i = b + 32 * u + lane;
            if (i < e) {
                v[u] = StreamVal1<VT>::load(val, i, pol);
                c[u] = __ldg(cb + (32 * u) / ZCHUNK) + (int32_t)ldg_stream_b16(col16 + i, pol);
            }
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (b + 32 * u + lane < e) acc[u & 3] = fmaf(v[u], __ldg(x + c[u]), acc[u & 3]);
    }
    float sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    return sum;
}

// The rows of a warp-row launch, passed to f in order.  Without a list: rows
// warp0, warp0 + stride, ... that the mask keeps.  With the window list (mask.woff):
// list items in runs of WIN_RUN consecutive items, run warp0, warp0 + stride, ...; the
// items of a run are consecutive rows of one window segment or of the next ones, so
// the segment is searched once per run and then followed item by item.
constexpr int WIN_RUN = 4;
template <typename F> __device__ __forceinline__ void for_rows(const RowParams &p, int64_t warp0, F &&f) {
    if (!p.mask.woff) {
        for (int64_t r = warp0; r < p.n_rows; r += p.stride)
            if (row_needed(p.mask, r)) f(r);
        return;
    }
    const int64_t n_items = (int64_t)__ldg(p.mask.woff + p.mask.nseg);
    for (int64_t c0 = warp0 * WIN_RUN; c0 < n_items; c0 += p.stride * WIN_RUN) {
        int lo = 0, hi = p.mask.nseg; // woff[lo] <= c0 < woff[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(p.mask.woff + mid) <= c0) lo = mid;
            else hi = mid;
        }
        int64_t seg_end = __ldg(p.mask.woff + lo + 1);
        int64_t r = (int64_t)lo * p.mask.n_cols + __ldg(p.mask.win + lo).x + (c0 - __ldg(p.mask.woff + lo));
        const int64_t c1 = min(c0 + WIN_RUN, n_items);
        for (int64_t i = c0; i < c1; ++i, ++r) {
            while (i == seg_end) { // the next segment with a row (empty windows have none)
                ++lo;
                seg_end = __ldg(p.mask.woff + lo + 1);
                r = (int64_t)lo * p.mask.n_cols + __ldg(p.mask.win + lo).x;
            }
            f(r);
        }
    }
}

template <int THREADS, int UNROLL, typename VT>
__global__ void __launch_bounds__(THREADS) spmv_warp_row_z_kernel(RowParams p) {
    if (p.skip && *p.skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
    if (warp0 >= p.stride) return; // warp-uniform
    const uint64_t pol = l2_evict_first_policy();
    for_rows(p, warp0, [&](int64_t r) {
        float sum = warp_row_sum_z<UNROLL, VT>(p.rowptr, p.cptr, p.cbase, p.col16, p.val, p.x, r, lane, pol);
        if (lane == 0) {
            if (p.row_scale) sum *= p.row_scale[r];
            p.y[p.row_ids ? p.row_ids[r] : r] = sum;
        }
    });
}

template <int THREADS, int UNROLL, typename VT>
__global__ void __launch_bounds__(THREADS) spmv_warp_row_c_kernel(RowParams p) {
    if (p.skip && *p.skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
    if (warp0 >= p.stride) return; // warp-uniform
    const uint64_t pol = l2_evict_first_policy();
    for_rows(p, warp0, [&](int64_t r) {
        float sum = warp_row_sum_c<UNROLL, VT>(p.rowptr, p.col, p.val, p.x, r, lane, pol);
        if (lane == 0) {
            if (p.row_scale) sum *= p.row_scale[r];
            p.y[p.row_ids ? p.row_ids[r] : r] = sum;
        }
    });
}

template <int THREADS, int UNROLL, typename VT>
__global__ void __launch_bounds__(THREADS) spmv_warp_row_kernel(RowParams p) {
    if (p.skip && *p.skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
    if (warp0 >= p.stride) return; // warp-uniform
    const uint64_t pol = l2_evict_first_policy();
    for_rows(p, warp0, [&](int64_t r) {
        float sum = warp_row_sum<UNROLL, VT>(p.rowptr, p.col, p.val, p.x, r, lane, pol);
        if (lane == 0) {
            if (p.row_scale) sum *= p.row_scale[r];
            p.y[p.row_ids ? p.row_ids[r] : r] = sum;
        }
    });
}

// Several plans' matrices in one launch: global row g belongs to plan p with
// row_off[p] <= g < row_off[p + 1] (row g - row_off[p] of that plan).  A warp
// looks its plan up when it crosses into another plan's range.
template <int THREADS, int UNROLL, typename VT, bool CONSEC>
__global__ void __launch_bounds__(THREADS)
    spmv_rows_batched_kernel(const SpmvPlan *__restrict__ plans, const int64_t *__restrict__ row_off, int32_t n_plans,
                             int64_t total_rows, int64_t stride) {
    __shared__ int64_t soff[VMAT_MAX_BATCH + 1];
    for (int i = threadIdx.x; i <= n_plans; i += THREADS) soff[i] = row_off[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
    if (warp0 >= stride) return; // warp-uniform, after the block's only barrier
    const uint64_t pol = l2_evict_first_policy();
    int64_t lo = 0, hi = 0;
    SpmvPlan P;
    bool skip = true;
    for (int64_t gr = warp0; gr < total_rows; gr += stride) {
        if (gr < lo || gr >= hi) {
            int a = 0, b = n_plans; // soff[a] <= gr < soff[b]
            while (b - a > 1) {
                const int m = (a + b) >> 1;
                if (soff[m] <= gr) a = m;
                else b = m;
            }
            P = plans[a];
            lo = soff[a];
            hi = soff[a + 1];
            skip = P.skip && *P.skip;
        }
        if (skip) continue;
        const int64_t r = gr - lo;
        if (!row_needed(P.mask, r)) continue;
        float sum = CONSEC ? warp_row_sum_c<UNROLL, VT>(P.rowptr, P.col, P.val, P.x, r, lane, pol)
                           : warp_row_sum<UNROLL, VT>(P.rowptr, P.col, P.val, P.x, r, lane, pol);
        if (lane == 0) {
            if (P.row_scale) sum *= P.row_scale[r];
            P.y[P.row_ids ? P.row_ids[r] : r] = sum;
        }
    }
}

// Adds tile carries to their rows.  Tile b's carry belongs to row tile_row[b + 1];
// the first tile of each run of equal keys sums the run left to right.  Rows not in
// the mask are skipped (their tiles may not have run).
__global__ void spmv_fixup(const int32_t *tile_row, const float *carry_val, int32_t n_tiles,
                           const int32_t *tile_list, const int32_t *n_list, int32_t n_rows, float *y,
                           const int32_t *row_ids, const float *row_scale, RowMask mask) {
    const int32_t n_work = tile_list ? *n_list : n_tiles;
    for (int32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < n_work; w += gridDim.x * blockDim.x) {
        const int32_t b = tile_list ? tile_list[w] : w;
        const int32_t key = tile_row[b + 1];
        if (key >= n_rows) continue;
        if (!row_needed(mask, key)) continue;
        if (b > 0 && tile_row[b] == key) continue;
        float sum = carry_val[b];
        for (int32_t bb = b + 1; bb < n_tiles && tile_row[bb + 1] == key; ++bb) sum += carry_val[bb];
        if (row_scale) sum *= row_scale[key];
        y[row_ids ? row_ids[key] : key] += sum;
    }
}

// tile_row[b] = largest r with rowptr[r] <= b * tile (tile_row[0] = 0, tile_row[n_tiles] = n_rows).
__global__ void compute_tile_rows(const int64_t *rowptr, int32_t n_rows, int32_t tile, int32_t n_tiles,
                                  int32_t *tile_row) {
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= n_tiles; b += gridDim.x * blockDim.x) {
        if (b == 0) {
            tile_row[0] = 0;
            continue;
        }
        const int64_t a = (int64_t)b * tile;
        int32_t lo = 0, hi = n_rows;
        while (lo < hi) {
            int32_t mid = (int32_t)(((int64_t)lo + hi + 1) >> 1);
            if (rowptr[mid] <= a) lo = mid;
            else hi = mid - 1;
        }
        tile_row[b] = lo;
    }
}

// A tile is active when its row range [tile_row[b], tile_row[b+1]] meets a row in the mask.
__global__ void flag_active_tiles(const int32_t *tile_row, int32_t n_tiles, int32_t n_rows, RowMask mask,
                                  int32_t *flag) {
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_tiles; b += gridDim.x * blockDim.x) {
        const int32_t r0 = tile_row[b];
        const int32_t r1 = min(tile_row[b + 1], n_rows - 1);
        int32_t f = 0;
        if (mask.win) {
            for (int32_t r = r0; r <= r1 && !f; ++r) f = row_needed(mask, r) ? 1 : 0;
        } else {
            for (int32_t k = r0 / mask.bpc; k <= r1 / mask.bpc && !f; ++k) f = mask.cp_active[k] != 0;
        }
        flag[b] = f;
    }
}

__global__ void compact_tiles(const int32_t *flag, const int64_t *off, int32_t n_tiles, int32_t *list,
                              int32_t *n_list) {
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_tiles; b += gridDim.x * blockDim.x)
        if (flag[b]) list[off[b]] = b;
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_list = (int32_t)off[n_tiles];
}

__global__ void scale_vector(const float *x, const float *s, float *out, int32_t n) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = x[i] * s[i];
}

// ---------------------------------------------------------------------------
// Configurations and dispatch
// ---------------------------------------------------------------------------
struct Cfg {
    int family; // 0 = tile-segmented, 1 = warp per row (4-entry lane chunks), 2 = warp per row (consecutive
                // lanes), 3 = as 2 reading the 16-bit column index
    int threads, e, stages; // tile: E entries per thread, STAGES bulk-copy stages; warp-row: e = unroll
};
static const Cfg kCfgs[] = {{0, 256, 16, 2}, {0, 256, 8, 3}, {0, 512, 8, 2}, {0, 128, 16, 3},
                            {1, 256, 2, 0},  {1, 256, 1, 0}, {1, 512, 4, 0}, {1, 256, 4, 0},
                            {1, 256, 8, 0}, {2, 256, 4, 0}, {2, 256, 8, 0}, {2, 512, 4, 0},
                            {3, 256, 4, 0}, {3, 256, 8, 0}, {3, 512, 4, 0}};
constexpr int N_CFG = 15;

using TileFn = void (*)(SpmvParams);
using RowFn = void (*)(RowParams);
using RowBatchFn = void (*)(const SpmvPlan *, const int64_t *, int32_t, int64_t, int64_t);

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Row stride of a warp-row launch with n_warps warps: the largest s <= n_warps that
// is coprime with every MLC column count in cols[0..n).  A warp's rows r, r + s, ...
// then cycle through every beamlet column instead of keeping one (n_warps is a
// multiple of the warps per block, and so often of n_cols), which keeps the warps
// balanced when the leaf-travel windows leave whole columns out of a pass.
static int64_t coprime_stride(int64_t n_warps, const int32_t *cols, int n) {
    for (int64_t st = n_warps; st > n_warps / 2 && st > 1; --st) {
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) ok = cols[i] <= 1 || gcd64(st, cols[i]) == 1;
        if (ok) return st;
    }
    return std::max<int64_t>(n_warps, 1);
}

template <typename VT> TileFn tile_kernel_for(int cfg) {
    switch (cfg) {
    case 0: return spmv_tile_kernel<256, 16, 2, VT>;
    case 1: return spmv_tile_kernel<256, 8, 3, VT>;
    case 2: return spmv_tile_kernel<512, 8, 2, VT>;
    default: return spmv_tile_kernel<128, 16, 3, VT>;
    }
}

template <typename VT> RowFn row_kernel_for(int cfg) {
    switch (cfg) {
    case 4: return spmv_warp_row_kernel<256, 2, VT>;
    case 5: return spmv_warp_row_kernel<256, 1, VT>;
    case 7: return spmv_warp_row_kernel<256, 4, VT>;
    case 8: return spmv_warp_row_kernel<256, 8, VT>;
    case 9: return spmv_warp_row_c_kernel<256, 4, VT>;
    case 10: return spmv_warp_row_c_kernel<256, 8, VT>;
    case 11: return spmv_warp_row_c_kernel<512, 4, VT>;
    case 12: return spmv_warp_row_z_kernel<256, 4, VT>;
    case 13: return spmv_warp_row_z_kernel<256, 8, VT>;
    case 14: return spmv_warp_row_z_kernel<512, 4, VT>;
    default: return spmv_warp_row_kernel<512, 4, VT>;
    }
}

template <typename VT> int smem_for(int cfg) {
    switch (cfg) {
    case 0: return TileShape<256, 16, 2, VT>::SMEM;
    case 1: return TileShape<256, 8, 3, VT>::SMEM;
    case 2: return TileShape<512, 8, 2, VT>::SMEM;
    case 3: return TileShape<128, 16, 3, VT>::SMEM;
    default: return 0;
    }
}

struct Launch {
    TileFn tile = nullptr;
    RowFn row = nullptr;
    int threads = 0, smem = 0, blocks_per_sm = 0;
};

template <typename VT> static void pick(int cfg, Launch &n) {
    if (kCfgs[cfg].family == 0) {
        n.tile = tile_kernel_for<VT>(cfg);
        n.smem = smem_for<VT>(cfg);
    } else {
        n.row = row_kernel_for<VT>(cfg);
        n.smem = 0;
    }
}

static vmat_status launch_info(vmat_dtype dt, int cfg, Launch *out) {
    static Launch cache[3][N_CFG];
    static int cached_dev[3][N_CFG];
    int dev;
    VMAT_CUDA(cudaGetDevice(&dev));
    Launch &L = cache[dt][cfg];
    if ((L.tile || L.row) && cached_dev[dt][cfg] == dev) {
        *out = L;
        return VMAT_OK;
    }
    Launch n;
    n.threads = kCfgs[cfg].threads;
    if (dt == VMAT_F32) pick<float>(cfg, n);
    else if (dt == VMAT_BF16) pick<__nv_bfloat16>(cfg, n);
    else pick<__nv_fp8_e4m3>(cfg, n);
    if (n.tile) {
        VMAT_CUDA(cudaFuncSetAttribute(n.tile, cudaFuncAttributeMaxDynamicSharedMemorySize, n.smem));
        VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n.blocks_per_sm, n.tile, n.threads, n.smem));
    } else {
        VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n.blocks_per_sm, n.row, n.threads, 0));
    }
    if (n.blocks_per_sm < 1) return set_error(VMAT_ECUDA, "spmv: configuration %d does not fit on an SM", cfg);
    L = n;
    cached_dev[dt][cfg] = dev;
    *out = n;
    return VMAT_OK;
}

int spmv_n_configs() { return N_CFG; }
bool spmv_config_index16(int cfg) { return cfg >= 0 && cfg < N_CFG && kCfgs[cfg].family == 3; }
int spmv_default_config() { return 4; }
int32_t spmv_config_tile(int cfg) { return kCfgs[cfg].family == 0 ? kCfgs[cfg].threads * kCfgs[cfg].e : 0; }

vmat_status spmv_prepare_tiles(CsrMat &m, int cfg, cudaStream_t s) {
    if (kCfgs[cfg].family == 3 && !m.col16 && m.nnz > 0)
        return set_error(VMAT_EUNSUPPORTED, "spmv: configuration %d reads the 16-bit column index, which this matrix "
                                            "does not hold (build with index16, chunks spanning < 65536 columns)", cfg);
    if (kCfgs[cfg].family != 0) { // warp per row: no tile structure needed
        m.cfg = cfg;
        m.tile = 0;
        return VMAT_OK;
    }
    const int32_t tile = spmv_config_tile(cfg);
    const int32_t n_tiles = (int32_t)std::max<int64_t>(1, (m.nnz + tile - 1) / tile);
    if ((int64_t)n_tiles * tile > m.nnz_pad) return set_error(VMAT_ECUDA, "spmv: padding smaller than a tile");
    if (m.tile_row && m.n_tiles != n_tiles) {
        cudaFree(m.tile_row);
        cudaFree(m.carry_val);
        cudaFree(m.tile_flag);
        cudaFree(m.tile_list);
        cudaFree(m.n_list);
        m.tile_row = m.tile_flag = m.tile_list = m.n_list = nullptr;
        m.carry_val = nullptr;
    }
    if (!m.tile_row) {
        VMAT_CUDA(cudaMalloc(&m.tile_row, (size_t)(n_tiles + 1) * 4));
        VMAT_CUDA(cudaMalloc(&m.carry_val, (size_t)n_tiles * 4));
        VMAT_CUDA(cudaMalloc(&m.tile_flag, (size_t)(n_tiles + 1) * 4));
        VMAT_CUDA(cudaMalloc(&m.tile_list, (size_t)n_tiles * 4));
        // n_list[0] = count; 8-byte aligned int64 offsets of the tile scan follow at byte 8
        VMAT_CUDA(cudaMalloc(&m.n_list, 8 + 8 * (size_t)(n_tiles + 1)));
    }
    m.cfg = cfg;
    m.tile = tile;
    m.n_tiles = n_tiles;
    compute_tile_rows<<<std::max(1, std::min(1024, (n_tiles + 256) / 256)), 256, 0, s>>>(m.rowptr, m.n_rows, tile,
                                                                                       n_tiles, m.tile_row);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status spmv_run(const Ddc &h, const CsrMat &m, const float *x, float *y, const float *row_scale, RowMask mask,
                     cudaStream_t s, const int32_t *skip) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    Launch L;
    VMAT_TRY(launch_info(h.dtype, m.cfg, &L));
    if (L.row) {
        RowParams p;
        p.rowptr = m.rowptr;
        p.col = m.col;
        p.val = m.val;
        p.x = x;
        p.y = y;
        p.row_scale = row_scale;
        p.row_ids = m.row_ids;
        p.mask = mask;
        p.n_rows = m.n_rows;
        p.skip = skip;
        p.col16 = m.col16;
        p.cbase = m.cbase;
        p.cptr = m.cptr;
        if (kCfgs[m.cfg].family == 3 && !m.col16 && m.n_rows > 0)
            return set_error(VMAT_ESTATE, "spmv: configuration %d needs the 16-bit column index", m.cfg);
        const int64_t warps = std::max<int64_t>(1, m.n_rows);
        const int64_t want = (warps * 32 + L.threads - 1) / L.threads;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->n_sm * L.blocks_per_sm));
        const int64_t n_warps = (int64_t)grid * L.threads / 32;
        p.stride = mask.win && !mask.woff ? coprime_stride(n_warps, &mask.n_cols, 1) : n_warps;
        L.row<<<grid, L.threads, 0, s>>>(p);
        VMAT_LAUNCH_CHECK();
        return VMAT_OK;
    }
    const int32_t *list = nullptr;
    int32_t *n_list = nullptr;
    if (mask.cp_active || mask.win) {
        // ordered list of active tiles: flags, exclusive scan, compaction
        int64_t *off = reinterpret_cast<int64_t *>(m.n_list + 2);
        int g = std::max(1, std::min(ctx->n_sm * 8, (m.n_tiles + 255) / 256));
        flag_active_tiles<<<g, 256, 0, s>>>(m.tile_row, m.n_tiles, m.n_rows, mask, m.tile_flag);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(scan_counts(m.tile_flag, off, m.n_tiles, s));
        compact_tiles<<<g, 256, 0, s>>>(m.tile_flag, off, m.n_tiles, m.tile_list, m.n_list);
        VMAT_LAUNCH_CHECK();
        list = m.tile_list;
        n_list = m.n_list;
    }
    SpmvParams p;
    p.rowptr = m.rowptr;
    p.col = m.col;
    p.val = m.val;
    p.x = x;
    p.y = y;
    p.row_scale = row_scale;
    p.row_ids = m.row_ids;
    p.tile_row = m.tile_row;
    p.tile_list = list;
    p.n_list = n_list;
    p.n_tiles = m.n_tiles;
    p.n_rows = m.n_rows;
    p.nnz = m.nnz;
    p.carry_val = m.carry_val;
    p.status = ctx->status;
    p.skip = skip;
    const int grid = std::max(1, std::min(m.n_tiles, ctx->n_sm * L.blocks_per_sm));
    L.tile<<<grid, L.threads, L.smem, s>>>(p);
    VMAT_LAUNCH_CHECK();
    const int gf = std::max(1, std::min(ctx->n_sm * 4, (m.n_tiles + 255) / 256));
    spmv_fixup<<<gf, 256, 0, s>>>(m.tile_row, m.carry_val, m.n_tiles, list, n_list, m.n_rows, y, m.row_ids,
                                  row_scale, mask);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

template <typename VT> static RowBatchFn batched_kernel_for(int cfg) {
    switch (cfg) {
    case 4: return spmv_rows_batched_kernel<256, 2, VT, false>;
    case 5: return spmv_rows_batched_kernel<256, 1, VT, false>;
    case 6: return spmv_rows_batched_kernel<512, 4, VT, false>;
    case 7: return spmv_rows_batched_kernel<256, 4, VT, false>;
    case 8: return spmv_rows_batched_kernel<256, 8, VT, false>;
    case 9: return spmv_rows_batched_kernel<256, 4, VT, true>;
    case 10: return spmv_rows_batched_kernel<256, 8, VT, true>;
    case 11: return spmv_rows_batched_kernel<512, 4, VT, true>;
    default: return nullptr;
    }
}

bool spmv_batched_config(int cfg) {
    return cfg >= 0 && cfg < N_CFG && (kCfgs[cfg].family == 1 || kCfgs[cfg].family == 2);
}

vmat_status spmv_rows_batched(vmat_dtype dt, int cfg, const SpmvPlan *plans, const int64_t *row_off, int32_t n_plans,
                              int64_t total_rows, cudaStream_t s, const int32_t *cols, int n_cols) {
    if (!spmv_batched_config(cfg)) return set_error(VMAT_EINVAL, "spmv_rows_batched: configuration %d is not warp-row", cfg);
    if (n_plans < 1 || n_plans > VMAT_MAX_BATCH) return set_error(VMAT_EINVAL, "spmv_rows_batched: bad plan count");
    if (total_rows <= 0) return VMAT_OK;
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    RowBatchFn fn = dt == VMAT_F32 ? batched_kernel_for<float>(cfg)
                    : dt == VMAT_BF16 ? batched_kernel_for<__nv_bfloat16>(cfg)
                                      : batched_kernel_for<__nv_fp8_e4m3>(cfg);
    const int threads = kCfgs[cfg].threads;
    int bps = 1;
    VMAT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, threads, 0));
    const int64_t want = (total_rows * 32 + threads - 1) / threads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)ctx->n_sm * std::max(bps, 1)));
    fn<<<grid, threads, 0, s>>>(plans, row_off, n_plans, total_rows,
                                coprime_stride((int64_t)grid * threads / 32, cols, cols ? n_cols : 0));
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status dose_forward_impl(const Ddc &h, const float *x, float *d, bool compact, cudaStream_t s) {
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    const float *xin = x;
    if (h.dtype == VMAT_FP8E4M3) { // columns of CSR(D) carry the per-beamlet scale: use s o x
        scale_vector<<<std::max(1, std::min(ctx->n_sm * 8, (h.J + 255) / 256)), 256, 0, s>>>(x, h.scale, h.xs, h.J);
        VMAT_LAUNCH_CHECK();
        xin = h.xs;
    }
    if (compact) {
        CsrMat m = h.D;
        m.row_ids = nullptr;
        return spmv_run(h, m, xin, d, nullptr, all_rows(), s);
    }
    VMAT_CUDA(cudaMemsetAsync(d, 0, (size_t)h.V * 4, s));
    return spmv_run(h, h.D, xin, d, nullptr, all_rows(), s);
}

// g in voxel order to brick order: a thread per voxel (positions of the padding are never read).
__global__ void g_to_brick_kernel(const float *__restrict__ g, int32_t V, BrickGrid b, float *__restrict__ gb) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x)
        gb[brick_pos(b, v)] = g[v];
}

vmat_status g_for_dt(const Ddc &h, const float *g, Scratch &ws, const float **out, cudaStream_t s) {
    if (!h.brick.on()) {
        *out = g;
        return VMAT_OK;
    }
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    VMAT_TRY(ws.alloc((size_t)h.brick.n_pos * 4, s));
    float *gb = static_cast<float *>(ws.ptr);
    g_to_brick_kernel<<<std::max(1, std::min(ctx->n_sm * 8, (h.V + 255) / 256)), 256, 0, s>>>(g, h.V, h.brick, gb);
    VMAT_LAUNCH_CHECK();
    *out = gb;
    return VMAT_OK;
}

vmat_status spmv_autotune(Ddc &h, cudaStream_t s) {
    // Time every configuration on the handle's own matrices and keep the fastest.
    for (CsrMat *m : {&h.Dt, &h.D}) {
        const bool isDt = m == &h.Dt;
        if (isDt ? !h.built_Dt : !h.built_D) continue;
        float *x = nullptr, *y = nullptr;
        const int32_t nin = isDt ? m->n_cols : h.J;
        const int32_t nout = isDt ? h.J : h.V;
        VMAT_CUDA(cudaMalloc(&x, (size_t)nin * 4));
        VMAT_CUDA(cudaMalloc(&y, (size_t)nout * 4));
        VMAT_CUDA(cudaMemsetAsync(x, 0, (size_t)nin * 4, s));
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        int best = m->cfg;
        float best_ms = 1e30f;
        for (int cfg = 0; cfg < N_CFG; ++cfg) {
            if (kCfgs[cfg].family == 3 && !m->col16) continue;
            vmat_status st = spmv_prepare_tiles(*m, cfg, s);
            if (st != VMAT_OK) break;
            float ms_total = 0.f;
            for (int rep = 0; rep < 6; ++rep) {
                cudaEventRecord(a, s);
                st = isDt ? spmv_run(h, *m, x, y, h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr, all_rows(), s)
                          : dose_forward_impl(h, x, y, false, s);
                cudaEventRecord(b, s);
                cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep >= 2) ms_total += ms;
                if (st != VMAT_OK) break;
            }
            if (st == VMAT_OK && ms_total < best_ms) {
                best_ms = ms_total;
                best = cfg;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaFree(x);
        cudaFree(y);
        VMAT_TRY(spmv_prepare_tiles(*m, best, s));
    }
    VMAT_CUDA(cudaStreamSynchronize(s));
    h.tuned = true;
    h.win_ncols = h.win_nseg = 0;
    return VMAT_OK;
}

// Window [n_cols / 4, n_cols / 4 + max(1, n_cols / 2)) on every MLC row: a typical pass of the
// plan reads about half of the unoccupied CPs' rows, in runs of neighbouring beamlets.
__global__ void half_windows_kernel(short2 *win, int32_t nseg, int32_t n_cols) {
    const short lo = (short)(n_cols / 4), hi = (short)(n_cols / 4 + max(1, n_cols / 2));
    for (int32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nseg; q += gridDim.x * blockDim.x)
        win[q] = make_short2(lo, hi);
}

vmat_status ddc_window_config(Ddc &h, int32_t n_cols, int32_t nseg, cudaStream_t s, int *cfg) {
    *cfg = h.Dt.cfg;
    if (!h.tuned || h.Dt.nnz == 0) return VMAT_OK;
    if (h.win_ncols == n_cols && h.win_nseg == nseg) {
        *cfg = h.win_cfg;
        return VMAT_OK;
    }
    DevBuf bw, bo, bx, by;
    VMAT_CUDA(bw.alloc((size_t)nseg * sizeof(short2)));
    VMAT_CUDA(bo.alloc((size_t)(nseg + 1) * 4));
    VMAT_CUDA(bx.alloc((size_t)h.Dt.n_cols * 4));
    VMAT_CUDA(by.alloc((size_t)h.J * 4));
    VMAT_CUDA(cudaMemsetAsync(bx.p, 0, (size_t)h.Dt.n_cols * 4, s));
    short2 *win = static_cast<short2 *>(bw.p);
    int32_t *woff = static_cast<int32_t *>(bo.p);
    half_windows_kernel<<<std::max(1, std::min(1024, (nseg + 255) / 256)), 256, 0, s>>>(win, nseg, n_cols);
    VMAT_LAUNCH_CHECK();
    VMAT_TRY(window_offsets(win, nseg, woff, nullptr, s));
    const RowMask mask{nullptr, win, n_cols, n_cols, woff, nseg}; // no CP mask: bpc unused
    cudaEvent_t a, b;
    VMAT_CUDA(cudaEventCreate(&a));
    VMAT_CUDA(cudaEventCreate(&b));
    int best = h.Dt.cfg;
    float best_ms = 1e30f;
    for (int c = 0; c < N_CFG; ++c) {
        const int fam = kCfgs[c].family;
        if (c != h.Dt.cfg && !(fam == 1 || fam == 2 || (fam == 3 && h.Dt.col16))) continue;
        CsrMat m = h.Dt;
        m.cfg = c; // a warp-row configuration reads no tile structure; the handle's own has its tiles
        float tot = 0.f;
        vmat_status st = VMAT_OK;
        for (int rep = 0; rep < 4 && st == VMAT_OK; ++rep) {
            cudaEventRecord(a, s);
            st = spmv_run(h, m, static_cast<const float *>(bx.p), static_cast<float *>(by.p),
                          h.dtype == VMAT_FP8E4M3 ? h.scale : nullptr, mask, s);
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (rep >= 1) tot += ms;
        }
        if (st == VMAT_OK && tot < best_ms) {
            best_ms = tot;
            best = c;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    VMAT_CUDA(cudaStreamSynchronize(s));
    clear_error();
    h.win_cfg = best;
    h.win_ncols = n_cols;
    h.win_nseg = nseg;
    *cfg = best;
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" {

vmat_status dose_forward(vmat_ddc hd, const float *x, float *d, void *stream) {
    clear_error();
    if (!hd || !x || !d) return set_error(VMAT_EINVAL, "dose_forward: NULL argument");
    Ddc *h = as_ddc(hd);
    if (!h->built_D) return set_error(VMAT_ESTATE, "dose_forward: CSR(D) not built");
    return dose_forward_impl(*h, x, d, false, as_stream(stream));
}

vmat_status beamlet_price(vmat_ddc hd, const float *g, float *pi, const uint8_t *cp_active, int32_t beamlets_per_cp,
                          void *stream) {
    clear_error();
    if (!hd || !g || !pi) return set_error(VMAT_EINVAL, "beamlet_price: NULL argument");
    Ddc *h = as_ddc(hd);
    if (!h->built_Dt) return set_error(VMAT_ESTATE, "beamlet_price: CSR(D^T) not built");
    if (cp_active && (beamlets_per_cp <= 0 || h->J % beamlets_per_cp != 0))
        return set_error(VMAT_EINVAL, "beamlet_price: beamlets_per_cp (%d) must divide J (%d)", beamlets_per_cp, h->J);
    cudaStream_t s = as_stream(stream);
    Scratch gws;
    const float *gd;
    VMAT_TRY(g_for_dt(*h, g, gws, &gd, s));
    return spmv_run(*h, h->Dt, gd, pi, h->dtype == VMAT_FP8E4M3 ? h->scale : nullptr,
                    RowMask{cp_active, nullptr, cp_active ? beamlets_per_cp : 1, 1}, s);
}

vmat_status beamlet_price_windowed(vmat_ddc hd, const vmat_mlc *mlc, const uint8_t *occupied, const int16_t *leaves,
                                   const float *g, float *pi, void *stream) {
    clear_error();
    if (!hd || !g || !pi || !occupied || !leaves) return set_error(VMAT_EINVAL, "beamlet_price_windowed: NULL argument");
    VMAT_TRY(validate_mlc(mlc));
    Ddc *h = as_ddc(hd);
    if (!h->built_Dt) return set_error(VMAT_ESTATE, "beamlet_price_windowed: CSR(D^T) not built");
    if ((int64_t)mlc->K * mlc->n_rows * mlc->n_cols != h->J)
        return set_error(VMAT_EINVAL, "beamlet_price_windowed: K*n_rows*n_cols != J");
    PricingGeom pg;
    VMAT_TRY(pricing_geom(mlc, &pg));
    cudaStream_t s = as_stream(stream);
    const int32_t nseg = mlc->K * mlc->n_rows;
    Scratch ws;
    VMAT_TRY(ws.alloc((size_t)nseg * sizeof(short2) + (size_t)(nseg + 1) * sizeof(int32_t), s));
    short2 *win = static_cast<short2 *>(ws.ptr);
    int32_t *woff = reinterpret_cast<int32_t *>(win + nseg);
    VMAT_TRY(price_windows(pg, occupied, leaves, win, h->Dt.rowptr, nullptr, nullptr, nullptr, s));
    VMAT_TRY(window_offsets(win, nseg, woff, nullptr, s));
    Scratch gws;
    const float *gd;
    VMAT_TRY(g_for_dt(*h, g, gws, &gd, s));
    return spmv_run(*h, h->Dt, gd, pi, h->dtype == VMAT_FP8E4M3 ? h->scale : nullptr,
                    RowMask{nullptr, win, mlc->n_rows * mlc->n_cols, mlc->n_cols, woff, nseg}, s);
}

} // extern "C"
