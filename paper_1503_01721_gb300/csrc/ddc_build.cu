// ddc_build: COO -> CSR(D^T) (beamlet rows) and CSR(D) (non-empty voxel rows).
//
// Section 2.2.2 of the paper keeps D as COO on the host and converts it to a
// CSR of D^T on the GPU at initialisation.  Here both orientations are built on
// the device: counting sort by row (histogram, scan, atomic scatter), then a
// per-row bitonic sort by column so that the layout does not depend on the
// scatter order, then optional BF16 / FP8-E4M3 quantisation.
#include <limits.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace vmat {

namespace {

constexpr int BUILD_THREADS = 256;
constexpr int SORT_SMEM_CAP_MAX = 16384; // entries (key + value = 128 KB)

int sort_smem_cap() {
    // A smaller cap (power of two >= 32) can be forced to exercise the long-row path.
    const char *e = getenv("VMAT_SORT_SMEM_CAP");
    if (e) {
        int v = atoi(e);
        if (v >= 32 && v <= SORT_SMEM_CAP_MAX && (v & (v - 1)) == 0) return v;
    }
    return SORT_SMEM_CAP_MAX;
}

// Validates the COO, counts entries per voxel and per beamlet, and sets bad[1]
// unless the entries are in column order (beamlets nondecreasing, voxels strictly
// increasing within a beamlet: the order a dose engine writes per-beamlet columns
// in).  Lanes with the same beamlet add their count with one atomic (column-ordered
// input has runs of equal beamlets).
__global__ void coo_check_hist(const int32_t *__restrict__ vox, const int32_t *__restrict__ blt,
                               const float *__restrict__ val, int64_t nnz, int32_t V, int32_t J, int32_t *cnt_vox,
                               int32_t *cnt_blt, unsigned *colmax_bits, int32_t *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    bool unordered = false;
    // every lane runs the same number of rounds (warp-wide matches inside)
    const int64_t rounds = (nnz + stride - 1) / stride;
    for (int64_t q = 0; q < rounds; ++q) {
        const int64_t e = q * stride + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        const bool in = e < nnz;
        int32_t i = in ? vox[e] : 0, j = in ? blt[e] : -1;
        const float v = in ? val[e] : 0.f;
        const bool ok = in && i >= 0 && i < V && j >= 0 && j < J && isfinite(v);
        if (in && !ok) atomicOr(bad, DEV_INDEX);
        if (in && e + 1 < nnz) {
            const int32_t j1 = blt[e + 1];
            unordered = unordered || j1 < j || (j1 == j && vox[e + 1] <= i);
        }
        if (ok) atomicAdd(&cnt_vox[i], 1);
        const int key = ok ? j : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (ok && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&cnt_blt[j], __popc(peers));
        if (ok && colmax_bits) atomicMax(&colmax_bits[j], __float_as_uint(fabsf(v)));
    }
    if (__any_sync(0xffffffffu, unordered) && lane == 0) atomicOr(bad + 1, 1);
}

__global__ void flag_nonzero(const int32_t *cnt, int32_t n, int32_t *flag) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = cnt[i] > 0 ? 1 : 0;
}

// Brick order: the voxel at brick position p (the inverse of brick_pos), or -1 for a position
// of the padding.
__device__ __forceinline__ int32_t brick_voxel(const BrickGrid &b, int64_t p) {
    const int64_t brick = p >> 5;
    const int32_t in = (int32_t)(p & 31);
    const int32_t bx = (int32_t)(brick % b.nbx), by = (int32_t)((brick / b.nbx) % b.nby);
    const int32_t bz = (int32_t)(brick / ((int64_t)b.nbx * b.nby));
    const int32_t x = 4 * bx + (in & 3), y = 4 * by + ((in >> 2) & 3), z = 2 * bz + (in >> 4);
    if (x >= b.nx || y >= b.ny || z >= b.nz) return -1;
    return (z * b.ny + y) * b.nx + x;
}

__global__ void flag_nonzero_brick(const int32_t *cnt, BrickGrid b, int32_t *flag) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < b.n_pos; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = brick_voxel(b, p);
        flag[p] = v >= 0 && cnt[v] > 0 ? 1 : 0;
    }
}

// The compact rows of CSR(D) in brick order: off = the exclusive scan of flag_nonzero_brick.
__global__ void compact_voxels_brick(const int32_t *cnt_vox, const int64_t *off, BrickGrid b, int32_t *act_vox,
                                     int32_t *vox2act, int32_t *cnt_act) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < b.n_pos; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = brick_voxel(b, p);
        if (v < 0) continue;
        const int32_t c = cnt_vox[v];
        if (c > 0) {
            const int32_t a = (int32_t)off[p];
            act_vox[a] = v;
            vox2act[v] = a;
            cnt_act[a] = c;
        } else {
            vox2act[v] = -1;
        }
    }
}

__global__ void compact_voxels(const int32_t *cnt_vox, const int64_t *off, int32_t V, int32_t *act_vox,
                               int32_t *vox2act, int32_t *cnt_act) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < V; v += gridDim.x * blockDim.x) {
        int32_t c = cnt_vox[v];
        if (c > 0) {
            int32_t a = (int32_t)off[v];
            act_vox[a] = v;
            vox2act[v] = a;
            cnt_act[a] = c;
        } else {
            vox2act[v] = -1;
        }
    }
}

__global__ void coo_scatter(const int32_t *__restrict__ vox, const int32_t *__restrict__ blt,
                            const float *__restrict__ val, int64_t nnz, const int64_t *rp_t, int32_t *cur_t,
                            int32_t *col_t, float *val_t, const int64_t *rp_d, const int32_t *vox2act, int32_t *cur_d,
                            int32_t *col_d, float *val_d) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        int32_t i = vox[e], j = blt[e];
        float v = val[e];
        if (col_t) {
            int64_t p = rp_t[j] + atomicAdd(&cur_t[j], 1);
            col_t[p] = i;
            val_t[p] = v;
        }
        if (col_d) {
            int32_t a = vox2act[i];
            int64_t q = rp_d[a] + atomicAdd(&cur_d[a], 1);
            col_d[q] = j;
            val_d[q] = v;
        }
    }
}

// ---- Stable LSD radix sort by compact voxel index (CSR(D) of a column-ordered COO).
// Sorting the column-ordered entries by voxel with a stable sort leaves each voxel's
// entries in beamlet order: no per-row sort.  7-bit digits; a block sorts a tile of
// RS_TILE entries: per-tile digit counts, one exclusive scan over (digit, tile), then
// a scatter whose in-tile ranks keep the input order (warp match per 32 entries,
// warp counters, a prefix over the warps).
constexpr int RS_BITS = 7, RS_BUCKETS = 1 << RS_BITS, RS_THREADS = 256, RS_ITEMS = 8;
constexpr int RS_WARPS = RS_THREADS / 32, RS_TILE = RS_THREADS * RS_ITEMS;

// Key of entry e: the pass-0 input is the COO (key = compact index of its voxel),
// later passes read the previous pass's keys.
__device__ __forceinline__ int32_t rs_key(const int32_t *keys, const int32_t *vox, const int32_t *vox2act, int64_t e) {
    return keys ? keys[e] : vox2act[vox[e]];
}

__global__ void __launch_bounds__(RS_THREADS)
    rs_hist(const int32_t *__restrict__ keys, const int32_t *__restrict__ vox, const int32_t *__restrict__ vox2act,
            int64_t n, int shift, int64_t n_tiles, int32_t *__restrict__ hist) {
    __shared__ int32_t c[RS_BUCKETS];
    for (int d = threadIdx.x; d < RS_BUCKETS; d += RS_THREADS) c[d] = 0;
    __syncthreads();
    const int64_t t = blockIdx.x, base = t * RS_TILE;
    for (int u = 0; u < RS_ITEMS; ++u) {
        const int64_t e = base + (int64_t)u * RS_THREADS + threadIdx.x;
        if (e < n) atomicAdd(&c[(rs_key(keys, vox, vox2act, e) >> shift) & (RS_BUCKETS - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BUCKETS; d += RS_THREADS) hist[(int64_t)d * n_tiles + t] = c[d];
}

__global__ void __launch_bounds__(RS_THREADS)
    rs_scatter(const int32_t *__restrict__ keys, const int32_t *__restrict__ vox, const int32_t *__restrict__ vox2act,
               const int32_t *__restrict__ pay, const float *__restrict__ val, int64_t n, int shift,
               const int64_t *__restrict__ off, int64_t n_tiles, int32_t *keys_out, int32_t *pay_out,
               float *val_out) {
    __shared__ int32_t wcnt[RS_WARPS][RS_BUCKETS];
    __shared__ int32_t woff[RS_WARPS][RS_BUCKETS];
    __shared__ int32_t bstart[RS_BUCKETS + 1];
    extern __shared__ __align__(16) int32_t rs_dyn[]; // the tile in sorted order: keys, payloads, values
    int32_t *sk = rs_dyn, *sp = rs_dyn + RS_TILE;
    float *sv = reinterpret_cast<float *>(rs_dyn + 2 * RS_TILE);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BUCKETS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    // warp w takes entries [base, base + 32 RS_ITEMS) of the tile, 32 consecutive per round
    const int64_t t = blockIdx.x, base = t * RS_TILE + (int64_t)wid * 32 * RS_ITEMS;
    const unsigned below = (1u << lane) - 1u;
    int32_t key[RS_ITEMS], pj[RS_ITEMS], rk[RS_ITEMS];
    float pv[RS_ITEMS];
#pragma unroll
    for (int u = 0; u < RS_ITEMS; ++u) {
        const int64_t e = base + (int64_t)u * 32 + lane;
        const bool ok = e < n;
        key[u] = ok ? rs_key(keys, vox, vox2act, e) : 0;
        pj[u] = ok ? pay[e] : 0;
        pv[u] = ok ? val[e] : 0.f;
        const int d = ok ? (key[u] >> shift) & (RS_BUCKETS - 1) : RS_BUCKETS; // past the end: no digit
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int lower = __popc(peers & below);
        const int cur = ok ? wcnt[wid][d] : 0;
        __syncwarp();
        rk[u] = cur + lower;
        if (ok && lower == 0) wcnt[wid][d] = cur + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < RS_BUCKETS; d += RS_THREADS) {
        int32_t acc = 0;
        for (int w = 0; w < RS_WARPS; ++w) {
            woff[w][d] = acc;
            acc += wcnt[w][d];
        }
        bstart[d + 1] = acc; // the bucket's size in this tile, scanned below
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bstart[0] = 0;
        for (int d = 0; d < RS_BUCKETS; ++d) bstart[d + 1] += bstart[d];
    }
    __syncthreads();
    // the tile in sorted order in shared memory, then written out with consecutive
    // threads on consecutive positions (each bucket's run is contiguous in the output)
#pragma unroll
    for (int u = 0; u < RS_ITEMS; ++u) {
        const int64_t e = base + (int64_t)u * 32 + lane;
        if (e < n) {
            const int d = (key[u] >> shift) & (RS_BUCKETS - 1);
            const int li = bstart[d] + woff[wid][d] + rk[u];
            sk[li] = key[u];
            sp[li] = pj[u];
            sv[li] = pv[u];
        }
    }
    __syncthreads();
    const int cnt = bstart[RS_BUCKETS];
    for (int li = threadIdx.x; li < cnt; li += RS_THREADS) {
        const int32_t kk = sk[li];
        const int d = (kk >> shift) & (RS_BUCKETS - 1);
        const int64_t pos = off[(int64_t)d * n_tiles + t] + (li - bstart[d]);
        if (keys_out) keys_out[pos] = kk;
        pay_out[pos] = sp[li];
        val_out[pos] = sv[li];
    }
}

// Bitonic network over P (a power of two) keys with their values; thread t of a stage
// takes pair t: the lower index i = 2 t - (t mod stride) and i + stride.
__device__ __forceinline__ void bitonic_smem(int32_t *k, float *v, int P) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1)), j = i + stride;
                const bool up = (i & size) == 0;
                const int32_t a = k[i], b = k[j];
                if ((a > b) == up) {
                    k[i] = b;
                    k[j] = a;
                    const float w = v[i];
                    v[i] = v[j];
                    v[j] = w;
                }
            }
            __syncthreads();
        }
    }
}

// Column (voxel) of every entry to its brick position.
__global__ void cols_to_brick(int32_t *col, int64_t n, BrickGrid b) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        col[e] = brick_pos(b, col[e]);
}

__global__ void map_to_brick(const int32_t *vox, int32_t n, BrickGrid b, int32_t *pos) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        pos[i] = brick_pos(b, vox[i]);
}

// Rows of up to RR_CAP entries: stable LSD radix sort by column in shared memory, a block
// per row, 8-bit digits of (col - the row's least col), as many passes as the row's column
// range needs.  Warp w holds entries [w RR_CAP / RR_WARPS, (w + 1) RR_CAP / RR_WARPS) of the
// row, 32 consecutive per round; a warp's running digit counts (match_any ranks) and the
// counts of the warps before it place each entry after every earlier entry of its digit,
// so each pass is stable and the result is the row sorted by column (ties, which the
// build rejects as duplicates, keep their order).  Sets DEV_DUPLICATE on equal neighbours.
constexpr int RR_THREADS = 256, RR_WARPS = RR_THREADS / 32, RR_CAP = 2048, RR_ITEMS = RR_CAP / RR_THREADS;
__global__ void __launch_bounds__(RR_THREADS)
    row_radix_sort(const int64_t *rowptr, int32_t *col, float *val, int32_t n_rows, int32_t *bad) {
    __shared__ int32_t wcnt[RR_WARPS][256];
    __shared__ int32_t bstart[256];
    __shared__ int32_t wsum[RR_WARPS];
    __shared__ int32_t red_min[RR_WARPS], red_max[RR_WARPS];
    extern __shared__ __align__(16) unsigned char rr_dyn[];
    int32_t *const ka = reinterpret_cast<int32_t *>(rr_dyn), *const kz = ka + RR_CAP;
    float *const va = reinterpret_cast<float *>(rr_dyn) + 2 * RR_CAP, *const vz = va + RR_CAP;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    for (int32_t r = blockIdx.x; r < n_rows; r += gridDim.x) {
        const int64_t s = rowptr[r];
        const int n = (int)(rowptr[r + 1] - s);
        if (n < 2 || n > RR_CAP) continue;
        int32_t kmin = INT_MAX, kmax = INT_MIN;
        for (int i = threadIdx.x; i < n; i += RR_THREADS) {
            const int32_t k = col[s + i];
            ka[i] = k;
            va[i] = val[s + i];
            kmin = min(kmin, k);
            kmax = max(kmax, k);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, d));
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, d));
        }
        if (lane == 0) {
            red_min[wid] = kmin;
            red_max[wid] = kmax;
        }
        __syncthreads();
        kmin = red_min[0];
        kmax = red_max[0];
        for (int w = 1; w < RR_WARPS; ++w) {
            kmin = min(kmin, red_min[w]);
            kmax = max(kmax, red_max[w]);
        }
        const uint32_t range = (uint32_t)(kmax - kmin);
        int32_t *kin = ka, *kout = kz;
        float *vin = va, *vout = vz;
        for (int shift = 0; shift < 32 && (shift == 0 || (range >> shift) != 0); shift += 8) {
            for (int i = threadIdx.x; i < RR_WARPS * 256; i += RR_THREADS) (&wcnt[0][0])[i] = 0;
            __syncthreads();
            int32_t key[RR_ITEMS], rk[RR_ITEMS];
            float v[RR_ITEMS];
#pragma unroll
            for (int u = 0; u < RR_ITEMS; ++u) {
                const int e = wid * (RR_CAP / RR_WARPS) + u * 32 + lane;
                const bool ok = e < n;
                key[u] = ok ? kin[e] : 0;
                v[u] = ok ? vin[e] : 0.f;
                const int d = ok ? (int)(((uint32_t)(key[u] - kmin) >> shift) & 255u) : 256;
                const unsigned peers = __match_any_sync(0xffffffffu, d);
                const int lower = __popc(peers & below);
                const int c0 = ok ? wcnt[wid][d] : 0;
                __syncwarp();
                rk[u] = c0 + lower;
                if (ok && lower == 0) wcnt[wid][d] = c0 + __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            // digit t: offsets of the warps within it, its total, then an exclusive scan of the totals
            const int t = threadIdx.x; // RR_THREADS == 256 digits
            int32_t acc = 0;
            for (int w = 0; w < RR_WARPS; ++w) {
                const int32_t c = wcnt[w][t];
                wcnt[w][t] = acc;
                acc += c;
            }
            int32_t inc = acc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t o = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += o;
            }
            if (lane == 31) wsum[wid] = inc;
            __syncthreads();
            int32_t before = 0;
            for (int w = 0; w < wid; ++w) before += wsum[w];
            bstart[t] = before + inc - acc;
            __syncthreads();
#pragma unroll
            for (int u = 0; u < RR_ITEMS; ++u) {
                const int e = wid * (RR_CAP / RR_WARPS) + u * 32 + lane;
                if (e < n) {
                    const int d = (int)(((uint32_t)(key[u] - kmin) >> shift) & 255u);
                    const int pos = bstart[d] + wcnt[wid][d] + rk[u];
                    kout[pos] = key[u];
                    vout[pos] = v[u];
                }
            }
            __syncthreads();
            int32_t *kt = kin;
            kin = kout;
            kout = kt;
            float *vt = vin;
            vin = vout;
            vout = vt;
        }
        for (int i = threadIdx.x; i < n; i += RR_THREADS) {
            const int32_t k = kin[i];
            col[s + i] = k;
            val[s + i] = vin[i];
            if (i > 0 && k == kin[i - 1]) atomicOr(bad, DEV_DUPLICATE);
        }
        __syncthreads();
    }
}

// Sorts the rows with lo < n <= cap entries (n >= 2), a block per row in shared memory.
__global__ void row_sort_smem(const int64_t *rowptr, int32_t *col, float *val, int32_t n_rows, int lo, int cap,
                              int32_t *bad) {
    extern __shared__ __align__(16) unsigned char sm[];
    int32_t *k = reinterpret_cast<int32_t *>(sm);
    float *v = reinterpret_cast<float *>(k + cap);
    for (int32_t r = blockIdx.x; r < n_rows; r += gridDim.x) {
        int64_t s = rowptr[r];
        int n = (int)(rowptr[r + 1] - s);
        if (n < 2 || n <= lo || n > cap) continue;
        int P = 1;
        while (P < n) P <<= 1;
        for (int i = threadIdx.x; i < P; i += blockDim.x) {
            k[i] = i < n ? col[s + i] : INT_MAX;
            v[i] = i < n ? val[s + i] : 0.f;
        }
        __syncthreads();
        bitonic_smem(k, v, P);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            col[s + i] = k[i];
            val[s + i] = v[i];
            if (i > 0 && k[i] == k[i - 1]) atomicOr(bad, DEV_DUPLICATE);
        }
        __syncthreads();
    }
}

__global__ void list_long_rows(const int64_t *rowptr, int32_t n_rows, int cap, int32_t *list, int32_t *n_list) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += gridDim.x * blockDim.x)
        if (rowptr[r + 1] - rowptr[r] > cap) list[atomicAdd(n_list, 1)] = r;
}

// Rows longer than the shared-memory cap: bitonic network over a global buffer,
// one block per row (the block's __syncthreads orders its global accesses).
__global__ void row_sort_global(const int64_t *rowptr, int32_t *col, float *val, const int32_t *list,
                                int32_t n_long, int32_t *kbuf, float *vbuf, int64_t pmax, int32_t *bad) {
    int32_t *k = kbuf + (int64_t)blockIdx.x * pmax;
    float *v = vbuf + (int64_t)blockIdx.x * pmax;
    for (int32_t t = blockIdx.x; t < n_long; t += gridDim.x) {
        int32_t r = list[t];
        int64_t s = rowptr[r];
        int64_t n = rowptr[r + 1] - s;
        int64_t P = 1;
        while (P < n) P <<= 1;
        for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
            k[i] = i < n ? col[s + i] : INT_MAX;
            v[i] = i < n ? val[s + i] : 0.f;
        }
        __syncthreads();
        for (int64_t size = 2; size <= P; size <<= 1) {
            for (int64_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (int64_t i = threadIdx.x; i < P; i += blockDim.x) {
                    int64_t j = i ^ stride;
                    if (j > i) {
                        bool up = (i & size) == 0;
                        int32_t a = k[i], b = k[j];
                        if ((a > b) == up) {
                            k[i] = b;
                            k[j] = a;
                            float tv = v[i];
                            v[i] = v[j];
                            v[j] = tv;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            col[s + i] = k[i];
            val[s + i] = v[i];
            if (i > 0 && k[i] == k[i - 1]) atomicOr(bad, DEV_DUPLICATE);
        }
        __syncthreads();
    }
}

__global__ void max_count(const int32_t *cnt, int32_t n, int32_t *out) {
    int32_t m = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, cnt[i]);
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// s_j = least power of two with 448 * s_j >= max_i |D_ij| (1 for an empty beamlet).
__global__ void fp8_scales(const unsigned *colmax_bits, int32_t J, float *scale) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
        float m = __uint_as_float(colmax_bits[j]);
        float s = 1.f;
        if (m > 0.f) {
            int e;
            frexpf(m / 448.f, &e);
            s = ldexpf(1.f, e);
            while (448.f * s < m) s *= 2.f;
            while (448.f * (s * 0.5f) >= m) s *= 0.5f;
        }
        scale[j] = s;
    }
}

__global__ void to_bf16(const float *in, __nv_bfloat16 *out, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = __float2bfloat16_rn(in[e]);
}

// FP8 with the scale of column col[e] (CSR(D): columns are beamlets).
__global__ void to_fp8_by_col(const float *in, const int32_t *col, const float *scale, uint8_t *out, int64_t n) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = (uint8_t)__nv_cvt_float_to_fp8(in[e] / scale[col[e]], __NV_SATFINITE, __NV_E4M3);
}

// FP8 with the scale of the row (CSR(D^T): rows are beamlets); one warp per row.
__global__ void to_fp8_by_row(const float *in, const int64_t *rowptr, int32_t n_rows, const float *scale,
                              uint8_t *out) {
    const int lane = threadIdx.x & 31;
    for (int32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += (gridDim.x * blockDim.x) >> 5) {
        float s = scale[r];
        for (int64_t e = rowptr[r] + lane; e < rowptr[r + 1]; e += 32)
            out[e] = (uint8_t)__nv_cvt_float_to_fp8(in[e] / s, __NV_SATFINITE, __NV_E4M3);
    }
}

int grid_for(int64_t n, int n_sm) {
    int64_t g = (n + BUILD_THREADS - 1) / BUILD_THREADS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)n_sm * 16));
}

int64_t round_pad(int64_t nnz) { return ((std::max<int64_t>(nnz, 1) + NNZ_PAD - 1) / NNZ_PAD) * NNZ_PAD; }

// Sort each row of a CSR by column, check duplicates.
// CSR(D) of a column-ordered COO: entries sorted by compact voxel index (stable), the
// beamlet into col, the value into val.  Passes of RS_BITS bits over the key's width.
// reuse (optional): three nnz-entry device arrays the call may overwrite after the first
// pass has read the input (the COO itself, when it is not kept), used as ping-pong space.
vmat_status radix_by_voxel(const int32_t *vox, const int32_t *blt, const float *cval, const int32_t *vox2act,
                           int64_t nnz, int32_t n_keys, int32_t *col, float *val, cudaStream_t s,
                           int32_t *reuse_k = nullptr, int32_t *reuse_p = nullptr, float *reuse_v = nullptr) {
    if (nnz == 0) return VMAT_OK;
    int bits = 1;
    while (bits < 31 && (1 << bits) < n_keys) ++bits;
    const int passes = (bits + RS_BITS - 1) / RS_BITS;
    const int64_t n_tiles = (nnz + RS_TILE - 1) / RS_TILE;
    if (n_tiles > INT32_MAX) return set_error(VMAT_EUNSUPPORTED, "ddc_build: too many nonzeros for the radix pass");
    DevBuf hist, off, ka, kb, pa, va;
    VMAT_CUDA(hist.alloc((size_t)RS_BUCKETS * n_tiles * 4));
    VMAT_CUDA(off.alloc(((size_t)RS_BUCKETS * n_tiles + 1) * 8));
    // ping-pong through the outputs: pass q writes to (col, val) when passes - 1 - q is even,
    // else to the temporaries (pa, va), so the last pass lands in (col, val)
    // The input is read only by pass 0, so the A set may be the input's own arrays when pass 0
    // writes to the outputs instead (passes - 1 even: an odd number of passes, at least 3).
    const bool reuse = reuse_k && reuse_p && reuse_v && passes >= 3 && (passes & 1);
    if (passes > 1 && !reuse) {
        VMAT_CUDA(ka.alloc((size_t)nnz * 4));
        VMAT_CUDA(pa.alloc((size_t)nnz * 4));
        VMAT_CUDA(va.alloc((size_t)nnz * 4));
    }
    if (passes > 2) VMAT_CUDA(kb.alloc((size_t)nnz * 4));
    int32_t *A_k = reuse ? reuse_k : (int32_t *)ka.p, *A_p = reuse ? reuse_p : (int32_t *)pa.p;
    float *A_v = reuse ? reuse_v : (float *)va.p;
    // the sorted tile (48 KB) comes on top of the static counters: above the default per-block limit
    VMAT_CUDA(cudaFuncSetAttribute(rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * RS_TILE * 4));
    const int32_t *kin = nullptr, *pin = blt;
    const float *vin = cval;
    for (int q = 0; q < passes; ++q) {
        const int shift = q * RS_BITS;
        const bool last = q == passes - 1, to_out = ((passes - 1 - q) & 1) == 0;
        int32_t *kout = last ? nullptr : (to_out ? (int32_t *)kb.p : A_k);
        int32_t *pout = to_out ? col : A_p;
        float *vout = to_out ? val : A_v;
        rs_hist<<<(unsigned)n_tiles, RS_THREADS, 0, s>>>(kin, vox, vox2act, nnz, shift, n_tiles, (int32_t *)hist.p);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(scan_counts((const int32_t *)hist.p, (int64_t *)off.p, (int64_t)RS_BUCKETS * n_tiles, s));
        rs_scatter<<<(unsigned)n_tiles, RS_THREADS, 3 * RS_TILE * 4, s>>>(kin, vox, vox2act, pin, vin, nnz, shift,
                                                                          (const int64_t *)off.p, n_tiles, kout,
                                                                          pout, vout);
        VMAT_LAUNCH_CHECK();
        kin = kout;
        pin = pout;
        vin = vout;
    }
    VMAT_CUDA(cudaStreamSynchronize(s)); // the ping-pong buffers are freed on return
    return VMAT_OK;
}

vmat_status longest_row(const int32_t *cnt, int32_t n_rows, int n_sm, cudaStream_t s, int32_t *max_row) {
    *max_row = 0;
    if (n_rows == 0) return VMAT_OK;
    DevBuf bmax;
    VMAT_CUDA(bmax.alloc(sizeof(int32_t)));
    VMAT_CUDA(cudaMemsetAsync(bmax.p, 0, sizeof(int32_t), s));
    max_count<<<grid_for(n_rows, n_sm), BUILD_THREADS, 0, s>>>(cnt, n_rows, (int32_t *)bmax.p);
    VMAT_LAUNCH_CHECK();
    VMAT_CUDA(cudaMemcpyAsync(max_row, bmax.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    return VMAT_OK;
}

vmat_status sort_rows(const int64_t *rowptr, const int32_t *cnt, int32_t n_rows, int32_t *col, float *val,
                      int32_t *bad, int n_sm, cudaStream_t s, int32_t *max_row) {
    *max_row = 0;
    if (n_rows == 0) return VMAT_OK;
    int32_t *dmax = nullptr;
    DevBuf bmax;
    VMAT_CUDA(bmax.alloc(2 * sizeof(int32_t)));
    dmax = (int32_t *)bmax.p;
    VMAT_CUDA(cudaMemsetAsync(dmax, 0, 2 * sizeof(int32_t), s));
    max_count<<<grid_for(n_rows, n_sm), BUILD_THREADS, 0, s>>>(cnt, n_rows, dmax);
    VMAT_LAUNCH_CHECK();
    int32_t maxlen = 0;
    VMAT_CUDA(cudaMemcpyAsync(&maxlen, dmax, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    *max_row = maxlen;
    if (maxlen < 2) return VMAT_OK;
    int cap_max = sort_smem_cap();
    int cap = 32;
    while (cap < maxlen && cap < cap_max) cap <<= 1;
    // rows up to RR_CAP entries by the radix sort (unless a smaller cap is forced), the longer
    // ones (up to cap) by the bitonic network in a second launch, so that a few long rows do not
    // set every block's shared memory
    int grid = (int)std::min<int64_t>(n_rows, (int64_t)n_sm * 8);
    int cap1 = 0;
    if (cap_max >= RR_CAP) {
        cap1 = RR_CAP;
        VMAT_CUDA(cudaFuncSetAttribute(row_radix_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, RR_CAP * 16));
        row_radix_sort<<<grid, RR_THREADS, (size_t)RR_CAP * 16, s>>>(rowptr, col, val, n_rows, bad);
        VMAT_LAUNCH_CHECK();
    }
    if (cap > cap1) {
        VMAT_CUDA(cudaFuncSetAttribute(row_sort_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, cap * 8));
        row_sort_smem<<<grid, BUILD_THREADS, (size_t)cap * 8, s>>>(rowptr, col, val, n_rows, cap1, cap, bad);
        VMAT_LAUNCH_CHECK();
    }
    if (maxlen > cap) {
        DevBuf blist;
        VMAT_CUDA(blist.alloc((size_t)n_rows * 4));
        int32_t *list = (int32_t *)blist.p;
        list_long_rows<<<grid_for(n_rows, n_sm), BUILD_THREADS, 0, s>>>(rowptr, n_rows, cap, list, dmax + 1);
        VMAT_LAUNCH_CHECK();
        int32_t n_long = 0;
        VMAT_CUDA(cudaMemcpyAsync(&n_long, dmax + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        VMAT_CUDA(cudaStreamSynchronize(s));
        int64_t pmax = 1;
        while (pmax < maxlen) pmax <<= 1;
        int gl = std::min<int32_t>(n_long, 64);
        DevBuf kb, vb;
        VMAT_CUDA(kb.alloc((size_t)gl * pmax * 4));
        VMAT_CUDA(vb.alloc((size_t)gl * pmax * 4));
        row_sort_global<<<gl, 1024, 0, s>>>(rowptr, col, val, list, n_long, (int32_t *)kb.p, (float *)vb.p, pmax,
                                            bad);
        VMAT_LAUNCH_CHECK();
        VMAT_CUDA(cudaStreamSynchronize(s));
    }
    return VMAT_OK;
}

// Chunks of ZCHUNK entries per row (the last one ragged).
__global__ void chunk_counts(const int64_t *__restrict__ rowptr, int32_t n_rows, int32_t *cnt) {
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rows; r += gridDim.x * blockDim.x)
        cnt[r] = (int32_t)((rowptr[r + 1] - rowptr[r] + ZCHUNK - 1) / ZCHUNK);
}

// A warp per row: each chunk's base is its first column (rows are sorted), each
// entry stores its offset from that base; bad is set when an offset needs more
// than 16 bits.
__global__ void fill_index16(const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                             const int64_t *__restrict__ cptr, int32_t n_rows, int32_t *cbase, uint16_t *col16,
                             int32_t *bad) {
    const int lane = threadIdx.x & 31;
    for (int32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += (gridDim.x * blockDim.x) >> 5) {
        const int64_t s = rowptr[r], e = rowptr[r + 1], c0 = cptr[r];
        bool ok = true;
        for (int64_t i = s + lane; i < e; i += 32) {
            const int64_t t = (i - s) / ZCHUNK;
            const int32_t base = col[s + t * ZCHUNK];
            const int32_t off = col[i] - base;
            ok = ok && off >= 0 && off <= 65535;
            col16[i] = (uint16_t)off;
            if (i - s == t * ZCHUNK) cbase[c0 + t] = base;
        }
        if (__any_sync(0xffffffffu, !ok) && lane == 0) *bad = 1;
    }
}

} // namespace

vmat_status csr_build_index16(CsrMat &m, int n_sm, cudaStream_t s) {
    if (m.n_rows <= 0 || m.nnz <= 0) return VMAT_OK;
    DevBuf b_cnt, b_cptr, b_base, b_c16, b_bad;
    VMAT_CUDA(b_cnt.alloc((size_t)m.n_rows * 4));
    VMAT_CUDA(b_cptr.alloc((size_t)(m.n_rows + 1) * 8));
    VMAT_CUDA(b_bad.alloc(8)); // [0]: invalid or duplicate entries, [1]: not in column order
    chunk_counts<<<grid_for(m.n_rows, n_sm), BUILD_THREADS, 0, s>>>(m.rowptr, m.n_rows, (int32_t *)b_cnt.p);
    VMAT_LAUNCH_CHECK();
    VMAT_TRY(scan_counts((int32_t *)b_cnt.p, (int64_t *)b_cptr.p, m.n_rows, s));
    int64_t n_chunks = 0;
    VMAT_CUDA(cudaMemcpyAsync(&n_chunks, (int64_t *)b_cptr.p + m.n_rows, 8, cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaMemsetAsync(b_bad.p, 0, 4, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    VMAT_CUDA(b_base.alloc((size_t)std::max<int64_t>(n_chunks, 1) * 4));
    VMAT_CUDA(b_c16.alloc((size_t)m.nnz * 2));
    fill_index16<<<grid_for((int64_t)m.n_rows * 32, n_sm), BUILD_THREADS, 0, s>>>(
        m.rowptr, m.col, (const int64_t *)b_cptr.p, m.n_rows, (int32_t *)b_base.p, (uint16_t *)b_c16.p,
        (int32_t *)b_bad.p);
    VMAT_LAUNCH_CHECK();
    int32_t bad = 0;
    VMAT_CUDA(cudaMemcpyAsync(&bad, b_bad.p, 4, cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    if (bad) return VMAT_OK; // some chunk spans 65536 columns or more: this matrix keeps 32-bit indices only
    m.cptr = (int64_t *)b_cptr.release();
    m.cbase = (int32_t *)b_base.release();
    m.col16 = (uint16_t *)b_c16.release();
    m.n_chunks = n_chunks;
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" vmat_status ddc_build(vmat_ddc hd, const vmat_build_opts *opts_in, void *stream) {
    clear_error();
    if (!hd) return set_error(VMAT_EINVAL, "ddc_build: handle is NULL");
    Ddc *h = as_ddc(hd);
    vmat_build_opts opts = {VMAT_F32, 1, 1, -1, 0, 0, 0, -1, 0, {0, 0, 0}};
    if (opts_in) opts = *opts_in;
    BrickGrid brick;
    if (opts.vox_grid[0] || opts.vox_grid[1] || opts.vox_grid[2]) {
        const int32_t nx = opts.vox_grid[0], ny = opts.vox_grid[1], nz = opts.vox_grid[2];
        if (nx <= 0 || ny <= 0 || nz <= 0 || (int64_t)nx * ny * nz != (int64_t)h->V)
            return set_error(VMAT_EINVAL, "ddc_build: vox_grid {%d, %d, %d} does not give V = %d voxels", nx, ny, nz,
                             h->V);
        brick.nx = nx;
        brick.ny = ny;
        brick.nz = nz;
        brick.nbx = (nx + 3) / 4;
        brick.nby = (ny + 3) / 4;
        brick.n_pos = (int64_t)brick.nbx * brick.nby * ((nz + 1) / 2) * 32;
        if (brick.n_pos > INT32_MAX) return set_error(VMAT_EINVAL, "ddc_build: vox_grid padded to bricks exceeds 2^31 voxels");
    }
    if (opts.dtype != VMAT_F32 && opts.dtype != VMAT_BF16 && opts.dtype != VMAT_FP8E4M3)
        return set_error(VMAT_EINVAL, "ddc_build: unknown dtype %d", (int)opts.dtype);
    if (!opts.build_D && !opts.build_Dt) return set_error(VMAT_EINVAL, "ddc_build: nothing to build");
    if (opts.tile_cfg >= spmv_n_configs() || opts.tile_cfg_Dt >= spmv_n_configs())
        return set_error(VMAT_EINVAL, "ddc_build: tile_cfg / tile_cfg_Dt out of range");
    if (!h->coo_vox) return set_error(VMAT_ESTATE, "ddc_build: the COO copy was released by an earlier build");
    DeviceCtx *ctx;
    VMAT_TRY(device_ctx(&ctx));
    cudaStream_t s = as_stream(stream);
    const int n_sm = ctx->n_sm;
    const int32_t V = h->V, J = h->J;
    const int64_t nnz = h->nnz;

    // drop an earlier build
    {
        Ddc keep = *h;
        h->coo_vox = nullptr;
        h->coo_blt = nullptr;
        h->coo_val = nullptr;
        h->free_all();
        h->coo_vox = keep.coo_vox;
        h->coo_blt = keep.coo_blt;
        h->coo_val = keep.coo_val;
        h->built_D = h->built_Dt = false;
    }

    cudaEvent_t e0, e1;
    VMAT_CUDA(cudaEventCreate(&e0));
    VMAT_CUDA(cudaEventCreate(&e1));
    VMAT_CUDA(cudaEventRecord(e0, s));

    DevBuf b_cnt_vox, b_cnt_blt, b_colmax, b_bad, b_flag, b_off, b_cnt_act, b_cur_t, b_cur_d;
    DevBuf b_rp_t, b_col_t, b_val_t, b_rp_d, b_col_d, b_val_d, b_act, b_v2a, b_scale;
    VMAT_CUDA(b_cnt_vox.alloc((size_t)V * 4));
    VMAT_CUDA(b_cnt_blt.alloc((size_t)J * 4));
    VMAT_CUDA(b_bad.alloc(8)); // [0]: invalid or duplicate entries, [1]: not in column order
    const bool fp8 = opts.dtype == VMAT_FP8E4M3;
    if (fp8) VMAT_CUDA(b_colmax.alloc((size_t)J * 4));
    int32_t *cnt_vox = (int32_t *)b_cnt_vox.p, *cnt_blt = (int32_t *)b_cnt_blt.p, *bad = (int32_t *)b_bad.p;
    VMAT_CUDA(cudaMemsetAsync(cnt_vox, 0, (size_t)V * 4, s));
    VMAT_CUDA(cudaMemsetAsync(cnt_blt, 0, (size_t)J * 4, s));
    VMAT_CUDA(cudaMemsetAsync(bad, 0, 8, s));
    if (fp8) VMAT_CUDA(cudaMemsetAsync(b_colmax.p, 0, (size_t)J * 4, s));
    if (nnz > 0) {
        coo_check_hist<<<grid_for(nnz, n_sm), BUILD_THREADS, 0, s>>>(h->coo_vox, h->coo_blt, h->coo_val, nnz, V, J,
                                                                      cnt_vox, cnt_blt, (unsigned *)b_colmax.p, bad);
        VMAT_LAUNCH_CHECK();
    }
    int32_t hbad[2] = {0, 0};
    VMAT_CUDA(cudaMemcpyAsync(hbad, bad, 8, cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    if (hbad[0]) return set_error(VMAT_EINVAL, "ddc_build: COO entry with voxel/beamlet index out of range or a non-finite value");
    // column-ordered input: CSR(D^T) is the COO's voxel and value arrays as they are
    const bool csc = nnz > 0 && hbad[1] == 0;

    const int64_t pad = round_pad(nnz);
    const int vb = value_bytes(opts.dtype);

    // ---- CSR(D^T): rows = beamlets
    if (opts.build_Dt) {
        VMAT_CUDA(b_rp_t.alloc((size_t)(J + 1) * 8));
        VMAT_TRY(scan_counts(cnt_blt, (int64_t *)b_rp_t.p, J, s));
        VMAT_CUDA(b_col_t.alloc((size_t)pad * 4));
        VMAT_CUDA(b_val_t.alloc((size_t)pad * 4));
        // every entry is written below; only the padding needs zeros
        VMAT_CUDA(cudaMemsetAsync((int32_t *)b_col_t.p + nnz, 0, (size_t)(pad - nnz) * 4, s));
        VMAT_CUDA(cudaMemsetAsync((float *)b_val_t.p + nnz, 0, (size_t)(pad - nnz) * 4, s));
        if (csc) {
            VMAT_CUDA(cudaMemcpyAsync(b_col_t.p, h->coo_vox, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
            VMAT_CUDA(cudaMemcpyAsync(b_val_t.p, h->coo_val, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s));
        } else {
            VMAT_CUDA(b_cur_t.alloc((size_t)J * 4));
            VMAT_CUDA(cudaMemsetAsync(b_cur_t.p, 0, (size_t)J * 4, s));
        }
    }
    // ---- CSR(D): rows = voxels with at least one entry
    int32_t n_active = 0;
    if (opts.build_D) {
        // compact rows in voxel order, or in brick order with vox_grid (then a 32-voxel tile of
        // the master problem is a 4 x 4 x 2 brick, and g is written almost in order)
        const int32_t npos = brick.on() ? (int32_t)brick.n_pos : V;
        VMAT_CUDA(b_flag.alloc((size_t)npos * 4));
        VMAT_CUDA(b_off.alloc((size_t)(npos + 1) * 8));
        if (brick.on())
            flag_nonzero_brick<<<grid_for(npos, n_sm), BUILD_THREADS, 0, s>>>(cnt_vox, brick, (int32_t *)b_flag.p);
        else
            flag_nonzero<<<grid_for(V, n_sm), BUILD_THREADS, 0, s>>>(cnt_vox, V, (int32_t *)b_flag.p);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(scan_counts((int32_t *)b_flag.p, (int64_t *)b_off.p, npos, s));
        int64_t na = 0;
        VMAT_CUDA(cudaMemcpyAsync(&na, (int64_t *)b_off.p + npos, 8, cudaMemcpyDeviceToHost, s));
        VMAT_CUDA(cudaStreamSynchronize(s));
        n_active = (int32_t)na;
        VMAT_CUDA(b_act.alloc((size_t)std::max(n_active, 1) * 4));
        VMAT_CUDA(b_v2a.alloc((size_t)V * 4));
        VMAT_CUDA(b_cnt_act.alloc((size_t)std::max(n_active, 1) * 4));
        if (brick.on())
            compact_voxels_brick<<<grid_for(npos, n_sm), BUILD_THREADS, 0, s>>>(
                cnt_vox, (int64_t *)b_off.p, brick, (int32_t *)b_act.p, (int32_t *)b_v2a.p, (int32_t *)b_cnt_act.p);
        else
            compact_voxels<<<grid_for(V, n_sm), BUILD_THREADS, 0, s>>>(cnt_vox, (int64_t *)b_off.p, V,
                                                                      (int32_t *)b_act.p, (int32_t *)b_v2a.p,
                                                                      (int32_t *)b_cnt_act.p);
        VMAT_LAUNCH_CHECK();
        VMAT_CUDA(b_rp_d.alloc((size_t)(n_active + 1) * 8));
        VMAT_TRY(scan_counts((int32_t *)b_cnt_act.p, (int64_t *)b_rp_d.p, n_active, s));
        VMAT_CUDA(b_col_d.alloc((size_t)pad * 4));
        VMAT_CUDA(b_val_d.alloc((size_t)pad * 4));
        VMAT_CUDA(cudaMemsetAsync((int32_t *)b_col_d.p + nnz, 0, (size_t)(pad - nnz) * 4, s));
        VMAT_CUDA(cudaMemsetAsync((float *)b_val_d.p + nnz, 0, (size_t)(pad - nnz) * 4, s));
        VMAT_CUDA(b_cur_d.alloc((size_t)std::max(n_active, 1) * 4));
        VMAT_CUDA(cudaMemsetAsync(b_cur_d.p, 0, (size_t)std::max(n_active, 1) * 4, s));
    }
    // column-ordered input: CSR(D^T) was copied, CSR(D) is a stable sort by voxel (rows come out in
    // beamlet order); otherwise an atomic scatter into rows, then a sort of each row by column
    const bool scatter_t = opts.build_Dt && !csc, scatter_d = opts.build_D && !csc;
    if (nnz > 0 && (scatter_t || scatter_d)) {
        coo_scatter<<<grid_for(nnz, n_sm), BUILD_THREADS, 0, s>>>(
            h->coo_vox, h->coo_blt, h->coo_val, nnz, (int64_t *)b_rp_t.p, (int32_t *)b_cur_t.p,
            scatter_t ? (int32_t *)b_col_t.p : nullptr, (float *)b_val_t.p, (int64_t *)b_rp_d.p, (int32_t *)b_v2a.p,
            (int32_t *)b_cur_d.p, scatter_d ? (int32_t *)b_col_d.p : nullptr, (float *)b_val_d.p);
        VMAT_LAUNCH_CHECK();
    }
    int32_t max_row_t = 0, max_row_d = 0;
    if (scatter_t)
        VMAT_TRY(sort_rows((int64_t *)b_rp_t.p, cnt_blt, J, (int32_t *)b_col_t.p, (float *)b_val_t.p, bad, n_sm, s,
                           &max_row_t));
    else if (opts.build_Dt && !brick.on())
        VMAT_TRY(longest_row(cnt_blt, J, n_sm, s, &max_row_t)); // already in order: nothing to sort
    if (opts.build_Dt && brick.on() && nnz > 0) { // columns to brick positions, each row sorted again by them
        cols_to_brick<<<grid_for(nnz, n_sm), BUILD_THREADS, 0, s>>>((int32_t *)b_col_t.p, nnz, brick);
        VMAT_LAUNCH_CHECK();
        VMAT_TRY(sort_rows((int64_t *)b_rp_t.p, cnt_blt, J, (int32_t *)b_col_t.p, (float *)b_val_t.p, bad, n_sm, s,
                           &max_row_t));
    }
    if (scatter_d) {
        VMAT_TRY(sort_rows((int64_t *)b_rp_d.p, (int32_t *)b_cnt_act.p, n_active, (int32_t *)b_col_d.p,
                           (float *)b_val_d.p, bad, n_sm, s, &max_row_d));
    } else if (opts.build_D) {
        VMAT_TRY(radix_by_voxel(h->coo_vox, h->coo_blt, h->coo_val, (const int32_t *)b_v2a.p, nnz, n_active,
                                (int32_t *)b_col_d.p, (float *)b_val_d.p, s,
                                opts.keep_coo ? nullptr : h->coo_vox, opts.keep_coo ? nullptr : h->coo_blt,
                                opts.keep_coo ? nullptr : h->coo_val));
        VMAT_TRY(longest_row((int32_t *)b_cnt_act.p, n_active, n_sm, s, &max_row_d));
    }
    VMAT_CUDA(cudaMemcpyAsync(hbad, bad, 4, cudaMemcpyDeviceToHost, s));
    VMAT_CUDA(cudaStreamSynchronize(s));
    if (hbad[0] & DEV_DUPLICATE) return set_error(VMAT_EINVAL, "ddc_build: duplicate (voxel, beamlet) entry in the COO input");

    // ---- quantisation
    if (fp8) {
        VMAT_CUDA(b_scale.alloc((size_t)J * 4));
        fp8_scales<<<grid_for(J, n_sm), BUILD_THREADS, 0, s>>>((unsigned *)b_colmax.p, J, (float *)b_scale.p);
        VMAT_LAUNCH_CHECK();
    }
    auto quantise = [&](DevBuf &bval, const int32_t *col, const int64_t *rowptr, int32_t n_rows, bool by_row,
                        void **out) -> vmat_status {
        if (opts.dtype == VMAT_F32) {
            *out = bval.release();
            return VMAT_OK;
        }
        DevBuf q;
        VMAT_CUDA(q.alloc((size_t)pad * vb));
        VMAT_CUDA(cudaMemsetAsync(q.p, 0, (size_t)pad * vb, s));
        if (opts.dtype == VMAT_BF16) {
            to_bf16<<<grid_for(nnz, n_sm), BUILD_THREADS, 0, s>>>((float *)bval.p, (__nv_bfloat16 *)q.p, nnz);
        } else if (by_row) {
            to_fp8_by_row<<<grid_for((int64_t)n_rows * 32, n_sm), BUILD_THREADS, 0, s>>>(
                (float *)bval.p, rowptr, n_rows, (float *)b_scale.p, (uint8_t *)q.p);
        } else {
            to_fp8_by_col<<<grid_for(nnz, n_sm), BUILD_THREADS, 0, s>>>((float *)bval.p, col, (float *)b_scale.p,
                                                                         (uint8_t *)q.p, nnz);
        }
        VMAT_LAUNCH_CHECK();
        VMAT_CUDA(cudaStreamSynchronize(s));
        *out = q.release();
        return VMAT_OK;
    };

    int cfg = opts.tile_cfg >= 0 ? opts.tile_cfg : spmv_default_config();
    const int cfg_dt = opts.tile_cfg_Dt >= 0 ? opts.tile_cfg_Dt : cfg;
    if (opts.build_Dt) {
        CsrMat &m = h->Dt;
        m.n_rows = J;
        m.n_cols = brick.on() ? (int32_t)brick.n_pos : V;
        m.nnz = nnz;
        m.nnz_pad = pad;
        VMAT_TRY(quantise(b_val_t, (int32_t *)b_col_t.p, (int64_t *)b_rp_t.p, J, true, &m.val));
        m.rowptr = (int64_t *)b_rp_t.release();
        m.col = (int32_t *)b_col_t.release();
        m.row_ids = nullptr;
        m.max_row = max_row_t;
        if (opts.index16) VMAT_TRY(csr_build_index16(m, n_sm, s));
        VMAT_TRY(spmv_prepare_tiles(m, cfg_dt, s));
        h->built_Dt = true;
    }
    if (opts.build_D) {
        CsrMat &m = h->D;
        m.n_rows = n_active;
        m.n_cols = J;
        m.nnz = nnz;
        m.nnz_pad = pad;
        VMAT_TRY(quantise(b_val_d, (int32_t *)b_col_d.p, (int64_t *)b_rp_d.p, n_active, false, &m.val));
        // FP32 refinement: the FP32 values stay beside the stored ones
        if (opts.refine_f32 && opts.dtype != VMAT_F32) h->D_val_f32 = (float *)b_val_d.release();
        m.rowptr = (int64_t *)b_rp_d.release();
        m.col = (int32_t *)b_col_d.release();
        h->act_vox = (int32_t *)b_act.release();
        h->vox2act = (int32_t *)b_v2a.release();
        h->n_active = n_active;
        if (brick.on()) {
            VMAT_CUDA(cudaMalloc(&h->act_gpos, (size_t)std::max(n_active, 1) * 4));
            if (n_active > 0) {
                map_to_brick<<<grid_for(n_active, n_sm), BUILD_THREADS, 0, s>>>(h->act_vox, n_active, brick,
                                                                                h->act_gpos);
                VMAT_LAUNCH_CHECK();
            }
        }
        m.row_ids = h->act_vox;
        m.max_row = max_row_d;
        if (opts.index16) VMAT_TRY(csr_build_index16(m, n_sm, s));
        VMAT_TRY(spmv_prepare_tiles(m, cfg, s));
        h->built_D = true;
    }
    if (fp8) {
        h->scale = (float *)b_scale.release();
        VMAT_CUDA(cudaMalloc(&h->xs, (size_t)J * 4));
    }
    h->dtype = opts.dtype;
    h->brick = brick;
    if (!opts.keep_coo) {
        VMAT_CUDA(cudaStreamSynchronize(s));
        cudaFree(h->coo_vox);
        cudaFree(h->coo_blt);
        cudaFree(h->coo_val);
        h->coo_vox = h->coo_blt = nullptr;
        h->coo_val = nullptr;
    }
    VMAT_CUDA(cudaEventRecord(e1, s));
    VMAT_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    h->build_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (opts.autotune) VMAT_TRY(spmv_autotune(*h, s));
    return VMAT_OK;
}
