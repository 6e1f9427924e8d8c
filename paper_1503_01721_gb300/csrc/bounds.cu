// Fluence-rate bounds of the master problem (Eq. 6) from the delivery limits of
// Eq. 2: gantry speed in [S^L, S^U], its change between control points at most
// Delta S per CP step, dose rate in [R^L, R^U], and a gantry slow enough for
// the leaves to move from one aperture to the next.
//
// A placed CP's speed is the speed over the interval to the next placed CP of
// its arc (m steps of cp_step degrees).  If its leaves move d columns at most,
// the interval must last d / leaf_speed seconds, so s_k <= m cp_step leaf_speed
// / d.  Along an arc the speed-change limit makes the largest speed allowed at
// k the min-plus propagation S^U_k = min_j (S_hat_j + Delta S |k - j|) of the
// per-interval caps S_hat_j = min(S^U, S^U_{j,j'}), and the smallest speed
// stays S^L.  Then R^L / S^U_k <= y_k <= R^U / S^L.
//
// One block handles one plan (the work is O(n^2 + n n_rows) for n placed
// apertures, microseconds): threads over apertures find each one's next CP and
// its largest leaf move, then each one's propagated bound.  Every float64
// operation is an explicitly rounded intrinsic (no contraction into FMAs), so
// the result is the same float64 expression evaluated in the same order.
#include <math.h>

#include "internal.cuh"

namespace vmat {

namespace {

constexpr int BOUNDS_THREADS = 256;

__host__ __device__ constexpr size_t bounds_smem(int n) { return (size_t)n * 16; }

__device__ void bounds_block(const BoundsGeom &g, int n, const int32_t *__restrict__ cps,
                             const int16_t *__restrict__ leaves, float *lo, float *hi, unsigned char *sm) {
    double *S_hat = reinterpret_cast<double *>(sm);
    int32_t *cp = reinterpret_cast<int32_t *>(S_hat + n);
    int32_t *arc = cp + n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int k = cps[t];
        int a = -1;
        if (k >= 0 && k < g.K) {
            a = 0;
            while (a + 1 < g.n_arcs && g.arc_first[a + 1] <= k) ++a;
        }
        cp[t] = k;
        arc[t] = a;
    }
    __syncthreads();
    if (!g.has_machine) {
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            lo[t] = 0.f;
            hi[t] = INFINITY;
        }
        return;
    }
    // per-interval caps
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int a = arc[t], k = cp[t];
        double S = g.s_max;
        if (a >= 0) {
            int u_next = -1, k_next = 0;
            for (int u = 0; u < n; ++u)
                if (arc[u] == a && cp[u] > k && (u_next < 0 || cp[u] < k_next)) {
                    u_next = u;
                    k_next = cp[u];
                }
            if (u_next >= 0) {
                const int16_t *la = leaves + (int64_t)t * g.n_rows * 2;
                const int16_t *lb = leaves + (int64_t)u_next * g.n_rows * 2;
                int d = 0;
                for (int i = 0; i < 2 * g.n_rows; ++i) d = max(d, abs((int)la[i] - (int)lb[i]));
                if (d > 0) {
                    const double cap = __ddiv_rn(__dmul_rn(__dmul_rn((double)(k_next - k), g.step), g.v_leaf), (double)d);
                    S = fmin(S, cap);
                }
            }
        }
        S_hat[t] = S;
    }
    __syncthreads();
    // propagated bounds and the fluence-rate box
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int a = arc[t], k = cp[t];
        if (a < 0) {
            lo[t] = 0.f;
            hi[t] = INFINITY;
            continue;
        }
        double SU = INFINITY;
        for (int u = 0; u < n; ++u)
            if (arc[u] == a) SU = fmin(SU, __dadd_rn(S_hat[u], __dmul_rn(g.ds, (double)abs(k - cp[u]))));
        lo[t] = __double2float_rn(__ddiv_rn(g.r_min, SU));
        hi[t] = g.s_min > 0.0 ? __double2float_rn(__ddiv_rn(g.r_max, g.s_min)) : INFINITY;
    }
}

__global__ void __launch_bounds__(BOUNDS_THREADS)
    fluence_bounds_kernel(BoundsGeom g, int32_t n, const int32_t *cps, const int16_t *leaves, float *lo, float *hi,
                          const int32_t *skip) {
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char sm[];
    bounds_block(g, n, cps, leaves, lo, hi, sm);
}

__global__ void __launch_bounds__(BOUNDS_THREADS) fluence_bounds_batched_kernel(const BoundsPlan *plans, int32_t n) {
    const BoundsPlan &p = plans[blockIdx.x];
    if (!p.lo || (p.skip && *p.skip)) return;
    extern __shared__ __align__(16) unsigned char sm[];
    bounds_block(p.g, n, p.cps, p.leaves, p.lo, p.hi, sm);
}

vmat_status bounds_attributes() {
    static bool done = false;
    if (!done) {
        const int mx = (int)bounds_smem(BOUNDS_MAX_AP);
        VMAT_CUDA(cudaFuncSetAttribute(fluence_bounds_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        VMAT_CUDA(cudaFuncSetAttribute(fluence_bounds_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        done = true;
    }
    return VMAT_OK;
}

} // namespace

vmat_status bounds_geom(const vmat_mlc *mlc, BoundsGeom *g) {
    if (mlc->n_arcs > MAX_ARCS) return set_error(VMAT_EUNSUPPORTED, "fluence bounds: more than %d arcs", MAX_ARCS);
    *g = BoundsGeom{};
    g->K = mlc->K;
    g->n_rows = mlc->n_rows;
    g->n_arcs = mlc->n_arcs;
    for (int a = 0; a < mlc->n_arcs; ++a) g->arc_first[a] = mlc->arc_first_cp[a];
    g->arc_first[mlc->n_arcs] = mlc->K;
    if (const vmat_machine *m = mlc->machine) {
        g->has_machine = 1;
        g->step = m->cp_step_deg;
        g->s_min = m->speed_min;
        g->s_max = m->speed_max;
        g->ds = m->speed_step_max;
        g->r_min = m->rate_min;
        g->r_max = m->rate_max;
        g->v_leaf = m->leaf_speed_cols;
    }
    return VMAT_OK;
}

vmat_status fluence_bounds_enqueue(const BoundsGeom &g, int32_t n, const int32_t *cps, const int16_t *leaves,
                                   float *lo, float *hi, const int32_t *skip, cudaStream_t s) {
    if (n <= 0) return VMAT_OK;
    if (n > BOUNDS_MAX_AP) return set_error(VMAT_EINVAL, "fluence bounds: more than %d apertures", BOUNDS_MAX_AP);
    VMAT_TRY(bounds_attributes());
    fluence_bounds_kernel<<<1, BOUNDS_THREADS, bounds_smem(n), s>>>(g, n, cps, leaves, lo, hi, skip);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

vmat_status fluence_bounds_batched(const BoundsPlan *plans, int32_t n_plans, int32_t n, cudaStream_t s) {
    if (n <= 0 || n_plans <= 0) return VMAT_OK;
    if (n > BOUNDS_MAX_AP) return set_error(VMAT_EINVAL, "fluence bounds: more than %d apertures", BOUNDS_MAX_AP);
    VMAT_TRY(bounds_attributes());
    fluence_bounds_batched_kernel<<<n_plans, BOUNDS_THREADS, bounds_smem(n), s>>>(plans, n);
    VMAT_LAUNCH_CHECK();
    return VMAT_OK;
}

} // namespace vmat

using namespace vmat;

extern "C" vmat_status fluence_bounds(const vmat_mlc *mlc, int32_t n_ap, const int32_t *cps, const int16_t *leaves,
                                      float *lo, float *hi, void *stream) {
    clear_error();
    VMAT_TRY(validate_mlc(mlc));
    if (n_ap < 0 || n_ap > BOUNDS_MAX_AP)
        return set_error(VMAT_EINVAL, "fluence_bounds: n_ap must be in [0, %d]", BOUNDS_MAX_AP);
    if (n_ap == 0) return VMAT_OK;
    if (!cps || !leaves || !lo || !hi) return set_error(VMAT_EINVAL, "fluence_bounds: NULL array");
    BoundsGeom g;
    VMAT_TRY(bounds_geom(mlc, &g));
    return fluence_bounds_enqueue(g, n_ap, cps, leaves, lo, hi, nullptr, as_stream(stream));
}
