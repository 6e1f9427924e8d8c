/*
 * Seeded synthetic pencil-beam dose-deposition-coefficient (DDC) generator.
 *
 * This module produces INPUT data only.  It holds none of the optimisation
 * arithmetic (no objective, no SpMV, no pricing); both the FP64 oracle and the
 * CUDA path consume the arrays it writes, so neither depends on the other.
 *
 * Geometry (voxel units): voxel centres sit on integer coordinates
 * (x, y, z), x fastest, voxel index i = (z*ny + y)*nx + x.  The isocentre is
 * the grid centre.  The gantry rotates about z; control point k of arc a has
 * angle theta = kk*360/n_cp + a*arc_offset_deg (kk = k mod n_cp).  The beam
 * travels along b = (cos theta, sin theta, 0); leaf columns run along
 * u = (-sin theta, cos theta, 0) and leaf rows along z.  Beamlet (k, r, c)
 * is a parallel pencil whose axis passes through
 *   iso + (c - (n_cols-1)/2)*pitch*u + (r - (n_rows-1)/2)*pitch*z_hat.
 * Its beamlet index is j = (k*n_rows + r)*n_cols + c, so the beamlets of one
 * control point are contiguous (the MLC layout the paper's pricing step walks,
 * Section 2.2.2).
 *
 * For a voxel at along-axis coordinate t and lateral distance rho (voxel
 * units) the deposited value is exp(-q) with
 *   q = mu_per_vox * (t - t_entry) + rho^2 / (2 sigma^2),
 * t_entry being where the beamlet axis enters the grid box.  Entries with
 * q > ln(1/cutoff) (value below cutoff times the beamlet's unit peak) and
 * voxels upstream of the entry point are dropped.  The keep test is done on q,
 * so no libm call decides which entries exist.  With trunc_vox > 0 the entries
 * farther than trunc_vox from the beamlet axis are dropped too (the paper's
 * truncated matrix of its method S1: a cone of radius gamma about each
 * beamlet's axis, a cylinder for these parallel beamlets).
 *
 * Output is COO, beamlet-major, voxel index ascending within each beamlet.
 * Every beamlet is generated independently, so the result does not depend on
 * the number of OpenMP threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    int32_t nx, ny, nz;
    double h_mm;
    int32_t n_cp;
    int32_t n_arcs;
    double arc_offset_deg;
    int32_t n_rows, n_cols;
    double pitch_vox;
    double mu_per_vox;
    double sigma_vox;
    double cutoff;
    double trunc_vox; /* > 0: also drop entries farther than this from the beamlet axis */
} synth_geom;

typedef struct {
    double p0[3];   /* a point on the beamlet axis */
    double b[3];    /* unit direction of travel */
    double t_entry; /* axis parameter where the axis enters the box */
    double t_max;   /* last axis parameter that can pass the keep test */
    int hit;        /* 0 when the axis misses the grid box */
} beamlet_axis;

static void axis_of(const synth_geom *g, int64_t j, beamlet_axis *ax)
{
    const double PI = 3.14159265358979323846;
    int64_t per_cp = (int64_t)g->n_rows * g->n_cols;
    int64_t k = j / per_cp;
    int64_t rem = j % per_cp;
    int32_t r = (int32_t)(rem / g->n_cols);
    int32_t c = (int32_t)(rem % g->n_cols);
    int32_t arc = (int32_t)(k / g->n_cp);
    int32_t kk = (int32_t)(k % g->n_cp);
    double theta = ((double)kk * 360.0 / (double)g->n_cp + (double)arc * g->arc_offset_deg) * PI / 180.0;
    double ct = cos(theta), st = sin(theta);
    double iso[3] = {0.5 * (g->nx - 1), 0.5 * (g->ny - 1), 0.5 * (g->nz - 1)};
    double off_c = ((double)c - 0.5 * (g->n_cols - 1)) * g->pitch_vox;
    double off_r = ((double)r - 0.5 * (g->n_rows - 1)) * g->pitch_vox;
    ax->b[0] = ct;
    ax->b[1] = st;
    ax->b[2] = 0.0;
    ax->p0[0] = iso[0] - st * off_c;
    ax->p0[1] = iso[1] + ct * off_c;
    ax->p0[2] = iso[2] + off_r;

    double lo[3] = {-0.5, -0.5, -0.5};
    double hi[3] = {g->nx - 0.5, g->ny - 0.5, g->nz - 0.5};
    double t0 = -1e300, t1 = 1e300;
    ax->hit = 1;
    for (int a = 0; a < 3; ++a) {
        double d = ax->b[a];
        if (fabs(d) < 1e-12) {
            if (ax->p0[a] < lo[a] || ax->p0[a] > hi[a]) ax->hit = 0;
            continue;
        }
        double ta = (lo[a] - ax->p0[a]) / d;
        double tb = (hi[a] - ax->p0[a]) / d;
        double tn = ta < tb ? ta : tb;
        double tf = ta < tb ? tb : ta;
        if (tn > t0) t0 = tn;
        if (tf < t1) t1 = tf;
    }
    if (!(t0 < t1)) ax->hit = 0;
    ax->t_entry = t0;
    double qmax = log(1.0 / g->cutoff);
    ax->t_max = t0 + qmax / g->mu_per_vox;
}

/* Count (vox == NULL) or write the entries of beamlet j; returns the count. */
static int64_t beamlet_entries(const synth_geom *g, int64_t j, int32_t *vox, float *val)
{
    beamlet_axis ax;
    axis_of(g, j, &ax);
    if (!ax.hit) return 0;
    const double qmax = log(1.0 / g->cutoff);
    const double inv2s2 = 1.0 / (2.0 * g->sigma_vox * g->sigma_vox);
    const double att = g->mu_per_vox;
    const double rho_max = g->sigma_vox * sqrt(2.0 * qmax);
    double bmin[3], bmax[3];
    for (int a = 0; a < 3; ++a) {
        double e0 = ax.p0[a] + ax.t_entry * ax.b[a];
        double e1 = ax.p0[a] + ax.t_max * ax.b[a];
        bmin[a] = (e0 < e1 ? e0 : e1) - rho_max;
        bmax[a] = (e0 < e1 ? e1 : e0) + rho_max;
    }
    int32_t n[3] = {g->nx, g->ny, g->nz};
    int32_t i0[3], i1[3];
    for (int a = 0; a < 3; ++a) {
        double f0 = ceil(bmin[a]), f1 = floor(bmax[a]);
        i0[a] = f0 < 0 ? 0 : (int32_t)f0;
        i1[a] = f1 > n[a] - 1 ? n[a] - 1 : (int32_t)f1;
    }
    int64_t cnt = 0;
    for (int32_t z = i0[2]; z <= i1[2]; ++z) {
        for (int32_t y = i0[1]; y <= i1[1]; ++y) {
            for (int32_t x = i0[0]; x <= i1[0]; ++x) {
                double w0 = x - ax.p0[0], w1 = y - ax.p0[1], w2 = z - ax.p0[2];
                double t = w0 * ax.b[0] + w1 * ax.b[1] + w2 * ax.b[2];
                if (t < ax.t_entry) continue;
                double l0 = w0 - t * ax.b[0], l1 = w1 - t * ax.b[1], l2 = w2 - t * ax.b[2];
                double rho2 = l0 * l0 + l1 * l1 + l2 * l2;
                if (g->trunc_vox > 0.0 && rho2 > g->trunc_vox * g->trunc_vox) continue;
                double q = att * (t - ax.t_entry) + rho2 * inv2s2;
                if (q > qmax) continue;
                if (vox) {
                    vox[cnt] = (int32_t)(((int64_t)z * g->ny + y) * g->nx + x);
                    val[cnt] = (float)exp(-q);
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

int64_t synth_n_beamlets(const synth_geom *g)
{
    return (int64_t)g->n_cp * g->n_arcs * g->n_rows * g->n_cols;
}

/* Per-beamlet entry counts; returns the total number of entries. */
int64_t synth_count(const synth_geom *g, int64_t *counts)
{
    int64_t J = synth_n_beamlets(g);
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t j = 0; j < J; ++j) {
        counts[j] = beamlet_entries(g, j, NULL, NULL);
        total += counts[j];
    }
    return total;
}

/* Counts for a list of beamlets js[0..n) (geometry of beamlet js[t]). */
int64_t synth_count_list(const synth_geom *g, const int64_t *js, int64_t n, int64_t *counts)
{
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : total)
    for (int64_t t = 0; t < n; ++t) {
        counts[t] = beamlet_entries(g, js[t], NULL, NULL);
        total += counts[t];
    }
    return total;
}

/* COO of a list of beamlets; entries of js[t] get beamlet index t. */
int synth_fill_list(const synth_geom *g, const int64_t *js, int64_t n, const int64_t *offsets, int32_t *vox,
                    int32_t *blt, float *val)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        int64_t o = offsets[t];
        int64_t c = beamlet_entries(g, js[t], vox + o, val + o);
        if (c != offsets[t + 1] - o) bad |= 1;
        for (int64_t e = 0; e < c; ++e) blt[o + e] = (int32_t)t;
    }
    return bad ? -1 : 0;
}

/* Fill COO arrays; offsets[j] is where beamlet j's entries start (J+1 entries). */
int synth_fill(const synth_geom *g, const int64_t *offsets, int32_t *vox, int32_t *blt, float *val)
{
    int64_t J = synth_n_beamlets(g);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t j = 0; j < J; ++j) {
        int64_t o = offsets[j];
        int64_t n = beamlet_entries(g, j, vox + o, val + o);
        if (n != offsets[j + 1] - o) bad |= 1;
        for (int64_t e = 0; e < n; ++e) blt[o + e] = (int32_t)j;
    }
    return bad ? -1 : 0;
}
