/*
 * cyl_oracle.c -- FP64 CPU oracle for cylindrical-grid SART.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
 * leg are its only users.  Nothing here is shared with, or called by, the CUDA path.
 *
 * Written to be checked by eye against the paper, not to be fast:
 *   - every crossing of a ray with a radial shell, an azimuthal wedge plane and an axial
 *     slab plane is collected, the list is SORTED, and each piece between consecutive
 *     crossings is assigned to the voxel containing its midpoint (definition of t_jl,
 *     Sec. 2.2 below Eq. 6: the intersection length of ray j with voxel l);
 *   - projection, back-projection and row sums are plain sums over those rows;
 *   - SART follows Eq. 7 literally: residual over the subset, divided by the row sum,
 *     back-projected, divided by the column sum over the subset, scaled by lambda.
 * The CUDA path walks crossings incrementally instead of sorting, so the two share no
 * algorithm beyond the geometry both take from the paper.
 */
#include "cyl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing the oracle on one core). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Sec. 2, Eq. 1: the pose's three intrinsic zxz Euler angles give the object's
 * orientation O = Rz(alpha) Rx(beta) Rz(gamma), so gamma is the spin about the object's
 * own axis (the "internal rotation" of Sec. 2.1, azimuthal phase).  The alignment
 * X' = R X + T takes scanner coordinates into the object frame, so R = O^T. */
void orc_pose_matrix(double alpha, double beta, double gamma, double R[9])
{
    double ca = cos(alpha), sa = sin(alpha);
    double cb = cos(beta), sb = sin(beta);
    double cg = cos(gamma), sg = sin(gamma);
    double Rz_a[9] = {ca, -sa, 0, sa, ca, 0, 0, 0, 1};
    double Rx_b[9] = {1, 0, 0, 0, cb, -sb, 0, sb, cb};
    double Rz_g[9] = {cg, -sg, 0, sg, cg, 0, 0, 0, 1};
    double M[9], O[9];
    int i, j, k;
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) {
            M[3 * i + j] = 0.0;
            for (k = 0; k < 3; ++k) M[3 * i + j] += Rz_a[3 * i + k] * Rx_b[3 * k + j];
        }
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) {
            O[3 * i + j] = 0.0;
            for (k = 0; k < 3; ++k) O[3 * i + j] += M[3 * i + k] * Rz_g[3 * k + j];
        }
    for (i = 0; i < 3; ++i)
        for (j = 0; j < 3; ++j) R[3 * i + j] = O[3 * j + i];
}

/* Lab point -> stage (rotate by -phi about z) -> object frame (Eq. 1).  T is the
 * object's position in stage coordinates ("translates the object along the three
 * spatial coordinates"), so the alignment reads X' = R (X - T). */
static void lab_to_object(const orc_setup *s, double phi, const double lab[3], double out[3])
{
    double R[9], st[3];
    double c = cos(phi), sn = sin(phi);
    st[0] = c * lab[0] + sn * lab[1] - s->tx;
    st[1] = -sn * lab[0] + c * lab[1] - s->ty;
    st[2] = lab[2] - s->tz;
    orc_pose_matrix(s->alpha, s->beta, s->gamma, R);
    out[0] = R[0] * st[0] + R[1] * st[1] + R[2] * st[2];
    out[1] = R[3] * st[0] + R[4] * st[1] + R[5] * st[2];
    out[2] = R[6] * st[0] + R[7] * st[1] + R[8] * st[2];
}

void orc_ray(const orc_setup *s, int p, int iu, int iv, double S[3], double D[3])
{
    double src[3] = {-s->sod, 0.0, 0.0};
    double pix[3];
    if (s->frames) {
        /* general trajectory: the projection's own source and detector, no stage turn */
        const double *f = s->frames + 12 * (long)p;
        int k;
        for (k = 0; k < 3; ++k) {
            src[k] = f[k];
            pix[k] = f[3 + k] + iu * f[6 + k] + iv * f[9 + k];
        }
        lab_to_object(s, 0.0, src, S);
        lab_to_object(s, 0.0, pix, D);
        return;
    }
    pix[0] = s->sdd - s->sod;
    pix[1] = (iu - 0.5 * (s->det_w - 1)) * s->pitch_u + s->off_u;
    pix[2] = (iv - 0.5 * (s->det_h - 1)) * s->pitch_v + s->off_v;
    lab_to_object(s, s->angles[p], src, S);
    lab_to_object(s, s->angles[p], pix, D);
}

/* Both roots of a t^2 + 2 b t + c = 0 with disc = b^2 - a c > 0, without cancellation. */
static void stable_roots(double a, double b, double c, double disc, double *t1, double *t2)
{
    double q = -(b + copysign(sqrt(disc), b));
    double r1 = q / a, r2 = c / q;
    *t1 = r1 < r2 ? r1 : r2;
    *t2 = r1 < r2 ? r2 : r1;
}

int orc_clip(const orc_setup *s, const double o[3], const double d[3], double *t_in, double *t_out)
{
    double lo = 0.0, hi = 1.0;
    double a = d[0] * d[0] + d[1] * d[1];
    double b = o[0] * d[0] + o[1] * d[1];
    double c = o[0] * o[0] + o[1] * o[1] - s->radius * s->radius;
    double m = o[0] * d[1] - o[1] * d[0];
    double half = 0.5 * s->height;
    if (a == 0.0) {
        if (c > 0.0) return 0;
    } else {
        /* b^2 - a c written as a R^2 - m^2 (m = z component of o x d): same value,
         * without the cancellation of two large squares when the source is far away */
        double disc = a * s->radius * s->radius - m * m, t1, t2;
        if (disc <= 0.0) return 0;
        stable_roots(a, b, c, disc, &t1, &t2);
        if (t1 > lo) lo = t1;
        if (t2 < hi) hi = t2;
    }
    if (d[2] == 0.0) {
        if (o[2] < -half || o[2] > half) return 0;
    } else {
        double z1 = (-half - o[2]) / d[2], z2 = (half - o[2]) / d[2];
        if (z1 > z2) { double tmp = z1; z1 = z2; z2 = tmp; }
        if (z1 > lo) lo = z1;
        if (z2 < hi) hi = z2;
    }
    if (!(hi > lo)) return 0;
    *t_in = lo;
    *t_out = hi;
    return 1;
}

static int cmp_double(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

static int max_crossings(const orc_setup *s)
{
    return 2 * s->n_r + s->n_theta + s->n_h + 4;
}

int orc_ray_row(const orc_setup *s, const double S[3], const double D[3], long *idx, double *len, int cap)
{
    double d[3] = {D[0] - S[0], D[1] - S[1], D[2] - S[2]};
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double t_in, t_out;
    double dr = s->radius / s->n_r, dth = 2.0 * ORC_PI / s->n_theta, dh = s->height / s->n_h;
    double *t;
    int nt = 0, k, n = 0;
    if (!orc_clip(s, S, d, &t_in, &t_out)) return 0;
    t = (double *)malloc(sizeof(double) * (size_t)max_crossings(s));
    if (!t) return -1;
    t[nt++] = t_in;
    t[nt++] = t_out;
    {   /* radial shells r = r_k, k = 1 .. N_r-1: roots of |P_xy(t)|^2 = r_k^2 */
        double a = d[0] * d[0] + d[1] * d[1];
        double b = S[0] * d[0] + S[1] * d[1];
        double m = S[0] * d[1] - S[1] * d[0];
        if (a > 0.0)
            for (k = 1; k < s->n_r; ++k) {
                double rk = k * dr;
                double c = S[0] * S[0] + S[1] * S[1] - rk * rk;
                double disc = a * rk * rk - m * m, t1, t2;   /* = b^2 - a c */
                if (disc <= 0.0) continue;
                stable_roots(a, b, c, disc, &t1, &t2);
                if (t1 > t_in && t1 < t_out) t[nt++] = t1;
                if (t2 > t_in && t2 < t_out) t[nt++] = t2;
            }
    }
    if (s->n_theta > 1)   /* wedge half-planes theta = theta_k through the z' axis */
        for (k = 0; k < s->n_theta; ++k) {
            double th = k * dth, ck = cos(th), sk = sin(th);
            double nd = -sk * d[0] + ck * d[1];
            double no = -sk * S[0] + ck * S[1];
            double tk, px, py;
            if (nd == 0.0) continue;
            tk = -no / nd;
            px = S[0] + tk * d[0];
            py = S[1] + tk * d[1];
            if (ck * px + sk * py <= 0.0) continue;   /* the opposite half-plane */
            if (tk > t_in && tk < t_out) t[nt++] = tk;
        }
    if (d[2] != 0.0)      /* axial slab planes h = h_k, k = 1 .. N_h-1 */
        for (k = 1; k < s->n_h; ++k) {
            double hk = -0.5 * s->height + k * dh;
            double tk = (hk - S[2]) / d[2];
            if (tk > t_in && tk < t_out) t[nt++] = tk;
        }
    qsort(t, (size_t)nt, sizeof(double), cmp_double);
    for (k = 0; k + 1 < nt; ++k) {
        double ta = t[k], tb = t[k + 1], tm, px, py, pz, r, th;
        long ir, ith, ih;
        if (!(tb > ta)) continue;
        tm = 0.5 * (ta + tb);
        px = S[0] + tm * d[0];
        py = S[1] + tm * d[1];
        pz = S[2] + tm * d[2];
        r = sqrt(px * px + py * py);
        th = atan2(py, px);
        if (th < 0.0) th += 2.0 * ORC_PI;
        ir = (long)floor(r / dr);
        ith = (long)floor(th / dth);
        ih = (long)floor((pz + 0.5 * s->height) / dh);
        if (ir < 0) ir = 0;
        if (ir >= s->n_r) ir = s->n_r - 1;
        if (ith < 0) ith = 0;
        if (ith >= s->n_theta) ith = s->n_theta - 1;
        if (ih < 0) ih = 0;
        if (ih >= s->n_h) ih = s->n_h - 1;
        if (n >= cap) { free(t); return -1; }
        idx[n] = (ih * s->n_theta + ith) * (long)s->n_r + ir;
        len[n] = (tb - ta) * dn;
        ++n;
    }
    free(t);
    return n;
}

static long n_vox(const orc_setup *s) { return (long)s->n_h * s->n_theta * s->n_r; }

int orc_project(const orc_setup *s, const double *x, int p0, int np, double *q)
{
    long npix = (long)s->det_w * s->det_h, nrays = npix * np, j;
    int cap = max_crossings(s), err = 0;
#pragma omp parallel
    {
        long *idx = (long *)malloc(sizeof(long) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (j = 0; j < nrays; ++j) {
            int p = p0 + (int)(j / npix), pix = (int)(j % npix), n, k;
            double S[3], D[3], acc = 0.0;
            orc_ray(s, p, pix % s->det_w, pix / s->det_w, S, D);
            n = (idx && len) ? orc_ray_row(s, S, D, idx, len, cap) : -1;
            if (n < 0) {
#pragma omp atomic write
                err = 1;
                n = 0;
            }
            for (k = 0; k < n; ++k) acc += len[k] * x[idx[k]];
            q[j] = acc;
        }
        free(idx);
        free(len);
    }
    return err ? -1 : 0;
}

int orc_row_sums(const orc_setup *s, int p0, int np, double *L)
{
    long npix = (long)s->det_w * s->det_h, nrays = npix * np, j;
    int cap = max_crossings(s), err = 0;
#pragma omp parallel
    {
        long *idx = (long *)malloc(sizeof(long) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (j = 0; j < nrays; ++j) {
            int p = p0 + (int)(j / npix), pix = (int)(j % npix), n, k;
            double S[3], D[3], acc = 0.0;
            orc_ray(s, p, pix % s->det_w, pix / s->det_w, S, D);
            n = (idx && len) ? orc_ray_row(s, S, D, idx, len, cap) : -1;
            if (n < 0) {
#pragma omp atomic write
                err = 1;
                n = 0;
            }
            for (k = 0; k < n; ++k) acc += len[k];
            L[j] = acc;
        }
        free(idx);
        free(len);
    }
    return err ? -1 : 0;
}

int orc_row_nnz(const orc_setup *s, int p0, int np, long *nnz)
{
    long npix = (long)s->det_w * s->det_h, nrays = npix * np, j;
    int cap = max_crossings(s), err = 0;
#pragma omp parallel
    {
        long *idx = (long *)malloc(sizeof(long) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
#pragma omp for schedule(dynamic, 64)
        for (j = 0; j < nrays; ++j) {
            int p = p0 + (int)(j / npix), pix = (int)(j % npix), n;
            double S[3], D[3];
            orc_ray(s, p, pix % s->det_w, pix / s->det_w, S, D);
            n = (idx && len) ? orc_ray_row(s, S, D, idx, len, cap) : -1;
            if (n < 0) {
#pragma omp atomic write
                err = 1;
                n = 0;
            }
            nnz[j] = n;
        }
        free(idx);
        free(len);
    }
    return err ? -1 : 0;
}

/* A^T y: every thread scatters its rays into a private volume; the partial volumes are
 * summed at the end. */
int orc_backproject(const orc_setup *s, const double *y, int p0, int np, double *out)
{
    long npix = (long)s->det_w * s->det_h, nrays = npix * np, V = n_vox(s), j, m;
    int cap = max_crossings(s), nthr = orc_num_threads(), err = 0, t;
    double *part = (double *)calloc((size_t)nthr * (size_t)V, sizeof(double));
    if (!part) return -1;
#pragma omp parallel
    {
        int tid = 0;
        long *idx = (long *)malloc(sizeof(long) * (size_t)cap);
        double *len = (double *)malloc(sizeof(double) * (size_t)cap);
        double *mine;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        mine = part + (size_t)tid * (size_t)V;
#pragma omp for schedule(dynamic, 64)
        for (j = 0; j < nrays; ++j) {
            int p = p0 + (int)(j / npix), pix = (int)(j % npix), n, k;
            double S[3], D[3];
            if (y[j] == 0.0) continue;
            orc_ray(s, p, pix % s->det_w, pix / s->det_w, S, D);
            n = (idx && len) ? orc_ray_row(s, S, D, idx, len, cap) : -1;
            if (n < 0) {
#pragma omp atomic write
                err = 1;
                n = 0;
            }
            for (k = 0; k < n; ++k) mine[idx[k]] += len[k] * y[j];
        }
        free(idx);
        free(len);
    }
    for (m = 0; m < V; ++m) {
        double acc = 0.0;
        for (t = 0; t < nthr; ++t) acc += part[(size_t)t * (size_t)V + (size_t)m];
        out[m] = acc;
    }
    free(part);
    return err ? -1 : 0;
}

/* Eq. 7, one subset at a time:
 *   mu_m += lambda * w_hat_m * [sum_{j in OS} t_jm (p_j - sum_l t_jl mu_l) / sum_l t_jl]
 *                              / [sum_{j in OS} t_jm]. */
int orc_sart(const orc_setup *s, const double *p, const double *x0, const double *w,
             int n_iter, int subset_size, double lambda, int clamp_nonneg, int weight_mode,
             double *x)
{
    long npix = (long)s->det_w * s->det_h, V = n_vox(s), m, j;
    double *q, *L, *res, *ones, *num, *den, *what = NULL;
    int it, p0, err = 0;
    if (subset_size < 1) subset_size = 1;
    q = (double *)malloc(sizeof(double) * (size_t)(npix * subset_size));
    L = (double *)malloc(sizeof(double) * (size_t)(npix * subset_size));
    res = (double *)malloc(sizeof(double) * (size_t)(npix * subset_size));
    ones = (double *)malloc(sizeof(double) * (size_t)(npix * subset_size));
    num = (double *)malloc(sizeof(double) * (size_t)V);
    den = (double *)malloc(sizeof(double) * (size_t)V);
    if (!q || !L || !res || !ones || !num || !den) { err = -1; goto done; }
    for (m = 0; m < V; ++m) x[m] = x0 ? x0[m] : 0.0;
    if (w) {
        double wmax = 0.0;
        what = (double *)malloc(sizeof(double) * (size_t)V);
        if (!what) { err = -1; goto done; }
        for (m = 0; m < V; ++m) if (w[m] > wmax) wmax = w[m];
        for (m = 0; m < V; ++m)
            what[m] = (weight_mode == 1) ? (wmax > 0.0 ? w[m] / wmax : 0.0) : w[m];
    }
    for (j = 0; j < npix * subset_size; ++j) ones[j] = 1.0;
    /* The row and column sums of Eq. 7 are floored at eps (2^-16 of the grid radius, far
     * below any voxel size): r_j = (p_j - q_j) / max(L_j, eps) and
     * x_m += lambda w_m num_m / max(den_m, eps).  Rays and voxels met by chords of eps or
     * more are updated exactly as in Eq. 7; a ray or voxel that is only grazed moves by a
     * share (chord / eps)^2 of its plain update instead of by the whole residual of the ray
     * that grazes it, however short the chord.  The paper's t_jl counts equidistant samples
     * (Sec. 2.2), which a grazing chord does not receive. */
    const double eps = ldexp(s->radius, -16);
    for (it = 0; it < n_iter; ++it) {
        for (p0 = 0; p0 < s->n_proj; p0 += subset_size) {
            int np = s->n_proj - p0 < subset_size ? s->n_proj - p0 : subset_size;
            long nr = npix * np;
            if (orc_project(s, x, p0, np, q) || orc_row_sums(s, p0, np, L)) { err = -1; goto done; }
            for (j = 0; j < nr; ++j)
                res[j] = L[j] > 0.0 ? (p[(long)p0 * npix + j] - q[j]) / (L[j] > eps ? L[j] : eps) : 0.0;
            if (orc_backproject(s, res, p0, np, num) || orc_backproject(s, ones, p0, np, den)) {
                err = -1;
                goto done;
            }
            for (m = 0; m < V; ++m) {
                if (den[m] > 0.0) {
                    double wm = what ? what[m] : 1.0;
                    x[m] += lambda * wm * num[m] / (den[m] > eps ? den[m] : eps);
                    if (clamp_nonneg && x[m] < 0.0) x[m] = 0.0;
                }
            }
        }
    }
done:
    free(q); free(L); free(res); free(ones); free(num); free(den); free(what);
    return err;
}

void orc_log_transform(const double *I, double I0, long n, double *p)
{
    long i;
    for (i = 0; i < n; ++i) {
        double v = I[i] < 1.0 ? 1.0 : I[i];
        p[i] = -log(v / I0);
    }
}
