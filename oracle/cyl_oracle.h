/*
 * cyl_oracle.h -- FP64 CPU oracle for cylindrical-grid SART (test infrastructure).
 *
 * This is the checker, not the product: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header or
 * table with the CUDA path.
 *
 * What it computes (Goethals, Heyndrickx, Boone, "Fast tomographic inspection of
 * cylindrical objects"):
 *   - pose: X' = R X + T with R built from intrinsic zxz Euler angles (Sec. 2, Eq. 1);
 *   - cylindrical coordinates r, theta, h about the z' axis (Eq. 2, theta read as atan2
 *     in [0, 2 pi));
 *   - the linear model p_j = sum_l t_jl mu_l with t_jl the exact length of ray j inside
 *     voxel l (Sec. 2.2, Eq. 6);
 *   - the SART update of Eq. 7 over ordered subsets of projections.
 *
 * Conventions the paper leaves open (the same ones the CUDA path documents):
 *   source at (-SOD, 0, 0); detector plane x = SDD - SOD, u along +y, v along +z;
 *   pixel (iu, iv) centre at (SDD-SOD, (iu-(W-1)/2) pu + off_u, (iv-(H-1)/2) pv + off_v);
 *   stage coordinates X = Rz(-phi_p) X_lab; object coordinates X' = R (X - T) with
 *   R = (Rz(alpha) Rx(beta) Rz(gamma))^T and T the object position in stage
 *   coordinates, so gamma spins the object about its own axis;
 *   grid r_k = k R/N_r, theta_k = 2 pi k/N_theta, h_k = -H/2 + k H/N_h,
 *   voxel l = (ih * N_theta + itheta) * N_r + ir;  sinogram [p][iv][iu].
 */
#ifndef CYL_ORACLE_H
#define CYL_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n_h, n_theta, n_r;      /* grid divisions */
    double radius, height;      /* grid cylinder, mm */
    double sod, sdd;            /* source-object and source-detector distance, mm */
    int n_proj, det_w, det_h;   /* projections, detector columns (u) and rows (v) */
    double pitch_u, pitch_v;    /* pixel pitch, mm */
    double off_u, off_v;        /* detector offset, mm */
    const double *angles;       /* n_proj stage angles phi_p, radians */
    double alpha, beta, gamma;  /* zxz Euler angles, radians */
    double tx, ty, tz;          /* object position T in stage coordinates, mm */
    const double *frames;       /* NULL (circular scan), or n_proj x 12 lab-frame source S,
                                   pixel (0, 0) centre D0 and pixel steps du, dv, mm: a
                                   general trajectory, no stage rotation */
} orc_setup;

/* Alignment matrix R of X' = R X + T, row-major: the transpose of the object's
 * orientation Rz(alpha) Rx(beta) Rz(gamma) (intrinsic zxz, gamma = spin about the axis). */
void orc_pose_matrix(double alpha, double beta, double gamma, double R[9]);

/* Source S' and pixel centre D' of ray (p, iu, iv) in object coordinates. */
void orc_ray(const orc_setup *s, int p, int iu, int iv, double S[3], double D[3]);

/* Clip the segment o + t d, t in [0,1], to the grid cylinder {r <= R, |h| <= H/2}.
 * Returns 1 and the interval if non-empty, else 0. */
int orc_clip(const orc_setup *s, const double o[3], const double d[3],
             double *t_in, double *t_out);

/* Row j of the system matrix: voxel indices and intersection lengths (mm) of the
 * segment S' -> D', in order along the ray.  Returns the entry count, or -1 if more
 * than cap entries would be written. */
int orc_ray_row(const orc_setup *s, const double S[3], const double D[3],
                long *idx, double *len, int cap);

/* q = A x for projections p0 .. p0+np-1 (q holds np*H*W values). */
int orc_project(const orc_setup *s, const double *x, int p0, int np, double *q);

/* out = A^T y for projections p0 .. p0+np-1 (out holds N_h*N_theta*N_r values). */
int orc_backproject(const orc_setup *s, const double *y, int p0, int np, double *out);

/* Row sums L_j = sum_l t_jl for projections p0 .. p0+np-1. */
int orc_row_sums(const orc_setup *s, int p0, int np, double *L);

/* Number of entries of each row list: pieces of positive length between consecutive
 * crossings (a voxel entered twice counts twice). */
int orc_row_nnz(const orc_setup *s, int p0, int np, long *nnz);

/* SART of Eq. 7.  x0 may be NULL (zeros), w may be NULL (all ones).
 * weight_mode 1: w_hat = w / max(w); 0: w_hat = w.  Subsets are runs of subset_size
 * consecutive projections in index order; one iteration is one sweep over all of them.
 * Row and column sums are floored at eps = 2^-16 radius in the normalisations (a grazed
 * ray or voxel moves by (chord / eps)^2 of its plain update; see orc_sart). */
int orc_sart(const orc_setup *s, const double *p, const double *x0, const double *w,
             int n_iter, int subset_size, double lambda, int clamp_nonneg,
             int weight_mode, double *x);

/* Eq. 6 log transform: p = -ln(max(I, 1) / I0), elementwise. */
void orc_log_transform(const double *I, double I0, long n, double *p);

int orc_num_threads(void);
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
