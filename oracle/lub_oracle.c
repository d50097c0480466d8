/*
 * Plain FP64 CPU oracle for the lubrication correction of Janoschek, Harting
 * and Toschi, "Accurate lubrication corrections for spherical and
 * non-spherical particles in discretized fluid simulations" (arXiv:1308.6482).
 *
 * TEST INFRASTRUCTURE.  This library is the reference the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA library, and it never reads anything the CUDA library wrote.
 *
 * Everything is plain double precision, written in the order and notation of
 * the paper, with no blocking, fusion or reordering:
 *
 *   orc_candidates     pair pre-filters of Sec. III A (centre distance and the
 *                      plane test against R_c), plus plane walls.
 *   orc_closest        points of closest approach y*_i, y*_j and the signed
 *                      gap h (Sec. III A, including the overlap extension).
 *                      The result has a plain definition: the common-normal
 *                      points, i.e. the maximiser over unit n of
 *                      g(n) = n.d - sigma_i(n) - sigma_j(n) (support-function
 *                      duality for convex bodies; max g = minimum distance
 *                      when separated, minus the penetration depth when
 *                      overlapping).  It is solved by safeguarded Newton with
 *                      back-tracking, certified afterwards.
 *   orc_pair_force     local principal frames and radii of curvature
 *                      (Eqs. lub:spheroid, lub:curvature-directions,
 *                      lub:curvature-radii), cubic coefficients Gamma_0,
 *                      Gamma_2 (Sec. III B), the combined-gap eigenproblem,
 *                      the cubic-coefficient rotation m_i and the rescaled
 *                      kappa_i (Appendix), the 16 elements of K (Appendix,
 *                      Eqs. app:first-element .. app:last-element), the
 *                      cut-off difference K~ (Eq. lub:resistance-correction),
 *                      the clipped gap and Hookean repulsion (Eqs. lub:frep,
 *                      lub:model), and the rigid-body transforms of Sec. III B
 *                      (V_i = v_i + w_i x (y*_i - r_i), t_i = T_i + ... x F_i).
 *   orc_apply          per-particle sums, with Newton's third law of
 *                      Eq. lub:resistance for particle j.
 *   orc_links          the link-based lubrication of Ding and Aidun that the
 *                      paper compares against (Sec. II, Eq. methods:dlub),
 *                      by brute force over the lattice sites and D3Q19 links
 *                      of a pair (readings in the section's comment).
 *
 * Readings of the paper that the code takes (each is also a test):
 *   - x1 is the unit vector along d y~/dp (increasing p), x3 the outward
 *     normal of i (the direction of h), x2 = x3 x x1.  For j, x1' is the unit
 *     vector along d y~_j/dp_j and x1' = cos(phi) x1 + sin(phi) x2.
 *   - l1 = (cos chi, -sin chi), l2 = (sin chi, cos chi); lambda_1 belongs to
 *     l1.  The labelling of the two eigenvalues is free.
 *   - Cut-offs: Delta_n for (3,3), Delta_r for (4,4),(4,5),(5,4),(5,5),
 *     Delta_t for every other non-zero element.
 *   - A wall is always the j side, with zero curvature, zero cubic terms,
 *     phi = 0 and zero velocity.
 *   - With h_c = 0 a pair with h <= 0 contributes nothing (status OVERLAP).
 *   - The appendix signs of K13, K23, K34, K35 are used as printed.
 *
 * The joint overall sign of the pair (K13, K23) and of the pair (K34, K35),
 * which the exchange symmetry cannot see, is pinned (with the elements'
 * values) by lubrication theory solved numerically: the Reynolds equation
 * for a squeeze between the exact spheroid surfaces, the ln h coefficient of
 * the force and torque on i taken from two small gaps (the thin-film tests).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* status bits (same meaning as the library's, defined independently) */
#define ORC_ST_OVERLAP    1
#define ORC_ST_NOCONV     2
#define ORC_ST_DEGENERATE 4

typedef struct {
    int64_t n;
    const double *x, *y, *z;
    const double *qw, *qx, *qy, *qz;
    const double *r_par, *r_perp;
    const double *vx, *vy, *vz, *wx, *wy, *wz;
} orc_particles;

typedef struct {
    double L[3];
    int32_t periodic[3];
    int32_t n_walls;
    double wall_z[2];
    int32_t wall_dir[2];
} orc_domain;

typedef struct {
    double mu, delta_n, delta_t, delta_r, h_c, eps_c, list_cutoff;
    double model;  /* 0: all elements of K~; 1: "normal only" (K~33 alone, Sec. IV C) */
} orc_params;

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

static void normalize3(double a[3])
{
    double l = norm3(a);
    a[0] /= l;
    a[1] /= l;
    a[2] /= l;
}

/* ------------------------------------------------------------------ */
/* particle shape: centre, body rotation Q (columns = body axes in the */
/* lab frame), semi-axes R_perp (body x, y) and R_par (body z, the     */
/* axis of rotational symmetry), Eq. lub:spheroid.                     */
/* ------------------------------------------------------------------ */
typedef struct {
    double r[3];
    double Q[3][3];
    double Rpar, Rperp;
} shape_t;

static void load_shape(const orc_particles *P, int64_t k, shape_t *s)
{
    double w = P->qw[k], x = P->qx[k], y = P->qy[k], z = P->qz[k];
    /* rotation of the normalised quaternion (scalar first) */
    double t = 2.0 / (w * w + x * x + y * y + z * z);
    s->Q[0][0] = 1.0 - t * (y * y + z * z);
    s->Q[0][1] = t * (x * y - w * z);
    s->Q[0][2] = t * (x * z + w * y);
    s->Q[1][0] = t * (x * y + w * z);
    s->Q[1][1] = 1.0 - t * (x * x + z * z);
    s->Q[1][2] = t * (y * z - w * x);
    s->Q[2][0] = t * (x * z - w * y);
    s->Q[2][1] = t * (y * z + w * x);
    s->Q[2][2] = 1.0 - t * (x * x + y * y);
    s->r[0] = P->x[k];
    s->r[1] = P->y[k];
    s->r[2] = P->z[k];
    s->Rpar = P->r_par[k];
    s->Rperp = P->r_perp[k];
}

static void to_body(const shape_t *s, const double a[3], double b[3])
{
    for (int i = 0; i < 3; ++i)
        b[i] = s->Q[0][i] * a[0] + s->Q[1][i] * a[1] + s->Q[2][i] * a[2];
}

static void to_lab(const shape_t *s, const double b[3], double a[3])
{
    for (int i = 0; i < 3; ++i)
        a[i] = s->Q[i][0] * b[0] + s->Q[i][1] * b[1] + s->Q[i][2] * b[2];
}

static double rmax(const shape_t *s) { return s->Rpar > s->Rperp ? s->Rpar : s->Rperp; }

/* Half-width of the spheroid along the (not necessarily unit) direction n:
 * sigma(n) = sqrt(n^T Q D Q^T n), D = diag(Rperp^2, Rperp^2, Rpar^2).
 * This is the support function: max over surface points y of (y - r).n. */
static double support(const shape_t *s, const double n[3])
{
    double b[3];
    to_body(s, n, b);
    double a2 = s->Rperp * s->Rperp, c2 = s->Rpar * s->Rpar;
    return sqrt(a2 * (b[0] * b[0] + b[1] * b[1]) + c2 * b[2] * b[2]);
}

/* Surface point with outward normal along n: r + Q D Q^T n / sigma(n). */
static void support_point(const shape_t *s, const double n[3], double y[3])
{
    double b[3], e[3];
    to_body(s, n, b);
    double a2 = s->Rperp * s->Rperp, c2 = s->Rpar * s->Rpar;
    double sg = sqrt(a2 * (b[0] * b[0] + b[1] * b[1]) + c2 * b[2] * b[2]);
    double yb[3] = {a2 * b[0] / sg, a2 * b[1] / sg, c2 * b[2] / sg};
    to_lab(s, yb, e);
    for (int i = 0; i < 3; ++i) y[i] = s->r[i] + e[i];
}

/* minimum-image separation d = r_j - r_i */
static void min_image(const orc_domain *D, const double ri[3], const double rj[3], double d[3])
{
    for (int k = 0; k < 3; ++k) {
        d[k] = rj[k] - ri[k];
        if (D->periodic[k]) d[k] -= D->L[k] * floor(d[k] / D->L[k] + 0.5);
    }
}

/* ------------------------------------------------------------------ */
/* Candidate pairs: pre-filters of Sec. III A.                         */
/*  (1) reject r_ij > Rmax_i + Rmax_j + Delta_L                         */
/*  (2) reject if particle i lies entirely beyond the plane normal to  */
/*      r_ij at distance R_c,j = Rmax_j + Delta_L from r_j towards i,  */
/*      i.e. r_ij - sigma_i(r^_ij) > R_c,j, or vice versa.             */
/* Walls: exact gap of a particle and the plane z = wall_z,            */
/*  h = dir (z_i - wall_z) - sigma_i(e_z) < Delta_L.                    */
/* Output order: particle pairs by (i, j), i < j; then wall pairs by   */
/* (i, wall), wall w stored as j = -1 - w.                             */
/* Returns the number of candidates; only the first cap are written.   */
/* ------------------------------------------------------------------ */
int64_t orc_candidates(const orc_particles *P, const orc_domain *D, double list_cutoff,
                       int32_t *pi, int32_t *pj, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t i = 0; i < P->n; ++i) {
        shape_t si;
        load_shape(P, i, &si);
        for (int64_t j = i + 1; j < P->n; ++j) {
            shape_t sj;
            load_shape(P, j, &sj);
            double d[3];
            min_image(D, si.r, sj.r, d);
            double rij = norm3(d);
            if (rij > rmax(&si) + rmax(&sj) + list_cutoff) continue;
            if (rij > 0.0) {
                double e[3] = {-d[0] / rij, -d[1] / rij, -d[2] / rij}; /* from j towards i */
                if (rij - support(&si, e) > rmax(&sj) + list_cutoff) continue;
                if (rij - support(&sj, e) > rmax(&si) + list_cutoff) continue;
            }
            if (cnt < cap) {
                pi[cnt] = (int32_t)i;
                pj[cnt] = (int32_t)j;
            }
            ++cnt;
        }
    }
    for (int64_t i = 0; i < P->n; ++i) {
        shape_t si;
        load_shape(P, i, &si);
        for (int w = 0; w < D->n_walls; ++w) {
            double ez[3] = {0.0, 0.0, 1.0};
            double h = D->wall_dir[w] * (si.r[2] - D->wall_z[w]) - support(&si, ez);
            if (h < list_cutoff) {
                if (cnt < cap) {
                    pi[cnt] = (int32_t)i;
                    pj[cnt] = -1 - w;
                }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Closest points.                                                     */
/* ------------------------------------------------------------------ */

/* g(n) = n.d - sigma_i(n) - sigma_j(n) for unit n, with its gradient   */
/* and Hessian in R^3.  grad sigma = M n / sigma,                      */
/* Hess sigma = M / sigma - (M n)(M n)^T / sigma^3, M = Q D Q^T.         */
static double g_eval(const shape_t *si, const shape_t *sj, const double d[3], const double n[3],
                     double grad[3], double H[3][3])
{
    double g = dot3(n, d);
    if (grad) {
        grad[0] = d[0];
        grad[1] = d[1];
        grad[2] = d[2];
    }
    if (H) memset(H, 0, 9 * sizeof(double));
    const shape_t *ss[2] = {si, sj};
    for (int k = 0; k < 2; ++k) {
        const shape_t *s = ss[k];
        double M[3][3];
        double dd[3] = {s->Rperp * s->Rperp, s->Rperp * s->Rperp, s->Rpar * s->Rpar};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                M[a][b] = 0.0;
                for (int c = 0; c < 3; ++c) M[a][b] += s->Q[a][c] * dd[c] * s->Q[b][c];
            }
        double Mn[3];
        for (int a = 0; a < 3; ++a) Mn[a] = M[a][0] * n[0] + M[a][1] * n[1] + M[a][2] * n[2];
        double sg = sqrt(dot3(n, Mn));
        g -= sg;
        if (grad)
            for (int a = 0; a < 3; ++a) grad[a] -= Mn[a] / sg;
        if (H)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    H[a][b] -= M[a][b] / sg - Mn[a] * Mn[b] / (sg * sg * sg);
    }
    return g;
}

/* an orthonormal pair (t1, t2) spanning the plane normal to unit n */
static void tangent_basis(const double n[3], double t1[3], double t2[3])
{
    double a[3] = {1.0, 0.0, 0.0};
    if (fabs(n[0]) > 0.6) {
        a[0] = 0.0;
        a[1] = 1.0;
    }
    double s = dot3(a, n);
    for (int k = 0; k < 3; ++k) t1[k] = a[k] - s * n[k];
    normalize3(t1);
    cross3(n, t1, t2);
}

/* Safeguarded Newton ascent of g on the unit sphere from n (in/out).
 * Returns the final g; *resid receives the tangential gradient norm. */
static double newton_on_sphere(const shape_t *si, const shape_t *sj, const double d[3], double n[3],
                               double scale, double *resid)
{
    double grad[3], H[3][3];
    double g = g_eval(si, sj, d, n, grad, H);
    double res = 0.0;
    for (int it = 0; it < 200; ++it) {
        double t1[3], t2[3];
        tangent_basis(n, t1, t2);
        double gt[2] = {dot3(t1, grad), dot3(t2, grad)};
        res = sqrt(gt[0] * gt[0] + gt[1] * gt[1]);
        if (res <= 1e-14 * scale) break;
        /* Hessian of g(n + a t1 + b t2)/|n + a t1 + b t2| at a = b = 0 */
        double Ht1[3], Ht2[3];
        for (int a = 0; a < 3; ++a) {
            Ht1[a] = H[a][0] * t1[0] + H[a][1] * t1[1] + H[a][2] * t1[2];
            Ht2[a] = H[a][0] * t2[0] + H[a][1] * t2[1] + H[a][2] * t2[2];
        }
        double gn = dot3(n, grad);
        double h11 = dot3(t1, Ht1) - gn, h12 = dot3(t1, Ht2), h22 = dot3(t2, Ht2) - gn;
        double det = h11 * h22 - h12 * h12;
        double s[2];
        if (h11 < 0.0 && det > 0.0) {
            s[0] = -(h22 * gt[0] - h12 * gt[1]) / det;
            s[1] = -(-h12 * gt[0] + h11 * gt[1]) / det;
        } else {
            double hs = fabs(h11) + fabs(h22) + fabs(h12) + scale;
            s[0] = gt[0] / hs;
            s[1] = gt[1] / hs;
        }
        double sl = sqrt(s[0] * s[0] + s[1] * s[1]);
        if (sl > 0.5) {
            s[0] *= 0.5 / sl;
            s[1] *= 0.5 / sl;
        }
        /* back-tracking on g */
        int accepted = 0;
        for (int bt = 0; bt < 60; ++bt) {
            double m[3];
            for (int k = 0; k < 3; ++k) m[k] = n[k] + s[0] * t1[k] + s[1] * t2[k];
            normalize3(m);
            double gm = g_eval(si, sj, d, m, NULL, NULL);
            if (gm >= g - 1e-15 * scale) {
                n[0] = m[0];
                n[1] = m[1];
                n[2] = m[2];
                accepted = 1;
                break;
            }
            s[0] *= 0.5;
            s[1] *= 0.5;
        }
        g = g_eval(si, sj, d, n, grad, H);
        if (!accepted) break;
    }
    {
        double t1[3], t2[3];
        tangent_basis(n, t1, t2);
        double a = dot3(t1, grad), b = dot3(t2, grad);
        res = sqrt(a * a + b * b);
    }
    *resid = res;
    return g;
}

/* Closest points of one candidate pair.  Outputs: unit normal n (outward  */
/* normal of i at y*_i, pointing from i to j), signed gap h, y*_i, y*_j    */
/* (with y*_j - y*_i = h n), status bits.                                  */
static int closest_one(const orc_particles *P, const orc_domain *D, int32_t i, int32_t j,
                       double n[3], double *h, double yi[3], double yj[3])
{
    shape_t si;
    load_shape(P, i, &si);
    int st = 0;
    if (!(si.Rpar > 0.0) || !(si.Rperp > 0.0)) st |= ORC_ST_DEGENERATE;
    if (j < 0) {
        /* plane wall: n = -dir e_z, closest point = support point along n */
        int w = -1 - j;
        double dir = D->wall_dir[w];
        n[0] = 0.0;
        n[1] = 0.0;
        n[2] = -dir;
        double ez[3] = {0.0, 0.0, 1.0};
        *h = dir * (si.r[2] - D->wall_z[w]) - support(&si, ez);
        support_point(&si, n, yi);
        for (int k = 0; k < 3; ++k) yj[k] = yi[k] + (*h) * n[k];
        if (*h <= 0.0) st |= ORC_ST_OVERLAP;
        return st;
    }
    shape_t sj;
    load_shape(P, j, &sj);
    if (!(sj.Rpar > 0.0) || !(sj.Rperp > 0.0)) st |= ORC_ST_DEGENERATE;
    double d[3];
    min_image(D, si.r, sj.r, d);
    double dl = norm3(d);
    if (!(dl > 0.0) || (st & ORC_ST_DEGENERATE)) {
        n[0] = n[1] = n[2] = 0.0;
        *h = 0.0;
        yi[0] = yi[1] = yi[2] = yj[0] = yj[1] = yj[2] = 0.0;
        return st | ORC_ST_DEGENERATE;
    }
    /* place j at its minimum image relative to i */
    for (int k = 0; k < 3; ++k) sj.r[k] = si.r[k] + d[k];
    double scale = dl + rmax(&si) + rmax(&sj);

    double best[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
    double res;
    double gbest = newton_on_sphere(&si, &sj, d, best, scale, &res);
    if (gbest <= 0.0) {
        /* Overlap: g is no longer concave on the sphere, so search all
         * directions (Fibonacci sphere) and polish the best sample. */
        const int ns = 4000;
        double gs = -1e300, ns_best[3] = {0, 0, 1};
        for (int k = 0; k < ns; ++k) {
            double zc = 1.0 - (2.0 * k + 1.0) / ns;
            double rc = sqrt(1.0 - zc * zc);
            double ph = k * ORC_PI * (3.0 - sqrt(5.0));
            double m[3] = {rc * cos(ph), rc * sin(ph), zc};
            double gm = g_eval(&si, &sj, d, m, NULL, NULL);
            if (gm > gs) {
                gs = gm;
                ns_best[0] = m[0];
                ns_best[1] = m[1];
                ns_best[2] = m[2];
            }
        }
        double res2;
        double g2 = newton_on_sphere(&si, &sj, d, ns_best, scale, &res2);
        if (g2 > gbest + 1e-12 * scale) {
            gbest = g2;
            res = res2;
            best[0] = ns_best[0];
            best[1] = ns_best[1];
            best[2] = ns_best[2];
        }
    }
    n[0] = best[0];
    n[1] = best[1];
    n[2] = best[2];
    *h = gbest;
    support_point(&si, n, yi);
    double mn[3] = {-n[0], -n[1], -n[2]};
    support_point(&sj, mn, yj);
    /* certificate: y*_j - y*_i must equal h n (common normal) */
    double err = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = (yj[k] - yi[k]) - (*h) * n[k];
        err += e * e;
    }
    if (sqrt(err) > 1e-10 * scale || res > 1e-10 * scale) st |= ORC_ST_NOCONV;
    /* the consistency checks of Sec. III A: normals point to the other centre */
    if (!(dot3(n, d) > 0.0)) st |= ORC_ST_NOCONV;
    if (*h <= 0.0) st |= ORC_ST_OVERLAP;
    return st;
}

void orc_closest(const orc_particles *P, const orc_domain *D, int64_t np, const int32_t *pi,
                 const int32_t *pj, double *n /*[np][3]*/, double *h, double *yi /*[np][3]*/,
                 double *yj /*[np][3]*/, int32_t *status)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < np; ++k)
        status[k] = closest_one(P, D, pi[k], pj[k], n + 3 * k, h + k, yi + 3 * k, yj + 3 * k);
}

/* ------------------------------------------------------------------ */
/* Local surface geometry at a surface point y of a spheroid, given    */
/* the outward unit normal nrm there.                                  */
/* Eq. lub:spheroid: y~(p,q) = (Rperp cos p cos q, Rperp cos p sin q,   */
/*                              Rpar sin p)                             */
/* Eq. lub:curvature-directions: s~1 = d y~/dp                          */
/* Eq. lub:curvature-radii: S1 = s1^3/(Rpar Rperp), S2 = Rperp s1/Rpar, */
/*   s1 = sqrt(Rperp^2 sin^2 p + Rpar^2 cos^2 p)                         */
/* Sec. III B: Gamma_0, Gamma_2 (Gamma_1 = Gamma_3 = 0).                */
/* ------------------------------------------------------------------ */
typedef struct {
    double x1[3];   /* unit principal direction along d y~/dp, orthogonal to nrm */
    double S1, S2;  /* radii of curvature along x1 and the other principal direction */
    double G[4];    /* Gamma_0..Gamma_3 */
    double p, q;
} surf_t;

static void surface_geometry(const shape_t *s, const double y[3], const double nrm[3], surf_t *o)
{
    double rel[3] = {y[0] - s->r[0], y[1] - s->r[1], y[2] - s->r[2]};
    double yb[3];
    to_body(s, rel, yb);
    double Rp = s->Rpar, Rq = s->Rperp;
    double p = atan2(yb[2] / Rp, sqrt(yb[0] * yb[0] + yb[1] * yb[1]) / Rq);
    double q = atan2(yb[1], yb[0]);
    double sp = sin(p), cp = cos(p), sq = sin(q), cq = cos(q);
    double s1 = sqrt(Rq * Rq * sp * sp + Rp * Rp * cp * cp);
    double s1b[3] = {-Rq * sp * cq, -Rq * sp * sq, Rp * cp};
    double x1[3];
    to_lab(s, s1b, x1);
    double a = dot3(x1, nrm);
    for (int k = 0; k < 3; ++k) x1[k] -= a * nrm[k];
    normalize3(x1);
    o->x1[0] = x1[0];
    o->x1[1] = x1[1];
    o->x1[2] = x1[2];
    o->S1 = s1 * s1 * s1 / (Rp * Rq);
    o->S2 = Rq * s1 / Rp;
    double s1_4 = s1 * s1 * s1 * s1;
    o->G[0] = (Rp * Rp - Rq * Rq) * Rp * Rq * sp * cp / (2.0 * s1_4 * s1 * s1);
    o->G[1] = 0.0;
    o->G[2] = (Rp * Rp - Rq * Rq) * Rp * sp * cp / (2.0 * Rq * s1_4);
    o->G[3] = 0.0;
    o->p = p;
    o->q = q;
}

/* Appendix: cubic coefficients a_0..a_3 given in a frame rotated by alpha, */
/* expressed in the unrotated frame: m_i(alpha, a_0, a_1, a_2, a_3).        */
static void m_rot(double al, const double a[4], double m[4])
{
    double c = cos(al), s = sin(al);
    m[0] = a[0] * c * c * c - a[1] * s * c * c + a[2] * s * s * c - a[3] * s * s * s;
    m[1] = a[0] * 3.0 * s * c * c + a[1] * (c * c * c - 2.0 * s * s * c) +
           a[2] * (s * s * s - 2.0 * s * c * c) + a[3] * 3.0 * s * s * c;
    m[2] = a[0] * 3.0 * c * s * s + a[1] * (2.0 * c * c * s - s * s * s) +
           a[2] * (c * c * c - 2.0 * c * s * s) - a[3] * (3.0 * c * c * s);
    m[3] = a[0] * s * s * s + a[1] * c * s * s + a[2] * c * c * s + a[3] * c * c * c;
}

/* Geometry of a pair at its closest points, plus K split into its ln h and */
/* 1/h coefficients: K_gd(h) = Lcoef[g][d] ln h + Hcoef33 / h (only (3,3)). */
typedef struct {
    double x1[3], x2[3], x3[3];
    double S1, S2, S1p, S2p; /* S1p, S2p infinite for a wall (stored as 0 curvature below) */
    double c1, c2, c1p, c2p; /* curvatures 1/S */
    double G[4], Gp[4];
    double phi, lam1, lam2, chi;
    double kappa[4];
    double Lcoef[6][6];
    double Hcoef33;
} pairgeom_t;

static void pair_geometry(const shape_t *si, const shape_t *sj /* NULL for a wall */, const double n[3],
                          const double yi[3], const double yj[3], pairgeom_t *G)
{
    memset(G, 0, sizeof(*G));
    surf_t a;
    surface_geometry(si, yi, n, &a);
    for (int k = 0; k < 3; ++k) {
        G->x3[k] = n[k];
        G->x1[k] = a.x1[k];
    }
    cross3(G->x3, G->x1, G->x2);
    G->S1 = a.S1;
    G->S2 = a.S2;
    G->c1 = 1.0 / a.S1;
    G->c2 = 1.0 / a.S2;
    for (int k = 0; k < 4; ++k) G->G[k] = a.G[k];
    if (sj) {
        surf_t b;
        double mn[3] = {-n[0], -n[1], -n[2]};
        surface_geometry(sj, yj, mn, &b);
        G->S1p = b.S1;
        G->S2p = b.S2;
        G->c1p = 1.0 / b.S1;
        G->c2p = 1.0 / b.S2;
        for (int k = 0; k < 4; ++k) G->Gp[k] = b.G[k];
        G->phi = atan2(dot3(b.x1, G->x2), dot3(b.x1, G->x1));
    } else {
        G->S1p = INFINITY;
        G->S2p = INFINITY;
        G->c1p = 0.0;
        G->c2p = 0.0;
        G->phi = 0.0;
    }
    /* combined-gap matrix (Appendix) */
    double cf = cos(G->phi), sf = sin(G->phi);
    double A11 = 0.5 * G->c1 + 0.5 * cf * cf * G->c1p + 0.5 * sf * sf * G->c2p;
    double A12 = 0.5 * sf * cf * (G->c1p - G->c2p);
    double A22 = 0.5 * G->c2 + 0.5 * sf * sf * G->c1p + 0.5 * cf * cf * G->c2p;
    double mid = 0.5 * (A11 + A22);
    double rad = sqrt(0.25 * (A11 - A22) * (A11 - A22) + A12 * A12);
    double l1 = mid + rad, l2 = mid - rad;
    /* eigenvector of lambda_2, l2 = (sin chi, cos chi) */
    double v0a = A12, v1a = l2 - A11;
    double v0b = l2 - A22, v1b = A12;
    double v0, v1;
    if (v0a * v0a + v1a * v1a >= v0b * v0b + v1b * v1b) {
        v0 = v0a;
        v1 = v1a;
    } else {
        v0 = v0b;
        v1 = v1b;
    }
    double chi = (v0 == 0.0 && v1 == 0.0) ? 0.0 : atan2(v0, v1);
    G->lam1 = l1;
    G->lam2 = l2;
    G->chi = chi;
    /* cubic terms: beta = m(phi, Gamma'), k = Gamma + beta,
       kappa_i = m_i(chi, k) / (sqrt(l1)^(3-i) sqrt(l2)^i) */
    double beta[4], kk[4], mk[4];
    m_rot(G->phi, G->Gp, beta);
    for (int k = 0; k < 4; ++k) kk[k] = G->G[k] + beta[k];
    m_rot(chi, kk, mk);
    double r1 = sqrt(l1), r2 = sqrt(l2);
    G->kappa[0] = mk[0] / (r1 * r1 * r1);
    G->kappa[1] = mk[1] / (r1 * r1 * r2);
    G->kappa[2] = mk[2] / (r1 * r2 * r2);
    G->kappa[3] = mk[3] / (r2 * r2 * r2);

    /* Elements of K, Eqs. app:first-element .. app:last-element, written with
       (1 - lambda S)/S = c - lambda (c = 1/S).  Lcoef multiplies ln h. */
    double cx = cos(chi), sx = sin(chi), c2x = cx * cx, s2x = sx * sx, scx = sx * cx;
    double sq = sqrt(l1 * l2);
    double D1 = (3.0 * l1 + 2.0 * l2) * l1; /* (3 l1 + 2 l2) l1 */
    double D2 = (2.0 * l1 + 3.0 * l2) * l2; /* (2 l1 + 3 l2) l2 */
    double c1 = G->c1, c2 = G->c2;
    const double *ka = G->kappa;
    const double *Ga = G->G;
    double pi = ORC_PI;
    double L[6][6];
    memset(L, 0, sizeof(L));
    /* K11 */
    L[0][0] = -pi / sq * (3.0 * c2x * (c1 - l1) * (c1 - l1) / D1 + 3.0 * s2x * (c1 - l2) * (c1 - l2) / D2 + 1.0);
    /* K12 */
    L[0][1] = 3.0 * pi / sq * scx * ((c1 - l1) * (c2 - l1) / D1 - (c1 - l2) * (c2 - l2) / D2);
    /* K13 */
    {
        double pre = -3.0 * pi / (2.0 * sq * (l1 + l2));
        double t1 = (2.0 * r1 * (3.0 * ka[0] * l1 + ka[2] * l2) -
                     1.5 * c1 / r1 * ((7.0 * l1 + 2.0 * l2) * ka[0] + (l1 + 2.0 * l2) * ka[2])) *
                    cx / (3.0 * l1 + 2.0 * l2);
        double t2 = (2.0 * r2 * (ka[1] * l1 + 3.0 * ka[3] * l2) -
                     1.5 * c1 / r2 * ((2.0 * l1 + l2) * ka[1] + (2.0 * l1 + 7.0 * l2) * ka[3])) *
                    sx / (2.0 * l1 + 3.0 * l2);
        double t3 = 3.0 * Ga[0] * (c2x / l1 + s2x / l2) + 2.0 * Ga[1] * scx * (1.0 / l2 - 1.0 / l1) +
                    Ga[2] * (s2x / l1 + c2x / l2);
        L[0][2] = pre * (t1 + t2 + t3);
    }
    /* K14 */
    L[0][3] = 3.0 * pi / sq * scx * ((c1 - l1) / D1 - (c1 - l2) / D2);
    /* K15 */
    L[0][4] = 3.0 * pi / sq * (c2x * (c1 - l1) / D1 + s2x * (c1 - l2) / D2);
    /* K22 */
    L[1][1] = -pi / sq * (3.0 * s2x * (c2 - l1) * (c2 - l1) / D1 + 3.0 * c2x * (c2 - l2) * (c2 - l2) / D2 + 1.0);
    /* K23 */
    {
        double pre = -3.0 * pi / (2.0 * sq * (l1 + l2));
        double t1 = (-2.0 * r1 * (3.0 * ka[0] * l1 + ka[2] * l2) +
                     1.5 * c2 / r1 * ((7.0 * l1 + 2.0 * l2) * ka[0] + (l1 + 2.0 * l2) * ka[2])) *
                    sx / (3.0 * l1 + 2.0 * l2);
        double t2 = (2.0 * r2 * (ka[1] * l1 + 3.0 * ka[3] * l2) -
                     1.5 * c2 / r2 * ((2.0 * l1 + l2) * ka[1] + (2.0 * l1 + 7.0 * l2) * ka[3])) *
                    cx / (2.0 * l1 + 3.0 * l2);
        double t3 = 3.0 * Ga[3] * (s2x / l1 + c2x / l2) + 2.0 * Ga[2] * scx * (1.0 / l2 - 1.0 / l1) +
                    Ga[1] * (c2x / l1 + s2x / l2);
        L[1][2] = pre * (t1 + t2 + t3);
    }
    /* K24 */
    L[1][3] = -3.0 * pi / sq * (s2x * (c2 - l1) / D1 + c2x * (c2 - l2) / D2);
    /* K25 */
    L[1][4] = 3.0 * pi / sq * scx * (-(c2 - l1) / D1 + (c2 - l2) / D2);
    /* K33: 1/h term only (the ln h part of Claeys & Brady's (2.20) is omitted,
       as in the paper) */
    G->Hcoef33 = 3.0 * pi / (sq * (l1 + l2));
    /* K34, K35 */
    {
        double pre = 9.0 * pi / (4.0 * sq * (l1 + l2));
        double Bq = ((2.0 * l1 + l2) * ka[1] + (2.0 * l1 + 7.0 * l2) * ka[3]) / (r2 * (2.0 * l1 + 3.0 * l2));
        double Aq = ((l1 + 2.0 * l2) * ka[2] + (7.0 * l1 + 2.0 * l2) * ka[0]) / (r1 * (3.0 * l1 + 2.0 * l2));
        L[2][3] = pre * (Bq * cx - Aq * sx);
        L[2][4] = -pre * (Aq * cx + Bq * sx);
    }
    /* K36 */
    L[2][5] = -3.0 * pi / (2.0 * sq * (l1 + l2)) * scx * (c1 - c2) * (1.0 / l1 - 1.0 / l2);
    /* K44, K45, K55 */
    L[3][3] = -3.0 * pi / sq * (s2x / D1 + c2x / D2);
    L[3][4] = 3.0 * pi / sq * scx * (-1.0 / D1 + 1.0 / D2);
    L[4][4] = -3.0 * pi / sq * (c2x / D1 + s2x / D2);
    /* symmetry of K */
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < r; ++c) L[r][c] = L[c][r];
    memcpy(G->Lcoef, L, sizeof(L));
}

/* cut-off of element (g, d), Sec. III B and Eq. results:cutoffs */
static double cutoff_of(const orc_params *p, int g, int d)
{
    if (g == 2 && d == 2) return p->delta_n;
    if ((g == 3 || g == 4) && (d == 3 || d == 4)) return p->delta_r;
    return p->delta_t;
}

/* K~(h) of Eq. lub:resistance-correction, evaluated at the gap he. */
static void ktilde(const pairgeom_t *G, const orc_params *p, double he, double Kt[6][6])
{
    for (int g = 0; g < 6; ++g)
        for (int d = 0; d < 6; ++d) {
            double D = cutoff_of(p, g, d);
            double v = 0.0;
            if (p->model == 1.0 && !(g == 2 && d == 2)) {
                v = 0.0;
            } else if (he < D) {
                if (g == 2 && d == 2)
                    v = G->Hcoef33 * (1.0 / he - 1.0 / D);
                else
                    v = G->Lcoef[g][d] * (log(he) - log(D));
            }
            Kt[g][d] = v;
        }
}

/* One pair: F_i, T_i in the lab frame (T_i about y*_i), the lever arms
 * y*_i - r_i and y*_j - r_j, K~ (6x6, local frame) and geometry summary.
 * Returns the status bits it adds (OVERLAP when h_c = 0 and h <= 0). */
static int pair_force_one(const orc_particles *P, const orc_domain *Dm, const orc_params *prm, int32_t i,
                          int32_t j, const double n[3], double h, const double yi[3], const double yj[3],
                          double FT[6], double lever[6], double Ktout[36], double geom[40])
{
    for (int k = 0; k < 6; ++k) FT[k] = 0.0;
    shape_t si, sj;
    load_shape(P, i, &si);
    double ri[3] = {si.r[0], si.r[1], si.r[2]};
    double rj[3] = {0.0, 0.0, 0.0};
    if (j >= 0) {
        /* image of r_j nearest to r_i */
        load_shape(P, j, &sj);
        double d[3];
        min_image(Dm, si.r, sj.r, d);
        for (int k = 0; k < 3; ++k) rj[k] = sj.r[k] = ri[k] + d[k];
    }
    for (int k = 0; k < 3; ++k) {
        lever[k] = yi[k] - ri[k];
        lever[3 + k] = (j >= 0) ? yj[k] - rj[k] : 0.0;
    }
    if (Ktout) memset(Ktout, 0, 36 * sizeof(double));
    if (geom) memset(geom, 0, 40 * sizeof(double));
    int st = 0;
    double he = h;
    if (prm->h_c > 0.0) {
        if (he < prm->h_c) he = prm->h_c;
    } else if (h <= 0.0) {
        return ORC_ST_OVERLAP;
    }
    pairgeom_t G;
    pair_geometry(&si, j >= 0 ? &sj : NULL, n, yi, yj, &G);
    double Kt[6][6];
    ktilde(&G, prm, he, Kt);

    /* surface velocities, Sec. III B: V = v + w x (y* - r), Omega = w */
    double vi[3] = {P->vx[i], P->vy[i], P->vz[i]}, wi[3] = {P->wx[i], P->wy[i], P->wz[i]};
    double Vi[3], Vj[3] = {0, 0, 0}, Wj[3] = {0, 0, 0};
    cross3(wi, lever, Vi);
    for (int k = 0; k < 3; ++k) Vi[k] += vi[k];
    if (j >= 0) {
        double vj[3] = {P->vx[j], P->vy[j], P->vz[j]};
        double wj[3] = {P->wx[j], P->wy[j], P->wz[j]};
        cross3(wj, lever + 3, Vj);
        for (int k = 0; k < 3; ++k) {
            Vj[k] += vj[k];
            Wj[k] = wj[k];
        }
    }
    const double *ax[3] = {G.x1, G.x2, G.x3};
    double u[6];
    for (int a = 0; a < 3; ++a) {
        double dv[3] = {Vj[0] - Vi[0], Vj[1] - Vi[1], Vj[2] - Vi[2]};
        double dw[3] = {Wj[0] - wi[0], Wj[1] - wi[1], Wj[2] - wi[2]};
        u[a] = dot3(ax[a], dv);
        u[3 + a] = dot3(ax[a], dw);
    }
    /* Eq. lub:model */
    double Fb[6];
    for (int g = 0; g < 6; ++g) {
        Fb[g] = 0.0;
        for (int d = 0; d < 6; ++d) Fb[g] += prm->mu * Kt[g][d] * u[d];
    }
    if (prm->h_c > 0.0 && h <= prm->h_c) {
        double Fr = (h > 0.0) ? prm->eps_c * (prm->h_c - h) : prm->eps_c * prm->h_c;
        Fb[2] -= Fr;
    }
    for (int k = 0; k < 3; ++k) {
        FT[k] = Fb[0] * G.x1[k] + Fb[1] * G.x2[k] + Fb[2] * G.x3[k];
        FT[3 + k] = Fb[3] * G.x1[k] + Fb[4] * G.x2[k] + Fb[5] * G.x3[k];
    }
    if (Ktout)
        for (int g = 0; g < 6; ++g)
            for (int d = 0; d < 6; ++d) Ktout[6 * g + d] = Kt[g][d];
    if (geom) {
        geom[0] = G.S1;
        geom[1] = G.S2;
        geom[2] = G.S1p;
        geom[3] = G.S2p;
        geom[4] = G.G[0];
        geom[5] = G.G[2];
        geom[6] = G.Gp[0];
        geom[7] = G.Gp[2];
        geom[8] = G.phi;
        geom[9] = G.lam1;
        geom[10] = G.lam2;
        geom[11] = G.chi;
        for (int k = 0; k < 4; ++k) geom[12 + k] = G.kappa[k];
        for (int k = 0; k < 3; ++k) {
            geom[16 + k] = G.x1[k];
            geom[19 + k] = G.x2[k];
            geom[22 + k] = G.x3[k];
        }
        geom[25] = G.Hcoef33;
        geom[26] = he;
        for (int k = 0; k < 6; ++k) geom[27 + k] = u[k];
    }
    return st;
}

void orc_pair_force(const orc_particles *P, const orc_domain *D, const orc_params *prm, int64_t np,
                    const int32_t *pi, const int32_t *pj, const double *n, const double *h,
                    const double *yi, const double *yj, double *FT /*[np][6]*/,
                    double *lever /*[np][6]*/, double *Kt /*[np][36] or NULL*/,
                    double *geom /*[np][40] or NULL*/, int32_t *status /* |= */)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < np; ++k) {
        int st = pair_force_one(P, D, prm, pi[k], pj[k], n + 3 * k, h[k], yi + 3 * k, yj + 3 * k,
                                FT + 6 * k, lever + 6 * k, Kt ? Kt + 36 * k : NULL,
                                geom ? geom + 40 * k : NULL);
        if (status) status[k] |= st;
    }
}

/* Per-particle force and torque, Sec. III B and Eq. lub:resistance:
 *   f_i += F_i,  t_i += T_i + (y*_i - r_i) x F_i,
 *   f_j -= F_i,  t_j += -T_i + (y*_j - r_j) x (-F_i).
 * Wall sides are dropped.  force, torque: [n][3], zeroed here. */
void orc_apply(int64_t nparticles, int64_t np, const int32_t *pi, const int32_t *pj, const double *FT,
               const double *lever, double *force, double *torque)
{
    memset(force, 0, 3 * nparticles * sizeof(double));
    memset(torque, 0, 3 * nparticles * sizeof(double));
    for (int64_t k = 0; k < np; ++k) {
        const double *F = FT + 6 * k, *T = FT + 6 * k + 3;
        const double *li = lever + 6 * k, *lj = lever + 6 * k + 3;
        int32_t i = pi[k], j = pj[k];
        double c[3];
        cross3(li, F, c);
        for (int a = 0; a < 3; ++a) {
            force[3 * i + a] += F[a];
            torque[3 * i + a] += T[a] + c[a];
        }
        if (j >= 0) {
            double mF[3] = {-F[0], -F[1], -F[2]};
            cross3(lj, mF, c);
            for (int a = 0; a < 3; ++a) {
                force[3 * j + a] -= F[a];
                torque[3 * j + a] += -T[a] + c[a];
            }
        }
    }
}

/* convenience for tests: the surface geometry of one particle at a point */
void orc_surface_geometry(const orc_particles *P, int64_t k, const double y[3], const double nrm[3],
                          double out[8] /* x1[3], S1, S2, G0, G2, p */)
{
    shape_t s;
    load_shape(P, k, &s);
    surf_t o;
    surface_geometry(&s, y, nrm, &o);
    out[0] = o.x1[0];
    out[1] = o.x1[1];
    out[2] = o.x1[2];
    out[3] = o.S1;
    out[4] = o.S2;
    out[5] = o.G[0];
    out[6] = o.G[2];
    out[7] = o.p;
}

/* convenience for tests: g(n) of a pair (i, j) at unit n */
double orc_g(const orc_particles *P, const orc_domain *D, int32_t i, int32_t j, const double n[3])
{
    shape_t si, sj;
    load_shape(P, i, &si);
    load_shape(P, j, &sj);
    double d[3];
    min_image(D, si.r, sj.r, d);
    for (int k = 0; k < 3; ++k) sj.r[k] = si.r[k] + d[k];
    return g_eval(&si, &sj, d, n, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* Learned warm start: the oracle's plain FP64 copy of the network used  */
/* to check the GPU's training kernels (features, forward, backward).    */
/* ------------------------------------------------------------------ */

/* Surface parameters (p, q) of Eq. lub:spheroid of the point y on particle k:
 * y~ = Q^T (y - r); sin p = y~_3 / R_par, cos p = |y~_12| / R_perp, q = atan2. */
void orc_surface_pq(const orc_particles *P, int64_t k, const double y[3], double pq[2])
{
    shape_t s;
    load_shape(P, k, &s);
    double rel[3] = {y[0] - s.r[0], y[1] - s.r[1], y[2] - s.r[2]};
    double yb[3];
    to_body(&s, rel, yb);
    pq[0] = atan2(yb[2] / s.Rpar, sqrt(yb[0] * yb[0] + yb[1] * yb[1]) / s.Rperp);
    pq[1] = atan2(yb[1], yb[0]);
}

/* The 12 input features of a pair (i, j).  They describe the pair up to
 * the motions that leave the targets unchanged: rigid motions of the pair,
 * rotations of i about its symmetry axis and of j about its own.  Frame: i's
 * body frame turned about its axis until d = r_j - r_i (minimum image) lies
 * in the half-plane y = 0, x >= 0 (unturned when d lies on the axis).
 *   [0]     rho / R_perp,i: distance of d from i's axis
 *   [1]     d_z / R_perp,i: component of d along i's axis
 *   [2..4]  j's symmetry axis in that frame
 *   [5..8]  ln R_par,i, ln R_perp,i, ln R_par,j, ln R_perp,j
 *   [9]     asinh(g(d^)/a): the support-function gap estimate along the line
 *           of centres, g = |d| - sigma_i(d^) - sigma_j(d^), over the smallest
 *           semi-axis a of the pair
 *   [10,11] ln(sigma_i(d^) / R_perp,i), ln(sigma_j(d^) / R_perp,j): the
 *           half-widths along the line of centres. */
void orc_mlp_features(const orc_particles *P, const orc_domain *D, int64_t np, const int32_t *pi,
                      const int32_t *pj, double *feat)
{
    for (int64_t k = 0; k < np; ++k) {
        int32_t i = pi[k], j = pj[k];
        shape_t si, sj;
        load_shape(P, i, &si);
        load_shape(P, j, &sj);
        double d[3];
        min_image(D, si.r, sj.r, d);
        double db[3];
        to_body(&si, d, db);
        const double rho = sqrt(db[0] * db[0] + db[1] * db[1]);
        const double c = rho > 0.0 ? db[0] / rho : 1.0, s = rho > 0.0 ? db[1] / rho : 0.0;
        double oj[3] = {sj.Q[0][2], sj.Q[1][2], sj.Q[2][2]}, ob[3];
        to_body(&si, oj, ob);
        double *f = feat + 12 * k;
        f[0] = rho / si.Rperp;
        f[1] = db[2] / si.Rperp;
        f[2] = c * ob[0] + s * ob[1];
        f[3] = -s * ob[0] + c * ob[1];
        f[4] = ob[2];
        f[5] = log(si.Rpar);
        f[6] = log(si.Rperp);
        f[7] = log(sj.Rpar);
        f[8] = log(sj.Rperp);
        double dl = norm3(d);
        double e[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
        const double wi = support(&si, e), wj = support(&sj, e);
        double a = si.Rpar;
        if (si.Rperp < a) a = si.Rperp;
        if (sj.Rpar < a) a = sj.Rpar;
        if (sj.Rperp < a) a = sj.Rperp;
        f[9] = asinh((dl - wi - wj) / a);
        f[10] = log(wi / si.Rperp);
        f[11] = log(wj / sj.Rperp);
    }
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static double gelu_d(double x)
{
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * ORC_PI);
}

/* wrap an angle difference to (-pi, pi] */
static double wrap_pi(double x) { return x - 2.0 * ORC_PI * floor(x / (2.0 * ORC_PI) + 0.5); }

/* The network 12 -> 128 -> 128 -> 4 with GELU: h1 = gelu(W1 x + b1),
 * h2 = gelu(W2 h1 + b2), y = W3 h2 + b3 (row-major W[out][in]).  x are the
 * standardised features.  Loss: the mean over the batch of
 *   1/2 sum_o w_o r_o^2,  r = (y0 - t0, wrap(y1 - t1), y2 - t2, wrap(y3 - t3)),
 * with per-sample weights w (all 1 if wgt is NULL).
 * Returns the loss; writes the gradients (if gW1 != NULL) and outputs (if out
 * != NULL).  nb = batch size. */
double orc_mlp_loss_grad(int64_t nb, const double *x, const double *tgt, const double *wgt, const double *W1,
                         const double *b1,
                         const double *W2, const double *b2, const double *W3, const double *b3, double *gW1,
                         double *gb1, double *gW2, double *gb2, double *gW3, double *gb3, double *out)
{
    enum { NI = 12, NH = 128, NO = 4 };
    if (gW1) {
        memset(gW1, 0, sizeof(double) * NH * NI);
        memset(gb1, 0, sizeof(double) * NH);
        memset(gW2, 0, sizeof(double) * NH * NH);
        memset(gb2, 0, sizeof(double) * NH);
        memset(gW3, 0, sizeof(double) * NO * NH);
        memset(gb3, 0, sizeof(double) * NO);
    }
    double loss = 0.0;
    for (int64_t s = 0; s < nb; ++s) {
        const double *xs = x + NI * s;
        double z1[NH], h1[NH], z2[NH], h2[NH], y[NO];
        for (int o = 0; o < NH; ++o) {
            double a = b1[o];
            for (int k = 0; k < NI; ++k) a += W1[o * NI + k] * xs[k];
            z1[o] = a;
            h1[o] = gelu(a);
        }
        for (int o = 0; o < NH; ++o) {
            double a = b2[o];
            for (int k = 0; k < NH; ++k) a += W2[o * NH + k] * h1[k];
            z2[o] = a;
            h2[o] = gelu(a);
        }
        for (int o = 0; o < NO; ++o) {
            double a = b3[o];
            for (int k = 0; k < NH; ++k) a += W3[o * NH + k] * h2[k];
            y[o] = a;
        }
        if (out)
            for (int o = 0; o < NO; ++o) out[NO * s + o] = y[o];
        const double *t = tgt + NO * s;
        double r[NO] = {y[0] - t[0], wrap_pi(y[1] - t[1]), y[2] - t[2], wrap_pi(y[3] - t[3])};
        double w[NO] = {1.0, 1.0, 1.0, 1.0};
        if (wgt)
            for (int o = 0; o < NO; ++o) w[o] = wgt[NO * s + o];
        for (int o = 0; o < NO; ++o) loss += 0.5 * w[o] * r[o] * r[o];
        if (!gW1) continue;
        /* backward (d loss / d y = w r / nb) */
        double dy[NO], dh2[NH], dz2[NH], dh1[NH], dz1[NH];
        for (int o = 0; o < NO; ++o) dy[o] = w[o] * r[o] / (double)nb;
        for (int o = 0; o < NO; ++o) {
            gb3[o] += dy[o];
            for (int k = 0; k < NH; ++k) gW3[o * NH + k] += dy[o] * h2[k];
        }
        for (int k = 0; k < NH; ++k) {
            double a = 0.0;
            for (int o = 0; o < NO; ++o) a += W3[o * NH + k] * dy[o];
            dh2[k] = a;
            dz2[k] = a * gelu_d(z2[k]);
        }
        for (int o = 0; o < NH; ++o) {
            gb2[o] += dz2[o];
            for (int k = 0; k < NH; ++k) gW2[o * NH + k] += dz2[o] * h1[k];
        }
        for (int k = 0; k < NH; ++k) {
            double a = 0.0;
            for (int o = 0; o < NH; ++o) a += W2[o * NH + k] * dz2[o];
            dh1[k] = a;
            dz1[k] = a * gelu_d(z1[k]);
        }
        for (int o = 0; o < NH; ++o) {
            gb1[o] += dz1[o];
            for (int k = 0; k < NI; ++k) gW1[o * NI + k] += dz1[o] * xs[k];
        }
    }
    return loss / (double)nb;
}

/* (p_i, q_i, p_j, q_j) of np pairs from their closest points (labels of the
 * learned warm start); out [np][4] */
void orc_pq_labels(const orc_particles *P, int64_t np, const int32_t *pi, const int32_t *pj, const double *yi,
                   const double *yj, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < np; ++k) {
        orc_surface_pq(P, pi[k], yi + 3 * k, out + 4 * k);
        orc_surface_pq(P, pj[k], yj + 3 * k, out + 4 * k + 2);
    }
}

/* Surface parameters (p, q) of the line-of-centres start: the support point
 * of i along d^ and of j along -d^ (d = r_j - r_i); out [np][4].  The network
 * learns the closest points' parameters as corrections to these; a zero
 * correction gives back the start n = d^ exactly. */
void orc_mlp_baseline(const orc_particles *P, const orc_domain *D, int64_t np, const int32_t *pi, const int32_t *pj,
                      double *out)
{
    for (int64_t k = 0; k < np; ++k) {
        shape_t si, sj;
        load_shape(P, pi[k], &si);
        load_shape(P, pj[k], &sj);
        double d[3];
        min_image(D, si.r, sj.r, d);
        double l = norm3(d);
        double e[3] = {d[0] / l, d[1] / l, d[2] / l}, me[3] = {-e[0], -e[1], -e[2]};
        double y[3];
        support_point(&si, e, y);
        orc_surface_pq(P, pi[k], y, out + 4 * k);
        support_point(&sj, me, y);
        orc_surface_pq(P, pj[k], y, out + 4 * k + 2);
    }
}

/* ------------------------------------------------------------------ */
/* Link-based lubrication of Ding and Aidun, as the paper summarises  */
/* it in Sec. II (Eq. methods:dlub), for comparison with the          */
/* contact-based corrections.  For every D3Q19 link c_r (18 nonzero   */
/* lattice vectors, c_r = 1 or sqrt 2) that ends on a site of          */
/* particle i and stems from a site of particle j, or from a fluid    */
/* site midway along 2 c_r from a site of j, a partial force on i     */
/*   df = -3 qbar mu / (2 c_r^2 lambda*) c^ (c^ . (v_bi - v_bj))        */
/*        (1 / h*^2 - 1 / c_r^2),        applied where h* < c_r,        */
/* and -df on j.  h* is the distance along the link (or pair of links) */
/* between the point where it leaves j's surface and the point where  */
/* it enters i's; v_b are the rigid-body velocities there; lambda* is */
/* the mean of the two surfaces' mean curvatures there.               */
/* Readings: lattice sites are the integer points of the box          */
/* coordinates (spacing 1); a site belongs to a particle when it lies */
/* in or on its spheroid, and to neither when it lies in both (then   */
/* it is no stem); particle j is taken at its minimum image from i; a */
/* fluid site lies in neither particle of the pair; only 0 < h* < c_r */
/* counts (h* <= 0: the surfaces overlap along the link); the forces  */
/* act at the two intersection points (torques about the centres);    */
/* walls give nothing.  Brute force: every site of i's bounding box,  */
/* every link.                                                         */
/* ------------------------------------------------------------------ */
static int in_spheroid(const shape_t *s, const double x[3])
{
    double u[3] = {x[0] - s->r[0], x[1] - s->r[1], x[2] - s->r[2]}, b[3];
    to_body(s, u, b);
    double a2 = s->Rperp * s->Rperp, c2 = s->Rpar * s->Rpar;
    return b[0] * b[0] / a2 + b[1] * b[1] / a2 + b[2] * b[2] / c2 <= 1.0;
}

/* the line x0 + t e (|e| = 1) meets the spheroid's surface at t_lo <= t_hi;
   returns 0 when it misses */
static int line_surface(const shape_t *s, const double x0[3], const double e[3], double *t_lo, double *t_hi)
{
    double u[3] = {x0[0] - s->r[0], x0[1] - s->r[1], x0[2] - s->r[2]}, ub[3], eb[3];
    to_body(s, u, ub);
    to_body(s, e, eb);
    double R2[3] = {s->Rperp * s->Rperp, s->Rperp * s->Rperp, s->Rpar * s->Rpar};
    double A = 0.0, B = 0.0, C = -1.0;
    for (int k = 0; k < 3; ++k) {
        A += eb[k] * eb[k] / R2[k];
        B += 2.0 * ub[k] * eb[k] / R2[k];
        C += ub[k] * ub[k] / R2[k];
    }
    double disc = B * B - 4.0 * A * C;
    if (disc < 0.0) return 0;
    double sq = sqrt(disc);
    *t_lo = (-B - sq) / (2.0 * A);
    *t_hi = (-B + sq) / (2.0 * A);
    return 1;
}

/* mean curvature (1/S1 + 1/S2) / 2 at the surface point y (radii of
   curvature of Eq. lub:curvature-radii) */
static double mean_curvature(const shape_t *s, const double y[3])
{
    double rel[3] = {y[0] - s->r[0], y[1] - s->r[1], y[2] - s->r[2]}, yb[3];
    to_body(s, rel, yb);
    double Rp = s->Rpar, Rq = s->Rperp;
    double p = atan2(yb[2] / Rp, sqrt(yb[0] * yb[0] + yb[1] * yb[1]) / Rq);
    double sp = sin(p), cp = cos(p);
    double s1 = sqrt(Rq * Rq * sp * sp + Rp * Rp * cp * cp);
    double S1 = s1 * s1 * s1 / (Rp * Rq), S2 = Rq * s1 / Rp;
    return 0.5 * (1.0 / S1 + 1.0 / S2);
}

static const int orc_d3q19[18][3] = {{1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                                     {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1},
                                     {1, 0, -1}, {-1, 0, 1},  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

/* one pair: force on i F[3], torques on i and j about their centres T[6],
   number of contributing links */
static int links_one(const orc_particles *P, const orc_domain *D, double mu, double qbar, int32_t i, int32_t j,
                     double F[3], double T[6])
{
    for (int k = 0; k < 3; ++k) F[k] = 0.0;
    for (int k = 0; k < 6; ++k) T[k] = 0.0;
    if (j < 0 || i < 0 || i >= P->n || j >= P->n || i == j) return 0;
    shape_t si, sj;
    load_shape(P, i, &si);
    load_shape(P, j, &sj);
    double d[3];
    min_image(D, si.r, sj.r, d);
    for (int k = 0; k < 3; ++k) sj.r[k] = si.r[k] + d[k];
    const double vi[3] = {P->vx[i], P->vy[i], P->vz[i]}, wi[3] = {P->wx[i], P->wy[i], P->wz[i]};
    const double vj[3] = {P->vx[j], P->vy[j], P->vz[j]}, wj[3] = {P->wx[j], P->wy[j], P->wz[j]};
    int64_t lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        double ek[3] = {0.0, 0.0, 0.0};
        ek[k] = 1.0;
        double w = support(&si, ek);
        lo[k] = (int64_t)ceil(si.r[k] - w);
        hi[k] = (int64_t)floor(si.r[k] + w);
    }
    int nlinks = 0;
    for (int64_t a = lo[0]; a <= hi[0]; ++a)
        for (int64_t b = lo[1]; b <= hi[1]; ++b)
            for (int64_t c = lo[2]; c <= hi[2]; ++c) {
                double x[3] = {(double)a, (double)b, (double)c};
                if (!in_spheroid(&si, x)) continue;
                for (int r = 0; r < 18; ++r) {
                    const double cv[3] = {(double)orc_d3q19[r][0], (double)orc_d3q19[r][1],
                                          (double)orc_d3q19[r][2]};
                    double y1[3] = {x[0] - cv[0], x[1] - cv[1], x[2] - cv[2]};
                    double y2[3] = {x[0] - 2.0 * cv[0], x[1] - 2.0 * cv[1], x[2] - 2.0 * cv[2]};
                    int kind = 0;
                    const int y1i = in_spheroid(&si, y1), y1j = in_spheroid(&sj, y1);
                    if (y1j && !y1i)
                        kind = 1;
                    else if (!y1j && !y1i && in_spheroid(&sj, y2) && !in_spheroid(&si, y2))
                        kind = 2;
                    if (!kind) continue;
                    const double cr = norm3(cv);
                    const double e[3] = {cv[0] / cr, cv[1] / cr, cv[2] / cr};
                    const double *x0 = kind == 1 ? y1 : y2;
                    double tjl, tjh, til, tih;
                    if (!line_surface(&sj, x0, e, &tjl, &tjh) || !line_surface(&si, x0, e, &til, &tih)) continue;
                    const double hstar = til - tjh;
                    if (!(hstar > 0.0 && hstar < cr)) continue;
                    double pi_[3], pj_[3];
                    for (int k = 0; k < 3; ++k) {
                        pi_[k] = x0[k] + til * e[k];
                        pj_[k] = x0[k] + tjh * e[k];
                    }
                    double ri[3] = {pi_[0] - si.r[0], pi_[1] - si.r[1], pi_[2] - si.r[2]};
                    double rj[3] = {pj_[0] - sj.r[0], pj_[1] - sj.r[1], pj_[2] - sj.r[2]};
                    double wri[3], wrj[3];
                    cross3(wi, ri, wri);
                    cross3(wj, rj, wrj);
                    double dv[3];
                    for (int k = 0; k < 3; ++k) dv[k] = (vi[k] + wri[k]) - (vj[k] + wrj[k]);
                    const double lam = 0.5 * (mean_curvature(&si, pi_) + mean_curvature(&sj, pj_));
                    const double coef =
                        -3.0 * qbar * mu / (2.0 * cr * cr * lam) * (1.0 / (hstar * hstar) - 1.0 / (cr * cr)) *
                        dot3(e, dv);
                    double df[3] = {coef * e[0], coef * e[1], coef * e[2]}, mdf[3] = {-df[0], -df[1], -df[2]};
                    double ti[3], tj[3];
                    cross3(ri, df, ti);
                    cross3(rj, mdf, tj);
                    for (int k = 0; k < 3; ++k) {
                        F[k] += df[k];
                        T[k] += ti[k];
                        T[3 + k] += tj[k];
                    }
                    ++nlinks;
                }
            }
    return nlinks;
}

/* per pair: force on i F[np][3], torques on i and j T[np][6], links[np] */
void orc_links(const orc_particles *P, const orc_domain *D, double mu, double qbar, int64_t np, const int32_t *pi,
               const int32_t *pj, double *F, double *T, int32_t *links)
{
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t k = 0; k < np; ++k) links[k] = links_one(P, D, mu, qbar, pi[k], pj[k], F + 3 * k, T + 6 * k);
}
