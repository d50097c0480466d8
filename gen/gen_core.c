/*
 * Seeded synthetic input generator: random sequential placement of spheroids
 * in a box, optionally attached to an already placed particle at a drawn gap.
 *
 * Input generation only.  It holds none of the lubrication method's
 * arithmetic: it draws poses, places a new particle either uniformly or in
 * contact with a parent at a requested surface gap (a particle placed so that
 * its surface point with normal -n sits at distance h along n from the
 * parent's surface point with normal n), and rejects overlaps with the
 * Perram-Wertheim contact function
 *     F = max_{0<l<1} l (1-l) d^T [(1-l) M_a + l M_b]^{-1} d,
 * which is >= 1 exactly when two ellipsoids do not overlap
 * (M = Q diag(Rperp^2, Rperp^2, Rpar^2) Q^T).  The drawn gap is a property
 * of the input distribution; expected results never come from here.
 *
 * Random numbers: xoshiro256** seeded by splitmix64, so a seed gives the
 * same draws on every machine.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GPI 3.14159265358979323846

typedef struct {
    uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t *x)
{
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t next_u64(rng_t *r)
{
    uint64_t *s = r->s;
    uint64_t res = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return res;
}

static double uni(rng_t *r) { return (double)(next_u64(r) >> 11) * (1.0 / 9007199254740992.0); }

static void rng_seed(rng_t *r, uint64_t seed)
{
    uint64_t x = seed;
    for (int k = 0; k < 4; ++k) r->s[k] = splitmix64(&x);
}

/* uniform random rotation (Shoemake), rounded to float as stored */
static void rand_quat(rng_t *r, float q[4])
{
    double u1 = uni(r), u2 = uni(r), u3 = uni(r);
    double a = sqrt(1.0 - u1), b = sqrt(u1);
    q[0] = (float)(b * cos(2.0 * GPI * u3));
    q[1] = (float)(a * sin(2.0 * GPI * u2));
    q[2] = (float)(a * cos(2.0 * GPI * u2));
    q[3] = (float)(b * sin(2.0 * GPI * u3));
}

static void rand_dir(rng_t *r, double n[3])
{
    double z = 2.0 * uni(r) - 1.0, ph = 2.0 * GPI * uni(r), s = sqrt(1.0 - z * z);
    n[0] = s * cos(ph);
    n[1] = s * sin(ph);
    n[2] = z;
}

/* M = Q diag(a2, a2, c2) Q^T from a (float) quaternion, normalised */
static void shape_matrix(const float qf[4], double a, double c, double M[3][3])
{
    double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
    double t = 2.0 / (w * w + x * x + y * y + z * z);
    double Q[3][3] = {{1.0 - t * (y * y + z * z), t * (x * y - w * z), t * (x * z + w * y)},
                      {t * (x * y + w * z), 1.0 - t * (x * x + z * z), t * (y * z - w * x)},
                      {t * (x * z - w * y), t * (y * z + w * x), 1.0 - t * (x * x + y * y)}};
    double dd[3] = {a * a, a * a, c * c};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            M[i][j] = 0.0;
            for (int k = 0; k < 3; ++k) M[i][j] += Q[i][k] * dd[k] * Q[j][k];
        }
}

static void matvec(const double M[3][3], const double v[3], double o[3])
{
    for (int i = 0; i < 3; ++i) o[i] = M[i][0] * v[0] + M[i][1] * v[1] + M[i][2] * v[2];
}

static double quad(const double M[3][3], const double v[3])
{
    double o[3];
    matvec(M, v, o);
    return v[0] * o[0] + v[1] * o[1] + v[2] * o[2];
}

/* d^T A^{-1} d for symmetric positive definite 3x3 A (Cramer) */
static double solve_quad(const double A[3][3], const double d[3])
{
    double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    double inv[3][3];
    inv[0][0] = c00 / det;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    inv[1][0] = c01 / det;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    inv[2][0] = c02 / det;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    return quad(inv, d);
}

/* Perram-Wertheim contact function (golden-section maximisation over l) */
static double pw_contact(const double Ma[3][3], const double Mb[3][3], const double d[3])
{
    double lo = 0.0, hi = 1.0;
    const double gr = 0.6180339887498949;
    double x1 = hi - gr * (hi - lo), x2 = lo + gr * (hi - lo);
    double A[3][3];
#define PWF(l, out)                                                                     \
    do {                                                                                \
        for (int i_ = 0; i_ < 3; ++i_)                                                  \
            for (int j_ = 0; j_ < 3; ++j_) A[i_][j_] = (1.0 - (l)) * Ma[i_][j_] + (l) * Mb[i_][j_]; \
        (out) = (l) * (1.0 - (l)) * solve_quad(A, d);                                   \
    } while (0)
    double f1, f2;
    PWF(x1, f1);
    PWF(x2, f2);
    for (int it = 0; it < 80; ++it) {
        if (f1 < f2) {
            lo = x1;
            x1 = x2;
            f1 = f2;
            x2 = lo + gr * (hi - lo);
            PWF(x2, f2);
        } else {
            hi = x2;
            x2 = x1;
            f2 = f1;
            x1 = hi - gr * (hi - lo);
            PWF(x1, f1);
        }
    }
#undef PWF
    return f1 > f2 ? f1 : f2;
}

/*
 * Random sequential placement.
 *   N particles with given semi-axes (r_par, r_perp, per particle, in order).
 *   Box [0,L)^3; periodic flags per axis; up to two plane walls at z = wall_z
 *   with fluid side wall_dir (+1: z > wall_z).
 *   Each particle (after the first) is, with probability attach_prob,
 *   attached to a random placed particle at a gap drawn log-uniform in
 *   [gap_lo, gap_hi]; otherwise placed uniformly.  Overlaps (PW < 1 + pw_eps)
 *   and wall contacts (gap to a wall < wall_min) are rejected.
 * Outputs x, y, z (double) and q (float, [N][4], scalar first).
 * Returns the number placed (N on success).
 */
int64_t gen_rsa(int64_t N, const double L[3], const int32_t periodic[3], int32_t n_walls,
                const double wall_z[2], const int32_t wall_dir[2], const float *r_par,
                const float *r_perp, double attach_prob, double gap_lo, double gap_hi,
                double wall_min, int64_t max_attempts, uint64_t seed, double *x, double *y,
                double *z, float *q)
{
    rng_t rng;
    rng_seed(&rng, seed);
    double rmax_all = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        double m = r_par[k] > r_perp[k] ? r_par[k] : r_perp[k];
        if (m > rmax_all) rmax_all = m;
    }
    /* cell grid for overlap candidates: cell >= 2 rmax */
    int nc[3];
    double cs[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(L[a] / (2.0 * rmax_all));
        if (nc[a] < 1) nc[a] = 1;
        if (nc[a] > 512) nc[a] = 512;
        cs[a] = L[a] / nc[a];
    }
    int64_t ncell = (int64_t)nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    double(*Ms)[3][3] = malloc(sizeof(double[3][3]) * (N > 0 ? N : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    int64_t placed = 0;
    for (int64_t k = 0; k < N; ++k) {
        double a = r_perp[k], c = r_par[k];
        double rk = a > c ? a : c;
        int ok = 0;
        for (int64_t att = 0; att < max_attempts && !ok; ++att) {
            float qk[4];
            rand_quat(&rng, qk);
            double M[3][3];
            shape_matrix(qk, a, c, M);
            double r[3];
            if (placed > 0 && uni(&rng) < attach_prob) {
                int64_t par = (int64_t)(uni(&rng) * placed);
                if (par >= placed) par = placed - 1;
                double n[3];
                rand_dir(&rng, n);
                double h = exp(log(gap_lo) + uni(&rng) * (log(gap_hi) - log(gap_lo)));
                double Mn_p[3], Mn_k[3];
                matvec(Ms[par], n, Mn_p);
                matvec(M, n, Mn_k);
                double sp = sqrt(quad(Ms[par], n)), sk = sqrt(quad(M, n));
                double rp[3] = {x[par], y[par], z[par]};
                for (int t = 0; t < 3; ++t) r[t] = rp[t] + Mn_p[t] / sp + h * n[t] + Mn_k[t] / sk;
            } else {
                for (int t = 0; t < 3; ++t) r[t] = uni(&rng) * L[t];
            }
            /* wrap periodic axes; reject outside non-periodic extent */
            int inside = 1;
            for (int t = 0; t < 3; ++t) {
                if (periodic[t])
                    r[t] -= L[t] * floor(r[t] / L[t]);
                else if (r[t] < 0.0 || r[t] >= L[t])
                    inside = 0;
            }
            if (!inside) continue;
            /* walls */
            double ez[3] = {0.0, 0.0, 1.0};
            double sz = sqrt(quad(M, ez));
            for (int w = 0; w < n_walls && inside; ++w)
                if (wall_dir[w] * (r[2] - wall_z[w]) - sz < wall_min) inside = 0;
            if (!inside) continue;
            /* overlaps with placed neighbours */
            int ci[3];
            for (int t = 0; t < 3; ++t) {
                ci[t] = (int)floor(r[t] / cs[t]);
                if (ci[t] < 0) ci[t] = 0;
                if (ci[t] >= nc[t]) ci[t] = nc[t] - 1;
            }
            int clash = 0;
            for (int dx = -1; dx <= 1 && !clash; ++dx)
                for (int dy = -1; dy <= 1 && !clash; ++dy)
                    for (int dz = -1; dz <= 1 && !clash; ++dz) {
                        int cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
                        int skip = 0;
                        for (int t = 0; t < 3; ++t) {
                            if (cc[t] < 0 || cc[t] >= nc[t]) {
                                if (periodic[t])
                                    cc[t] = (cc[t] + nc[t]) % nc[t];
                                else
                                    skip = 1;
                            }
                        }
                        if (skip) continue;
                        /* with fewer than 3 cells along an axis the same cell can
                           recur; duplicates only repeat the same test */
                        int64_t cell = ((int64_t)cc[0] * nc[1] + cc[1]) * nc[2] + cc[2];
                        for (int64_t m = head[cell]; m >= 0 && !clash; m = next[m]) {
                            double d[3] = {x[m] - r[0], y[m] - r[1], z[m] - r[2]};
                            for (int t = 0; t < 3; ++t)
                                if (periodic[t]) d[t] -= L[t] * floor(d[t] / L[t] + 0.5);
                            double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                            double rm = r_par[m] > r_perp[m] ? r_par[m] : r_perp[m];
                            if (dist >= rk + rm) continue;
                            if (dist < 1e-9) {
                                clash = 1;
                                break;
                            }
                            if (pw_contact(M, Ms[m], d) < 1.0 + 1e-12) clash = 1;
                        }
                    }
            if (clash) continue;
            x[k] = r[0];
            y[k] = r[1];
            z[k] = r[2];
            for (int t = 0; t < 4; ++t) q[4 * k + t] = qk[t];
            memcpy(Ms[k], M, sizeof(M));
            int64_t cell = ((int64_t)ci[0] * nc[1] + ci[1]) * nc[2] + ci[2];
            next[k] = head[cell];
            head[cell] = k;
            ok = 1;
        }
        if (!ok) break;
        placed = k + 1;
    }
    free(head);
    free(next);
    free(Ms);
    return placed;
}

/* ---------------------------------------------------------------------------
 * Growth packing, for suspensions denser than random sequential placement
 * reaches (it jams near Phi = 0.4 for these spheroids).  The particles start
 * at a fraction s0 of their linear size, placed one by one at random (easy at
 * that size), and grow: every step multiplies all sizes by (1 + g), then
 * relaxation sweeps push overlapping particles apart, with walls, by a
 * Hookean repulsion proportional to the overlap depth acting at the contact
 * point, in the overdamped limit of damped motion (the displacement and the
 * rotation of a sweep are proportional to the summed force and torque; no
 * inertia, no velocities kept).  The growth goes on to s_over slightly above
 * 1; there the sweeps continue until nothing overlaps, and the sizes are
 * reset to 1, which leaves every gap at least about (s_over - 1) times the
 * particle sizes.  g adapts: it grows while the sweeps keep the overlaps
 * small and shrinks when they do not.
 *
 * Overlap from the Perram-Wertheim contact function of the scaled shapes,
 * F(l) = l (1 - l) d^T G(l)^{-1} d, G(l) = (1 - l) A + l B, maximised over
 * l in (0, 1) (concave: Newton on F'(l) = 0, bisection safeguard): the bodies
 * overlap exactly when F < 1, the depth along the centre line is
 * |d| (1/sqrt(F) - 1) (exact for spheres), and at the maximiser the contact
 * point is r_i + (1 - l) A x with x = G^{-1} d, where both surfaces have
 * normal x / |x| (from i towards j).
 *
 * Deterministic: every sweep computes all pushes from the positions of the
 * sweep before (Jacobi), each particle summing over its neighbours in a fixed
 * order, so the result does not depend on the number of threads.
 * ------------------------------------------------------------------------- */

/* x = G^{-1} d for symmetric positive definite G (Cramer); returns d.x */
static double solve3(const double G[3][3], const double d[3], double x[3])
{
    double c00 = G[1][1] * G[2][2] - G[1][2] * G[2][1];
    double c01 = G[1][2] * G[2][0] - G[1][0] * G[2][2];
    double c02 = G[1][0] * G[2][1] - G[1][1] * G[2][0];
    double det = G[0][0] * c00 + G[0][1] * c01 + G[0][2] * c02;
    double inv[3][3];
    inv[0][0] = c00;
    inv[0][1] = G[0][2] * G[2][1] - G[0][1] * G[2][2];
    inv[0][2] = G[0][1] * G[1][2] - G[0][2] * G[1][1];
    inv[1][0] = c01;
    inv[1][1] = G[0][0] * G[2][2] - G[0][2] * G[2][0];
    inv[1][2] = G[0][2] * G[1][0] - G[0][0] * G[1][2];
    inv[2][0] = c02;
    inv[2][1] = G[0][1] * G[2][0] - G[0][0] * G[2][1];
    inv[2][2] = G[0][0] * G[1][1] - G[0][1] * G[1][0];
    for (int i = 0; i < 3; ++i) x[i] = (inv[i][0] * d[0] + inv[i][1] * d[1] + inv[i][2] * d[2]) / det;
    return d[0] * x[0] + d[1] * x[1] + d[2] * x[2];
}

/* PW maximisation; returns F, sets l and x = G(l)^{-1} d */
static double pw_newton(const double A[3][3], const double B[3][3], const double d[3], double *lam, double x[3])
{
    double BA[3][3], G[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) BA[i][j] = B[i][j] - A[i][j];
    double lo = 0.0, hi = 1.0, l = 0.5, F = 0.0;
    for (int it = 0; it < 30; ++it) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) G[i][j] = A[i][j] + l * BA[i][j];
        const double dx = solve3(G, d, x);
        double Bx[3], y[3];
        matvec(BA, x, Bx);
        const double xBx = x[0] * Bx[0] + x[1] * Bx[1] + x[2] * Bx[2];
        solve3(G, Bx, y); /* y = G^{-1} (B - A) x */
        const double yBx = y[0] * Bx[0] + y[1] * Bx[1] + y[2] * Bx[2];
        F = l * (1.0 - l) * dx;
        const double F1 = (1.0 - 2.0 * l) * dx - l * (1.0 - l) * xBx;
        const double F2 = -2.0 * dx - 2.0 * (1.0 - 2.0 * l) * xBx + 2.0 * l * (1.0 - l) * yBx;
        if (F1 > 0.0) lo = l; else hi = l;
        double ln = (F2 < 0.0) ? l - F1 / F2 : 0.5 * (lo + hi);
        if (!(ln > lo && ln < hi)) ln = 0.5 * (lo + hi);
        if (fabs(ln - l) < 1e-12 || hi - lo < 1e-12) {
            l = ln;
            break;
        }
        l = ln;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G[i][j] = A[i][j] + l * BA[i][j];
    F = l * (1.0 - l) * solve3(G, d, x);
    *lam = l;
    return F;
}

typedef struct {
    int nc[3];
    double cs[3];
    int64_t *head, *next;
} grid_t;

static void grid_fill(grid_t *g, int64_t N, const double *pos, const double L[3], double range)
{
    for (int a = 0; a < 3; ++a) {
        g->nc[a] = (int)floor(L[a] / range);
        if (g->nc[a] < 1) g->nc[a] = 1;
        if (g->nc[a] > 256) g->nc[a] = 256;
        g->cs[a] = L[a] / g->nc[a];
    }
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    for (int64_t c = 0; c < ncell; ++c) g->head[c] = -1;
    for (int64_t k = N - 1; k >= 0; --k) {
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            ci[a] = (int)floor(pos[3 * k + a] / g->cs[a]);
            if (ci[a] < 0) ci[a] = 0;
            if (ci[a] >= g->nc[a]) ci[a] = g->nc[a] - 1;
        }
        int64_t c = ((int64_t)ci[0] * g->nc[1] + ci[1]) * g->nc[2] + ci[2];
        g->next[k] = g->head[c];
        g->head[c] = k;
    }
}

static double maxd(double a, double b) { return a > b ? a : b; }

/* pairs are pushed apart while their gap is below this fraction of the
   smaller semi-axes (so that the sweeps end with no overlap left, instead of
   approaching contact from the overlapping side) */
#define GROW_SKIN 1e-3
/* growth continues while the deepest overlap after a sweep stays below this
   fraction of the smaller semi-axis, and slows down above three times it */
#define GROW_LOOSE 0.1

/* one relaxation sweep at scale s: pushes from the current state into dr, dth;
   returns the largest overlap depth relative to the particle sizes */
static double grow_sweep(int64_t N, const double L[3], const int32_t periodic[3], int32_t n_walls,
                         const double wall_z[2], const int32_t wall_dir[2], const float *r_par, const float *r_perp,
                         double s, const double *pos, double (*M)[3][3], const grid_t *g, double *dr, double *dth,
                         int64_t *n_over)
{
    double worst = 0.0;
    int64_t over = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(max : worst) reduction(+ : over)
    for (int64_t i = 0; i < N; ++i) {
        const double ri = maxd(r_par[i], r_perp[i]), rmin = r_par[i] < r_perp[i] ? r_par[i] : r_perp[i];
        double A[3][3], f[3] = {0, 0, 0}, t[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) A[a][b] = s * s * M[i][a][b];
        int ci[3];
        for (int a = 0; a < 3; ++a) {
            ci[a] = (int)floor(pos[3 * i + a] / g->cs[a]);
            if (ci[a] < 0) ci[a] = 0;
            if (ci[a] >= g->nc[a]) ci[a] = g->nc[a] - 1;
        }
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    int cc[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz}, skip = 0;
                    for (int a = 0; a < 3; ++a)
                        if (cc[a] < 0 || cc[a] >= g->nc[a]) {
                            if (periodic[a]) cc[a] = (cc[a] + g->nc[a]) % g->nc[a];
                            else skip = 1;
                        }
                    if (skip) continue;
                    /* a cell met twice (fewer than 3 cells along an axis) is tested once */
                    int dup = 0;
                    const int small = g->nc[0] < 3 || g->nc[1] < 3 || g->nc[2] < 3;
                    for (int ex = -1; small && ex <= dx && !dup; ++ex)
                        for (int ey = -1; ey <= 1 && !dup; ++ey)
                            for (int ez = -1; ez <= 1 && !dup; ++ez) {
                                if (ex == dx && (ey > dy || (ey == dy && ez >= dz))) continue;
                                int ee[3] = {ci[0] + ex, ci[1] + ey, ci[2] + ez}, sk = 0;
                                for (int a = 0; a < 3; ++a)
                                    if (ee[a] < 0 || ee[a] >= g->nc[a]) {
                                        if (periodic[a]) ee[a] = (ee[a] + g->nc[a]) % g->nc[a];
                                        else sk = 1;
                                    }
                                if (!sk && ee[0] == cc[0] && ee[1] == cc[1] && ee[2] == cc[2]) dup = 1;
                            }
                    if (dup) continue;
                    int64_t cell = ((int64_t)cc[0] * g->nc[1] + cc[1]) * g->nc[2] + cc[2];
                    for (int64_t j = g->head[cell]; j >= 0; j = g->next[j]) {
                        if (j == i) continue;
                        double d[3];
                        for (int a = 0; a < 3; ++a) {
                            d[a] = pos[3 * j + a] - pos[3 * i + a];
                            if (periodic[a]) d[a] -= L[a] * floor(d[a] / L[a] + 0.5);
                        }
                        const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        const double rj = maxd(r_par[j], r_perp[j]);
                        const double rminj = r_par[j] < r_perp[j] ? r_par[j] : r_perp[j];
                        const double skin = GROW_SKIN * s * 0.5 * (rmin + rminj);
                        if (dist >= s * (ri + rj) + skin) continue;
                        double B[3][3];
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) B[a][b] = s * s * M[j][a][b];
                        if (dist > 0.0) {
                            /* half-widths along the centre line: no overlap when they fit */
                            const double e[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
                            if (dist > sqrt(quad(A, e)) + sqrt(quad(B, e)) + skin) continue;
                        }
                        double lam, x[3], n[3];
                        double depth, Fpw;
                        if (dist > 0.0) {
                            Fpw = pw_newton(A, B, d, &lam, x);
                            const double h = dist * (1.0 - 1.0 / sqrt(Fpw));  /* gap estimate */
                            if (h >= skin) continue;
                            if (h < 0.0) ++over;
                            depth = skin - h;
                        } else {
                            ++over;
                            lam = 0.5;
                            x[0] = 1.0; x[1] = 0.0; x[2] = 0.0;
                            depth = s * (ri + rj);
                        }
                        const double xn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
                        for (int a = 0; a < 3; ++a) n[a] = x[a] / xn;
                        double rho[3];
                        matvec(A, x, rho);
                        for (int a = 0; a < 3; ++a) rho[a] *= (1.0 - lam);
                        /* push on i: half the depth, away from j, at the contact point */
                        const double pf[3] = {-0.5 * depth * n[0], -0.5 * depth * n[1], -0.5 * depth * n[2]};
                        for (int a = 0; a < 3; ++a) f[a] += pf[a];
                        t[0] += rho[1] * pf[2] - rho[2] * pf[1];
                        t[1] += rho[2] * pf[0] - rho[0] * pf[2];
                        t[2] += rho[0] * pf[1] - rho[1] * pf[0];
                        const double rel = depth / (s * rmin);
                        if (rel > worst) worst = rel;
                    }
                }
        /* walls: the support extent of the scaled body along z */
        for (int w = 0; w < n_walls; ++w) {
            const double ez[3] = {0.0, 0.0, 1.0};
            const double sz = sqrt(quad(A, ez));
            const double skin = GROW_SKIN * s * rmin;
            const double hw = wall_dir[w] * (pos[3 * i + 2] - wall_z[w]) - sz - skin;
            if (hw >= 0.0) continue;
            if (hw + skin < 0.0) ++over;
            double Mz[3];
            matvec(A, ez, Mz);
            const double rho[3] = {-wall_dir[w] * Mz[0] / sz, -wall_dir[w] * Mz[1] / sz, -wall_dir[w] * Mz[2] / sz};
            const double pf[3] = {0.0, 0.0, -hw * wall_dir[w]};
            f[2] += pf[2];
            t[0] += rho[1] * pf[2];
            t[1] += -rho[0] * pf[2];
            const double rel = -hw / (s * rmin);
            if (rel > worst) worst = rel;
        }
        /* overdamped response, under-relaxed and clamped (several contacts at once) */
        double fl = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        const double cap = 0.1 * s * rmin, c1 = fl * 0.6 > cap ? cap / fl : 0.6;
        for (int a = 0; a < 3; ++a) dr[3 * i + a] = c1 * f[a];
        const double ir2 = 1.0 / (s * s * ri * ri);
        double tl = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]) * 0.3 * ir2;
        const double c2 = tl > 0.05 ? 0.05 / tl : 1.0;
        for (int a = 0; a < 3; ++a) dth[3 * i + a] = c2 * 0.3 * ir2 * t[a];
    }
    *n_over = over;
    return worst;
}

/*
 * Returns the number of particles (N) on success; -1 when the first
 * placement at s0 stalls; -2 - k when k pairs or wall contacts still overlap
 * after max_sweeps.  Outputs x, y, z (double) and q ([N][4] float, scalar
 * first); *sweeps_out = relaxation sweeps used.
 */
int64_t gen_grow(int64_t N, const double L[3], const int32_t periodic[3], int32_t n_walls, const double wall_z[2],
                 const int32_t wall_dir[2], const float *r_par, const float *r_perp, double s0, double s_over,
                 double g0, int64_t max_sweeps, uint64_t seed, double *x, double *y, double *z, float *q,
                 int64_t *sweeps_out)
{
    if (N <= 0) return 0;
    float *sp = (float *)malloc(sizeof(float) * N), *sq = (float *)malloc(sizeof(float) * N);
    double rmax = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        sp[k] = (float)(s0 * r_par[k]);
        sq[k] = (float)(s0 * r_perp[k]);
        rmax = maxd(rmax, maxd(r_par[k], r_perp[k]));
    }
    /* walls: keep centres at least a full-size half-width away while placing */
    const int64_t placed = gen_rsa(N, L, periodic, n_walls, wall_z, wall_dir, sp, sq, 0.0, 1e-4, 1.0, 0.0, 100000,
                                   seed, x, y, z, q);
    free(sp);
    free(sq);
    if (placed != N) return -1;
    double *pos = (double *)malloc(sizeof(double) * 3 * N), *dr = (double *)malloc(sizeof(double) * 3 * N),
           *dth = (double *)malloc(sizeof(double) * 3 * N), *qd = (double *)malloc(sizeof(double) * 4 * N);
    double(*M)[3][3] = malloc(sizeof(double[3][3]) * N);
    grid_t gr;
    int64_t ncell_max = 1;
    for (int a = 0; a < 3; ++a) {
        int nc = (int)floor(L[a] / (2.0 * s0 * rmax));
        ncell_max *= nc < 1 ? 1 : (nc > 256 ? 256 : nc);
    }
    gr.head = (int64_t *)malloc(sizeof(int64_t) * ncell_max);
    gr.next = (int64_t *)malloc(sizeof(int64_t) * N);
    for (int64_t k = 0; k < N; ++k) {
        pos[3 * k] = x[k];
        pos[3 * k + 1] = y[k];
        pos[3 * k + 2] = z[k];
        for (int a = 0; a < 4; ++a) qd[4 * k + a] = q[4 * k + a];
    }
    double s = s0, g = g0;
    int64_t sweeps = 0, n_over = 0;
    int done = 0;
    while (!done && sweeps < max_sweeps) {
        const int at_top = s >= s_over;
        /* shape matrices from the current orientations, cells for range 2 s Rmax */
        for (int64_t k = 0; k < N; ++k) {
            double w = qd[4 * k], a = qd[4 * k + 1], b = qd[4 * k + 2], c = qd[4 * k + 3];
            double t = 2.0 / (w * w + a * a + b * b + c * c);
            double Q[3][3] = {{1.0 - t * (b * b + c * c), t * (a * b - w * c), t * (a * c + w * b)},
                              {t * (a * b + w * c), 1.0 - t * (a * a + c * c), t * (b * c - w * a)},
                              {t * (a * c - w * b), t * (b * c + w * a), 1.0 - t * (a * a + b * b)}};
            double dd[3] = {(double)r_perp[k] * r_perp[k], (double)r_perp[k] * r_perp[k], (double)r_par[k] * r_par[k]};
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    M[k][i][j] = 0.0;
                    for (int m = 0; m < 3; ++m) M[k][i][j] += Q[i][m] * dd[m] * Q[j][m];
                }
        }
        grid_fill(&gr, N, pos, L, 2.0 * s * rmax * 1.0000001);
        const double worst = grow_sweep(N, L, periodic, n_walls, wall_z, wall_dir, r_par, r_perp, s, pos, M, &gr, dr,
                                        dth, &n_over);
        ++sweeps;
        if (at_top && n_over == 0) {
            done = 1;
            break;
        }
        /* apply the pushes */
        for (int64_t k = 0; k < N; ++k) {
            for (int a = 0; a < 3; ++a) {
                double v = pos[3 * k + a] + dr[3 * k + a];
                if (periodic[a]) v -= L[a] * floor(v / L[a]);
                else if (v < 0.0) v = 0.0;
                else if (v >= L[a]) v = L[a] * (1.0 - 1e-12);
                pos[3 * k + a] = v;
            }
            const double th[3] = {dth[3 * k], dth[3 * k + 1], dth[3 * k + 2]};
            const double ang = sqrt(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
            if (ang > 0.0) {
                const double cs = cos(0.5 * ang), sn = sin(0.5 * ang) / ang;
                const double r0 = cs, r1 = sn * th[0], r2 = sn * th[1], r3 = sn * th[2];
                const double q0 = qd[4 * k], q1 = qd[4 * k + 1], q2 = qd[4 * k + 2], q3 = qd[4 * k + 3];
                double n0 = r0 * q0 - r1 * q1 - r2 * q2 - r3 * q3, n1 = r0 * q1 + r1 * q0 + r2 * q3 - r3 * q2;
                double n2 = r0 * q2 - r1 * q3 + r2 * q0 + r3 * q1, n3 = r0 * q3 + r1 * q2 - r2 * q1 + r3 * q0;
                const double nn = 1.0 / sqrt(n0 * n0 + n1 * n1 + n2 * n2 + n3 * n3);
                qd[4 * k] = n0 * nn;
                qd[4 * k + 1] = n1 * nn;
                qd[4 * k + 2] = n2 * nn;
                qd[4 * k + 3] = n3 * nn;
            }
        }
        /* grow while the overlaps stay small */
        if (!at_top) {
            if (worst < GROW_LOOSE) {
                s *= 1.0 + g;
                if (s > s_over) s = s_over;
                g = g * 1.25 > 0.02 ? 0.02 : g * 1.25;
            } else if (worst > 3 * GROW_LOOSE) {
                g = g * 0.5 < 1e-4 ? 1e-4 : g * 0.5;
            }
        }
    }
    for (int64_t k = 0; k < N; ++k) {
        x[k] = pos[3 * k];
        y[k] = pos[3 * k + 1];
        z[k] = pos[3 * k + 2];
        for (int a = 0; a < 4; ++a) q[4 * k + a] = (float)qd[4 * k + a];
    }
    free(pos);
    free(dr);
    free(dth);
    free(qd);
    free(M);
    free(gr.head);
    free(gr.next);
    if (sweeps_out) *sweeps_out = sweeps;
    return done ? N : -2 - n_over;
}
