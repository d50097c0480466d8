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
