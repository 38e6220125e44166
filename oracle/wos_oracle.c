/*
 * wos_oracle.c -- plain FP64 CPU oracle of the extended Walk-on-Spheres toolbox build.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that
 * the CUDA path is checked against.  Only the tests, the smoke check and the timed
 * CPU baseline of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it computes (paper: "Extended Walk-on-Spheres Algorithm for Linear and
 * Nonlinear Elliptic Problems of Divergence-type"):
 *   - the WoS chain X_{k+1} = X_k + r(X_k) U_k                        (Sec. 2.1, eq. wos chain)
 *   - the matrix estimators A, B^(j), H, K^(j)                         (Sec. 2.3, eqs.
 *     Estimator_A, Estimator_B, Estimator_H, Estimator_K), fused per walk as in Algorithm 5,
 *     with the singular terms replaced by the samplers of Prop. 2.6 / Rem. 2.8:
 *       * d = 2 Green density: R = F^{-1}(u), F(t) = t^2 - t^2 ln t^2   (Prop. 2.6 (i.1))
 *       * d = 3 Green density: R = median of three uniforms ~ Beta(2,2) (Prop. 2.6 (i.2))
 *       * ball term: S = 1 - sqrt(u), weight sum_{k<d} S^k             (Prop. 2.6 (ii))
 *   - the Voronoi binning by nearest centre, ties to the lowest index (Sec. 2.3, "Example:
 *     Voronoi diagrams"), here by brute force over all centres.
 *
 * Readings of the paper taken here (each is listed in the design notes of the repository):
 *   - G := A/2 and gradG := B/2, so G is the inverse of -Laplace (G 1 = (1-|x|^2)/(2d) on
 *     the unit ball); H and gradH := K are unchanged.
 *   - the walk stops at the first X_k with r(X_k) < eps (eps-shell), or after max_steps
 *     work steps; the stopping point is binned into the boundary cells without projection
 *     (the boundary cells partition the closure of D).
 *   - a fresh source point Y is drawn at every step; the direction U_k and Y are drawn
 *     independently per (node, walk, step) from Philox4x32-10.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random
 * numbers: as easy as 1, 2, 3"), key = (seed_lo, seed_hi), counter =
 * (walk l, step k, node i, tag<<24 | instance<<8 | slot); uniform u = ((x>>9)+0.5)/2^23.
 * Step k >= 0 (k = 0 at x_i): d = 2 slot 0 = (radius of Y, angle of Y, angle of U, -);
 * d = 3 slot 0 = (three uniforms of the median, z of Y), slot 1 = (phi of Y, z of U, phi of U, -).
 * Ball term: step word 0xFFFFFFFF, slot 0 = (S, angle / z, phi, -).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- Philox4x32-10 */
static void orc_philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        orc_philox_round(c, k0, k1);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

double oracle_u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* ---------------------------------------------------------------- samplers (Prop. 2.6) */
/* d = 2: radius R with CDF F(t) = t^2 - t^2 ln t^2 (proof of Prop. 2.6 (i.1)).
 * Write t^2 = e^{-L}; then F = (1+L) e^{-L} = u, i.e. g(L) = log1p(L) - L + a = 0 with
 * a = -ln u.  g is decreasing on L >= 0, g(a) >= 0 and g(a + sqrt(2a)) <= 0 (because
 * 1 + t + t^2/2 <= e^t), so plain bisection on [a, a + sqrt(2a)] gives L to full precision.
 * This equals R = exp((1 + W_{-1}(-u/e))/2) of Prop. 2.6 (i.1) with L = -(1 + W_{-1}). */
double oracle_green_radius_2d(double u) {
    double a = -log(u);
    double lo = a, hi = a + sqrt(2.0 * a);
    for (int it = 0; it < 200 && hi > lo; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double g = log1p(mid) - mid + a;
        if (g > 0.0) lo = mid; else hi = mid;
    }
    return exp(-0.25 * (lo + hi));
}

static double orc_med3(double a, double b, double c) {
    double mn = a < b ? a : b, mx = a < b ? b : a;
    double t = mx < c ? mx : c;
    return mn > t ? mn : t;
}

static void orc_dir2(double u, double out[2]) {
    double th = 2.0 * ORC_PI * u;
    out[0] = cos(th); out[1] = sin(th);
}

static void orc_dir3(double uz, double uphi, double out[3]) {
    double z = 1.0 - 2.0 * uz;
    double rho = sqrt(fmax(0.0, 1.0 - z * z));
    double ph = 2.0 * ORC_PI * uphi;
    out[0] = rho * cos(ph); out[1] = rho * sin(ph); out[2] = z;
}

/* ---------------------------------------------------------------- distance to the boundary */
/* r(x) of eq. (r).  kind 0: ball, params = centre (d), radius.  kind 1: box, params = lo (d),
 * hi (d).  kind 2: closed polygon (d = 2), params = vertices x0,y0,x1,y1,...: the distance to
 * the nearest edge, with the sign of an even-odd inside test (Rem. 2.14 (i) allows any
 * such distance). */
static double orc_sdf(int dim, int kind, const double* prm, int64_t nprm, const double* x) {
    if (kind == 0) {
        double s = 0.0;
        for (int c = 0; c < dim; ++c) { double t = x[c] - prm[c]; s += t * t; }
        return prm[dim] - sqrt(s);
    } else if (kind == 1) {
        double r = INFINITY;
        for (int c = 0; c < dim; ++c) {
            double a = x[c] - prm[c], b = prm[dim + c] - x[c];
            if (a < r) r = a;
            if (b < r) r = b;
        }
        return r;
    } else {
        /* signed: positive inside (crossing-number test), negative outside */
        int64_t nv = nprm / 2;
        double best = INFINITY;
        int inside = 0;
        for (int64_t e = 0; e < nv; ++e) {
            double ax = prm[2 * e], ay = prm[2 * e + 1];
            int64_t f = (e + 1 == nv) ? 0 : e + 1;
            double bx = prm[2 * f], by = prm[2 * f + 1];
            double ex = bx - ax, ey = by - ay, px = x[0] - ax, py = x[1] - ay;
            double ee = ex * ex + ey * ey;
            double t = ee > 0.0 ? (px * ex + py * ey) / ee : 0.0;
            if (t < 0.0) t = 0.0;
            if (t > 1.0) t = 1.0;
            double dx = px - t * ex, dy = py - t * ey;
            double d2 = dx * dx + dy * dy;
            if (d2 < best) best = d2;
            if ((ay > x[1]) != (by > x[1])) {
                double xc = ax + (x[1] - ay) / (by - ay) * (bx - ax);
                if (x[0] < xc) inside = !inside;
            }
        }
        return inside ? sqrt(best) : -sqrt(best);
    }
}

double oracle_sdf(int dim, int kind, const double* prm, int64_t nprm, const double* x) {
    return orc_sdf(dim, kind, prm, nprm, x);
}

/* nearest centre, ties to the lowest index (Voronoi cells of Sec. 2.3) */
static int64_t orc_nearest(int dim, const double* q, const double* pts, int64_t np) {
    int64_t bj = 0;
    double best = INFINITY;
    for (int64_t j = 0; j < np; ++j) {
        double s = 0.0;
        for (int c = 0; c < dim; ++c) { double t = q[c] - pts[j * dim + c]; s += t * t; }
        if (s < best) { best = s; bj = j; }
    }
    return bj;
}

int64_t oracle_nearest(int dim, const double* q, const double* pts, int64_t np) {
    return orc_nearest(dim, q, pts, np);
}

/* digest of one interior binning for the per-walk records: Vigna's SplitMix64 output
 * function applied to (tag << 32 | cell), folded to 32 bits */
static uint32_t orc_cellmix(uint32_t tag, uint32_t cell) {
    uint64_t z = ((uint64_t)tag << 32) | (uint64_t)cell;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z = z ^ (z >> 31);
    return (uint32_t)(z ^ (z >> 32));
}

void oracle_philox_batch(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, int64_t count) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < count; ++t) oracle_philox4x32_10(ctr + 4 * t, key, out + 4 * t);
}

/* ---------------------------------------------------------------- toolbox rows */
typedef struct {
    int dim, sdf_kind;
    const double* sdf_params; int64_t n_sdf_params;
    const double* x; int64_t n;      /* W centres (walk starts), n x dim */
    const double* y; int64_t m;      /* V centres, m x dim */
    const double* z; int64_t p;      /* boundary centres, p x dim */
    int64_t walks;                   /* N */
    double eps;
    uint64_t seed;
    int64_t max_steps;
    uint32_t instance;
} oracle_spec;

static void orc_draw(const oracle_spec* s, uint32_t l, uint32_t k, uint32_t i, uint32_t slot,
                     double u[4]) {
    uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
    uint32_t ctr[4] = {l, k, i, ((s->instance & 0xFFFFu) << 8) | slot};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    for (int c = 0; c < 4; ++c) u[c] = oracle_u01(out[c]);
}

/*
 * One toolbox row per entry of rows[] (global node indices), all N walks of that node.
 * Outputs (row-major, r = position in rows[]):
 *   G     [nrows][m]         = A/2,   scaled by 1/N
 *   gradG [dim][nrows][m]    = B/2,   scaled by 1/N
 *   Hc    [nrows][p]         exit counts (H = Hc/N)
 *   gradH [dim][nrows][p]    = K,     scaled by 1/N
 * Optional per-walk records (NULL to skip), index r*N + l:
 *   rec_exit (boundary cell), rec_steps (work steps K after the first), rec_capped,
 *   rec_gmass (total G contribution of the walk, unscaled), rec_gradmass [.][dim],
 *   rec_w [.][dim] (X_1 - x_i), rec_vhash (XOR over the walk's interior binnings of
 *   cellmix(tag, cell): tag 0xFFFFFFFF for the ball term, k for the source of step k),
 *   rec_xexit [.][dim] (stopping point).  Grsum [nrows][m] (optional): sum of r/(2d N) over the
 *   same binnings as G (a diagnostic used to bound rounding differences, not an estimator).
 * stats[0] += total WoS steps (1 + K per walk), stats[1] += capped walks.
 * Returns 0, or -1 on invalid input (a node with r(x_i) <= 0).
 */
int oracle_walk_rows(const oracle_spec* s, const int64_t* rows, int64_t nrows,
                     double* G, double* gradG, int64_t* Hc, double* gradH,
                     int32_t* rec_exit, int32_t* rec_steps, int8_t* rec_capped,
                     double* rec_gmass, double* rec_gradmass, double* rec_w,
                     uint32_t* rec_vhash, double* rec_xexit, double* Grsum, int64_t* stats) {
    const int d = s->dim;
    const int64_t m = s->m, p = s->p, N = s->walks;
    int bad = 0;
    int64_t tot_steps = 0, tot_capped = 0;
    for (int64_t r = 0; r < nrows; ++r) {
        if (orc_sdf(d, s->sdf_kind, s->sdf_params, s->n_sdf_params, s->x + rows[r] * d) <= 0.0)
            bad = 1;
    }
    if (bad || d < 2 || d > 3) return -1;
    memset(G, 0, sizeof(double) * nrows * m);
    if (Grsum) memset(Grsum, 0, sizeof(double) * nrows * m);
    memset(gradG, 0, sizeof(double) * d * nrows * m);
    memset(Hc, 0, sizeof(int64_t) * nrows * p);
    memset(gradH, 0, sizeof(double) * d * nrows * p);

#pragma omp parallel for schedule(dynamic, 1) reduction(+ : tot_steps, tot_capped)
    for (int64_t r = 0; r < nrows; ++r) {
        const int64_t i = rows[r];
        const double* xi = s->x + i * d;
        const double r0 = orc_sdf(d, s->sdf_kind, s->sdf_params, s->n_sdf_params, xi);
        double* Grow = G + r * m;
        int64_t* Hrow = Hc + r * p;
        for (int64_t l = 0; l < N; ++l) {
            double u[4], v[4], Zb[3] = {0, 0, 0}, Zs[3] = {0, 0, 0}, U[3] = {0, 0, 0};
            double S, R, wsum, pt[3], X[3], w[3] = {0, 0, 0};
            double gmass = 0.0, gm[3] = {0, 0, 0};
            uint32_t vh = 0u;
            /* ball term of the first sphere (Prop. 2.6 (ii)): its own counter, step tag 0xFFFFFFFF */
            orc_draw(s, (uint32_t)l, 0xFFFFFFFFu, (uint32_t)i, 0u, u);
            S = 1.0 - sqrt(u[0]);
            if (d == 2) { orc_dir2(u[1], Zb); wsum = 1.0 + S; }
            else { orc_dir3(u[1], u[2], Zb); wsum = 1.0 + S + S * S; }
            for (int c = 0; c < d; ++c) pt[c] = xi[c] + r0 * S * Zb[c];
            int64_t jb = orc_nearest(d, pt, s->y, m);
            vh ^= orc_cellmix(0xFFFFFFFFu, (uint32_t)jb);
            for (int c = 0; c < d; ++c) {
                double a = 0.5 * r0 * wsum * Zb[c];
                gradG[((int64_t)c * nrows + r) * m + jb] += a;
                gm[c] += a;
            }
            /* the chain: step k draws the source Y_k (Green density) and the direction U_k;
             * step 0 starts at x_i with r = r0 and contributes to G only (k = 0 term of
             * eq. Estimator_A; eq. Estimator_B sums from s = 1) */
            for (int c = 0; c < d; ++c) X[c] = xi[c];
            int64_t k = 0;
            int capped = 0;
            for (;;) {
                double rk = orc_sdf(d, s->sdf_kind, s->sdf_params, s->n_sdf_params, X);
                if (k > 0 && rk < s->eps) break;
                if (k > s->max_steps) { capped = 1; break; }
                if (d == 2) {
                    orc_draw(s, (uint32_t)l, (uint32_t)k, (uint32_t)i, 0u, u);
                    R = oracle_green_radius_2d(u[0]);
                    orc_dir2(u[1], Zs);
                    orc_dir2(u[2], U);
                } else {
                    orc_draw(s, (uint32_t)l, (uint32_t)k, (uint32_t)i, 0u, u);
                    orc_draw(s, (uint32_t)l, (uint32_t)k, (uint32_t)i, 1u, v);
                    R = orc_med3(u[0], u[1], u[2]);
                    orc_dir3(u[3], v[0], Zs);
                    orc_dir3(v[1], v[2], U);
                }
                for (int c = 0; c < d; ++c) pt[c] = X[c] + rk * R * Zs[c];
                int64_t j = orc_nearest(d, pt, s->y, m);
                vh ^= orc_cellmix((uint32_t)k, (uint32_t)j);
                double r2 = rk * rk;
                Grow[j] += r2 / (2.0 * d);
                if (Grsum) Grsum[r * m + j] += rk / (2.0 * d);
                gmass += r2 / (2.0 * d);
                if (k > 0) {
                    for (int c = 0; c < d; ++c) {
                        double a = w[c] * r2 / (2.0 * r0 * r0);
                        gradG[((int64_t)c * nrows + r) * m + j] += a;
                        gm[c] += a;
                    }
                } else {
                    for (int c = 0; c < d; ++c) w[c] = rk * U[c];
                }
                for (int c = 0; c < d; ++c) X[c] += rk * U[c];
                ++k;
            }
            int64_t jz = orc_nearest(d, X, s->z, p);
            Hrow[jz] += 1;
            for (int c = 0; c < d; ++c)
                gradH[((int64_t)c * nrows + r) * p + jz] += (double)d / (r0 * r0) * w[c];
            tot_steps += k;          /* step 0 plus k-1 further steps */
            tot_capped += capped;
            int64_t ridx = r * N + l;
            if (rec_exit) rec_exit[ridx] = (int32_t)jz;
            if (rec_steps) rec_steps[ridx] = (int32_t)(k - 1);
            if (rec_capped) rec_capped[ridx] = (int8_t)capped;
            if (rec_gmass) rec_gmass[ridx] = gmass;
            if (rec_gradmass) for (int c = 0; c < d; ++c) rec_gradmass[ridx * d + c] = gm[c];
            if (rec_w) for (int c = 0; c < d; ++c) rec_w[ridx * d + c] = w[c];
            if (rec_vhash) rec_vhash[ridx] = vh;
            if (rec_xexit) for (int c = 0; c < d; ++c) rec_xexit[ridx * d + c] = X[c];
        }
    }
    const double invN = 1.0 / (double)N;
    for (int64_t t = 0; t < nrows * m; ++t) G[t] *= invN;
    if (Grsum) for (int64_t t = 0; t < nrows * m; ++t) Grsum[t] *= invN;
    for (int64_t t = 0; t < d * nrows * m; ++t) gradG[t] *= invN;
    for (int64_t t = 0; t < d * nrows * p; ++t) gradH[t] *= invN;
    if (stats) { stats[0] += tot_steps; stats[1] += tot_capped; }
    return 0;
}

/* ---------------------------------------------------------------- cell weights lambda_i */
/* lambda_i = lambda(W_i)/lambda(D) (Sec. 3.1) by Monte Carlo: uniform points in the bounding
 * box lo..hi, kept when r(x) > 0, binned to the nearest centre.  Counter of sample j:
 * (j_lo, j_hi, 0, 1<<24 | instance<<8); coordinates from the first dim uniforms. */
int oracle_cell_counts(int dim, int sdf_kind, const double* prm, int64_t nprm,
                       const double* y, int64_t m, const double* lo, const double* hi,
                       int64_t nsamples, uint64_t seed, uint32_t instance, int64_t* counts) {
    memset(counts, 0, sizeof(int64_t) * m);
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel
    {
        int64_t* local = (int64_t*)calloc((size_t)m, sizeof(int64_t));
#pragma omp for schedule(static)
        for (int64_t j = 0; j < nsamples; ++j) {
            uint32_t ctr[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), 0u,
                               (1u << 24) | ((instance & 0xFFFFu) << 8)};
            uint32_t out[4];
            oracle_philox4x32_10(ctr, key, out);
            double pt[3];
            for (int c = 0; c < dim; ++c) pt[c] = lo[c] + (hi[c] - lo[c]) * oracle_u01(out[c]);
            if (orc_sdf(dim, sdf_kind, prm, nprm, pt) > 0.0) local[orc_nearest(dim, pt, y, m)] += 1;
        }
#pragma omp critical
        for (int64_t t = 0; t < m; ++t) counts[t] += local[t];
        free(local);
    }
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
