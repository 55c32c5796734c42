/*
 * FP64 CPU oracle for the fast hyperspectral reconstruction (FHR) path of
 * "Fast Hyperspectral Neutron Tomography" (arXiv 2410.22500).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the FHR path computes.  It is called by the tests, by the
 * smoke check and by the benchmark's CPU-baseline leg, and by nothing else.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is double precision, written as plain loops in the order the
 * paper states the steps.  Loops whose iterations write disjoint outputs may
 * run on several host threads (OpenMP); every sum is still taken in one fixed
 * order, so each result is the same bit for bit whatever the thread count
 * (or_set_threads).  Each function cites the passage it
 * follows.  Where the paper is silent, the reading taken is stated beside the
 * code (and listed with the design notes of the project).
 *
 * Layouts (row-major C arrays):
 *   counts y   [Nv][Nr][Nc][Nk]      open beam y0 [Nr][Nc][Nk]
 *   P          [Np][Nk], pixel j = (v*Nc + c)*Nr + r   (the paper's p, Np x Nk)
 *   D          [Nk][K]   (the paper's D^s)              W [Np][K] (the paper's V^s)
 *   volume x   [N][N][Wl], element (iy, ix, w), w = r*K + j (slice r, channel j)
 *   sinogram   [Nv][Nc][Wl]  (equal to W viewed with Wl = Nr*K)
 *   x^h        [Nr][N][N][Nk]
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NOMEM -2

/* Host threads for the parallel loops (1 = serial); returns the count in use. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------
 * Normalisation.  Eq. (neglogattenuation): p = -log(y / y^o).
 * Appendix A, Eq. (off_corr_proof)/(back_offset): with a background pixel set
 * B, b_{v,k} = mean over (r,c) in B of -log(y/y^o), and p <- p - b.
 * Readings (paper silent): counts are clamped at 1 before the log so zero
 * counts stay finite; p is clamped at 0 afterwards because the factorisation
 * of Eq. (sub_extract_solve) needs p >= 0; a dead wavelength bin (mask [Nk])
 * gives p = 0 for every pixel.
 * Output pixel order is (v, c, r) so that P's rows, read K at a time, are the
 * subspace sinogram in [view][bin][slice] order.
 * ---------------------------------------------------------------------- */
int or_normalise(int Nv, int Nr, int Nc, int Nk,
                 const uint16_t *y, const uint16_t *y0,
                 const uint8_t *bg,   /* [Nr][Nc] or NULL */
                 const uint8_t *dead, /* [Nk] (per_pixel = 0) or [Nr][Nc][Nk] (per_pixel = 1), or NULL */
                 int per_pixel,
                 double *P,           /* [Nv*Nc*Nr][Nk] */
                 double *b_out)       /* [Nv][Nk] or NULL */
{
    if (Nv <= 0 || Nr <= 0 || Nc <= 0 || Nk <= 0) return OR_ERR_ARG;
    double *b = (double *)calloc((size_t)Nv * Nk, sizeof(double));
    if (!b) return OR_ERR_NOMEM;
    /* a dead entry (detector pixel (r, c), bin k) carries no measurement */
#define OR_DEAD(r, c, k) \
    (dead && (per_pixel ? dead[((size_t)(r) * Nc + (c)) * Nk + (k)] : dead[(k)]))
    if (bg) {
        /* Appendix A: b_{v,k} = mean of -log(y/y0) over the background pixels whose
           entry is live; 0 when there is none */
#pragma omp parallel for schedule(static)
        for (int v = 0; v < Nv; ++v)
            for (int k = 0; k < Nk; ++k) {
                double s = 0.0;
                long n = 0;
                for (int r = 0; r < Nr; ++r)
                    for (int c = 0; c < Nc; ++c) {
                        if (!bg[r * Nc + c] || OR_DEAD(r, c, k)) continue;
                        double yy = y[(((size_t)v * Nr + r) * Nc + c) * Nk + k];
                        double yo = y0[((size_t)r * Nc + c) * Nk + k];
                        s += log(dmax(yo, 1.0)) - log(dmax(yy, 1.0));
                        ++n;
                    }
                b[(size_t)v * Nk + k] = n > 0 ? s / (double)n : 0.0;
            }
    }
#pragma omp parallel for schedule(static)
    for (int v = 0; v < Nv; ++v)
        for (int r = 0; r < Nr; ++r)
            for (int c = 0; c < Nc; ++c) {
                size_t j = ((size_t)v * Nc + c) * Nr + r;
                for (int k = 0; k < Nk; ++k) {
                    double yy = y[(((size_t)v * Nr + r) * Nc + c) * Nk + k];
                    double yo = y0[((size_t)r * Nc + c) * Nk + k];
                    double p = log(dmax(yo, 1.0)) - log(dmax(yy, 1.0));
                    p -= b[(size_t)v * Nk + k];
                    p = dmax(p, 0.0);
                    if (OR_DEAD(r, c, k)) p = 0.0;
                    P[j * Nk + k] = p;
                }
            }
#undef OR_DEAD
    if (b_out) memcpy(b_out, b, sizeof(double) * (size_t)Nv * Nk);
    free(b);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Subspace extraction, Eq. (sub_extract_solve): min ||p - V D^T||_F^2 over
 * V >= 0, D >= 0, solved (Sec. III) by coordinate descent with fast HALS
 * updates.  Each half-step minimises the objective exactly over one
 * coordinate at a time (a 1-D nonnegative quadratic), coordinates in natural
 * order, Gauss-Seidel within a row:
 *   V row j:  v_js <- max(0, v_js + ((p_j D)_s - sum_t (D^T D)_{s,t} v_jt) / (D^T D)_{s,s})
 *   D row k:  d_ks <- max(0, d_ks + ((p^T V)_{k,s} - sum_t d_kt (V^T V)_{t,s}) / (V^T V)_{s,s})
 * A coordinate whose Gram diagonal is zero is left unchanged.
 * ---------------------------------------------------------------------- */
void or_gram(long rows, int K, const double *X, double *G)
{
    for (int s = 0; s < K; ++s)
        for (int t = 0; t < K; ++t) {
            double a = 0.0;
            for (long i = 0; i < rows; ++i) a += X[i * K + s] * X[i * K + t];
            G[s * K + t] = a;
        }
}

int or_hals_update_W(long Np, int Nk, int K, const double *P, const double *D, double *W)
{
    if (K <= 0 || K > 64) return OR_ERR_ARG;
    double G[64 * 64];
    or_gram(Nk, K, D, G);
#pragma omp parallel for schedule(static)
    for (long j = 0; j < Np; ++j) {
        double r[64];
        const double *p = P + j * Nk;
        double *w = W + j * K;
        for (int s = 0; s < K; ++s) {
            double a = 0.0;
            for (int k = 0; k < Nk; ++k) a += p[k] * D[(size_t)k * K + s];
            r[s] = a;
        }
        for (int s = 0; s < K; ++s) {
            double h = G[s * K + s];
            if (h == 0.0) continue;
            double g = r[s];
            for (int t = 0; t < K; ++t) g -= G[s * K + t] * w[t];
            w[s] = dmax(0.0, w[s] + g / h);
        }
    }
    return OR_OK;
}

int or_hals_update_D(long Np, int Nk, int K, const double *P, const double *W, double *D)
{
    if (K <= 0 || K > 64) return OR_ERR_ARG;
    double G[64 * 64];
    or_gram(Np, K, W, G);
    double *Q = (double *)calloc((size_t)Nk * K, sizeof(double));
    if (!Q) return OR_ERR_NOMEM;
    /* Q = p^T V: each Q[k][s] is summed over j = 0..Np-1 in that order; a thread
       takes a block of 16 bins at a time */
#pragma omp parallel for schedule(dynamic)
    for (int k0 = 0; k0 < Nk; k0 += 16) {
        const int k1 = k0 + 16 < Nk ? k0 + 16 : Nk;
        for (long j = 0; j < Np; ++j)
            for (int k = k0; k < k1; ++k) {
                double p = P[j * Nk + k];
                for (int s = 0; s < K; ++s) Q[(size_t)k * K + s] += p * W[j * K + s];
            }
    }
    for (int k = 0; k < Nk; ++k) {
        double *d = D + (size_t)k * K;
        for (int s = 0; s < K; ++s) {
            double h = G[s * K + s];
            if (h == 0.0) continue;
            double g = Q[(size_t)k * K + s];
            for (int t = 0; t < K; ++t) g -= d[t] * G[t * K + s];
            d[s] = dmax(0.0, d[s] + g / h);
        }
    }
    free(Q);
    return OR_OK;
}

/* Reading (paper silent): after each D half-step the columns of D are scaled
 * to unit L2 norm and the matching columns of V by the inverse factor, so the
 * product V D^T (and the objective) is unchanged.  Zero columns are kept. */
void or_normalise_columns(long Np, int Nk, int K, double *D, double *W, double *norms)
{
    for (int s = 0; s < K; ++s) {
        double a = 0.0;
        for (int k = 0; k < Nk; ++k) a += D[(size_t)k * K + s] * D[(size_t)k * K + s];
        double n = sqrt(a);
        if (norms) norms[s] = n;
        if (n > 0.0) {
            for (int k = 0; k < Nk; ++k) D[(size_t)k * K + s] /= n;
            for (long j = 0; j < Np; ++j) W[j * K + s] *= n;
        }
    }
}

/* ||p - V D^T||_F^2, evaluated entry by entry (Eq. sub_extract_solve, no 1/2). */
double or_objective(long Np, int Nk, int K, const double *P, const double *D, const double *W)
{
    /* the squared residuals of each pixel row are summed over k, and the row sums
       over j, each in ascending order */
    double *row = (double *)malloc(sizeof(double) * (size_t)(Np > 0 ? Np : 1));
    if (!row) return NAN;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < Np; ++j) {
        double fr = 0.0;
        for (int k = 0; k < Nk; ++k) {
            double e = P[j * Nk + k];
            for (int s = 0; s < K; ++s) e -= W[j * K + s] * D[(size_t)k * K + s];
            fr += e * e;
        }
        row[j] = fr;
    }
    double f = 0.0;
    for (long j = 0; j < Np; ++j) f += row[j];
    free(row);
    return f;
}

/* `iters` full iterations, each: V half-step, D half-step, column scaling,
 * objective.  obj[t] (if non-NULL) receives the objective after iteration t. */
int or_nmf(long Np, int Nk, int K, int iters, const double *P, double *D, double *W,
           double *obj)
{
    for (int t = 0; t < iters; ++t) {
        int e = or_hals_update_W(Np, Nk, K, P, D, W);
        if (e) return e;
        e = or_hals_update_D(Np, Nk, K, P, W, D);
        if (e) return e;
        or_normalise_columns(Np, Nk, K, D, W, NULL);
        if (obj) obj[t] = or_objective(Np, Nk, K, P, D, W);
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Clustering start for the NMF (not specified by the paper, whose Sec. III
 * uses NNDSVD; this is the library's added "clustering-initialised" mode).
 * Reading, stated in full because the paper gives none:
 *   1. sample S pixels, j_i = floor(i * Np / S), i = 0..S-1;
 *   2. k-means++ seeding: u_m is output m (0-based) of splitmix64 (Steele, Lea
 *      and Flood, OOPSLA 2014) started from state `seed`, scaled to [0, 1) by
 *      its top 53 bits.  Centre 0 is sample floor(u_0 S).  Centre m >= 1 is the
 *      first sample i whose running sum of d_i exceeds u_m * sum(d), where d_i
 *      is the squared distance of sample i to its nearest chosen centre (if
 *      every d_i is 0: sample floor(u_m S));
 *   3. `iters` Lloyd iterations: assign each sample to its nearest centre
 *      (lowest index on ties), then move each centre to the mean of its
 *      samples (a centre with no samples stays where it is);
 *   4. D0 column m = centre m; W0 = one HALS V half-step started from V = 0.
 * All distances and means in FP64.
 * ---------------------------------------------------------------------- */
static uint64_t splitmix64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* the first n outputs of splitmix64 from `seed` */
void or_splitmix64(uint64_t seed, int n, uint64_t *out)
{
    uint64_t st = seed;
    for (int i = 0; i < n; ++i) out[i] = splitmix64_next(&st);
}

static double sqdist(const double *a, const double *b, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        double d = a[k] - b[k];
        s += d * d;
    }
    return s;
}

/* The k-means++ pick: the first sample whose running sum of d (squared distances
 * to the nearest chosen centre) exceeds u times their total; when rounding leaves
 * none, the last sample with d > 0.  -1 when the total is 0. */
long or_kmpp_pick(const double *d, long S, double u)
{
    double tot = 0.0;
    for (long i = 0; i < S; ++i) tot += d[i];
    if (!(tot > 0.0)) return -1;
    double target = u * tot, run = 0.0;
    for (long i = 0; i < S; ++i) {
        run += d[i];
        if (run > target) return i;
    }
    for (long i = S - 1; i >= 0; --i)
        if (d[i] > 0.0) return i;
    return -1;
}

/* k-means on the sampled rows of P [Np][Nk].  C [K][Nk] receives the centres,
 * labels [S] (if non-NULL) the final assignment, cost [iters+1] (if non-NULL)
 * the sum of squared distances to the assigned centre before each centre
 * move and after the last one, seeds [K] (if non-NULL) the seeding samples. */
int or_kmeans(long Np, int Nk, const double *P, long S, int K, int iters, uint64_t seed, double *C,
              int *labels, double *cost, long *seeds)
{
    if (S < 1 || S > Np || K < 1 || K > S) return OR_ERR_ARG;
    double *X = (double *)malloc((size_t)S * Nk * sizeof(double));
    double *d = (double *)malloc((size_t)S * sizeof(double));
    int *lab = (int *)malloc((size_t)S * sizeof(int));
    double *acc = (double *)malloc((size_t)K * Nk * sizeof(double));
    long *cnt = (long *)malloc((size_t)K * sizeof(long));
    if (!X || !d || !lab || !acc || !cnt) {
        free(X); free(d); free(lab); free(acc); free(cnt);
        return OR_ERR_NOMEM;
    }
    for (long i = 0; i < S; ++i) {
        long j = (long)(((__int128)i * Np) / S);
        memcpy(X + (size_t)i * Nk, P + (size_t)j * Nk, (size_t)Nk * sizeof(double));
    }
    /* k-means++ seeding */
    uint64_t st = seed;
    for (int m = 0; m < K; ++m) {
        double u = (double)(splitmix64_next(&st) >> 11) * 0x1.0p-53;
        long pick = (long)(u * (double)S);
        if (m > 0) {
            for (long i = 0; i < S; ++i) {
                double e = sqdist(X + (size_t)i * Nk, C + (size_t)(m - 1) * Nk, Nk);
                d[i] = (m == 1 || e < d[i]) ? e : d[i];
            }
            const long q = or_kmpp_pick(d, S, u);
            if (q >= 0) pick = q;   /* all samples on chosen centres: keep the first-seed formula */
        }
        if (seeds) seeds[m] = pick;
        memcpy(C + (size_t)m * Nk, X + (size_t)pick * Nk, (size_t)Nk * sizeof(double));
    }
    /* Lloyd iterations */
    for (int it = 0; it <= iters; ++it) {
        double c = 0.0;
        for (long i = 0; i < S; ++i) {
            int best = 0;
            double bd = sqdist(X + (size_t)i * Nk, C, Nk);
            for (int m = 1; m < K; ++m) {
                double e = sqdist(X + (size_t)i * Nk, C + (size_t)m * Nk, Nk);
                if (e < bd) { bd = e; best = m; }
            }
            lab[i] = best;
            c += bd;
        }
        if (cost) cost[it] = c;
        if (it == iters) break;
        memset(acc, 0, (size_t)K * Nk * sizeof(double));
        memset(cnt, 0, (size_t)K * sizeof(long));
        for (long i = 0; i < S; ++i) {
            cnt[lab[i]]++;
            for (int k = 0; k < Nk; ++k) acc[(size_t)lab[i] * Nk + k] += X[(size_t)i * Nk + k];
        }
        for (int m = 0; m < K; ++m)
            if (cnt[m] > 0)
                for (int k = 0; k < Nk; ++k) C[(size_t)m * Nk + k] = acc[(size_t)m * Nk + k] / (double)cnt[m];
    }
    if (labels) memcpy(labels, lab, (size_t)S * sizeof(int));
    free(X); free(d); free(lab); free(acc); free(cnt);
    return OR_OK;
}

/* Clustering start: D0 [Nk][K] = k-means centres (transposed), W0 [Np][K] =
 * one HALS V half-step from zero with D0. */
int or_cluster_init(long Np, int Nk, const double *P, long S, int K, int iters, uint64_t seed, double *D0,
                    double *W0)
{
    double *C = (double *)malloc((size_t)K * Nk * sizeof(double));
    if (!C) return OR_ERR_NOMEM;
    int e = or_kmeans(Np, Nk, P, S, K, iters, seed, C, NULL, NULL, NULL);
    if (e) { free(C); return e; }
    for (int k = 0; k < Nk; ++k)
        for (int m = 0; m < K; ++m) D0[(size_t)k * K + m] = C[(size_t)m * Nk + k];
    free(C);
    memset(W0, 0, (size_t)Np * K * sizeof(double));
    return or_hals_update_W(Np, Nk, K, P, D0, W0);
}

/* ------------------------------------------------------------------------
 * Parallel-beam projector A of Eq. (porj_matd_rel) / Eq. (recon).  The paper
 * does not state its discretisation (it uses a library).  Reading: the strip
 * (area) model.  A_{(v,c),i} = area(pixel_i  intersect  strip_{v,c}) / du, with
 * strip_{v,c} = {(x,y): |x cos t_v + y sin t_v - u_c| <= du/2}, unit pixels and
 * unit bins (du = 1).  Two independent constructions are given: the closed
 * form below (integral of the pixel's trapezoidal footprint over the bin) and
 * polygon clipping (or_strip_area_polyclip) for brute-force checks.
 * ---------------------------------------------------------------------- */

/* Cumulative integral of the footprint of a unit square seen at direction
 * (cos t, sin t): the footprint is a trapezoid of total area 1, flat top of
 * height 1/hi for |s| <= (hi-lo)/2, linear to 0 at |s| = (hi+lo)/2, where
 * hi = max(|cos|,|sin|), lo = min(|cos|,|sin|). */
static double footprint_cdf(double s, double hi, double lo)
{
    double t2 = 0.5 * (hi + lo), t1 = 0.5 * (hi - lo);
    if (s <= -t2) return 0.0;
    if (s >= t2) return 1.0;
    if (s <= -t1) return (s + t2) * (s + t2) / (2.0 * hi * lo);
    if (s <= t1) return lo / (2.0 * hi) + (s + t1) / hi;
    return 1.0 - (t2 - s) * (t2 - s) / (2.0 * hi * lo);
}

double or_strip_area(double theta, double px, double py, double uc)
{
    double c = cos(theta), s = sin(theta);
    double a = fabs(c), b = fabs(s);
    double hi = dmax(a, b), lo = dmin(a, b);
    double u0 = px * c + py * s;
    return footprint_cdf(uc + 0.5 - u0, hi, lo) - footprint_cdf(uc - 0.5 - u0, hi, lo);
}

/* Sutherland-Hodgman clipping of a convex polygon by the half-plane
 * nx*x + ny*y <= d.  Returns the new vertex count. */
static int clip_halfplane(const double *in, int n, double nx, double ny, double d, double *out)
{
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const double *P = in + 2 * i, *Q = in + 2 * ((i + 1) % n);
        double fp = nx * P[0] + ny * P[1] - d, fq = nx * Q[0] + ny * Q[1] - d;
        if (fp <= 0) { out[2 * m] = P[0]; out[2 * m + 1] = P[1]; ++m; }
        if ((fp < 0 && fq > 0) || (fp > 0 && fq < 0)) {
            double tt = fp / (fp - fq);
            out[2 * m] = P[0] + tt * (Q[0] - P[0]);
            out[2 * m + 1] = P[1] + tt * (Q[1] - P[1]);
            ++m;
        }
    }
    return m;
}

double or_strip_area_polyclip(double theta, double px, double py, double uc)
{
    double A[32], B[32];
    double c = cos(theta), s = sin(theta);
    A[0] = px - 0.5; A[1] = py - 0.5;
    A[2] = px + 0.5; A[3] = py - 0.5;
    A[4] = px + 0.5; A[5] = py + 0.5;
    A[6] = px - 0.5; A[7] = py + 0.5;
    int n = clip_halfplane(A, 4, c, s, uc + 0.5, B);          /* u <= uc + 1/2 */
    n = clip_halfplane(B, n, -c, -s, -(uc - 0.5), A);          /* u >= uc - 1/2 */
    double area = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *P = A + 2 * i, *Q = A + 2 * ((i + 1) % n);
        area += P[0] * Q[1] - Q[0] * P[1];
    }
    return 0.5 * fabs(area);
}

static double pix_x(int ix, int N) { return ix - 0.5 * (N - 1); }
static double bin_u(int c, int Nc) { return c - 0.5 * (Nc - 1); }

/* Dense system matrix [Nv*Nc][N*N] (tiny cases only). */
void or_system_matrix(int N, int Nc, int Nv, const double *theta, int polyclip, double *A)
{
    for (int v = 0; v < Nv; ++v)
        for (int c = 0; c < Nc; ++c)
            for (int iy = 0; iy < N; ++iy)
                for (int ix = 0; ix < N; ++ix) {
                    double px = pix_x(ix, N), py = pix_x(iy, N), uc = bin_u(c, Nc);
                    A[((size_t)v * Nc + c) * N * N + (size_t)iy * N + ix] =
                        polyclip ? or_strip_area_polyclip(theta[v], px, py, uc)
                                 : or_strip_area(theta[v], px, py, uc);
                }
}

/* The bins a pixel's footprint can touch at angle theta: every c whose strip
 * centre lies within 1/2 + (|cos|+|sin|)/2 of the pixel's projected centre.
 * Outside that range the strip area is exactly zero. */
static void bin_range(double theta, double px, double py, int Nc, int *c0, int *c1)
{
    double c = cos(theta), s = sin(theta);
    double u0 = px * c + py * s;
    double half = 0.5 + 0.5 * (fabs(c) + fabs(s));
    double lo = u0 - half + 0.5 * (Nc - 1), hi = u0 + half + 0.5 * (Nc - 1);
    int a = (int)floor(lo), b = (int)ceil(hi);
    if (a < 0) a = 0;
    if (b > Nc - 1) b = Nc - 1;
    *c0 = a;
    *c1 = b;
}

/* y = A x over a vector of Wl values per pixel / per ray. */
void or_project(int N, int Nc, int Nv, const double *theta, int Wl, const double *x, double *y)
{
    memset(y, 0, sizeof(double) * (size_t)Nv * Nc * Wl);
#pragma omp parallel for schedule(dynamic)
    for (int v = 0; v < Nv; ++v)
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                double px = pix_x(ix, N), py = pix_x(iy, N);
                int c0, c1;
                bin_range(theta[v], px, py, Nc, &c0, &c1);
                const double *xi = x + ((size_t)iy * N + ix) * Wl;
                for (int c = c0; c <= c1; ++c) {
                    double a = or_strip_area(theta[v], px, py, bin_u(c, Nc));
                    if (a == 0.0) continue;
                    double *yr = y + ((size_t)v * Nc + c) * Wl;
                    for (int w = 0; w < Wl; ++w) yr[w] += a * xi[w];
                }
            }
}

/* x = A^T y (the exact transpose of or_project). */
void or_backproject(int N, int Nc, int Nv, const double *theta, int Wl, const double *y, double *x)
{
    memset(x, 0, sizeof(double) * (size_t)N * N * Wl);
    /* each pixel sums over views v, then bins c, in ascending order */
#pragma omp parallel for schedule(dynamic)
    for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix)
            for (int v = 0; v < Nv; ++v) {
                double px = pix_x(ix, N), py = pix_x(iy, N);
                int c0, c1;
                bin_range(theta[v], px, py, Nc, &c0, &c1);
                double *xi = x + ((size_t)iy * N + ix) * Wl;
                for (int c = c0; c <= c1; ++c) {
                    double a = or_strip_area(theta[v], px, py, bin_u(c, Nc));
                    if (a == 0.0) continue;
                    const double *yr = y + ((size_t)v * Nc + c) * Wl;
                    for (int w = 0; w < Wl; ++w) xi[w] += a * yr[w];
                }
            }
}

/* ------------------------------------------------------------------------
 * Filtered back-projection of the subspace sinograms (the "FHR with FBP"
 * variant, Sec. V / Table II), the paper's faster alternative to MBIR.
 * Reading (the paper names FBP without its discretisation): the textbook
 * parallel-beam FBP with the band-limited ramp (Ram-Lak) filter sampled at the
 * bin spacing tau = 1 (Kak and Slaney, Sec. 3.3.3):
 *   h[0] = 1 / (4 tau^2), h[n] = 0 for even n != 0, h[n] = -1 / (n pi tau)^2 odd;
 *   q[v][c] = tau * sum_c' h[c - c'] p[v][c'] (linear convolution, zero outside
 *   the detector);
 *   x = (pi / Nv) A^T q, with A^T the strip-area back-projector above.
 * ---------------------------------------------------------------------- */
double or_ramp(int n)
{
    if (n == 0) return 0.25;
    if (n % 2 == 0) return 0.0;
    return -1.0 / ((double)n * (double)n * M_PI * M_PI);
}

void or_ramp_filter(int Nv, int Nc, int Wl, const double *p, double *q)
{
#pragma omp parallel for schedule(static)
    for (int v = 0; v < Nv; ++v)
        for (int c = 0; c < Nc; ++c) {
            double *qo = q + ((size_t)v * Nc + c) * Wl;
            for (int w = 0; w < Wl; ++w) qo[w] = 0.0;
            for (int c2 = 0; c2 < Nc; ++c2) {
                double h = or_ramp(c - c2);
                if (h == 0.0) continue;
                const double *pi = p + ((size_t)v * Nc + c2) * Wl;
                for (int w = 0; w < Wl; ++w) qo[w] += h * pi[w];
            }
        }
}

int or_fbp(int N, int Nc, int Nv, const double *theta, int Wl, const double *p, double *x)
{
    double *q = (double *)malloc(sizeof(double) * (size_t)Nv * Nc * Wl);
    if (!q) return OR_ERR_NOMEM;
    or_ramp_filter(Nv, Nc, Wl, p, q);
    or_backproject(N, Nc, Nv, theta, Wl, q, x);
    const double sc = M_PI / (double)Nv;
    for (size_t i = 0; i < (size_t)N * N * Wl; ++i) x[i] *= sc;
    free(q);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * MBIR reconstruction of each subspace channel, Eq. (recon):
 *   x_j = argmin_x  1/(2 sigma_v^2) ||V_j - A x||^2 + h(x),
 * with the qGGMRF prior h (Sec. III; the paper gives no formula, it cites the
 * standard qGGMRF form):
 *   h(x) = sum over neighbour pairs {s,r} of b_sr rho(x_s - x_r),
 *   rho(d) = |d|^p / (p sigma_x^p) * u / (1 + u),  u = |d / (T sigma_x)|^(q-p).
 * Readings (paper silent; its solver is a library): solved by separable
 * quadratic surrogates (SQS) with the symmetric-bound surrogate of rho, so
 * every iteration decreases the cost; x >= 0 enforced by clamping; q = 2;
 * 8 in-plane neighbours (weight 1 edge, 1/sqrt2 diagonal) and 2 inter-slice
 * neighbours (weight 1) when Nr > 1, all weights divided by their sum;
 * voxels outside the volume are not neighbours.  `beta` scales h (1 = Eq.
 * recon; 0 removes the prior, used by tests).
 * Optional momentum: FISTA-style extrapolation of the SQS iterates.
 * ---------------------------------------------------------------------- */
typedef struct {
    double p, q, T, beta;
    int iters;
    int momentum;
} or_mbir_params;

/* rho(d) */
double or_qggmrf_rho(double d, double sx, double p, double q, double T)
{
    double a = fabs(d);
    double u = pow(a / (T * sx), q - p);
    return pow(a, p) / (p * pow(sx, p)) * u / (1.0 + u);
}

/* rho'(d)/d (the surrogate's half-curvature), finite at d = 0 for q = 2. */
double or_qggmrf_influence(double d, double sx, double p, double q, double T)
{
    double a = fabs(d);
    double u = pow(a / (T * sx), q - p);
    double lead = pow(a, q - 2.0) / (pow(sx, p) * pow(T * sx, q - p));
    return lead / (1.0 + u) * (1.0 + (q - p) / (p * (1.0 + u)));
}

/* neighbour offsets (dy, dx, dr) and raw weights */
static const int NB_OFF[10][3] = {
    {-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0},
    {-1, -1, 0}, {-1, 1, 0}, {1, -1, 0}, {1, 1, 0},
    {0, 0, -1}, {0, 0, 1}};

static void nb_weights(int Nr, double *bw, int *nnb)
{
    int n = Nr > 1 ? 10 : 8;
    double r2 = 1.0 / sqrt(2.0), z = 0.0;
    for (int i = 0; i < n; ++i) {
        bw[i] = (i >= 4 && i < 8) ? r2 : 1.0;
        z += bw[i];
    }
    for (int i = 0; i < n; ++i) bw[i] /= z;
    *nnb = n;
}

/* Cost of Eq. (recon) summed over channels: sum_j [ ||V_j - A x_j||^2 / (2 sv_j^2) + beta h_j(x_j) ]. */
double or_mbir_cost(int N, int Nr, int K, int Nc, int Nv, const double *theta, const double *V,
                    const double *sv, const double *sx, const or_mbir_params *prm, const double *x)
{
    int Wl = Nr * K;
    double *Ax = (double *)malloc(sizeof(double) * (size_t)Nv * Nc * Wl);
    if (!Ax) return NAN;
    or_project(N, Nc, Nv, theta, Wl, x, Ax);
    double f = 0.0;
    for (size_t i = 0; i < (size_t)Nv * Nc; ++i)
        for (int w = 0; w < Wl; ++w) {
            double e = V[i * Wl + w] - Ax[i * Wl + w];
            double s = sv[w % K];
            f += e * e / (2.0 * s * s);
        }
    free(Ax);
    double bw[10];
    int nnb;
    nb_weights(Nr, bw, &nnb);
    /* each unordered pair once: only the "forward" half of the offsets */
    const int fwd[5] = {1, 3, 6, 7, 9};
    for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix)
            for (int r = 0; r < Nr; ++r)
                for (int j = 0; j < K; ++j) {
                    double xs = x[((size_t)iy * N + ix) * Wl + r * K + j];
                    for (int q = 0; q < 5; ++q) {
                        int o = fwd[q];
                        if (o >= nnb) continue;
                        int yy = iy + NB_OFF[o][0], xx = ix + NB_OFF[o][1], rr = r + NB_OFF[o][2];
                        if (yy < 0 || yy >= N || xx < 0 || xx >= N || rr < 0 || rr >= Nr) continue;
                        double xr = x[((size_t)yy * N + xx) * Wl + rr * K + j];
                        f += prm->beta * bw[o] * or_qggmrf_rho(xs - xr, sx[j], prm->p, prm->q, prm->T);
                    }
                }
    return f;
}

/* One SQS step from z: returns x_new (may alias nothing). dA = A^T A 1 per pixel. */
static void sqs_step(int N, int Nr, int K, int Nc, int Nv, const double *theta, const double *V,
                     const double *sv, const double *sx, const or_mbir_params *prm,
                     const double *dA, const double *z, double *xnew, double *e, double *bp)
{
    int Wl = Nr * K;
    or_project(N, Nc, Nv, theta, Wl, z, e);
    for (size_t i = 0; i < (size_t)Nv * Nc * Wl; ++i) e[i] = V[i] - e[i];
    or_backproject(N, Nc, Nv, theta, Wl, e, bp);
    double bw[10];
    int nnb;
    nb_weights(Nr, bw, &nnb);
    /* every voxel's step reads z and bp only */
#pragma omp parallel for schedule(static)
    for (int iy = 0; iy < N; ++iy)
        for (int ix = 0; ix < N; ++ix)
            for (int r = 0; r < Nr; ++r)
                for (int j = 0; j < K; ++j) {
                    size_t idx = ((size_t)iy * N + ix) * Wl + r * K + j;
                    double s2 = sv[j] * sv[j];
                    double g = -bp[idx] / s2;
                    double d = dA[(size_t)iy * N + ix] / s2;
                    if (prm->beta != 0.0) {
                        for (int o = 0; o < nnb; ++o) {
                            int yy = iy + NB_OFF[o][0], xx = ix + NB_OFF[o][1], rr = r + NB_OFF[o][2];
                            if (yy < 0 || yy >= N || xx < 0 || xx >= N || rr < 0 || rr >= Nr) continue;
                            double dl = z[idx] - z[((size_t)yy * N + xx) * Wl + rr * K + j];
                            double wt = or_qggmrf_influence(dl, sx[j], prm->p, prm->q, prm->T);
                            g += prm->beta * bw[o] * dl * wt;
                            d += 2.0 * prm->beta * bw[o] * wt;
                        }
                    }
                    xnew[idx] = d > 0.0 ? dmax(0.0, z[idx] - g / d) : z[idx];
                }
}

int or_mbir(int N, int Nr, int K, int Nc, int Nv, const double *theta, const double *V,
            const double *sv, const double *sx, const or_mbir_params *prm, double *x,
            double *cost_hist)
{
    if (N <= 0 || Nr <= 0 || K <= 0 || Nc <= 0 || Nv <= 0 || !prm) return OR_ERR_ARG;
    int Wl = Nr * K;
    size_t nx = (size_t)N * N * Wl, ny = (size_t)Nv * Nc * Wl;
    double *dA = (double *)malloc(sizeof(double) * (size_t)N * N);
    double *ones = (double *)malloc(sizeof(double) * (size_t)N * N);
    double *A1 = (double *)malloc(sizeof(double) * (size_t)Nv * Nc);
    double *e = (double *)malloc(sizeof(double) * ny);
    double *bp = (double *)malloc(sizeof(double) * nx);
    double *xn = (double *)malloc(sizeof(double) * nx);
    double *z = (double *)malloc(sizeof(double) * nx);
    if (!dA || !ones || !A1 || !e || !bp || !xn || !z) {
        free(dA); free(ones); free(A1); free(e); free(bp); free(xn); free(z);
        return OR_ERR_NOMEM;
    }
    for (size_t i = 0; i < (size_t)N * N; ++i) ones[i] = 1.0;
    or_project(N, Nc, Nv, theta, 1, ones, A1);
    or_backproject(N, Nc, Nv, theta, 1, A1, dA);
    memcpy(z, x, sizeof(double) * nx);
    double t = 1.0;
    for (int it = 0; it < prm->iters; ++it) {
        sqs_step(N, Nr, K, Nc, Nv, theta, V, sv, sx, prm, dA, z, xn, e, bp);
        if (prm->momentum) {
            double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
            double a = (t - 1.0) / tn;
#pragma omp parallel for schedule(static)
            for (size_t i = 0; i < nx; ++i) {
                double zn = xn[i] + a * (xn[i] - x[i]);
                z[i] = dmax(zn, 0.0);
                x[i] = xn[i];
            }
            t = tn;
        } else {
            memcpy(x, xn, sizeof(double) * nx);
            memcpy(z, xn, sizeof(double) * nx);
        }
        if (cost_hist) cost_hist[it] = or_mbir_cost(N, Nr, K, Nc, Nv, theta, V, sv, sx, prm, x);
    }
    free(dA); free(ones); free(A1); free(e); free(bp); free(xn); free(z);
    return OR_OK;
}

/* Reading (paper silent on sigma_v, sigma_x): per channel j, from the
 * channel's sinogram V_j over all views, bins and slices:
 *   sigma_v = rms(V_j) * 10^(-snr_db/20),   sigma_x = 0.2 * mean(V_j) / Nc.
 * A channel whose sinogram is all zero gets sigma_v = sigma_x = 1. */
void or_mbir_sigmas(long rows, int K, const double *V, double snr_db, int Nc, double *sv, double *sx)
{
    for (int j = 0; j < K; ++j) {
        double s1 = 0.0, s2 = 0.0;
        for (long i = 0; i < rows; ++i) {
            double v = V[i * K + j];
            s1 += v;
            s2 += v * v;
        }
        double rms = sqrt(s2 / (double)rows), mean = s1 / (double)rows;
        if (rms > 0.0 && mean > 0.0) {
            sv[j] = rms * pow(10.0, -snr_db / 20.0);
            sx[j] = 0.2 * mean / (double)Nc;
        } else {
            sv[j] = 1.0;
            sx[j] = 1.0;
        }
    }
}

/* ------------------------------------------------------------------------
 * Subspace expansion, Eq. (sub_expansion): x^h = x^s (D^s)^T.
 * xs [N][N][Nr*K] (iy, ix, r*K+j) -> xh [Nr][N][N][Nk].
 * ---------------------------------------------------------------------- */
void or_expand(int N, int Nr, int K, int Nk, const double *xs, const double *D, double *xh)
{
#pragma omp parallel for schedule(static) collapse(2)
    for (int r = 0; r < Nr; ++r)
        for (int iy = 0; iy < N; ++iy)
            for (int ix = 0; ix < N; ++ix) {
                const double *a = xs + ((size_t)iy * N + ix) * Nr * K + (size_t)r * K;
                double *o = xh + (((size_t)r * N + iy) * N + ix) * Nk;
                for (int k = 0; k < Nk; ++k) {
                    double s = 0.0;
                    for (int j = 0; j < K; ++j) s += a[j] * D[(size_t)k * K + j];
                    o[k] = s;
                }
            }
}

/* ------------------------------------------------------------------------
 * Signal-to-noise ratios of the reconstructions (Sec. V-B).
 *   Eq. (snr_fhr): SNR = 10 log10( 1/(Nk Nm) sum_k sum_m (mu_{m,k} / sigma_k)^2 ),
 *     mu_{m,k} the mean of bin k of x^h over a region inside material m,
 *     sigma_k the standard deviation of bin k over a background region;
 *   Eq. (snr_fmd): SNR = 10 log10( 1/Nm sum_m (mu_m / sigma_m)^2 ),
 *     mu_m the mean of material image m over a region inside material m,
 *     sigma_m its standard deviation over a background region.
 * x [Nx][C]; roi [Nx]: 0 = in no region, m + 1 = inside material m (m < Nm),
 * 255 = background.  mode 0: Eq. (snr_fmd) (channel m of region m, C >= Nm);
 * mode 1: Eq. (snr_fhr) (every channel of every region).
 * Readings (paper silent): the regions are any voxel sets the caller marks
 * (the paper uses 20 x 20 pixel squares); sigma is the population standard
 * deviation (divided by the number of background voxels); log is base 10.
 * An empty region or background returns OR_ERR_ARG.
 * ---------------------------------------------------------------------- */
int or_snr(long Nx, int C, int Nm, int mode, const double *x, const uint8_t *roi, double *snr_db)
{
    if (Nx <= 0 || C <= 0 || Nm <= 0 || Nm > 254 || (mode == 0 && C < Nm)) return OR_ERR_ARG;
    double *mu = (double *)calloc((size_t)Nm * C, sizeof(double));
    double *bm = (double *)calloc((size_t)C, sizeof(double));
    double *sd = (double *)calloc((size_t)C, sizeof(double));
    long *cnt = (long *)calloc((size_t)Nm, sizeof(long));
    if (!mu || !bm || !sd || !cnt) {
        free(mu); free(bm); free(sd); free(cnt);
        return OR_ERR_NOMEM;
    }
    long nb = 0;
    for (long n = 0; n < Nx; ++n) {
        int r = roi[n];
        if (r == 255) {
            ++nb;
            for (int c = 0; c < C; ++c) bm[c] += x[n * C + c];
        } else if (r >= 1 && r <= Nm) {
            ++cnt[r - 1];
            for (int c = 0; c < C; ++c) mu[(size_t)(r - 1) * C + c] += x[n * C + c];
        }
    }
    int bad = nb == 0;
    for (int m = 0; m < Nm; ++m) bad |= cnt[m] == 0;
    if (bad) {
        free(mu); free(bm); free(sd); free(cnt);
        return OR_ERR_ARG;
    }
    for (int c = 0; c < C; ++c) bm[c] /= (double)nb;
    for (int m = 0; m < Nm; ++m)
        for (int c = 0; c < C; ++c) mu[(size_t)m * C + c] /= (double)cnt[m];
    /* standard deviation over the background, about its mean (two passes) */
    for (long n = 0; n < Nx; ++n)
        if (roi[n] == 255)
            for (int c = 0; c < C; ++c) {
                double d = x[n * C + c] - bm[c];
                sd[c] += d * d;
            }
    for (int c = 0; c < C; ++c) sd[c] = sqrt(sd[c] / (double)nb);
    double acc = 0.0;
    long terms = 0;
    for (int m = 0; m < Nm; ++m)
        for (int c = 0; c < C; ++c) {
            if (mode == 0 && c != m) continue;
            double q = mu[(size_t)m * C + c] / sd[c];
            acc += q * q;
            ++terms;
        }
    *snr_db = 10.0 * log10(acc / (double)terms);
    free(mu); free(bm); free(sd); free(cnt);
    return OR_OK;
}

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper; the library's added form): a
 * 3-layer MLP mapping a pixel's Nk-bin spectrum p to K nonnegative subspace
 * coefficients, trained by mean-squared error against coefficients that the
 * plain method produced.
 *   z1 = W1 p + b1,  a1 = gelu(z1)          (H1 units)
 *   z2 = W2 a1 + b2, a2 = gelu(z2)          (H2 units)
 *   z3 = W3 a2 + b3, y = softplus(z3)       (K outputs)
 * gelu(x) = x Phi(x) (exact, erf form); softplus(z) = log(1 + e^z), z for z > 20.
 * loss = mean over the M pixels and K outputs of (y - t)^2.
 * Parameters are packed [W1 (H1 x Nk), b1, W2 (H2 x H1), b2, W3 (K x H2), b3],
 * weights row-major [out][in].
 * ---------------------------------------------------------------------- */
static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }
static double gelu_d(double x)
{
    const double phi = exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * phi;
}
static double softplus(double z) { return z > 20.0 ? z : log1p(exp(z)); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

double or_gelu(double x) { return gelu(x); }
double or_softplus(double z) { return softplus(z); }

long or_mlp_nparams(int Nk, int H1, int H2, int K)
{
    return (long)H1 * Nk + H1 + (long)H2 * H1 + H2 + (long)K * H2 + K;
}

/* forward for M pixels; Y [M][K]; returns the loss if T != NULL */
double or_mlp_forward(int M, int Nk, int H1, int H2, int K, const double *prm, const double *X,
                      double *Y, const double *T)
{
    const double *W1 = prm, *b1 = W1 + (long)H1 * Nk, *W2 = b1 + H1, *b2 = W2 + (long)H2 * H1;
    const double *W3 = b2 + H2, *b3 = W3 + (long)K * H2;
    double *a1 = (double *)malloc(sizeof(double) * H1), *a2 = (double *)malloc(sizeof(double) * H2);
    double loss = 0.0;
    for (int m = 0; m < M; ++m) {
        const double *x = X + (long)m * Nk;
        for (int j = 0; j < H1; ++j) {
            double z = b1[j];
            for (int k = 0; k < Nk; ++k) z += W1[(long)j * Nk + k] * x[k];
            a1[j] = gelu(z);
        }
        for (int j = 0; j < H2; ++j) {
            double z = b2[j];
            for (int k = 0; k < H1; ++k) z += W2[(long)j * H1 + k] * a1[k];
            a2[j] = gelu(z);
        }
        for (int j = 0; j < K; ++j) {
            double z = b3[j];
            for (int k = 0; k < H2; ++k) z += W3[(long)j * H2 + k] * a2[k];
            double y = softplus(z);
            Y[(long)m * K + j] = y;
            if (T) loss += (y - T[(long)m * K + j]) * (y - T[(long)m * K + j]);
        }
    }
    free(a1);
    free(a2);
    return T ? loss / ((double)M * K) : 0.0;
}

/* loss and its gradient with respect to every packed parameter (G, same layout) */
double or_mlp_grad(int M, int Nk, int H1, int H2, int K, const double *prm, const double *X,
                   const double *T, double *G)
{
    const double *W1 = prm, *b1 = W1 + (long)H1 * Nk, *W2 = b1 + H1, *b2 = W2 + (long)H2 * H1;
    const double *W3 = b2 + H2, *b3 = W3 + (long)K * H2;
    long np = or_mlp_nparams(Nk, H1, H2, K);
    memset(G, 0, sizeof(double) * np);
    double *gW1 = G, *gb1 = gW1 + (long)H1 * Nk, *gW2 = gb1 + H1, *gb2 = gW2 + (long)H2 * H1;
    double *gW3 = gb2 + H2, *gb3 = gW3 + (long)K * H2;
    double *z1 = (double *)malloc(sizeof(double) * H1), *a1 = (double *)malloc(sizeof(double) * H1);
    double *z2 = (double *)malloc(sizeof(double) * H2), *a2 = (double *)malloc(sizeof(double) * H2);
    double *d1 = (double *)malloc(sizeof(double) * H1), *d2 = (double *)malloc(sizeof(double) * H2);
    double *d3 = (double *)malloc(sizeof(double) * K);
    double loss = 0.0, scale = 2.0 / ((double)M * K);
    for (int m = 0; m < M; ++m) {
        const double *x = X + (long)m * Nk;
        for (int j = 0; j < H1; ++j) {
            double z = b1[j];
            for (int k = 0; k < Nk; ++k) z += W1[(long)j * Nk + k] * x[k];
            z1[j] = z;
            a1[j] = gelu(z);
        }
        for (int j = 0; j < H2; ++j) {
            double z = b2[j];
            for (int k = 0; k < H1; ++k) z += W2[(long)j * H1 + k] * a1[k];
            z2[j] = z;
            a2[j] = gelu(z);
        }
        for (int j = 0; j < K; ++j) {
            double z = b3[j];
            for (int k = 0; k < H2; ++k) z += W3[(long)j * H2 + k] * a2[k];
            double y = softplus(z), e = y - T[(long)m * K + j];
            loss += e * e;
            d3[j] = scale * e * sigmoid(z);          /* d loss / d z3 */
        }
        for (int k = 0; k < H2; ++k) {
            double s = 0.0;
            for (int j = 0; j < K; ++j) s += W3[(long)j * H2 + k] * d3[j];
            d2[k] = s * gelu_d(z2[k]);               /* d loss / d z2 */
        }
        for (int k = 0; k < H1; ++k) {
            double s = 0.0;
            for (int j = 0; j < H2; ++j) s += W2[(long)j * H1 + k] * d2[j];
            d1[k] = s * gelu_d(z1[k]);               /* d loss / d z1 */
        }
        for (int j = 0; j < K; ++j) {
            gb3[j] += d3[j];
            for (int k = 0; k < H2; ++k) gW3[(long)j * H2 + k] += d3[j] * a2[k];
        }
        for (int j = 0; j < H2; ++j) {
            gb2[j] += d2[j];
            for (int k = 0; k < H1; ++k) gW2[(long)j * H1 + k] += d2[j] * a1[k];
        }
        for (int j = 0; j < H1; ++j) {
            gb1[j] += d1[j];
            for (int k = 0; k < Nk; ++k) gW1[(long)j * Nk + k] += d1[j] * x[k];
        }
    }
    free(z1); free(a1); free(z2); free(a2); free(d1); free(d2); free(d3);
    return loss / ((double)M * K);
}

/* AdamW (decoupled weight decay), step t >= 1:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps) + lr wd w */
void or_adamw(long n, double *w, const double *g, double *m, double *v, int t, double lr, double b1,
              double b2, double eps, double wd)
{
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        w[i] -= lr * (mh / (sqrt(vh) + eps) + wd * w[i]);
    }
}
