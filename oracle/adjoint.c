/*
 * Oracle: gradients of a linear functional of the camera image by
 * likelihood ratios along replayed paths (test infrastructure only; see
 * oracle.h).
 *
 * The camera image of Sec. 3.1.3 / Sec. 4.3 is a sum over photons of
 * next-event contributions c_j = W_j p_sr(mu_c,j) exp(-mu_ext l_j) at each
 * collision j, W_j = a^j (a = mu_s/mu_ext, Eq. 16) times any roulette boosts.
 * The path density is a product of flight densities mu_ext exp(-mu_ext s_i)
 * (Eq. 15) and polar-angle densities p(mu_i). For a parameter theta,
 *   dE[c_j]/dtheta = E[ c_j ( d log c_j/dtheta + sum over the flights and
 *                               scatterings before j of d log density/dtheta ) ]
 * with
 *   flight i:  d/dmu_s = d/dmu_a = 1/mu_ext - s_i
 *   W_j:       d/dmu_s = j (1/mu_s - 1/mu_ext),  d/dmu_a = -j/mu_ext
 *   transport: d/dmu_s = d/dmu_a = -l_j
 *   phase weights: p_w = p h_w / Z(w), h_w = sum_k w_k phi_k, Z_k = int p phi_k
 *   over the unweighted table p and Z(w) = sum_k w_k Z_k, so
 *   d log p_w(mu)/dw_k = phi_k(mu) / h_w(mu) - Z_k / Z(w) (at w = 1:
 *   phi_k(mu) - Z_k), both for the sampled angles mu_i (i < j) and for the
 *   camera density at mu_c,j. The walk samples p_w through its table, the
 *   unweighted table reweighted (oracle_phase_table_reweighted).
 * Flights that leave the cuvette carry no camera term and later terms of
 * the same photon do not depend on them. Each photon's path is simply
 * stored and summed afterwards.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

double oracle_hat(int n_w, int k, double mu)
{
    double h = 2.0 / (n_w - 1);
    double t = fabs(mu - (-1.0 + k * h)) / h;
    return t < 1.0 ? 1.0 - t : 0.0;
}

/* integral of phi_k over [a, b] (a < b), exactly: phi_k is piecewise linear
 * with breakpoints at the nodes, so integrate piece by piece. */
static double hat_integral(int n_w, int k, double a, double b)
{
    double h = 2.0 / (n_w - 1);
    double c = -1.0 + k * h;
    double pts[4] = {c - h, c, c + h};
    double s = 0.0, lo = a;
    for (int i = 0; i < 3 && lo < b; ++i) {
        double hi = fmin(b, pts[i]);
        if (hi > lo) {
            s += 0.5 * (oracle_hat(n_w, k, lo) + oracle_hat(n_w, k, hi)) * (hi - lo);
            lo = hi;
        }
    }
    if (b > lo)
        s += 0.5 * (oracle_hat(n_w, k, lo) + oracle_hat(n_w, k, b)) * (b - lo);
    return s;
}

void oracle_hat_integrals(const double *omu, int n_bins, int n_w, double *z)
{
    for (int k = 0; k < n_w; ++k) {
        double s = 0.0;
        for (int j = 0; j < n_bins; ++j) {
            double a = 1.0 - omu[j], b = 1.0 - omu[j + 1];
            double pdf = (1.0 / n_bins) / (omu[j] - omu[j + 1]);
            s += pdf * hat_integral(n_w, k, a, b);
        }
        z[k] = s;
    }
}

/* One photon's record. */
typedef struct {
    int n;          /* collisions */
    int cap;
    double *A;      /* adj[pix_j] * c_j */
    double *S;      /* prefix of flight scores up to flight j */
    double *l;      /* distance to the camera face */
    double *muc;    /* camera cosine d_y at collision j */
    double *mus;    /* polar cosine sampled at collision j (NAN: none) */
} rec_t;

static void rec_push(rec_t *R, double A, double S, double l, double muc)
{
    if (R->n == R->cap) {
        int nc = R->cap ? 2 * R->cap : 64;
        R->A = realloc(R->A, nc * sizeof(double));
        R->S = realloc(R->S, nc * sizeof(double));
        R->l = realloc(R->l, nc * sizeof(double));
        R->muc = realloc(R->muc, nc * sizeof(double));
        R->mus = realloc(R->mus, nc * sizeof(double));
        R->cap = nc;
    }
    R->A[R->n] = A;
    R->S[R->n] = S;
    R->l[R->n] = l;
    R->muc[R->n] = muc;
    R->mus[R->n] = NAN;
    R->n++;
}

static double hg_per_sr(double g, double mu)
{
    double t = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * M_PI * t * sqrt(t));
}

static double hg_sample(double g, double xi)
{
    if (fabs(g) < 1e-6)
        return 2.0 * xi - 1.0;
    double q = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
    return (1.0 + g * g - q * q) / (2.0 * g);
}

static int table_bin(const double *icdf, int n, double mu)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (icdf[mid] <= mu) lo = mid; else hi = mid;
    }
    return lo;
}

/* Walk photon p exactly as oracle_walk does, recording the collisions. */
static void replay(const oracle_walk_cfg *c, uint64_t p, const double *adj, rec_t *R)
{
    const uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
    const double mu_ext = c->mu_s + c->mu_a;
    const double lo[3] = {0.0, -0.5 * c->ly, -0.5 * c->lz};
    const double hi[3] = {c->lx, 0.5 * c->ly, 0.5 * c->lz};
    double r[3] = {0.0, 0.0, 0.0}, d[3] = {1.0, 0.0, 0.0}, w = 1.0, S = 0.0;
    uint32_t n_coll = 0;
    R->n = 0;
    if (c->beam_radius > 0.0) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u}, o[4];
        oracle_philox4x32_10(ctr, key, o);
        double rho = c->beam_radius * sqrt(oracle_uniform(o[0]));
        double psi = 2.0 * M_PI * oracle_uniform(o[1]);
        r[1] = rho * cos(psi);
        r[2] = rho * sin(psi);
    }
    for (uint32_t e = 0; e < c->max_events; ++e) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), e, 0u}, o[4];
        oracle_philox4x32_10(ctr, key, o);
        double u0 = oracle_uniform(o[0]), u1 = oracle_uniform(o[1]);
        double u2 = oracle_uniform(o[2]), u3 = oracle_uniform(o[3]);
        double s = -log(u0) / mu_ext;
        double sw = INFINITY;
        for (int i = 0; i < 3; ++i) {
            double t;
            if (d[i] > 0.0) t = (hi[i] - r[i]) / d[i];
            else if (d[i] < 0.0) t = (lo[i] - r[i]) / d[i];
            else continue;
            if (t < sw) sw = t;
        }
        if (s >= sw)
            return;
        for (int i = 0; i < 3; ++i) r[i] += s * d[i];
        n_coll++;
        S += 1.0 / mu_ext - s;
        w = w * (1.0 - c->mu_a / mu_ext);
        double muc = d[1], psr;
        if (c->phase_kind == ORACLE_PHASE_HG) {
            psr = hg_per_sr(c->hg_g, muc);
        } else {
            int nb = table_bin(c->icdf, c->n_bins, muc);
            psr = (1.0 / c->n_bins) / (c->omu[nb] - c->omu[nb + 1]) / (2.0 * M_PI);
        }
        double l = hi[1] - r[1];
        double nee = w * psr * exp(-mu_ext * l);
        double fx = r[0] / c->lx * c->nx, fz = (r[2] - lo[2]) / c->lz * c->nz;
        int ix = (int)floor(fx), iz = (int)floor(fz);
        if (ix < 0) ix = 0;
        if (ix > c->nx - 1) ix = c->nx - 1;
        if (iz < 0) iz = 0;
        if (iz > c->nz - 1) iz = c->nz - 1;
        rec_push(R, adj[iz * c->nx + ix] * nee, S, l, muc);
        if (c->max_scatter && n_coll >= c->max_scatter)
            return;
        double mu, omu;
        if (c->phase_kind == ORACLE_PHASE_HG) {
            mu = hg_sample(c->hg_g, u1);
            omu = 1.0 - mu;
        } else {
            double t = u1 * c->n_bins;
            int i = (int)floor(t);
            omu = c->omu[i] + (t - i) * (c->omu[i + 1] - c->omu[i]);
            mu = 1.0 - omu;
        }
        R->mus[R->n - 1] = mu;
        double st = sqrt(fmax(0.0, omu * (2.0 - omu)));
        double phi = 2.0 * M_PI * u2, cp = cos(phi), sp = sin(phi);
        double sg = copysign(1.0, d[2]), a = -1.0 / (sg + d[2]), b = d[0] * d[1] * a;
        double e1[3] = {1.0 + sg * d[0] * d[0] * a, sg * b, -sg * d[0]};
        double e2[3] = {b, sg + d[1] * d[1] * a, -d[1]};
        double nd[3];
        for (int i = 0; i < 3; ++i) nd[i] = mu * d[i] + st * (cp * e1[i] + sp * e2[i]);
        double nrm = sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
        for (int i = 0; i < 3; ++i) d[i] = nd[i] / nrm;
        if (w < c->rr_threshold) {
            if (u3 < c->rr_survival) w = w / c->rr_survival;
            else return;
        }
    }
}

typedef struct {
    const oracle_walk_cfg *c;
    const double *adj, *z, *w;   /* z: Z_k / Z(w); w: the weights */
    int n_w;
    uint64_t first, count;
    double *g, *g2;   /* [2 + n_w] */
    double value;
} ajob_t;

/* h_w(mu) = sum_k w_k phi_k(mu) */
static double h_w(int n_w, const double *w, double mu)
{
    double s = 0.0;
    for (int k = 0; k < n_w; ++k)
        s += w[k] * oracle_hat(n_w, k, mu);
    return s;
}

static void *adj_worker(void *arg)
{
    ajob_t *J = arg;
    const oracle_walk_cfg *c = J->c;
    const double mu_ext = c->mu_s + c->mu_a;
    const int m = 2 + J->n_w;
    double *pg = calloc((size_t)m, sizeof(double));
    rec_t R = {0};
    for (uint64_t k = 0; k < J->count; ++k) {
        replay(c, c->photon_offset + J->first + k, J->adj, &R);
        memset(pg, 0, (size_t)m * sizeof(double));
        for (int j = 0; j < R.n; ++j) {
            double jj = j + 1.0, A = R.A[j];
            J->value += A;
            pg[0] += A * (R.S[j] + jj * (1.0 / c->mu_s - 1.0 / mu_ext) - R.l[j]);
            pg[1] += A * (R.S[j] - jj / mu_ext - R.l[j]);
            for (int q = 0; q < J->n_w; ++q) {
                double t = oracle_hat(J->n_w, q, R.muc[j]) / h_w(J->n_w, J->w, R.muc[j]) - jj * J->z[q];
                for (int i = 0; i < j; ++i)
                    t += oracle_hat(J->n_w, q, R.mus[i]) / h_w(J->n_w, J->w, R.mus[i]);
                pg[2 + q] += A * t;
            }
        }
        for (int q = 0; q < m; ++q) {
            J->g[q] += pg[q];
            J->g2[q] += pg[q] * pg[q];
        }
    }
    free(pg);
    free(R.A); free(R.S); free(R.l); free(R.muc); free(R.mus);
    return NULL;
}

int oracle_adjoint(const oracle_walk_cfg *c, const double *adj, int n_w, double *grad, double *grad_sq,
                   double *value)
{
    return oracle_adjoint_weighted(c, adj, n_w, NULL, NULL, grad, grad_sq, value);
}

int oracle_adjoint_weighted(const oracle_walk_cfg *c, const double *adj, int n_w, const double *w,
                            const double *base_omu, double *grad, double *grad_sq, double *value)
{
    if (!c || !adj || !grad || !grad_sq || !value || n_w < 0 || n_w == 1 || !(c->mu_s > 0) || c->mu_a < 0)
        return -1;
    if (n_w > 0 && c->phase_kind != ORACLE_PHASE_MIE)
        return -1;
    if (c->phase_kind == ORACLE_PHASE_MIE && (!c->icdf || !c->omu))
        return -1;
    if (w && !base_omu)
        return -1;
    double *z = calloc((size_t)(n_w > 0 ? n_w : 1), sizeof(double));
    double *ws = malloc((size_t)(n_w > 0 ? n_w : 1) * sizeof(double));
    for (int k = 0; k < n_w; ++k) {
        ws[k] = w ? w[k] : 1.0;
        if (!(ws[k] > 0.0)) {
            free(z); free(ws);
            return -1;
        }
    }
    if (n_w > 0) {
        /* Z_k over the unweighted table, then Z_k / Z(w) */
        oracle_hat_integrals(base_omu ? base_omu : c->omu, c->n_bins, n_w, z);
        double zw = 0.0;
        for (int k = 0; k < n_w; ++k)
            zw += ws[k] * z[k];
        for (int k = 0; k < n_w; ++k)
            z[k] /= zw;
    }
    int T = c->n_threads > 0 ? c->n_threads : 1;
    if ((uint64_t)T > c->n_photons && c->n_photons > 0) T = (int)c->n_photons;
    if (T < 1) T = 1;
    ajob_t *jobs = calloc((size_t)T, sizeof *jobs);
    pthread_t *th = calloc((size_t)T, sizeof *th);
    for (int t = 0; t < T; ++t) {
        jobs[t].c = c;
        jobs[t].adj = adj;
        jobs[t].z = z;
        jobs[t].w = ws;
        jobs[t].n_w = n_w;
        jobs[t].first = c->n_photons * (uint64_t)t / (uint64_t)T;
        jobs[t].count = c->n_photons * (uint64_t)(t + 1) / (uint64_t)T - jobs[t].first;
        jobs[t].g = calloc((size_t)(2 + n_w), sizeof(double));
        jobs[t].g2 = calloc((size_t)(2 + n_w), sizeof(double));
        pthread_create(&th[t], NULL, adj_worker, &jobs[t]);
    }
    for (int t = 0; t < T; ++t) {
        pthread_join(th[t], NULL);
        for (int q = 0; q < 2 + n_w; ++q) {
            grad[q] += jobs[t].g[q];
            grad_sq[q] += jobs[t].g2[q];
        }
        *value += jobs[t].value;
        free(jobs[t].g);
        free(jobs[t].g2);
    }
    free(jobs);
    free(th);
    free(z);
    free(ws);
    return 0;
}

/* ------------------------------------------------------------------------
 * Gradient of L = sum adj * image with respect to the voxel densities n_v of
 * a heterogeneous medium (oracle_walk_cfg.density; delta tracking in
 * walk.c). The paths are the oracle walk's own, read from its traces of real
 * events. For a photon with real collisions at r_1..r_J (entry point r_0),
 * camera terms c_j and A_j = adj[pix_j] c_j, P_i = A_1 + .. + A_i:
 *   flight i (r_{i-1} -> r_i) has density mu_s(r_i) exp(-int mu_ext) times
 *   the scattering share, so d log / d n_v = [r_i in v] / n_v - k_ext l_i(v)
 *   (l_i(v): length of the flight inside voxel v), and it multiplies every
 *   later camera term: coefficient P_J - P_{i-1};
 *   camera term j: d log c_j / d n_v = -k_ext lc_j(v), lc_j(v) the length of
 *   the column from r_j up to y = +ly/2 inside v.
 * (With mu_a = 0 the point term 1/n_v equals k_ext / mu_ext; with mu_a > 0 it
 * is k_ext / mu_ext from the flight plus 1/n_v - k_ext / mu_ext from the
 * albedo k_sca n_v / mu_ext.) Roulette is held fixed. The escaping flight
 * precedes no camera term.
 * ------------------------------------------------------------------------ */

static int cmp_dbl(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

static void voxel_of(const oracle_walk_cfg *c, const double lo[3], const double r[3], int v[3])
{
    const double L[3] = {c->lx, c->ly, c->lz};
    const int g[3] = {c->gx, c->gy, c->gz};
    for (int i = 0; i < 3; ++i) {
        v[i] = (int)floor((r[i] - lo[i]) / L[i] * g[i]);
        if (v[i] < 0) v[i] = 0;
        if (v[i] > g[i] - 1) v[i] = g[i] - 1;
    }
}

/* grad[v] += coef * (length of the segment a -> b inside v), every v: the
 * segment is cut at every voxel plane it crosses and each piece is given to
 * the voxel holding its midpoint. */
static void segment_voxels(const oracle_walk_cfg *c, const double lo[3], const double a[3],
                           const double b[3], double coef, double *grad, double *ts, size_t ts_cap)
{
    const double L[3] = {c->lx, c->ly, c->lz};
    const int g[3] = {c->gx, c->gy, c->gz};
    double d[3], len = 0.0;
    for (int i = 0; i < 3; ++i) {
        d[i] = b[i] - a[i];
        len += d[i] * d[i];
    }
    len = sqrt(len);
    if (!(len > 0.0))
        return;
    size_t n = 0;
    ts[n++] = 0.0;
    ts[n++] = 1.0;
    for (int i = 0; i < 3; ++i) {
        if (d[i] == 0.0)
            continue;
        const double h = L[i] / g[i];
        double fa = (a[i] - lo[i]) / h, fb = (b[i] - lo[i]) / h;
        int k0 = (int)floor(fmin(fa, fb)) + 1, k1 = (int)ceil(fmax(fa, fb)) - 1;
        for (int k = k0; k <= k1 && n < ts_cap; ++k)
            ts[n++] = (lo[i] + k * h - a[i]) / d[i];
    }
    qsort(ts, n, sizeof *ts, cmp_dbl);
    for (size_t q = 0; q + 1 < n; ++q) {
        const double t0 = fmax(ts[q], 0.0), t1 = fmin(ts[q + 1], 1.0);
        if (!(t1 > t0))
            continue;
        double m[3];
        for (int i = 0; i < 3; ++i)
            m[i] = a[i] + 0.5 * (t0 + t1) * d[i];
        int v[3];
        voxel_of(c, lo, m, v);
        grad[((size_t)v[2] * c->gy + v[1]) * c->gx + v[0]] += coef * (t1 - t0) * len;
    }
}

/* The point term of a real collision in voxel vi followed by camera terms
 * B: the flight's density ends in mu_ext there (d log / d n_v = k_ext /
 * mu_ext) and, with absorption, the albedo k_sca n_v / mu_ext adds 1 / n_v -
 * k_ext / mu_ext. */
static void point_term(const oracle_walk_cfg *c, size_t vi, double B, double *grad)
{
    const double n_v = c->density[vi];
    const double mu = c->k_ext * n_v + c->mu_a;
    grad[vi] += B * c->k_ext / mu;
    if (c->mu_a > 0.0 && n_v > 0.0)
        grad[vi] += B * (1.0 / n_v - c->k_ext / mu);
}

/* Camera term Ai of a collision at height ry in voxel v: -Ai k_ext times the
 * length of its column up to the camera face inside each voxel it crosses
 * (the rest of its own voxel, then every voxel above). */
static void camera_column(const oracle_walk_cfg *c, const double lo[3], const int v[3], double ry, double Ai,
                          double *grad)
{
    const double vy = c->ly / c->gy;
    const size_t vi = ((size_t)v[2] * c->gy + v[1]) * c->gx + v[0];
    const double top = (v[1] == c->gy - 1) ? 0.5 * c->ly : lo[1] + (v[1] + 1) * vy;
    grad[vi] -= Ai * c->k_ext * (top - ry);
    for (int j = v[1] + 1; j < c->gy; ++j)
        grad[((size_t)v[2] * c->gy + j) * c->gx + v[0]] -= Ai * c->k_ext * vy;
}

int oracle_grid_adjoint(const oracle_walk_cfg *c, const double *adj, int max_events, double *grad,
                        double *value)
{
    if (!c || !c->density || !adj || !grad || !value || max_events < 2)
        return -1;
    const size_t nv = (size_t)c->gx * c->gy * c->gz;
    const double lo[3] = {0.0, -0.5 * c->ly, -0.5 * c->lz};
    const uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
    const uint64_t batch = 2048;
    oracle_trace_rec *tr = malloc(batch * (size_t)max_events * sizeof *tr);
    double *A = malloc((size_t)max_events * sizeof *A);
    const size_t ts_cap = (size_t)c->gx + c->gy + c->gz + 8;
    double *ts = malloc(ts_cap * sizeof *ts);
    if (!tr || !A || !ts) {
        free(tr); free(A); free(ts);
        return -1;
    }
    memset(grad, 0, nv * sizeof *grad);
    double val = 0.0;
    int rc = 0;
    for (uint64_t first = 0; first < c->n_photons && rc == 0; first += batch) {
        const uint64_t cnt = (c->n_photons - first < batch) ? c->n_photons - first : batch;
        oracle_walk_cfg cb = *c;
        cb.photon_offset = c->photon_offset + first;
        cb.n_photons = cnt;
        cb.nx = c->nx;
        oracle_walk_out out;
        memset(&out, 0, sizeof out);
        if (oracle_walk(&cb, &out, tr, (int)cnt, max_events)) {
            rc = -1;
            break;
        }
        for (uint64_t q = 0; q < cnt; ++q) {
            const oracle_trace_rec *R = tr + q * (size_t)max_events;
            const uint64_t p = cb.photon_offset + q;
            /* real collisions of the photon, and its camera terms */
            int J = 0, ended = 0;
            for (int e = 0; e < max_events; ++e) {
                const int st = (int)R[e].status;
                if (st < 0) { ended = 1; break; }
                if (st == 0 || st == 4 || st == 5) {
                    A[J++] = adj[(int)R[e].pix] * R[e].nee;
                    if (st != 0) { ended = 1; break; }
                } else {
                    ended = 1;   /* left the cuvette or truncated */
                    break;
                }
            }
            if (!ended) {
                rc = -1;   /* more real events than max_events */
                break;
            }
            double P = 0.0;
            for (int j = 0; j < J; ++j)
                P += A[j];
            val += P;
            double r0[3] = {0.0, 0.0, 0.0};
            if (c->beam_radius > 0.0) {
                uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u}, o[4];
                oracle_philox4x32_10(ctr, key, o);
                double rho = c->beam_radius * sqrt(oracle_uniform(o[0]));
                double psi = 2.0 * M_PI * oracle_uniform(o[1]);
                r0[1] = rho * cos(psi);
                r0[2] = rho * sin(psi);
            }
            double prev[3] = {r0[0], r0[1], r0[2]}, Pb = 0.0;
            for (int i = 0; i < J; ++i) {
                const double *ri = R[i].r;
                const double B = P - Pb;   /* camera terms from collision i on */
                int v[3];
                voxel_of(c, lo, ri, v);
                const size_t vi = ((size_t)v[2] * c->gy + v[1]) * c->gx + v[0];
                if (B != 0.0) {
                    /* flight: point term and transmission along the flight */
                    point_term(c, vi, B, grad);
                    segment_voxels(c, lo, prev, ri, -B * c->k_ext, grad, ts, ts_cap);
                }
                /* camera term i: its column up to the camera face */
                if (A[i] != 0.0)
                    camera_column(c, lo, v, ri[1], A[i], grad);
                Pb += A[i];
                for (int k = 0; k < 3; ++k)
                    prev[k] = ri[k];
            }
        }
    }
    free(tr); free(A); free(ts);
    *value = val;
    return rc;
}

/* ------------------------------------------------------------------------
 * The same gradient with the flights' transmission scored at null
 * collisions. Delta tracking samples tentative collisions from the
 * majorant's exponential (independent of the densities); each is real with
 * probability mu_ext / mubar and null otherwise. Along a photon's path the
 * log-density therefore depends on n_v through log(mu_ext / mubar) at every
 * real collision in v and log(1 - mu_ext / mubar) at every null collision
 * in v, whose derivatives are k_ext / mu_ext and -k_ext / (mubar - mu_ext).
 * With B the camera terms that follow a flight (all of them from its real
 * collision on), a null collision in that flight adds -B k_ext / (mubar -
 * mu_ext) at its voxel; the real collision's point term and the camera
 * columns are those of oracle_grid_adjoint. The paths are the oracle walk's
 * own with null collisions traced; mubar > mu_ext everywhere needs
 * majorant_scale > 1.
 * ------------------------------------------------------------------------ */
int oracle_grid_adjoint_nulls(const oracle_walk_cfg *c0, const double *adj, int max_events, double *grad,
                              double *value)
{
    if (!c0 || !c0->density || !adj || !grad || !value || max_events < 2 || !(c0->majorant_scale > 1.0))
        return -1;
    oracle_walk_cfg cfg = *c0;
    cfg.trace_nulls = 1;
    const oracle_walk_cfg *c = &cfg;
    const size_t nv = (size_t)c->gx * c->gy * c->gz;
    const double lo[3] = {0.0, -0.5 * c->ly, -0.5 * c->lz};
    const uint64_t batch = 1024;
    oracle_trace_rec *tr = malloc(batch * (size_t)max_events * sizeof *tr);
    if (!tr)
        return -1;
    memset(grad, 0, nv * sizeof *grad);
    double val = 0.0;
    int rc = 0;
    for (uint64_t first = 0; first < c->n_photons && rc == 0; first += batch) {
        const uint64_t cnt = (c->n_photons - first < batch) ? c->n_photons - first : batch;
        oracle_walk_cfg cb = *c;
        cb.photon_offset = c->photon_offset + first;
        cb.n_photons = cnt;
        oracle_walk_out out;
        memset(&out, 0, sizeof out);
        if (oracle_walk(&cb, &out, tr, (int)cnt, max_events)) {
            rc = -1;
            break;
        }
        for (uint64_t q = 0; q < cnt && rc == 0; ++q) {
            const oracle_trace_rec *R = tr + q * (size_t)max_events;
            /* the photon's camera terms, and where its records end */
            double P = 0.0;
            int n_rec = -1;
            for (int e = 0; e < max_events; ++e) {
                const int st = (int)R[e].status;
                if (st == 0 || st == 4 || st == 5)
                    P += adj[(int)R[e].pix] * R[e].nee;
                if (st == 0 || st == 7)
                    continue;
                n_rec = e;   /* the photon ended at record e */
                break;
            }
            if (n_rec < 0) {
                rc = -1;   /* more events than max_events */
                break;
            }
            val += P;
            double Pb = 0.0;   /* camera terms before the current flight */
            for (int e = 0; e <= n_rec; ++e) {
                const oracle_trace_rec *r = &R[e];
                const int st = (int)r->status;
                const double B = P - Pb;
                if (st == 7) {
                    if (B != 0.0)
                        grad[(size_t)r->pix] -= B * c->k_ext / (r->nee - r->w);
                    continue;
                }
                if (!(st == 0 || st == 4 || st == 5))
                    break;   /* left the cuvette or truncated: no camera term follows */
                int v[3];
                voxel_of(c, lo, r->r, v);
                const size_t vi = ((size_t)v[2] * c->gy + v[1]) * c->gx + v[0];
                const double A = adj[(int)r->pix] * r->nee;
                if (B != 0.0)
                    point_term(c, vi, B, grad);
                if (A != 0.0)
                    camera_column(c, lo, v, r->r[1], A, grad);
                Pb += A;
            }
        }
    }
    free(tr);
    *value = val;
    return rc;
}
