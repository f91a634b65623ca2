/*
 * Oracle: the photon random walk, double precision (test infrastructure
 * only; see oracle.h).
 *
 * Sec. 2.6 / Sec. 3.1.3: photons are independent; each one, launched along x
 * into the cuvette, repeats
 *   free path s = -ln(u) / mu_ext                                   (Eq. 15)
 *   boundary test: the cuvette walls are index matched, so a flight that
 *     reaches a wall leaves there (reflect: x = 0, far: x = lx, side: y/z)
 *   collision: implicit capture w <- w (1 - mu_abs/mu_ext)          (Eq. 16)
 *   next-event estimate for the 90-degree side camera (Sec. 4.3) on the
 *     y = +ly/2 face, looking along -y, orthographic:
 *       c = w p_sr(d_y) exp(-mu_ext (ly/2 - r_y)),
 *     p_sr the phase function per steradian, here the density of the same
 *     discretised table the walk samples (or Eq. 11 for H-G)
 *   scattering angle from the inverse-CDF table (Sec. 2.6), from the
 *     paper's 3000-angle cumulative distribution by binary search
 *     (Sec. 3.1.2), or from H-G with the same g (Sec. 3.1.3); azimuth phi
 *     uniform on [0, 2 pi)
 *   direction update in the orthonormal basis of Duff et al. (JCGT 6(1),
 *     2017), d' = mu d + sqrt(1 - mu^2) (cos phi e1 + sin phi e2)
 *   weight threshold (Sec. 3.1.3): below rr_threshold a photon survives with
 *     probability rr_survival and weight w / rr_survival, else it ends
 *     (rr_survival = 0 is the paper's plain cut at w < 0.001).
 * Event e of photon p draws its four uniforms from Philox4x32-10 with key
 * = seed and counter (p_lo, p_hi, e, 0): u0 free path, u1 polar angle,
 * u2 azimuth, u3 roulette. A finite beam draws its entry point from counter
 * (p_lo, p_hi, 0xFFFFFFFF, 0).
 * Tallies are plain double sums; per-photon squares give the variance.
 */
#include "oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double *image, *image_sq, *image_hits, *radial, *radial_sq;
    double totals[ORACLE_N_TOTALS], totals_sq[ORACLE_N_TOTALS];
    uint64_t steps, capped;
    /* per-photon scratch for the squares */
    int *hit_pix;
    double *hit_val;
    size_t hit_n, hit_cap;
} acc_t;

static void hit_push(acc_t *A, int pix, double v)
{
    if (A->hit_n == A->hit_cap) {
        size_t nc = A->hit_cap ? 2 * A->hit_cap : 256;
        A->hit_pix = realloc(A->hit_pix, nc * sizeof *A->hit_pix);
        A->hit_val = realloc(A->hit_val, nc * sizeof *A->hit_val);
        A->hit_cap = nc;
    }
    A->hit_pix[A->hit_n] = pix;
    A->hit_val[A->hit_n] = v;
    A->hit_n++;
}

/* Sum the photon's contributions per pixel, then add their squares. */
static void flush_photon_squares(acc_t *A)
{
    size_t n = A->hit_n;
    for (size_t i = 0; i < n; ++i) {
        if (A->hit_pix[i] < 0)
            continue;
        int pix = A->hit_pix[i];
        double s = A->hit_val[i];
        for (size_t j = i + 1; j < n; ++j)
            if (A->hit_pix[j] == pix) {
                s += A->hit_val[j];
                A->hit_pix[j] = -1;
            }
        A->image_sq[pix] += s * s;
    }
    A->hit_n = 0;
}

static double min2(double a, double b) { return a < b ? a : b; }

/* Distance of v to the nearest integer, in units of the grid size n. */
static double grid_margin(double v, int n)
{
    double f = v - floor(v);
    return min2(f, 1.0 - f) / n;
}

/* Eq. 11 per steradian. */
static double hg_per_sr(double g, double mu)
{
    double t = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * M_PI * t * sqrt(t));
}

/* Inverse of the H-G cumulative distribution in cos(theta). */
static double hg_sample(double g, double xi)
{
    if (fabs(g) < 1e-6)
        return 2.0 * xi - 1.0;
    double q = (1.0 - g * g) / (1.0 - g + 2.0 * g * xi);
    return (1.0 + g * g - q * q) / (2.0 * g);
}

/* Largest j in [0, n-1] with icdf[j] <= mu (plain bisection). */
static int table_bin(const double *icdf, int n, double mu)
{
    int lo = 0, hi = n; /* icdf[lo] <= mu holds for lo = 0 when mu >= -1 */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (icdf[mid] <= mu)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* Largest i in [0, n-1] with cdf[i] <= u (plain bisection; cdf[0] = 0). */
static int cdf_interval(const double *cdf, int n, double u)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (cdf[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* ---- heterogeneous medium (delta tracking) ------------------------------
 * The number density n is piecewise constant on a gx x gy x gz voxel grid
 * spanning the cuvette; mu_ext = k_ext n + mu_a and mu_s = k_sca n (Eq. 17
 * per voxel, mu_a a uniform background absorption). Free flights are sampled
 * by delta (Woodcock) tracking against a majorant that is constant on cells
 * of bx x by x bz voxels: the flight's optical depth tau = -ln u0 is spent
 * cell by cell at the cell's majorant; where it runs out, a tentative
 * collision is real with probability mu_ext / majorant (u3 decides), else
 * null (the photon goes on in the same direction with the next event's
 * numbers). A real collision reuses u3 for roulette as u3 * majorant /
 * mu_ext, uniform on [0, 1) given acceptance. The camera transmittance is
 * the exact optical depth of the voxel column above the collision. */

/* Voxel of r and mu_ext there; margin: distance to a voxel face. */
static double grid_mu(const oracle_walk_cfg *c, const double lo[3], const double r[3], int *ix,
                      int *iy, int *iz, double *margin)
{
    const double f[3] = {(r[0] - lo[0]) / c->lx * c->gx, (r[1] - lo[1]) / c->ly * c->gy,
                         (r[2] - lo[2]) / c->lz * c->gz};
    const int g[3] = {c->gx, c->gy, c->gz};
    int v[3];
    for (int i = 0; i < 3; ++i) {
        v[i] = (int)floor(f[i]);
        if (v[i] < 0) v[i] = 0;
        if (v[i] > g[i] - 1) v[i] = g[i] - 1;
        *margin = min2(*margin, grid_margin(f[i], g[i]));
    }
    *ix = v[0]; *iy = v[1]; *iz = v[2];
    return c->k_ext * c->density[((size_t)v[2] * c->gy + v[1]) * c->gx + v[0]] + c->mu_a;
}

/* One tentative flight spending tau. Returns 0 at a tentative collision (r
 * moved there, *mubar = the cell's majorant) or 1 when the flight reaches a
 * wall first (r on the wall, *face = its axis). */
static int delta_flight(const oracle_walk_cfg *c, const double *maj, const double lo[3],
                        const double hi[3], double r[3], const double d[3], double tau,
                        double *mubar, int *face, double *margin)
{
    const int g[3] = {c->gx, c->gy, c->gz};
    const int b[3] = {c->bx, c->by, c->bz};
    const double L[3] = {c->lx, c->ly, c->lz};
    int m[3], cell[3];
    for (int i = 0; i < 3; ++i) {
        m[i] = (g[i] + b[i] - 1) / b[i];
        double f = (r[i] - lo[i]) / L[i] * g[i] / b[i];
        cell[i] = (int)floor(f);
        if (cell[i] < 0) cell[i] = 0;
        if (cell[i] > m[i] - 1) cell[i] = m[i] - 1;
        if (d[i] != 0.0)
            *margin = min2(*margin, grid_margin(f, m[i]));
    }
    for (;;) {
        const double mb = maj[((size_t)cell[2] * m[1] + cell[1]) * m[0] + cell[0]];
        double t = INFINITY, t2 = INFINITY;
        int ax = -1;
        for (int i = 0; i < 3; ++i) {
            double plane, ti;
            if (d[i] > 0.0)
                plane = (cell[i] == m[i] - 1) ? hi[i] : lo[i] + (double)(cell[i] + 1) * b[i] * L[i] / g[i];
            else if (d[i] < 0.0)
                plane = (cell[i] == 0) ? lo[i] : lo[i] + (double)cell[i] * b[i] * L[i] / g[i];
            else
                continue;
            ti = (plane - r[i]) / d[i];
            if (ti < t) {
                t2 = t;
                t = ti;
                ax = i;
            } else if (ti < t2) {
                t2 = ti;
            }
        }
        if (mb * t > tau) {
            *margin = min2(*margin, (mb * t - tau) / tau);
            const double s = tau / mb;
            for (int i = 0; i < 3; ++i)
                r[i] += s * d[i];
            *mubar = mb;
            return 0;
        }
        if (tau > 0.0)
            *margin = min2(*margin, (tau - mb * t) / tau);
        if (isfinite(t2) && t > 0.0)
            *margin = min2(*margin, (t2 - t) / t);
        tau -= mb * t;
        for (int i = 0; i < 3; ++i)
            r[i] += t * d[i];
        cell[ax] += d[ax] > 0.0 ? 1 : -1;
        if (cell[ax] < 0 || cell[ax] >= m[ax]) {
            r[ax] = d[ax] > 0.0 ? hi[ax] : lo[ax];
            *face = ax;
            return 1;
        }
    }
}

/* Optical depth from r (in voxel ix, iy, iz) to the camera face y = +ly/2. */
static double column_depth(const oracle_walk_cfg *c, const double lo[3], const double hi[3],
                           const double r[3], int ix, int iy, int iz)
{
    const double vy = c->ly / c->gy;
    const double top = (iy == c->gy - 1) ? hi[1] : lo[1] + (iy + 1) * vy;
    const size_t row = (size_t)iz * c->gy;
    double od = (c->k_ext * c->density[(row + iy) * c->gx + ix] + c->mu_a) * (top - r[1]);
    for (int j = iy + 1; j < c->gy; ++j)
        od += (c->k_ext * c->density[(row + j) * c->gx + ix] + c->mu_a) * vy;
    return od;
}

static void run_photon(const oracle_walk_cfg *c, const double *maj, uint64_t p, acc_t *A,
                       oracle_trace_rec *tr, int n_tr_ev)
{
    const uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
    const double mu_ext = c->mu_s + c->mu_a;
    const double lo[3] = {0.0, -0.5 * c->ly, -0.5 * c->lz};
    const double hi[3] = {c->lx, 0.5 * c->ly, 0.5 * c->lz};
    double r[3] = {0.0, 0.0, 0.0}, d[3] = {1.0, 0.0, 0.0}, w = 1.0;
    double pt[ORACLE_N_TOTALS] = {0};
    uint32_t n_coll = 0;
    int rad_hit = -1;
    double rad_w = 0.0;

    if (c->beam_radius > 0.0) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u};
        uint32_t o[4];
        oracle_philox4x32_10(ctr, key, o);
        double rho = c->beam_radius * sqrt(oracle_uniform(o[0]));
        double psi = 2.0 * M_PI * oracle_uniform(o[1]);
        r[1] = rho * cos(psi);
        r[2] = rho * sin(psi);
    }

    const int het = c->density != NULL;
    uint32_t nrec = 0;   /* records written when null collisions are traced too */
    for (uint32_t e = 0;; ++e) {
        /* traces record the real events: every flight, or with delta
         * tracking every real collision and the exit (and, with
         * trace_nulls, every null collision in between) */
        const uint32_t ri = het ? (c->trace_nulls ? nrec : n_coll) : e;
        oracle_trace_rec *rec = (tr && ri < (uint32_t)n_tr_ev) ? &tr[ri] : NULL;
        if (e >= c->max_events) {
            pt[ORACLE_T_TRUNC] += w;
            A->capped++;
            if (rec) {
                memset(rec, 0, sizeof *rec);
                rec->status = 6;
                rec->pix = rec->nee_bin = rec->rad_bin = -1;
                rec->margin = INFINITY;
            }
            break;
        }
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), e, 0u};
        uint32_t o[4];
        oracle_philox4x32_10(ctr, key, o);
        double u0 = oracle_uniform(o[0]), u1 = oracle_uniform(o[1]);
        double u2 = oracle_uniform(o[2]), u3 = oracle_uniform(o[3]);
        A->steps++;

        int face = -1, escaped;
        double margin, mu_here = mu_ext, mubar = mu_ext, mua_here = c->mu_a;
        int vx = 0, vy = 0, vz = 0;
        if (het) {
            margin = INFINITY;
            escaped = delta_flight(c, maj, lo, hi, r, d, -log(u0), &mubar, &face, &margin);
            if (!escaped) {
                mu_here = grid_mu(c, lo, r, &vx, &vy, &vz, &margin);
                mua_here = mu_here - c->k_sca * c->density[((size_t)vz * c->gy + vy) * c->gx + vx];
                const double acc = mu_here / mubar;
                margin = min2(margin, fabs(u3 - acc));
                if (!(u3 < acc)) {   /* null collision */
                    if (c->trace_nulls) {
                        if (rec) {
                            memset(rec, 0, sizeof *rec);
                            rec->status = 7;
                            for (int i = 0; i < 3; ++i) {
                                rec->r[i] = r[i];
                                rec->d[i] = d[i];
                            }
                            rec->w = mu_here;
                            rec->nee = mubar;
                            rec->pix = (double)(((size_t)vz * c->gy + vy) * c->gx + vx);
                            rec->nee_bin = rec->rad_bin = -1;
                            rec->margin = margin;
                        }
                        nrec++;
                    }
                    continue;
                }
                u3 = u3 / acc;  /* uniform on [0, 1) given acceptance */
            }
        } else {
            /* Eq. 15 */
            double s = mu_ext > 0.0 ? -log(u0) / mu_ext : INFINITY;
            /* boundary: distance to the first wall along d */
            double sw = INFINITY, sw2 = INFINITY;
            for (int i = 0; i < 3; ++i) {
                double t;
                if (d[i] > 0.0)
                    t = (hi[i] - r[i]) / d[i];
                else if (d[i] < 0.0)
                    t = (lo[i] - r[i]) / d[i];
                else
                    continue;
                if (t < sw) {
                    sw2 = sw;
                    sw = t;
                    face = i;
                } else if (t < sw2) {
                    sw2 = t;
                }
            }
            margin = fabs(s - sw) / (sw > 0.0 ? sw : 1e-300);
            escaped = s >= sw;
            if (escaped) {
                for (int i = 0; i < 3; ++i)
                    r[i] += sw * d[i];
                if (isfinite(sw2))
                    margin = min2(margin, (sw2 - sw) / (sw > 0.0 ? sw : 1e-300));
            } else {
                for (int i = 0; i < 3; ++i)
                    r[i] += s * d[i];
            }
        }

        if (escaped) {
            double status;
            int rbin = -1;
            if (face == 0 && d[0] < 0.0) {
                pt[ORACLE_T_REFLECT] += w;
                status = 1;
            } else if (face == 0) {
                pt[ORACLE_T_FAR] += w;
                if (n_coll == 0)
                    pt[ORACLE_T_BALLISTIC] += w;
                double rho = sqrt(r[1] * r[1] + r[2] * r[2]);
                double fr = rho / c->r_max * c->n_radial;
                rbin = (int)floor(fr);
                if (rbin > c->n_radial - 1)
                    rbin = c->n_radial - 1;
                margin = min2(margin, grid_margin(fr, c->n_radial));
                rad_hit = rbin;
                rad_w = w;
                status = 2;
            } else {
                pt[ORACLE_T_SIDE] += w;
                if (face == 1 && d[1] > 0.0 && c->cone_cos > 0.0 && d[1] >= c->cone_cos)
                    pt[ORACLE_T_CONE] += w;
                status = 3;
            }
            if (rec) {
                rec->status = status;
                for (int i = 0; i < 3; ++i) {
                    rec->r[i] = r[i];
                    rec->d[i] = d[i];
                }
                rec->w = w;
                rec->nee = 0.0;
                rec->pix = -1;
                rec->nee_bin = -1;
                rec->rad_bin = rbin;
                rec->margin = margin;
            }
            break;
        }

        n_coll++;

        /* Eq. 16 */
        pt[ORACLE_T_ABSORB] += w * (mua_here / mu_here);
        w = w * (1.0 - mua_here / mu_here);

        /* camera: next-event estimate toward +y */
        double muc = d[1];
        double psr;
        int nbin = -1;
        if (c->phase_kind == ORACLE_PHASE_HG) {
            psr = hg_per_sr(c->hg_g, muc);
        } else if (c->phase_kind == ORACLE_PHASE_PAPER) {
            /* the sampled distribution is uniform in theta on each interval,
             * density (cdf[j+1] - cdf[j]) / dtheta per radian, hence that
             * divided by sin(theta) per unit cos(theta) */
            const int n = c->n_theta - 1;
            const double dth = M_PI / n;
            double thc = acos(fmax(-1.0, fmin(1.0, muc)));
            nbin = (int)floor(thc / dth);
            if (nbin > n - 1) nbin = n - 1;
            double stc = sin(thc);
            double pth = (c->cdf[nbin + 1] - c->cdf[nbin]) / dth;
            psr = stc > 0.0 ? pth / stc / (2.0 * M_PI) : 0.0;
            margin = min2(margin, min2(cos(nbin * dth) - muc, muc - cos((nbin + 1) * dth)));
        } else {
            nbin = table_bin(c->icdf, c->n_bins, muc);
            double pdf = (1.0 / c->n_bins) / (c->omu[nbin] - c->omu[nbin + 1]);
            psr = pdf / (2.0 * M_PI);
            margin = min2(margin, min2(muc - c->icdf[nbin], c->icdf[nbin + 1] - muc));
        }
        double od = het ? column_depth(c, lo, hi, r, vx, vy, vz) : mu_ext * (hi[1] - r[1]);
        double nee = w * psr * exp(-od);
        double fx = r[0] / c->lx * c->nx;
        double fz = (r[2] - lo[2]) / c->lz * c->nz;
        int ix = (int)floor(fx), iz = (int)floor(fz);
        if (ix < 0) ix = 0;
        if (ix > c->nx - 1) ix = c->nx - 1;
        if (iz < 0) iz = 0;
        if (iz > c->nz - 1) iz = c->nz - 1;
        margin = min2(margin, min2(grid_margin(fx, c->nx), grid_margin(fz, c->nz)));
        int pix = iz * c->nx + ix;
        A->image[pix] += nee;
        A->image_hits[pix] += 1.0;
        hit_push(A, pix, nee);

        double status = 0;
        if (c->max_scatter && n_coll >= c->max_scatter) {
            pt[ORACLE_T_TRUNC] += w;
            status = 5;
        } else {
            /* polar angle */
            double mu, omu;
            if (c->phase_kind == ORACLE_PHASE_HG) {
                mu = hg_sample(c->hg_g, u1);
                omu = 1.0 - mu;
            } else if (c->phase_kind == ORACLE_PHASE_PAPER) {
                /* binary search of the cumulative distribution, then linear
                 * interpolation in theta inside the interval (Sec. 3.1.2) */
                const int n = c->n_theta - 1;
                int i = cdf_interval(c->cdf, n, u1);
                double f = (u1 - c->cdf[i]) / (c->cdf[i + 1] - c->cdf[i]);
                margin = min2(margin, min2(u1 - c->cdf[i], c->cdf[i + 1] - u1));
                double th = (i + f) * (M_PI / n);
                double sh = sin(0.5 * th);
                omu = 2.0 * sh * sh;
                mu = cos(th);
            } else {
                double t = u1 * c->n_bins;
                int i = (int)floor(t);
                double f = t - i;
                omu = c->omu[i] + f * (c->omu[i + 1] - c->omu[i]);
                mu = 1.0 - omu;
            }
            double st = sqrt(fmax(0.0, omu * (2.0 - omu)));
            double phi = 2.0 * M_PI * u2;
            double cp = cos(phi), sp = sin(phi);
            /* Duff et al. basis around d */
            double sg = copysign(1.0, d[2]);
            double a = -1.0 / (sg + d[2]);
            double b = d[0] * d[1] * a;
            double e1[3] = {1.0 + sg * d[0] * d[0] * a, sg * b, -sg * d[0]};
            double e2[3] = {b, sg + d[1] * d[1] * a, -d[1]};
            double nd[3];
            for (int i = 0; i < 3; ++i)
                nd[i] = mu * d[i] + st * (cp * e1[i] + sp * e2[i]);
            double nrm = sqrt(nd[0] * nd[0] + nd[1] * nd[1] + nd[2] * nd[2]);
            for (int i = 0; i < 3; ++i)
                d[i] = nd[i] / nrm;

            /* weight threshold */
            if (w < c->rr_threshold) {
                margin = min2(margin, fabs(w - c->rr_threshold) / c->rr_threshold);
                if (het)
                    margin = min2(margin, fabs(u3 - c->rr_survival));
                if (u3 < c->rr_survival) {
                    double wn = w / c->rr_survival;
                    pt[ORACLE_T_ROULETTE] += w - wn;
                    w = wn;
                } else {
                    pt[ORACLE_T_ROULETTE] += w;
                    status = 4;
                }
            }
        }
        if (rec) {
            rec->status = status;
            for (int i = 0; i < 3; ++i) {
                rec->r[i] = r[i];
                rec->d[i] = d[i];
            }
            rec->w = (status == 4) ? 0.0 : w;
            rec->nee = nee;
            rec->pix = pix;
            rec->nee_bin = nbin;
            rec->rad_bin = -1;
            rec->margin = margin;
        }
        nrec++;
        if (status != 0)
            break;
    }

    for (int k = 0; k < ORACLE_N_TOTALS; ++k) {
        A->totals[k] += pt[k];
        A->totals_sq[k] += pt[k] * pt[k];
    }
    if (rad_hit >= 0) {
        A->radial[rad_hit] += rad_w;
        A->radial_sq[rad_hit] += rad_w * rad_w;
    }
    flush_photon_squares(A);
}

typedef struct {
    const oracle_walk_cfg *c;
    const double *maj;
    acc_t acc;
    uint64_t first, count;
    oracle_trace_rec *trace;
    int n_trace, n_trace_events;
    int fail;
} job_t;

static void *worker(void *arg)
{
    job_t *J = arg;
    const oracle_walk_cfg *c = J->c;
    for (uint64_t k = 0; k < J->count; ++k) {
        uint64_t rel = J->first + k;
        oracle_trace_rec *tr = NULL;
        if (J->trace && rel < (uint64_t)J->n_trace)
            tr = J->trace + rel * (uint64_t)J->n_trace_events;
        run_photon(c, J->maj, c->photon_offset + rel, &J->acc, tr, J->n_trace_events);
    }
    return NULL;
}

int oracle_walk(const oracle_walk_cfg *c, oracle_walk_out *out,
                oracle_trace_rec *trace, int n_trace, int n_trace_events)
{
    if (!c || !out || c->nx < 1 || c->nz < 1 || c->n_radial < 1 ||
        !(c->lx > 0) || !(c->ly > 0) || !(c->lz > 0) || c->mu_s < 0 ||
        c->mu_a < 0 || !(c->r_max > 0) || c->beam_radius < 0)
        return -1;
    if (c->phase_kind == ORACLE_PHASE_MIE && (!c->icdf || !c->omu || c->n_bins < 2))
        return -1;
    if (c->phase_kind == ORACLE_PHASE_PAPER && (!c->cdf || c->n_theta < 3))
        return -1;
    if (c->phase_kind < 0 || c->phase_kind > ORACLE_PHASE_PAPER)
        return -1;
    double *maj = NULL;
    if (c->density) {
        if (c->gx < 1 || c->gy < 1 || c->gz < 1 || c->bx < 1 || c->by < 1 || c->bz < 1 ||
            !(c->k_ext >= c->k_sca) || !(c->k_sca >= 0.0))
            return -1;
        const size_t nv = (size_t)c->gx * c->gy * c->gz;
        for (size_t i = 0; i < nv; ++i)
            if (!(c->density[i] >= 0.0) || !isfinite(c->density[i]))
                return -1;
        /* majorant of each cell: mu_ext at the densest voxel it holds */
        const int mx = (c->gx + c->bx - 1) / c->bx, my = (c->gy + c->by - 1) / c->by,
                  mz = (c->gz + c->bz - 1) / c->bz;
        maj = calloc((size_t)mx * my * mz, sizeof *maj);
        if (!maj)
            return -1;
        for (int z = 0; z < c->gz; ++z)
            for (int y = 0; y < c->gy; ++y)
                for (int x = 0; x < c->gx; ++x) {
                    double mu = c->k_ext * c->density[((size_t)z * c->gy + y) * c->gx + x] + c->mu_a;
                    double *q = &maj[((size_t)(z / c->bz) * my + y / c->by) * mx + x / c->bx];
                    if (mu > *q)
                        *q = mu;
                }
        if (c->majorant_scale > 0.0 && c->majorant_scale != 1.0) {
            if (!(c->majorant_scale > 1.0) || !isfinite(c->majorant_scale)) {
                free(maj);
                return -1;
            }
            for (size_t i = 0; i < (size_t)mx * my * mz; ++i)
                maj[i] *= c->majorant_scale;
        }
    } else if (!(c->mu_s + c->mu_a > 0.0)) {
        return -1;
    }
    if (c->phase_kind == ORACLE_PHASE_HG && !(c->hg_g > -1.0 && c->hg_g < 1.0))
        return -1;
    if (trace) {
        for (size_t i = 0; i < (size_t)n_trace * (size_t)n_trace_events; ++i) {
            memset(&trace[i], 0, sizeof trace[i]);
            trace[i].status = -1;
        }
    }
    int T = c->n_threads > 0 ? c->n_threads : 1;
    if ((uint64_t)T > c->n_photons && c->n_photons > 0)
        T = (int)c->n_photons;
    if (T < 1)
        T = 1;
    size_t npix = (size_t)c->nx * c->nz;
    job_t *jobs = calloc((size_t)T, sizeof *jobs);
    pthread_t *th = calloc((size_t)T, sizeof *th);
    if (!jobs || !th) {
        free(jobs);
        free(th);
        free(maj);
        return -1;
    }
    int rc = 0;
    for (int t = 0; t < T; ++t) {
        job_t *J = &jobs[t];
        J->c = c;
        J->maj = maj;
        J->first = c->n_photons * (uint64_t)t / (uint64_t)T;
        J->count = c->n_photons * (uint64_t)(t + 1) / (uint64_t)T - J->first;
        J->trace = trace;
        J->n_trace = n_trace;
        J->n_trace_events = n_trace_events;
        J->acc.image = calloc(npix, sizeof(double));
        J->acc.image_sq = calloc(npix, sizeof(double));
        J->acc.image_hits = calloc(npix, sizeof(double));
        J->acc.radial = calloc((size_t)c->n_radial, sizeof(double));
        J->acc.radial_sq = calloc((size_t)c->n_radial, sizeof(double));
        if (!J->acc.image || !J->acc.image_sq || !J->acc.image_hits || !J->acc.radial ||
            !J->acc.radial_sq)
            rc = -1;
    }
    if (rc == 0) {
        for (int t = 0; t < T; ++t)
            pthread_create(&th[t], NULL, worker, &jobs[t]);
        for (int t = 0; t < T; ++t)
            pthread_join(th[t], NULL);
        /* merge in thread order */
        for (int t = 0; t < T; ++t) {
            acc_t *A = &jobs[t].acc;
            for (size_t i = 0; i < npix; ++i) {
                if (out->image) out->image[i] += A->image[i];
                if (out->image_sq) out->image_sq[i] += A->image_sq[i];
                if (out->image_hits) out->image_hits[i] += A->image_hits[i];
            }
            for (int i = 0; i < c->n_radial; ++i) {
                if (out->radial) out->radial[i] += A->radial[i];
                if (out->radial_sq) out->radial_sq[i] += A->radial_sq[i];
            }
            for (int k = 0; k < ORACLE_N_TOTALS; ++k) {
                out->totals[k] += A->totals[k];
                out->totals_sq[k] += A->totals_sq[k];
            }
            out->steps += A->steps;
            out->capped += A->capped;
        }
    }
    for (int t = 0; t < T; ++t) {
        acc_t *A = &jobs[t].acc;
        free(A->image); free(A->image_sq); free(A->image_hits);
        free(A->radial); free(A->radial_sq);
        free(A->hit_pix); free(A->hit_val);
    }
    free(jobs);
    free(th);
    free(maj);
    return rc;
}
