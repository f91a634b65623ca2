/*
 * Oracle, single-precision mode (test infrastructure only; see oracle.h).
 *
 * The walk of Sec. 2.6 / Sec. 3.1.3 in a homogeneous medium, restated in
 * IEEE single precision with every fused multiply-add written out as fmaf
 * and the C library's correctly rounded or faithful logf / expf / sincosf /
 * sqrtf (the file is compiled without contraction, so nothing else fuses).
 * Same photons, events and Philox numbers as walk.c; traces only. Steps:
 *   free path s = -ln(u0) / mu_ext                                   (Eq. 15)
 *   the flight r + s d leaves through the first wall it reaches, else a
 *   collision there: w <- w mu_s / mu_ext                             (Eq. 16)
 *   camera term w p_sr(d_y) exp(-mu_ext (ly/2 - r_y)) on the y = +ly/2 face,
 *     p_sr the density of the sampled table per steradian, or Eq. 11 for H-G
 *   polar angle from the table by linear interpolation between its levels,
 *     or from the H-G inverse, written for 1 - cos(theta) without
 *     cancellation: 1 - mu = 2 (1-g)^2 (1-xi) (1+g xi) / (1-g+2g xi)^2
 *   azimuth 2 pi u2; d' = mu d + sin(theta) (cos phi e1 + sin phi e2) in the
 *     basis of Duff et al. (JCGT 6(1), 2017), renormalised
 *   weight threshold: below rr_threshold survive with rr_survival (w / it)
 * The table enters as the double-precision levels of 1 - cos(theta) rounded
 * to float, and the density of bin j as (1/n) / (omu_j - omu_{j+1})
 * computed in double and rounded. Trace records and margins as in walk.c.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static const float PI_F = 3.14159265358979323846f;

static double min2d(double a, double b) { return a < b ? a : b; }

static double grid_margin32(double v, int n)
{
    double f = v - floor(v);
    return min2d(f, 1.0 - f) / n;
}

/* Largest j in [0, n-1] with omu[j] >= om (omu decreasing from 2 to 0). */
static int bin_of_omu(const float *omu, int n, float om)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (omu[mid] >= om)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

static void put(oracle_trace_rec *rec, double status, const float r[3], const float d[3], float w,
                float nee, int pix, int nbin, int rbin, double margin)
{
    if (!rec)
        return;
    rec->status = status;
    for (int i = 0; i < 3; ++i) {
        rec->r[i] = r[i];
        rec->d[i] = d[i];
    }
    rec->w = w;
    rec->nee = nee;
    rec->pix = pix;
    rec->nee_bin = nbin;
    rec->rad_bin = rbin;
    rec->margin = margin;
}

static void photon32(const oracle_walk_cfg *c, const float *omu, const float *pdf, uint64_t p,
                     oracle_trace_rec *tr, int n_ev)
{
    const uint32_t key[2] = {(uint32_t)c->seed, (uint32_t)(c->seed >> 32)};
    /* the coefficients and the albedo of Eq. 16, each rounded once */
    const float mu_ext = (float)(c->mu_s + c->mu_a);
    const float albedo = (float)(c->mu_s / (c->mu_s + c->mu_a));
    const float lx = (float)c->lx, hy = 0.5f * (float)c->ly, hz = 0.5f * (float)c->lz;
    const float lo[3] = {0.0f, -hy, -hz}, hi[3] = {lx, hy, hz};
    const float g = (float)c->hg_g;
    const float thr = (float)c->rr_threshold, surv = (float)c->rr_survival;
    float r[3] = {0.0f, 0.0f, 0.0f}, d[3] = {1.0f, 0.0f, 0.0f}, w = 1.0f;
    uint32_t n_coll = 0;

    if (c->beam_radius > 0.0) {
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0xFFFFFFFFu, 0u};
        uint32_t o[4];
        oracle_philox4x32_10(ctr, key, o);
        float rho = (float)c->beam_radius * sqrtf((float)oracle_uniform(o[0]));
        float sp, cp;
        sincosf(2.0f * PI_F * (float)oracle_uniform(o[1]), &sp, &cp);
        r[1] = rho * cp;
        r[2] = rho * sp;
    }

    for (uint32_t e = 0;; ++e) {
        oracle_trace_rec *rec = (tr && e < (uint32_t)n_ev) ? &tr[e] : NULL;
        if (e >= c->max_events) {
            if (rec) {
                memset(rec, 0, sizeof *rec);
                rec->status = 6;
                rec->pix = rec->nee_bin = rec->rad_bin = -1;
                rec->margin = INFINITY;
            }
            break;
        }
        if (!rec)
            break;   /* nothing more is recorded */
        uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), e, 0u};
        uint32_t o[4];
        oracle_philox4x32_10(ctr, key, o);
        /* the uniforms (r >> 9) 2^-23 + 2^-24 are exact in single precision */
        const float u0 = (float)oracle_uniform(o[0]), u1 = (float)oracle_uniform(o[1]);
        const float u2 = (float)oracle_uniform(o[2]), u3 = (float)oracle_uniform(o[3]);

        /* Eq. 15 and the flight */
        const float s = -logf(u0) / mu_ext;
        float pnt[3];
        for (int i = 0; i < 3; ++i)
            pnt[i] = fmaf(s, d[i], r[i]);
        const int out = !(pnt[0] > 0.0f && pnt[0] < lx) || !(fabsf(pnt[1]) < hy) || !(fabsf(pnt[2]) < hz);

        /* distances to the walls along d: the first one is the exit */
        float sw = INFINITY, sw2 = INFINITY;
        int face = -1;
        for (int i = 0; i < 3; ++i) {
            float t;
            if (d[i] > 0.0f)
                t = (hi[i] - r[i]) / d[i];
            else if (d[i] < 0.0f)
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
        double margin = fabs((double)s - sw) / (sw > 0.0f ? sw : 1e-300);

        if (out) {
            float ex[3];
            for (int i = 0; i < 3; ++i)
                ex[i] = fmaf(sw, d[i], r[i]);
            if (isfinite(sw2))
                margin = min2d(margin, ((double)sw2 - sw) / (sw > 0.0f ? sw : 1e-300));
            int rbin = -1;
            double status;
            if (face == 0 && d[0] < 0.0f) {
                status = 1;
            } else if (face == 0) {
                const float rho = sqrtf(fmaf(ex[1], ex[1], ex[2] * ex[2]));
                const double fr = (double)rho / c->r_max * c->n_radial;
                rbin = (int)floor(fr);
                if (rbin > c->n_radial - 1)
                    rbin = c->n_radial - 1;
                margin = min2d(margin, grid_margin32(fr, c->n_radial));
                status = 2;
            } else {
                status = 3;
            }
            put(rec, status, ex, d, w, 0.0f, -1, -1, rbin, margin);
            break;
        }

        for (int i = 0; i < 3; ++i)
            r[i] = pnt[i];
        n_coll++;
        w = w * albedo;   /* Eq. 16 */

        /* camera */
        const float muc = d[1];
        float psr;
        int nbin = -1;
        if (c->phase_kind == ORACLE_PHASE_HG) {
            const float t = fmaf(2.0f * g, 1.0f - muc, (1.0f - g) * (1.0f - g));
            psr = (1.0f - g * g) / (4.0f * PI_F) / (t * sqrtf(t));
        } else {
            const float om = 1.0f - fminf(fmaxf(muc, -1.0f), 1.0f);
            nbin = bin_of_omu(omu, c->n_bins, om);
            psr = pdf[nbin] / (2.0f * PI_F);
            margin = min2d(margin, min2d((double)omu[nbin] - om, (double)om - omu[nbin + 1]));
        }
        const float nee = w * psr * expf(-mu_ext * (hy - r[1]));
        const double fx = (double)r[0] / c->lx * c->nx;
        /* rows measured from the axis: z = 0 is exactly row nz / 2 (the
           pixel-tie reading); hz, the float half-height, would round it */
        const double fz = (double)r[2] / c->lz * c->nz + 0.5 * c->nz;
        int ix = (int)floor(fx), iz = (int)floor(fz);
        if (ix > c->nx - 1) ix = c->nx - 1;
        if (iz > c->nz - 1) iz = c->nz - 1;
        if (ix < 0) ix = 0;
        if (iz < 0) iz = 0;
        margin = min2d(margin, min2d(grid_margin32(fx, c->nx), grid_margin32(fz, c->nz)));
        const int pix = iz * c->nx + ix;

        double status = 0;
        if (c->max_scatter && n_coll >= c->max_scatter) {
            status = 5;
        } else {
            /* polar angle as om = 1 - cos(theta) and op = 1 + cos(theta) */
            float om, op;
            if (c->phase_kind == ORACLE_PHASE_HG) {
                const float D = fmaf(2.0f * g, u1, 1.0f - g);
                om = 2.0f * (1.0f - g) * (1.0f - g) * (1.0f - u1) * fmaf(g, u1, 1.0f) / (D * D);
                /* the inverse of Eq. 11 written for 1 + cos(theta) too, so that
                   an angle near pi does not lose 1 + cos(theta) in 2 - om */
                op = 2.0f * (1.0f + g) * (1.0f + g) * u1 * fmaf(g, u1, 1.0f - g) / (D * D);
            } else {
                const float t = u1 * (float)c->n_bins;
                const int i = (int)t;
                const float f = t - (float)i;
                om = fmaf(f, omu[i + 1] - omu[i], omu[i]);
                op = 2.0f - om;
            }
            const float mu = om <= op ? 1.0f - om : op - 1.0f;
            const float st = sqrtf(fmaxf(om * op, 0.0f));
            float sp, cp;
            sincosf(2.0f * PI_F * u2, &sp, &cp);
            /* Duff et al. basis around d */
            const float sg = copysignf(1.0f, d[2]);
            const float a = -1.0f / (sg + d[2]);
            const float b = d[0] * d[1] * a;
            const float e1[3] = {fmaf(sg * d[0] * d[0], a, 1.0f), sg * b, -sg * d[0]};
            const float e2[3] = {b, fmaf(d[1] * d[1], a, sg), -d[1]};
            float nd[3];
            for (int i = 0; i < 3; ++i)
                nd[i] = fmaf(mu, d[i], st * fmaf(cp, e1[i], sp * e2[i]));
            const float nrm = sqrtf(fmaf(nd[0], nd[0], fmaf(nd[1], nd[1], nd[2] * nd[2])));
            for (int i = 0; i < 3; ++i)
                d[i] = nd[i] / nrm;
            /* weight threshold */
            if (w < thr) {
                margin = min2d(margin, fabs((double)w - thr) / thr);
                if (u3 < surv) {
                    w = w / surv;
                } else {
                    status = 4;
                }
            }
        }
        put(rec, status, r, d, status == 4 ? 0.0f : w, nee, pix, nbin, -1, margin);
        if (status != 0)
            break;
    }
}

int oracle_walk32_trace(const oracle_walk_cfg *c, oracle_trace_rec *trace, int n_trace, int n_trace_events)
{
    if (!c || !trace || n_trace < 0 || n_trace_events < 1 || c->density || !(c->mu_s > 0.0) ||
        c->mu_a < 0.0 || (c->phase_kind != ORACLE_PHASE_MIE && c->phase_kind != ORACLE_PHASE_HG) ||
        (c->phase_kind == ORACLE_PHASE_MIE && (!c->omu || c->n_bins < 2)) ||
        (c->phase_kind == ORACLE_PHASE_HG && !(c->hg_g > -1.0 && c->hg_g < 1.0)) || c->nx < 1 || c->nz < 1 ||
        c->n_radial < 1 || !(c->r_max > 0) || !(c->lx > 0) || !(c->ly > 0) || !(c->lz > 0) || c->beam_radius < 0)
        return -1;
    const int n = c->phase_kind == ORACLE_PHASE_MIE ? c->n_bins : 0;
    float *omu = NULL, *pdf = NULL;
    if (n) {
        omu = malloc(sizeof(float) * (n + 1));
        pdf = malloc(sizeof(float) * n);
        if (!omu || !pdf) {
            free(omu);
            free(pdf);
            return -1;
        }
        for (int j = 0; j <= n; ++j)
            omu[j] = (float)c->omu[j];
        for (int j = 0; j < n; ++j)
            pdf[j] = (float)((1.0 / n) / (c->omu[j] - c->omu[j + 1]));
    }
    memset(trace, 0, sizeof *trace * (size_t)n_trace * n_trace_events);
    for (size_t k = 0; k < (size_t)n_trace * n_trace_events; ++k)
        trace[k].status = -1;   /* no event */
    for (int k = 0; k < n_trace; ++k)
        photon32(c, omu, pdf, c->photon_offset + (uint64_t)k, trace + (size_t)k * n_trace_events, n_trace_events);
    free(omu);
    free(pdf);
    return 0;
}
