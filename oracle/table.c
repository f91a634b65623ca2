/*
 * Oracle: phase-function normalisation and inverse-CDF table (test
 * infrastructure only; see oracle.h).
 *
 * Sec. 3.1.2 precomputes the phase function on an angular grid and builds a
 * cumulative distribution function that Sec. 2.6 inverts to sample the
 * scattering angle. Steps, in that order:
 *   1. P(cos theta) on a fine uniform theta grid (Eq. 9, or Eq. 11 for H-G).
 *   2. Normalise so that (1/2) int_{-1}^{1} P dmu = 1, which is Eq. 10 for an
 *      azimuthally symmetric P (dOmega = 2 pi dmu). Composite Simpson in theta
 *      on the density F(theta) = (1/2) P(cos theta) sin theta.
 *   3. CDF(mu) = (1/2) int_{-1}^{mu} P dmu', accumulated from theta = pi.
 *   4. Invert at the equal-probability levels i / n_bins: inside the Simpson
 *      panel that holds the level, the integral of the panel's interpolating
 *      parabola is solved for theta by bisection.
 * The sampled distribution is the piecewise-linear inverse CDF through those
 * nodes, whose density on bin j is (1/n_bins) / (icdf[j+1] - icdf[j]); the
 * walk's camera estimate uses that same density.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>

/* Eq. 11 times 4 pi, in the cancellation-free form
 * 1 + g^2 - 2 g cos(theta) = (1-g)^2 + 4 g sin^2(theta/2). */
static double hg_phase(double g, double theta)
{
    double sh = sin(0.5 * theta);
    double t = (1.0 - g) * (1.0 - g) + 4.0 * g * sh * sh;
    return (1.0 - g * g) / (t * sqrt(t));
}

/* Integral over [0, s] of the parabola through (0,f0), (h,f1), (2h,f2). */
static double panel_partial(double f0, double f1, double f2, double h, double s)
{
    double c1 = (-3.0 * f0 + 4.0 * f1 - f2) / (4.0 * h);
    double c2 = (f0 - 2.0 * f1 + f2) / (6.0 * h * h);
    return s * (f0 + s * (c1 + s * c2));
}

static int build_table(int kind, double m_re, double m_im, double x, double hg_g, int n_w,
                       const double *wts, int n_bins, int n_fine, double *icdf, double *omu,
                       double *pdf, double *diag);
static int invert_density(double *F, const double *mu, int n_fine, int n_bins, double *icdf,
                          double *omu, double *pdf, double *diag);

int oracle_phase_table(int kind, double m_re, double m_im, double x,
                       double hg_g, int n_bins, int n_fine, double *icdf,
                       double *omu, double *pdf, double *diag)
{
    return build_table(kind, m_re, m_im, x, hg_g, 0, NULL, n_bins, n_fine, icdf, omu, pdf, diag);
}

int oracle_phase_table_weighted(int kind, double m_re, double m_im, double x,
                                double hg_g, int n_w, const double *w, int n_bins,
                                int n_fine, double *icdf, double *omu, double *pdf,
                                double *diag)
{
    if (n_w < 2 || !w)
        return -1;
    return build_table(kind, m_re, m_im, x, hg_g, n_w, w, n_bins, n_fine, icdf, omu, pdf, diag);
}

static int build_table(int kind, double m_re, double m_im, double x, double hg_g, int n_w,
                       const double *wts, int n_bins, int n_fine, double *icdf, double *omu,
                       double *pdf, double *diag)
{
    if (n_bins < 2 || n_fine < 4 || (n_fine & 1))
        return -1;
    if (kind == ORACLE_PHASE_HG && !(hg_g > -1.0 && hg_g < 1.0))
        return -1;
    if (kind != ORACLE_PHASE_HG && kind != ORACLE_PHASE_MIE)
        return -1;

    const double h = M_PI / n_fine;
    /* Node j sits at theta_j = pi - j h, so mu increases with j. */
    double *F = malloc((size_t)(n_fine + 1) * sizeof *F);
    double *mu = malloc((size_t)(n_fine + 1) * sizeof *mu);
    if (!F || !mu)
        goto fail;

    for (int j = 0; j <= n_fine; ++j)
        mu[j] = cos((double)(n_fine - j) * h);
    if (kind == ORACLE_PHASE_MIE) {
        if (oracle_mie_phase_raw(m_re, m_im, x, mu, n_fine + 1, F))
            goto fail;
    } else {
        for (int j = 0; j <= n_fine; ++j)
            F[j] = hg_phase(hg_g, (double)(n_fine - j) * h);
    }
    /* F <- (1/2) P sin(theta), times the hat weights h_w(cos theta) if any */
    for (int j = 0; j <= n_fine; ++j) {
        F[j] *= 0.5 * sin((double)(n_fine - j) * h);
        if (n_w) {
            double hw = 0.0;
            for (int k = 0; k < n_w; ++k)
                hw += wts[k] * oracle_hat(n_w, k, mu[j]);
            F[j] *= hw;
        }
    }
    int rc = invert_density(F, mu, n_fine, n_bins, icdf, omu, pdf, diag);
    free(F); free(mu);
    return rc;
fail:
    free(F); free(mu);
    return -1;
}

/* Steps 2-4 for a density F(theta_j) = (1/2) P(cos theta_j) sin theta_j on the
 * grid theta_j = pi - j pi / n_fine (mu[j] = cos theta_j). */
static int invert_density(double *F, const double *mu, int n_fine, int n_bins, double *icdf,
                          double *omu, double *pdf, double *diag)
{
    const double h = M_PI / n_fine;
    double *cum = malloc((size_t)(n_fine / 2 + 1) * sizeof *cum);
    double *t_icdf = malloc((size_t)(n_bins + 1) * sizeof *t_icdf);
    double *t_omu = malloc((size_t)(n_bins + 1) * sizeof *t_omu);
    if (!cum || !t_icdf || !t_omu)
        goto fail;

    /* Step 2/3: Simpson panels, cumulated from theta = pi. */
    cum[0] = 0.0;
    double gnum = 0.0;
    for (int p = 0; p < n_fine / 2; ++p) {
        int j = 2 * p;
        cum[p + 1] = cum[p] + h / 3.0 * (F[j] + 4.0 * F[j + 1] + F[j + 2]);
        gnum += h / 3.0 * (F[j] * mu[j] + 4.0 * F[j + 1] * mu[j + 1] +
                           F[j + 2] * mu[j + 2]);
    }
    const double Z = cum[n_fine / 2];
    if (!(Z > 0.0))
        goto fail;

    /* Step 4: inversion at levels i / n_bins. */
    t_icdf[0] = -1.0;
    t_omu[0] = 2.0;
    t_icdf[n_bins] = 1.0;
    t_omu[n_bins] = 0.0;
    int p = 0;
    for (int i = 1; i < n_bins; ++i) {
        double target = Z * ((double)i / n_bins);
        while (p < n_fine / 2 - 1 && cum[p + 1] <= target)
            ++p;
        int j = 2 * p;
        double want = target - cum[p];
        double lo = 0.0, hi = 2.0 * h;
        for (int it = 0; it < 200 && hi - lo > 1e-18 * h; ++it) {
            double mid = 0.5 * (lo + hi);
            if (panel_partial(F[j], F[j + 1], F[j + 2], h, mid) < want)
                lo = mid;
            else
                hi = mid;
        }
        double s = 0.5 * (lo + hi);
        /* theta = pi - (2 p h + s), written from the near end of the grid */
        double theta = (double)(n_fine - j) * h - s;
        double sh = sin(0.5 * theta);
        t_icdf[i] = cos(theta);
        t_omu[i] = 2.0 * sh * sh;
    }

    if (icdf)
        for (int i = 0; i <= n_bins; ++i) icdf[i] = t_icdf[i];
    if (omu)
        for (int i = 0; i <= n_bins; ++i) omu[i] = t_omu[i];
    if (pdf)
        for (int i = 0; i < n_bins; ++i)
            pdf[i] = (1.0 / n_bins) / (t_omu[i] - t_omu[i + 1]);
    if (diag) {
        double mean = 0.0;
        for (int i = 0; i < n_bins; ++i)
            mean += 0.5 * (t_icdf[i] + t_icdf[i + 1]);
        diag[0] = Z;
        diag[1] = gnum / Z;
        diag[2] = mean / n_bins;
        diag[3] = (double)n_fine;
    }
    free(cum); free(t_icdf); free(t_omu);
    return 0;
fail:
    free(cum); free(t_icdf); free(t_omu);
    return -1;
}

/*
 * A suspension of several particle kinds (for example the size bins of a
 * polydisperse sample) scatters with the mixture of their phase functions,
 * each weighted by its share of the scattering coefficient, n_i sigma_sca,i:
 * p = sum_i w_i p_i / sum_i w_i with every p_i normalised by Eq. 10. The
 * components are normalised on the same Simpson grid, summed, and the
 * mixture is tabulated by the same steps 2-4.
 */
int oracle_phase_table_mixture(int n_comp, const int *kind, const double *m_re,
                               const double *m_im, const double *x, const double *hg_g,
                               const double *w, int n_bins, int n_fine, double *icdf,
                               double *omu, double *pdf, double *diag)
{
    if (n_comp < 1 || n_bins < 2 || n_fine < 4 || (n_fine & 1))
        return -1;
    double wsum = 0.0;
    for (int i = 0; i < n_comp; ++i) {
        if (!(w[i] >= 0.0))
            return -1;
        if (kind[i] == ORACLE_PHASE_HG && !(hg_g[i] > -1.0 && hg_g[i] < 1.0))
            return -1;
        if (kind[i] != ORACLE_PHASE_HG && kind[i] != ORACLE_PHASE_MIE)
            return -1;
        wsum += w[i];
    }
    if (!(wsum > 0.0))
        return -1;
    const double h = M_PI / n_fine;
    double *F = calloc((size_t)(n_fine + 1), sizeof *F);
    double *G = malloc((size_t)(n_fine + 1) * sizeof *G);
    double *mu = malloc((size_t)(n_fine + 1) * sizeof *mu);
    int rc = -1;
    if (!F || !G || !mu)
        goto out;
    for (int j = 0; j <= n_fine; ++j)
        mu[j] = cos((double)(n_fine - j) * h);
    for (int i = 0; i < n_comp; ++i) {
        if (kind[i] == ORACLE_PHASE_MIE) {
            if (oracle_mie_phase_raw(m_re[i], m_im[i], x[i], mu, n_fine + 1, G))
                goto out;
        } else {
            for (int j = 0; j <= n_fine; ++j)
                G[j] = hg_phase(hg_g[i], (double)(n_fine - j) * h);
        }
        double Z = 0.0;
        for (int j = 0; j <= n_fine; ++j)
            G[j] *= 0.5 * sin((double)(n_fine - j) * h);
        for (int p = 0; p < n_fine / 2; ++p)
            Z += h / 3.0 * (G[2 * p] + 4.0 * G[2 * p + 1] + G[2 * p + 2]);
        if (!(Z > 0.0))
            goto out;
        for (int j = 0; j <= n_fine; ++j)
            F[j] += (w[i] / wsum) * G[j] / Z;
    }
    rc = invert_density(F, mu, n_fine, n_bins, icdf, omu, pdf, diag);
out:
    free(F); free(G); free(mu);
    return rc;
}

/*
 * The sampling scheme of Sec. 3.1.2 as printed: the phase function at
 * n_theta equally spaced scattering angles theta_i = i pi / (n_theta - 1),
 * i = 0 (forward) .. n_theta - 1 (backward), a cumulative distribution over
 * them, and a binary search of that distribution for each sample. The paper
 * does not say how the cumulative sum is formed; here it is the trapezoidal
 * rule on the density in theta, (1/2) P(cos theta) sin theta (Eq. 10 with
 * dOmega = 2 pi sin theta dtheta), divided by its total so that cdf[0] = 0
 * and cdf[n_theta - 1] = 1.
 */
int oracle_paper_cdf(int kind, double m_re, double m_im, double x, double hg_g,
                     int n_theta, double *cdf)
{
    if (n_theta < 3 || !cdf)
        return -1;
    if (kind == ORACLE_PHASE_HG && !(hg_g > -1.0 && hg_g < 1.0))
        return -1;
    if (kind != ORACLE_PHASE_HG && kind != ORACLE_PHASE_MIE)
        return -1;
    const int n = n_theta - 1;
    const double h = M_PI / n;
    double *F = malloc((size_t)n_theta * sizeof *F);
    double *mu = malloc((size_t)n_theta * sizeof *mu);
    if (!F || !mu) {
        free(F); free(mu);
        return -1;
    }
    for (int i = 0; i < n_theta; ++i)
        mu[i] = cos(i * h);
    if (kind == ORACLE_PHASE_MIE) {
        if (oracle_mie_phase_raw(m_re, m_im, x, mu, n_theta, F)) {
            free(F); free(mu);
            return -1;
        }
    } else {
        for (int i = 0; i < n_theta; ++i)
            F[i] = hg_phase(hg_g, i * h);
    }
    for (int i = 0; i < n_theta; ++i)
        F[i] *= 0.5 * sin(i * h);
    cdf[0] = 0.0;
    for (int i = 0; i < n; ++i)
        cdf[i + 1] = cdf[i] + 0.5 * h * (F[i] + F[i + 1]);
    const double Z = cdf[n];
    free(F); free(mu);
    if (!(Z > 0.0))
        return -1;
    for (int i = 1; i < n; ++i)
        cdf[i] /= Z;
    cdf[n] = 1.0;
    return 0;
}

/*
 * A tabulated phase function reweighted by hat-function weights: the
 * phase-table weights that the camera-image gradient is taken with respect
 * to. The table's own density p (pdf_j = (1/n) / (omu_j - omu_{j+1}) on bin j,
 * cos theta in [1 - omu_j, 1 - omu_{j+1}]) times h_w(mu) = sum_k w_k phi_k(mu)
 * is renormalised by Z(w) = int p h_w and inverted at the equal-probability
 * levels i / n_bins. Steps, in that order:
 *   1. the mass of each bin: p_j times the integral of h_w over the bin (h_w
 *      is linear between the hat nodes, so trapezoids piece by piece are
 *      exact);
 *   2. the running sum of the masses; its total is Z(w);
 *   3. for each level, the bin whose running sum brackets i Z(w) / n_bins,
 *      and inside it the point where the partial mass reaches the level, by
 *      bisection in 1 - cos theta.
 */
static double hw_at(int n_w, const double *w, double mu)
{
    /* only the two hats around mu are nonzero */
    double t = (mu + 1.0) * 0.5 * (n_w - 1);
    int k = (int)floor(t);
    if (k < 0) k = 0;
    if (k > n_w - 2) k = n_w - 2;
    return w[k] * oracle_hat(n_w, k, mu) + w[k + 1] * oracle_hat(n_w, k + 1, mu);
}

/* integral of h_w d(mu) over cos theta in [1 - va, 1 - vb], va >= vb given
 * in 1 - cos theta (the hat nodes sit at 1 - cos theta = 2 - 2k/(n_w - 1)) */
static double hw_integral(int n_w, const double *w, double va, double vb)
{
    const double hh = 2.0 / (n_w - 1);
    double s = 0.0, hi = va;
    for (int k = 0; k < n_w; ++k) {
        double vk = 2.0 - k * hh;
        if (vk < hi && vk > vb) {
            s += 0.5 * (hw_at(n_w, w, 1.0 - hi) + hw_at(n_w, w, 1.0 - vk)) * (hi - vk);
            hi = vk;
        }
    }
    s += 0.5 * (hw_at(n_w, w, 1.0 - hi) + hw_at(n_w, w, 1.0 - vb)) * (hi - vb);
    return s;
}

int oracle_phase_table_reweighted(const double *omu_base, int n_bins, int n_w, const double *w,
                                  double *icdf, double *omu, double *pdf, double *z_out)
{
    if (!omu_base || n_bins < 2 || n_w < 2 || !w || !omu)
        return -1;
    for (int k = 0; k < n_w; ++k)
        if (!(w[k] > 0.0) || !isfinite(w[k]))
            return -1;
    double *cum = malloc((size_t)(n_bins + 1) * sizeof *cum);
    double *p = malloc((size_t)n_bins * sizeof *p);
    if (!cum || !p) {
        free(cum); free(p);
        return -1;
    }
    cum[0] = 0.0;
    for (int j = 0; j < n_bins; ++j) {
        p[j] = (1.0 / n_bins) / (omu_base[j] - omu_base[j + 1]);
        cum[j + 1] = cum[j] + p[j] * hw_integral(n_w, w, omu_base[j], omu_base[j + 1]);
    }
    const double Z = cum[n_bins];
    omu[0] = 2.0;
    omu[n_bins] = 0.0;
    int j = 0;
    for (int i = 1; i < n_bins; ++i) {
        double target = ((double)i / n_bins) * Z;   /* level i of the weighted mass */
        while (j < n_bins - 1 && cum[j + 1] <= target)
            ++j;
        double want = target - cum[j];
        double a = omu_base[j + 1], b = omu_base[j];   /* partial mass from b down to v */
        for (int it = 0; it < 200; ++it) {
            double v = 0.5 * (a + b);
            if (!(v > a && v < b))
                break;
            if (p[j] * hw_integral(n_w, w, omu_base[j], v) < want) b = v; else a = v;
        }
        omu[i] = 0.5 * (a + b);
    }
    for (int i = 0; i < n_bins; ++i) {
        if (pdf)
            pdf[i] = (1.0 / n_bins) / (omu[i] - omu[i + 1]);
    }
    if (icdf)
        for (int i = 0; i <= n_bins; ++i)
            icdf[i] = 1.0 - omu[i];
    if (z_out)
        *z_out = Z;
    free(cum); free(p);
    return 0;
}
