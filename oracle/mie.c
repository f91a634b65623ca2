/*
 * Oracle: Lorenz-Mie quantities in double precision (test infrastructure
 * only; see oracle.h).
 *
 * Follows Sec. 2.2 (Eq. 3-9), Sec. 2.4 (Eq. 12) and Sec. 2.5 (Eq. 13-14).
 * Eq. 7-8 are evaluated in the algebraically equal logarithmic-derivative
 * form of Bohren & Huffman (the recurrence algorithm the paper adopts in
 * Sec. 2.5): with D_n(y) = psi_n'(y)/psi_n(y), y = m x,
 *     a_n = [(D_n/m + n/x) psi_n - psi_{n-1}] / [(D_n/m + n/x) xi_n - xi_{n-1}]
 *     b_n = [(m D_n + n/x) psi_n - psi_{n-1}] / [(m D_n + n/x) xi_n - xi_{n-1}]
 * D_n by downward recurrence (started high enough above max(nmax, |y|) that
 * the start value is forgotten), psi_n and chi_n by upward recurrence,
 * xi_n = psi_n - i chi_n.
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>

int oracle_mie_nmax(double x)
{
    return (int)ceil(x + 4.0 * cbrt(x) + 2.0);
}

/* Eq. 3 with the wavelength taken inside the medium. */
double oracle_size_parameter(double d_um, double n_medium, double lambda0_nm)
{
    double lambda_um = (lambda0_nm * 1e-3) / n_medium;
    return M_PI * d_um / lambda_um;
}

/* Eq. 7-8 (see file header for the form used). */
int oracle_mie_ab(double m_re, double m_im, double x, int nmax,
                  double *a_reim, double *b_reim)
{
    if (!(x > 0.0) || nmax < 1 || !(m_re > 0.0) || m_im < 0.0)
        return -1;
    double complex m = m_re + I * m_im;
    double complex y = m * x;
    /* The downward recurrence forgets its arbitrary start value only once it
     * runs through the evanescent region n > |y|, whose width grows like
     * |y|^(1/3); a fixed offset of ~15 leaves errors of 1e-6 at |y| ~ 120. */
    int nstart = (int)(fmax((double)nmax, cabs(y)) + 16.0 + 8.0 * cbrt(cabs(y)));
    double complex *D = malloc((size_t)(nstart + 1) * sizeof *D);
    if (!D)
        return -1;
    D[nstart] = 0.0;
    for (int n = nstart; n >= 1; --n)
        D[n - 1] = (double)n / y - 1.0 / (D[n] + (double)n / y);

    /* psi_{-1}, psi_0 and chi_{-1}, chi_0 */
    double psi_nm2 = cos(x), psi_nm1 = sin(x);
    double chi_nm2 = -sin(x), chi_nm1 = cos(x);
    for (int n = 1; n <= nmax; ++n) {
        double psi_n = (2.0 * n - 1.0) / x * psi_nm1 - psi_nm2;
        double chi_n = (2.0 * n - 1.0) / x * chi_nm1 - chi_nm2;
        double complex xi_n = psi_n - I * chi_n;
        double complex xi_nm1 = psi_nm1 - I * chi_nm1;
        double complex ta = D[n] / m + (double)n / x;
        double complex tb = m * D[n] + (double)n / x;
        double complex an = (ta * psi_n - psi_nm1) / (ta * xi_n - xi_nm1);
        double complex bn = (tb * psi_n - psi_nm1) / (tb * xi_n - xi_nm1);
        a_reim[2 * (n - 1)] = creal(an);
        a_reim[2 * (n - 1) + 1] = cimag(an);
        b_reim[2 * (n - 1)] = creal(bn);
        b_reim[2 * (n - 1) + 1] = cimag(bn);
        psi_nm2 = psi_nm1;
        psi_nm1 = psi_n;
        chi_nm2 = chi_nm1;
        chi_nm1 = chi_n;
    }
    free(D);
    return 0;
}

static int load_ab(double m_re, double m_im, double x, int *nmax_out,
                   double complex **a_out, double complex **b_out)
{
    int nmax = oracle_mie_nmax(x);
    double *ar = malloc((size_t)nmax * 2 * sizeof *ar);
    double *br = malloc((size_t)nmax * 2 * sizeof *br);
    double complex *a = malloc((size_t)(nmax + 1) * sizeof *a);
    double complex *b = malloc((size_t)(nmax + 1) * sizeof *b);
    if (!ar || !br || !a || !b || oracle_mie_ab(m_re, m_im, x, nmax, ar, br)) {
        free(ar); free(br); free(a); free(b);
        return -1;
    }
    for (int n = 1; n <= nmax; ++n) {
        a[n] = ar[2 * (n - 1)] + I * ar[2 * (n - 1) + 1];
        b[n] = br[2 * (n - 1)] + I * br[2 * (n - 1) + 1];
    }
    a[0] = b[0] = 0.0;
    free(ar);
    free(br);
    *nmax_out = nmax;
    *a_out = a;
    *b_out = b;
    return 0;
}

/* Eq. 13 for Q_ext; Q_sca is the matching sum of |a_n|^2 + |b_n|^2; the
 * asymmetry parameter g of Eq. 12 from the series
 *   g Q_sca = (4/x^2) sum_n [ n(n+2)/(n+1) Re(a_n a*_{n+1} + b_n b*_{n+1})
 *                             + (2n+1)/(n(n+1)) Re(a_n b*_n) ]. */
int oracle_mie_efficiencies(double m_re, double m_im, double x,
                            double *qext, double *qsca, double *g_series)
{
    int nmax;
    double complex *a, *b;
    if (load_ab(m_re, m_im, x, &nmax, &a, &b))
        return -1;
    double se = 0.0, ss = 0.0, sg = 0.0;
    for (int n = 1; n <= nmax; ++n) {
        se += (2.0 * n + 1.0) * creal(a[n] + b[n]);
        ss += (2.0 * n + 1.0) * (creal(a[n] * conj(a[n])) + creal(b[n] * conj(b[n])));
        if (n < nmax)
            sg += (double)n * (n + 2.0) / (n + 1.0) *
                  creal(a[n] * conj(a[n + 1]) + b[n] * conj(b[n + 1]));
        sg += (2.0 * n + 1.0) / ((double)n * (n + 1.0)) * creal(a[n] * conj(b[n]));
    }
    double qe = 2.0 / (x * x) * se;
    double qs = 2.0 / (x * x) * ss;
    if (qext) *qext = qe;
    if (qsca) *qsca = qs;
    if (g_series) *g_series = (4.0 / (x * x)) * sg / qs;
    free(a);
    free(b);
    return 0;
}

/* Eq. 5-6 with the angular functions from their upward recurrences
 *   pi_0 = 0, pi_1 = 1,
 *   pi_n = (2n-1)/(n-1) mu pi_{n-1} - n/(n-1) pi_{n-2},
 *   tau_n = n mu pi_n - (n+1) pi_{n-1}. */
static void s12_at(const double complex *a, const double complex *b, int nmax,
                   double mu, double complex *s1, double complex *s2)
{
    double complex S1 = 0.0, S2 = 0.0;
    double pi_nm2 = 0.0, pi_nm1 = 0.0;
    for (int n = 1; n <= nmax; ++n) {
        double pi_n = (n == 1) ? 1.0
                               : ((2.0 * n - 1.0) / (n - 1.0)) * mu * pi_nm1 -
                                     ((double)n / (n - 1.0)) * pi_nm2;
        double tau_n = n * mu * pi_n - (n + 1.0) * pi_nm1;
        double f = (2.0 * n + 1.0) / ((double)n * (n + 1.0));
        S1 += f * (a[n] * pi_n + b[n] * tau_n);
        S2 += f * (a[n] * tau_n + b[n] * pi_n);
        pi_nm2 = pi_nm1;
        pi_nm1 = pi_n;
    }
    *s1 = S1;
    *s2 = S2;
}

int oracle_mie_s12(double m_re, double m_im, double x, const double *mu,
                   int n_mu, double *s1_reim, double *s2_reim)
{
    int nmax;
    double complex *a, *b;
    if (load_ab(m_re, m_im, x, &nmax, &a, &b))
        return -1;
    for (int i = 0; i < n_mu; ++i) {
        double complex s1, s2;
        s12_at(a, b, nmax, mu[i], &s1, &s2);
        s1_reim[2 * i] = creal(s1);
        s1_reim[2 * i + 1] = cimag(s1);
        s2_reim[2 * i] = creal(s2);
        s2_reim[2 * i + 1] = cimag(s2);
    }
    free(a);
    free(b);
    return 0;
}

/* Eq. 9 up to its constant factor, which Eq. 10 removes. */
int oracle_mie_phase_raw(double m_re, double m_im, double x, const double *mu,
                         int n_mu, double *p)
{
    int nmax;
    double complex *a, *b;
    if (load_ab(m_re, m_im, x, &nmax, &a, &b))
        return -1;
    for (int i = 0; i < n_mu; ++i) {
        double complex s1, s2;
        s12_at(a, b, nmax, mu[i], &s1, &s2);
        p[i] = creal(s1 * conj(s1)) + creal(s2 * conj(s2));
    }
    free(a);
    free(b);
    return 0;
}

/* Eq. 14 (d in micrometres, result in mm^2). */
double oracle_cross_section_mm2(double q, double d_um)
{
    double d_mm = d_um * 1e-3;
    return q * M_PI * d_mm * d_mm / 4.0;
}

/* Eq. 17. */
double oracle_optical_depth(double n_per_mm3, double sigma_mm2, double l_mm)
{
    return n_per_mm3 * sigma_mm2 * l_mm;
}
