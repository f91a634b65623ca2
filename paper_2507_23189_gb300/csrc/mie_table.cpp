// Host-side Lorenz-Mie phase table (the engine's table builder).
//
// Sec. 3.1.2 precomputes the phase function and its cumulative distribution
// so that the walk samples the scattering angle by table lookup (Sec. 2.6).
// Everything here is double precision; only the packed output is rounded to
// single precision for the kernels.
//
//  * Mie coefficients a_n, b_n (Eq. 7-8) in the logarithmic-derivative form of
//    Bohren & Huffman (the paper's ref. [12], Sec. 2.5). D_N(mx) at the top of
//    the series comes from the continued fraction for psi_N / psi_{N-1}
//    (evaluated with the modified Lentz method), then D_n runs downward;
//    psi_n(x), chi_n(x) run upward. Series length: Wiscombe (1980).
//  * Efficiencies (Eq. 13), g (Eq. 12 via the cross-term series), cross
//    sections (Eq. 14).
//  * Phase function |S1|^2 + |S2|^2 (Eq. 5-6, 9) integrated over theta with
//    8-point Gauss-Legendre panels; normalisation (Eq. 10) by the total.
//  * Inverse CDF on n_bins equal-probability levels by safeguarded Newton
//    iteration on the exact integrand inside the panel holding each level.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "../../include/mcmie.h"
#include "table_format.h"

namespace {

using cplx = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// Wiscombe's recommended number of terms.
int series_length(double x)
{
    double n;
    if (x < 0.02)
        n = x + 4.0 * std::cbrt(x) + 1.0;
    else if (x <= 8.0)
        n = x + 4.0 * std::cbrt(x) + 1.0;
    else if (x < 4200.0)
        n = x + 4.05 * std::cbrt(x) + 2.0;
    else
        n = x + 4.0 * std::cbrt(x) + 2.0;
    int k = (int)std::lround(n);
    return k < 1 ? 1 : k;
}

// psi_N(z) / psi_{N-1}(z) = 1 / (b1 - 1 / (b2 - 1 / (b3 - ...))),
// b_k = (2N + 2k - 1) / z; modified Lentz.
cplx riccati_ratio(int N, cplx z)
{
    const double tiny = 1e-300, eps = 1e-17;
    cplx f = tiny, C = f, D = 0.0;
    for (int k = 1; k < 100000; ++k) {
        cplx b = (2.0 * N + 2.0 * k - 1.0) / z;
        double a = (k == 1) ? 1.0 : -1.0;
        D = b + a * D;
        if (std::abs(D) < tiny) D = tiny;
        C = b + a / C;
        if (std::abs(C) < tiny) C = tiny;
        D = 1.0 / D;
        cplx delta = C * D;
        f *= delta;
        if (std::abs(delta - 1.0) < eps) break;
    }
    return f;
}

struct MieSeries {
    int nmax = 0;
    std::vector<cplx> a, b;  // index 1..nmax
};

bool mie_series(cplx m, double x, MieSeries &S)
{
    int N = series_length(x);
    S.nmax = N;
    S.a.assign(N + 2, 0.0);
    S.b.assign(N + 2, 0.0);
    cplx z = m * x;
    // D_n(z), n = 0..N+1, from the exact top value downward
    int top = N + 1;
    std::vector<cplx> D(top + 1);
    D[top] = 1.0 / riccati_ratio(top, z) - (double)top / z;
    for (int n = top; n >= 1; --n)
        D[n - 1] = (double)n / z - 1.0 / (D[n] + (double)n / z);
    double psi0 = std::cos(x), psi1 = std::sin(x);   // psi_{n-2}, psi_{n-1}
    double chi0 = -std::sin(x), chi1 = std::cos(x);
    for (int n = 1; n <= N; ++n) {
        double fn = (2.0 * n - 1.0) / x;
        double psi = fn * psi1 - psi0;
        double chi = fn * chi1 - chi0;
        cplx xi(psi, -chi), xi1(psi1, -chi1);
        cplx ea = D[n] / m + (double)n / x;
        cplx eb = m * D[n] + (double)n / x;
        S.a[n] = (ea * psi - psi1) / (ea * xi - xi1);
        S.b[n] = (eb * psi - psi1) / (eb * xi - xi1);
        if (!std::isfinite(S.a[n].real()) || !std::isfinite(S.b[n].real())) return false;
        psi0 = psi1; psi1 = psi;
        chi0 = chi1; chi1 = chi;
    }
    return true;
}

// Unnormalised phase function |S1|^2 + |S2|^2 at cos(theta) = mu.
double phase_raw(const MieSeries &S, double mu)
{
    cplx s1 = 0.0, s2 = 0.0;
    double pm1 = 0.0, pm2 = 0.0;  // pi_{n-1}, pi_{n-2}
    for (int n = 1; n <= S.nmax; ++n) {
        double pn = (n == 1) ? 1.0 : ((2.0 * n - 1.0) * mu * pm1 - n * pm2) / (n - 1.0);
        double tn = n * mu * pn - (n + 1.0) * pm1;
        double w = (2.0 * n + 1.0) / (n * (n + 1.0));
        s1 += w * (S.a[n] * pn + S.b[n] * tn);
        s2 += w * (S.a[n] * tn + S.b[n] * pn);
        pm2 = pm1;
        pm1 = pn;
    }
    return std::norm(s1) + std::norm(s2);
}

// 8-point Gauss-Legendre on [-1, 1].
const double GL_X[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290,
                        -0.1834346424956498, 0.1834346424956498, 0.5255324099163290,
                        0.7966664774136267, 0.9602898564975363};
const double GL_W[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873,
                        0.3626837833783620, 0.3626837833783620, 0.3137066458778873,
                        0.2223810344533745, 0.1012285362903763};

// A phase function as a weighted sum of Mie components: density in theta
// sum_k c_k (1/2) P_k(cos t) sin t (a single particle is one component).
struct Mix {
    std::vector<const MieSeries *> S;
    std::vector<double> c;
    double dens(double t) const
    {
        const double mu = std::cos(t), st = std::sin(t);
        double v = 0.0;
        for (size_t k = 0; k < S.size(); ++k)
            if (c[k] != 0.0) v += c[k] * phase_raw(*S[k], mu);
        return 0.5 * v * st;
    }
    // Integral of the density over theta in [t0, t1].
    double integrate(double t0, double t1) const
    {
        double m = 0.5 * (t0 + t1), h = 0.5 * (t1 - t0), s = 0.0;
        for (int i = 0; i < 8; ++i) s += GL_W[i] * dens(m + h * GL_X[i]);
        return s * h;
    }
};

// The particle's Mie series and the quantities of mie_info (all but
// g_table). Returns MC_ERR_ARG for parameters out of range.
mc_status prepare(const mie_params *P, MieSeries &S, mie_info &I)
{
    if (!(P->diameter_um > 0.0) || !(P->n_medium > 0.0) || !(P->wavelength_nm > 0.0) ||
        !(P->n_particle_re > 0.0) || !(P->n_particle_im >= 0.0) || !std::isfinite(P->diameter_um) ||
        !std::isfinite(P->n_particle_re) || !std::isfinite(P->n_particle_im) ||
        !std::isfinite(P->wavelength_nm) || !std::isfinite(P->n_medium))
        return MC_ERR_ARG;
    const double x = kPi * P->diameter_um * P->n_medium / (P->wavelength_nm * 1e-3);
    if (!(x >= 1e-3) || x > 2000.0) return MC_ERR_ARG;
    const cplx m(P->n_particle_re / P->n_medium, P->n_particle_im / P->n_medium);
    if (!mie_series(m, x, S)) return MC_ERR_NUMERIC;

    double se = 0.0, ss = 0.0, sg = 0.0;
    for (int n = 1; n <= S.nmax; ++n) {
        se += (2.0 * n + 1.0) * (S.a[n] + S.b[n]).real();
        ss += (2.0 * n + 1.0) * (std::norm(S.a[n]) + std::norm(S.b[n]));
        sg += n * (n + 2.0) / (n + 1.0) *
                  (S.a[n] * std::conj(S.a[n + 1]) + S.b[n] * std::conj(S.b[n + 1])).real() +
              (2.0 * n + 1.0) / (n * (n + 1.0)) * (S.a[n] * std::conj(S.b[n])).real();
    }
    const double qext = 2.0 / (x * x) * se, qsca = 2.0 / (x * x) * ss;
    // Q_abs is exactly zero for a real index; the series difference only
    // carries rounding (of either sign), so keep it non-negative.
    const double qabs = (m.imag() > 0.0) ? std::fmax(qext - qsca, 0.0) : 0.0;
    I.x = x;
    I.m_re = m.real();
    I.m_im = m.imag();
    I.qext = qext;
    I.qsca = qsca;
    I.qabs = qabs;
    I.g = 4.0 / (x * x) * sg / qsca;
    I.g_table = 0.0;
    const double geo = kPi * (P->diameter_um * 1e-3) * (P->diameter_um * 1e-3) / 4.0;
    I.sigma_ext_mm2 = qext * geo;
    I.sigma_sca_mm2 = qsca * geo;
    I.sigma_abs_mm2 = qabs * geo;
    I.nmax = S.nmax;
    return MC_OK;
}


// Steps 2-4 for the density D: cumulative integral over theta on panels of
// 8-point Gauss-Legendre (enough panels for the oscillations of a series of
// nmax terms), the equal-probability levels by safeguarded Newton iteration,
// the packed single-precision blob and its camera-density guide.
mc_status build_levels(const Mix &D, int nmax, int n_bins, size_t bytes, mc_table_header &H, void *table,
                       double *omu64, double *pdf64, double *mean_out)
{
    const int n = n_bins;
    // Panels in theta, accumulated from theta = pi (mu = -1) toward 0.
    const int M = std::max(4 * n, 96 * nmax);
    const double h = kPi / M;
    std::vector<double> cum(M + 1);
    cum[0] = 0.0;
    for (int k = 0; k < M; ++k) {
        double t1 = kPi - k * h, t0 = kPi - (k + 1) * h;
        cum[k + 1] = cum[k] + D.integrate(t0, t1);
    }
    const double Z = cum[M];
    if (!(Z > 0.0) || !std::isfinite(Z)) return MC_ERR_NUMERIC;

    std::vector<double> theta(n + 1);
    theta[0] = kPi;
    theta[n] = 0.0;
    int k = 0;
    for (int i = 1; i < n; ++i) {
        double target = Z * ((double)i / n);
        while (k < M - 1 && cum[k + 1] <= target) ++k;
        // Panel k spans theta in [pi-(k+1)h, pi-kh]; cum rises as theta falls.
        double hi = kPi - k * h, lo = kPi - (k + 1) * h;
        if (k == M - 1) lo = 0.0;
        double want = target - cum[k];
        double a = lo, b = hi;  // C(b) = 0 <= want <= C(a)
        double t = 0.5 * (a + b);
        for (int it = 0; it < 60; ++it) {
            double c = D.integrate(t, hi) - want;
            if (c > 0) a = t; else b = t;   // too much mass: move toward hi
            double f = D.dens(t);
            double tn = (f > 0.0) ? t + c / f : 0.5 * (a + b);
            if (!(tn > a && tn < b)) tn = 0.5 * (a + b);
            if (std::fabs(tn - t) <= 1e-16 * (1.0 + std::fabs(t))) { t = tn; break; }
            t = tn;
        }
        theta[i] = t;
    }

    std::vector<double> omu(n + 1), pdf(n);
    for (int i = 0; i <= n; ++i) {
        double sh = std::sin(0.5 * theta[i]);
        omu[i] = 2.0 * sh * sh;
    }
    omu[0] = 2.0;
    omu[n] = 0.0;
    double mean = 0.0;
    for (int j = 0; j < n; ++j) {
        double w = omu[j] - omu[j + 1];
        if (!(w > 0.0)) return MC_ERR_NUMERIC;
        pdf[j] = (1.0 / n) / w;
        mean += 1.0 - 0.5 * (omu[j] + omu[j + 1]);
    }
    mean /= n;
    *mean_out = mean;

    if (omu64) std::memcpy(omu64, omu.data(), sizeof(double) * (n + 1));
    if (pdf64) std::memcpy(pdf64, pdf.data(), sizeof(double) * n);
    if (table) {
        unsigned char *blob = static_cast<unsigned char *>(table);
        std::memset(blob, 0, bytes);
        H.g_table = (float)mean;
        std::memcpy(blob, &H, sizeof H);
        float *fo = reinterpret_cast<float *>(blob + H.off_omu);
        float *fp = reinterpret_cast<float *>(blob + H.off_pdf);
        uint16_t *gd = reinterpret_cast<uint16_t *>(blob + H.off_guide);
        for (int i = 0; i <= n; ++i) fo[i] = (float)omu[i];
        for (int j = 0; j < n; ++j) fp[j] = (float)pdf[j];
        // guide[c] brackets the camera-density lookup. The kernel finds the
        // bin of a direction cosine m (float) as the largest j with
        // fo[j] >= 1 - m (float subtraction), starting from the cell
        // c = floor(fl(m + 1) * G/2). Both are monotone in m, so with lo(c) the
        // smallest float whose cell is c, guide[c] = bin(lo(c)) and
        // guide[c+1] bound the bins of every m in cell c. Computed here with
        // the same single-precision operations the kernel performs.
        const int G = H.n_guide;
        const float half_g = 0.5f * (float)G;
        auto cell_of = [&](float m) {
            volatile float t = m + 1.0f;
            return (int)std::floor((float)(t * half_g));
        };
        auto bin_of = [&](float m) {
            volatile float om = 1.0f - m;
            int lo = 0, hi = n - 1;   // fo[0] = 2 >= om always
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (fo[mid] >= om) lo = mid; else hi = mid - 1;
            }
            return lo;
        };
        // floats in increasing order <-> unsigned keys in increasing order
        auto key_of = [](float f) {
            uint32_t b;
            std::memcpy(&b, &f, 4);
            return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
        };
        auto float_of = [](uint32_t k) {
            uint32_t b = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
            float f;
            std::memcpy(&f, &b, 4);
            return f;
        };
        gd[0] = (uint16_t)bin_of(-1.0f);
        for (int c = 1; c < G; ++c) {
            // smallest float m in [-1, 1] with cell_of(m) >= c, by bisection on keys
            uint32_t lo = key_of(-1.0f), hi = key_of(1.0f);
            while (lo < hi) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (cell_of(float_of(mid)) >= c) hi = mid; else lo = mid + 1;
            }
            gd[c] = (uint16_t)bin_of(float_of(lo));
        }
        gd[G] = (uint16_t)bin_of(1.0f);
    }
    return MC_OK;
}

}  // namespace

extern "C" size_t mc_table_bytes(int n_bins) { return mc_table_layout(n_bins, nullptr); }

extern "C" mc_status mie_table_build(const mie_params *P, mie_info *info, void *table,
                                     double *omu64, double *pdf64)
{
    if (!P) return MC_ERR_ARG;
    mc_table_header H;
    size_t bytes = mc_table_layout(P->n_bins, &H);
    if (!bytes) return MC_ERR_ARG;
    MieSeries S;
    mie_info I;
    const mc_status st = prepare(P, S, I);
    if (st != MC_OK) return st;

    Mix D;
    D.S.push_back(&S);
    D.c.push_back(1.0);
    double mean = 0.0;
    const mc_status bs = build_levels(D, S.nmax, P->n_bins, bytes, H, table, omu64, pdf64, &mean);
    if (bs != MC_OK) return bs;
    if (info) {
        *info = I;
        info->g_table = mean;
    }
    return MC_OK;
}

extern "C" mc_status mc_medium_from_density(const mie_info *info, double nd, double mu_a_medium,
                                            mc_medium *out)
{
    if (!info || !out || !(nd >= 0.0) || !(mu_a_medium >= 0.0) || !std::isfinite(nd) ||
        !std::isfinite(mu_a_medium))
        return MC_ERR_ARG;
    // Eq. 17 per unit length: mu = n sigma.
    out->mu_s = nd * info->sigma_sca_mm2;
    out->mu_a = nd * std::fmax(info->sigma_abs_mm2, 0.0) + mu_a_medium;
    return MC_OK;
}

// Eq. 17 solved for the number density: OD = n sigma_e L gives n = OD /
// (sigma_e L), then the coefficients as mc_medium_from_density.
extern "C" mc_status mc_medium_from_optical_depth(const mie_info *info, double tau, double length_mm,
                                                  double mu_a_medium, mc_medium *out,
                                                  double *number_density_out)
{
    if (!info || !out || !std::isfinite(tau) || !(tau >= 0.0) || !std::isfinite(length_mm) ||
        !(length_mm > 0.0) || !std::isfinite(info->sigma_ext_mm2) || !(info->sigma_ext_mm2 > 0.0))
        return MC_ERR_ARG;
    const double nd = tau / (info->sigma_ext_mm2 * length_mm);
    if (!std::isfinite(nd)) return MC_ERR_ARG;
    const mc_status s = mc_medium_from_density(info, nd, mu_a_medium, out);
    if (s == MC_OK && number_density_out) *number_density_out = nd;
    return s;
}

// A suspension of several particle kinds (the size bins of a polydisperse
// sample, number fractions f_k) scatters with the mixture of their phase
// functions weighted by f_k sigma_sca,k (Eq. 14 per kind); each raw
// |S1|^2 + |S2|^2 integrates to x_k^2 Q_sca,k (its Eq. 10 normalisation).
extern "C" mc_status mie_mixture_table_build(const mie_params *P, const double *number_frac, int n_comp,
                                             mie_info *info, void *table, double *omu64, double *pdf64)
{
    if (!P || !number_frac || n_comp < 1 || n_comp > 256) return MC_ERR_ARG;
    const int n_bins = P[0].n_bins;
    mc_table_header H;
    const size_t bytes = mc_table_layout(n_bins, &H);
    if (!bytes) return MC_ERR_ARG;
    std::vector<MieSeries> S(n_comp);
    std::vector<mie_info> I(n_comp);
    double fsum = 0.0;
    for (int k = 0; k < n_comp; ++k) {
        if (P[k].n_bins != n_bins || !(number_frac[k] >= 0.0) || !std::isfinite(number_frac[k]))
            return MC_ERR_ARG;
        const mc_status st = prepare(&P[k], S[k], I[k]);
        if (st != MC_OK) return st;
        fsum += number_frac[k];
    }
    if (!(fsum > 0.0)) return MC_ERR_ARG;
    mie_info M = I[0];
    double se = 0.0, ss = 0.0, sa = 0.0, geo = 0.0, gs = 0.0;
    int nmax = 0;
    Mix D;
    for (int k = 0; k < n_comp; ++k) {
        const double f = number_frac[k] / fsum;
        se += f * I[k].sigma_ext_mm2;
        ss += f * I[k].sigma_sca_mm2;
        sa += f * I[k].sigma_abs_mm2;
        geo += f * kPi * (P[k].diameter_um * 1e-3) * (P[k].diameter_um * 1e-3) / 4.0;
        gs += f * I[k].sigma_sca_mm2 * I[k].g;
        nmax = std::max(nmax, S[k].nmax);
    }
    if (!(ss > 0.0)) return MC_ERR_NUMERIC;
    for (int k = 0; k < n_comp; ++k) {
        const double w = (number_frac[k] / fsum) * I[k].sigma_sca_mm2 / ss;
        D.S.push_back(&S[k]);
        D.c.push_back(w * 2.0 / (I[k].x * I[k].x * I[k].qsca));
    }
    double mean = 0.0;
    const mc_status bs = build_levels(D, nmax, n_bins, bytes, H, table, omu64, pdf64, &mean);
    if (bs != MC_OK) return bs;
    if (info) {
        M.sigma_ext_mm2 = se;
        M.sigma_sca_mm2 = ss;
        M.sigma_abs_mm2 = sa;
        M.qext = se / geo;
        M.qsca = ss / geo;
        M.qabs = sa / geo;
        M.g = gs / ss;
        M.g_table = mean;
        M.nmax = nmax;
        *info = M;
    }
    return MC_OK;
}

extern "C" size_t mc_paper_table_bytes(int n_theta) { return mc_paper_layout(n_theta, nullptr); }

// Sec. 3.1.2 as printed: the phase function at n_theta equally spaced angles,
// its cumulative distribution by the trapezoidal rule on (1/2) P sin(theta)
// (Eq. 10's measure), normalised by the total, and the search aids the
// kernel needs to sample it by bisection exactly as a double-precision
// search would decide.
extern "C" mc_status mie_paper_table_build(const mie_params *P, int n_theta, mie_info *info,
                                           void *table, double *cdf64)
{
    if (!P) return MC_ERR_ARG;
    mc_paper_header H;
    const size_t bytes = mc_paper_layout(n_theta, &H);
    if (!bytes) return MC_ERR_ARG;
    MieSeries S;
    mie_info I;
    const mc_status st = prepare(P, S, I);
    if (st != MC_OK) return st;

    const int n = n_theta - 1;
    const double dth = kPi / n;
    std::vector<double> F(n_theta), cdf(n_theta);
    for (int i = 0; i < n_theta; ++i) {
        const double t = i * dth;
        F[i] = 0.5 * phase_raw(S, std::cos(t)) * std::sin(t);
    }
    cdf[0] = 0.0;
    for (int i = 0; i < n; ++i) cdf[i + 1] = cdf[i] + 0.5 * dth * (F[i] + F[i + 1]);
    const double Z = cdf[n];
    if (!(Z > 0.0) || !std::isfinite(Z)) return MC_ERR_NUMERIC;
    for (int i = 1; i < n; ++i) cdf[i] /= Z;
    cdf[n] = 1.0;

    // mean cosine of the distribution that is uniform in theta on each interval
    double mean = 0.0;
    for (int i = 0; i < n; ++i)
        mean += (cdf[i + 1] - cdf[i]) * (std::sin((i + 1) * dth) - std::sin(i * dth)) / dth;
    if (info) {
        *info = I;
        info->g_table = mean;
    }
    if (cdf64) std::memcpy(cdf64, cdf.data(), sizeof(double) * n_theta);
    if (table) {
        unsigned char *blob = static_cast<unsigned char *>(table);
        std::memset(blob, 0, bytes);
        H.dtheta = (float)dth;
        H.g_table = (float)mean;
        std::memcpy(blob, &H, sizeof H);
        uint32_t *K = reinterpret_cast<uint32_t *>(blob + H.off_k);
        float *dl = reinterpret_cast<float *>(blob + H.off_dl);
        float *ri = reinterpret_cast<float *>(blob + H.off_ri);
        float *om = reinterpret_cast<float *>(blob + H.off_omu);
        float *pth = reinterpret_cast<float *>(blob + H.off_pth);
        const double q = 8388608.0;   // 2^23 uniform indices; u(k) = (k + 1/2) / q
        for (int i = 0; i <= n; ++i) {
            double kk = (i == n) ? q : std::ceil(cdf[i] * q - 0.5);
            if (kk < 0.0) kk = 0.0;
            if (kk > q) kk = q;
            K[i] = (uint32_t)kk;
            if (i < n) {
                // K[i] is the first index whose uniform reaches cdf_i
                const double u = (kk + 0.5) / q;
                if (!(u >= cdf[i]) || (kk > 0.0 && !((kk - 0.5) / q < cdf[i]))) return MC_ERR_NUMERIC;
                dl[i] = (float)(u - cdf[i]);
                const double w = cdf[i + 1] - cdf[i];
                ri[i] = w > 0.0 ? (float)(1.0 / w) : 0.0f;
                pth[i] = (float)(w / dth);
            }
        }
        for (int i = 0; i < n_theta; ++i) {
            const double sh = std::sin(0.5 * i * dth);
            om[i] = (float)(2.0 * sh * sh);
        }
        om[0] = 0.0f;
        om[n] = 2.0f;
        // guides: the last interval start at or below each bucket's lower end
        uint16_t *gq = reinterpret_cast<uint16_t *>(blob + H.off_gq);
        uint16_t *go = reinterpret_cast<uint16_t *>(blob + H.off_go);
        const uint32_t qstep = 8388608u / MC_PAPER_GUIDE;
        int iq = 0, io = 0;
        for (int b = 0; b <= MC_PAPER_GUIDE; ++b) {
            while (iq + 1 < n && K[iq + 1] <= (uint32_t)b * qstep) ++iq;
            gq[b] = (uint16_t)iq;
            const float edge = (float)b * (2.0f / MC_PAPER_GUIDE);   // exact: b / 2048
            while (io + 1 < n && om[io + 1] <= edge) ++io;
            go[b] = (uint16_t)io;
        }
    }
    return MC_OK;
}
