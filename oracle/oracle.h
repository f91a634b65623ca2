/*
 * Test oracle for the Monte Carlo / Lorenz-Mie photon-transport engine.
 *
 * THIS IS TEST INFRASTRUCTURE. It is a plain, slow, double-precision CPU
 * restatement of what the paper (arXiv 2507.23189) computes, written to check
 * the CUDA path against. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product library never does.
 * It shares no code, header, table or constant generator with the product.
 *
 * Contents
 *   mie.c     Mie coefficients a_n, b_n (Eq. 7-8, evaluated with the
 *             logarithmic-derivative recurrences of Bohren & Huffman, the
 *             paper's ref. [12] in Sec. 2.5), efficiencies (Eq. 13), amplitude
 *             functions S1/S2 (Eq. 5-6), phase function (Eq. 9), asymmetry
 *             parameter g (Eq. 12), cross section (Eq. 14), Eq. 17.
 *   table.c   normalisation (Eq. 10), cumulative distribution and its inverse
 *             on an equal-probability grid (Sec. 2.6, Sec. 3.1.2), and the
 *             paper's own 3000-angle cumulative distribution (Sec. 3.1.2).
 *   philox.c  Philox4x32-10 counter-based generator (Salmon et al., SC'11).
 *   walk.c    the photon random walk of Sec. 3.1.3 (Eq. 15, Eq. 16) with a
 *             next-event estimate for the 90-degree side camera (Sec. 4.3);
 *             optionally through a voxel density grid by delta tracking
 *             (the complex media the paper leaves to future work, Sec. 6).
 *   walk32.c  the homogeneous walk again in IEEE single precision with
 *             explicit fused multiply-adds (the FP32 mode), traces only.
 *
 * Parity status: every function here is pinned by the -m "not gpu" tests
 * (closed forms, invariants, an independent 50-digit evaluation of Eq. 7-8,
 * a library Philox); none is "parity unpinned".
 */
#ifndef MC_ORACLE_H
#define MC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- mie.c */

/* Wiscombe's series length: ceil(x + 4 x^(1/3) + 2). */
int oracle_mie_nmax(double x);

/* Size parameter x = pi d / lambda (Eq. 3) with lambda the wavelength in the
 * medium, lambda0 / n_medium. d in micrometres, lambda0 in nanometres. */
double oracle_size_parameter(double d_um, double n_medium, double lambda0_nm);

/* a_n, b_n for n = 1..nmax, stored interleaved as (re, im) pairs at index
 * 2*(n-1).  m = m_re + i m_im is the refractive index relative to the medium
 * (m_im >= 0 absorbs).  Returns 0, or -1 on bad arguments. */
int oracle_mie_ab(double m_re, double m_im, double x, int nmax,
                  double *a_reim, double *b_reim);

/* Efficiencies from the series: Eq. 13 for Q_ext, the matching sum of
 * |a_n|^2 + |b_n|^2 for Q_sca, and g from the cross-term series. */
int oracle_mie_efficiencies(double m_re, double m_im, double x,
                            double *qext, double *qsca, double *g_series);

/* S1 and S2 (Eq. 5-6) at n_mu cosines, (re, im) interleaved outputs. */
int oracle_mie_s12(double m_re, double m_im, double x, const double *mu,
                   int n_mu, double *s1_reim, double *s2_reim);

/* Raw phase function |S1|^2 + |S2|^2 (Eq. 9 without the constant 1/k^2). */
int oracle_mie_phase_raw(double m_re, double m_im, double x, const double *mu,
                         int n_mu, double *p);

/* Extinction cross section, Eq. 14: sigma = Q pi d^2 / 4, d in um, result
 * in mm^2. */
double oracle_cross_section_mm2(double q, double d_um);

/* Eq. 17: optical depth from number density (per mm^3), cross section (mm^2)
 * and path length (mm). */
double oracle_optical_depth(double n_per_mm3, double sigma_mm2, double l_mm);

/* --------------------------------------------------------------- table.c */

/* Phase-function kinds understood by the table builder. */
#define ORACLE_PHASE_MIE 0
#define ORACLE_PHASE_HG  1
#define ORACLE_PHASE_PAPER 2   /* walk only: the cdf of oracle_paper_cdf */

/* Build the equal-probability inverse CDF of a phase function.
 *   kind == ORACLE_PHASE_MIE: (m_re, m_im, x) select the Mie phase function.
 *   kind == ORACLE_PHASE_HG : hg_g selects Eq. 11.
 * n_fine (even) is the number of fine theta intervals on [0, pi].
 * Outputs (each may be NULL):
 *   icdf[n_bins+1]  cos(theta) at cumulative probability i / n_bins
 *   omu [n_bins+1]  1 - icdf, computed without cancellation
 *   pdf [n_bins]    density per unit cos(theta) of the piecewise-linear
 *                   inverse CDF, (1/n_bins) / (icdf[j+1] - icdf[j])
 *   diag[4]         {raw normalisation 1/2 int P dmu, g by quadrature,
 *                    mean of the tabulated distribution, n_fine}
 * Returns 0, or -1 on bad arguments. */
int oracle_phase_table(int kind, double m_re, double m_im, double x,
                       double hg_g, int n_bins, int n_fine, double *icdf,
                       double *omu, double *pdf, double *diag);

/* The same for the weighted phase function p(mu) h_w(mu) / Z(w),
 * h_w = sum_k w_k phi_k (hat functions of oracle_hat), n_w >= 2. */
int oracle_phase_table_weighted(int kind, double m_re, double m_im, double x,
                                double hg_g, int n_w, const double *w, int n_bins,
                                int n_fine, double *icdf, double *omu, double *pdf,
                                double *diag);

/* The table omu_base[n_bins + 1] (1 - cos theta at the levels, as
 * oracle_phase_table writes it) reweighted: its own piecewise-constant
 * density times h_w = sum_k w_k phi_k (n_w >= 2 hats of oracle_hat, every
 * w_k > 0), renormalised and inverted at the equal-probability levels.
 * Outputs icdf, omu [n_bins + 1] and pdf [n_bins] as oracle_phase_table
 * (icdf, pdf may be NULL); *z_out (may be NULL) receives Z(w) = int p h_w.
 * Returns 0, or -1 on bad arguments. */
int oracle_phase_table_reweighted(const double *omu_base, int n_bins, int n_w, const double *w,
                                  double *icdf, double *omu, double *pdf, double *z_out);

/* Table of a mixture of n_comp phase functions (kind[i], m[i], x[i] or
 * hg_g[i]), component i weighted by w[i] >= 0 (its share n_i sigma_sca,i of
 * the scattering coefficient) after each is normalised (Eq. 10). Outputs
 * as oracle_phase_table. */
int oracle_phase_table_mixture(int n_comp, const int *kind, const double *m_re,
                               const double *m_im, const double *x, const double *hg_g,
                               const double *w, int n_bins, int n_fine, double *icdf,
                               double *omu, double *pdf, double *diag);

/* The paper's own sampling table (Sec. 3.1.2): cdf[i], i < n_theta, the
 * cumulative probability of scattering angles up to theta_i = i pi /
 * (n_theta - 1) (trapezoidal rule on (1/2) P(cos theta) sin theta, normalised
 * so that cdf[0] = 0 and cdf[n_theta - 1] = 1). The walk samples it by binary
 * search and linear interpolation in theta (ORACLE_PHASE_PAPER). */
int oracle_paper_cdf(int kind, double m_re, double m_im, double x, double hg_g,
                     int n_theta, double *cdf);

/* -------------------------------------------------------------- philox.c */

/* Philox4x32 with 10 rounds: out = bijection(ctr) under key. */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                          uint32_t out[4]);

/* Batch form for tests: n counters (4 words each), one key. */
void oracle_philox4x32_10_n(const uint32_t *ctr, uint64_t n,
                            uint64_t seed, uint32_t *out);

/* The uniform in (0,1) the walk draws from one 32-bit output word. */
double oracle_uniform(uint32_t r);

/* ---------------------------------------------------------------- walk.c */

typedef struct {
    /* medium */
    double mu_s, mu_a;          /* mm^-1 */
    int phase_kind;             /* ORACLE_PHASE_MIE (table), _HG or _PAPER */
    double hg_g;
    const double *icdf;         /* [n_bins+1] when phase_kind == MIE */
    const double *omu;          /* [n_bins+1], 1 - icdf */
    int n_bins;
    const double *cdf;          /* [n_theta] when phase_kind == PAPER */
    int n_theta;
    /* geometry: x in [0,lx] (beam axis), y in [-ly/2,ly/2], z in [-lz/2,lz/2] */
    double lx, ly, lz;
    double beam_radius;         /* 0: pencil beam at (0,0,0) */
    /* side camera on y = +ly/2, columns along x, rows along z */
    int nx, nz;
    int n_radial;               /* far-face radial profile bins */
    double r_max;
    /* run */
    uint64_t n_photons, photon_offset, seed;
    double rr_threshold, rr_survival;
    uint32_t max_events;        /* flights per photon before truncation */
    uint32_t max_scatter;       /* 0: unlimited; else stop after that many collisions */
    double cone_cos;            /* > 0 enables the ORACLE_T_CONE tally */
    int n_threads;
    /* heterogeneous medium, delta tracking (density NULL: homogeneous).
     * density[gz][gy][gx]: particles per mm^3, constant on each voxel of the
     * cuvette; mu_ext = k_ext n + mu_a, mu_s = k_sca n (mu_s above unused);
     * majorants constant on cells of bx x by x bz voxels. Traces then record
     * real collisions and the exit only; max_events counts tentative ones. */
    const double *density;
    int gx, gy, gz;
    double k_ext, k_sca;
    int bx, by, bz;
    /* majorants: the largest mu_ext of each cell times majorant_scale (0 or
     * 1: the largest itself). trace_nulls != 0: traces of a heterogeneous
     * walk also record every null collision (status 7, in event order) */
    double majorant_scale;
    int trace_nulls;
} oracle_walk_cfg;

/* Totals, in weight units (one photon carries weight 1). */
enum {
    ORACLE_T_REFLECT = 0,   /* left through x = 0 */
    ORACLE_T_FAR = 1,       /* left through x = lx */
    ORACLE_T_SIDE = 2,      /* left through a y or z face */
    ORACLE_T_ABSORB = 3,    /* implicit capture, Eq. 16 */
    ORACLE_T_ROULETTE = 4,  /* net weight removed by roulette */
    ORACLE_T_TRUNC = 5,     /* weight left when max_events / max_scatter hit */
    ORACLE_T_BALLISTIC = 6, /* far-face weight with no collision */
    ORACLE_T_CONE = 7,      /* analog camera: weight leaving y = +ly/2 with
                               d_y >= cone_cos (test of the camera estimate) */
    ORACLE_N_TOTALS = 8
};

typedef struct {
    double *image, *image_sq;     /* [nz*nx] sum and sum of per-photon squares */
    double *image_hits;           /* [nz*nx] number of contributions (may be NULL) */
    double *radial, *radial_sq;   /* [n_radial] */
    double totals[ORACLE_N_TOTALS];
    double totals_sq[ORACLE_N_TOTALS];
    uint64_t steps;               /* sampled free flights */
    uint64_t capped;              /* photons stopped by max_events */
} oracle_walk_out;

/* Per-event trace record, double precision. */
typedef struct {
    double status;   /* 0 collided, 1 reflect, 2 far, 3 side, 4 roulette kill,
                        5 truncated (max_scatter), 6 capped (max_events),
                        7 null collision (trace_nulls; then w holds mu_ext at
                        the point, nee the majorant, pix the voxel index) */
    double r[3];     /* position after the flight (collision or exit point) */
    double d[3];     /* direction after the event */
    double w;        /* weight after the event */
    double nee;      /* camera contribution added at this event (0: none) */
    double pix;      /* pixel index of that contribution, -1: none */
    double nee_bin;  /* table bin used for the camera density, -1: none/HG */
    double rad_bin;  /* radial bin for a far-face exit, -1 otherwise */
    double margin;   /* smallest relative distance of any discrete decision
                        taken at this event to its threshold */
} oracle_trace_rec;

/* Run photons [photon_offset, photon_offset + n_photons). Tallies are
 * accumulated into out (caller zeroes them). If trace != NULL, the first
 * n_trace photons of the range record their first n_trace_events events into
 * trace[photon * n_trace_events + event] (unused records get status -1).
 * Returns 0, or -1 on bad arguments. */
int oracle_walk(const oracle_walk_cfg *cfg, oracle_walk_out *out,
                oracle_trace_rec *trace, int n_trace, int n_trace_events);

/* ---------------------------------------------------------- walk32.c */

/* The same walk in IEEE single precision with explicit fused multiply-adds
 * (the oracle's FP32 mode): homogeneous medium, table or H-G phase, the
 * first n_trace_events events of photons photon_offset .. + n_trace - 1
 * recorded as by oracle_walk (no tallies). Returns 0 or -1. */
int oracle_walk32_trace(const oracle_walk_cfg *cfg, oracle_trace_rec *trace, int n_trace,
                        int n_trace_events);

/* ---------------------------------------------------------- adjoint.c */

/* Hat functions for the phase-weight gradient: n_w nodes at
 * mu_k = -1 + 2k/(n_w-1); phi_k is 1 at mu_k and falls linearly to 0 at the
 * neighbouring nodes. */
double oracle_hat(int n_w, int k, double mu);

/* Z_k = int_{-1}^{1} p(mu) phi_k(mu) dmu for the tabulated density
 * (piecewise constant on the table bins), exactly. */
void oracle_hat_integrals(const double *omu, int n_bins, int n_w, double *z);

/* Gradient of L = sum_pix adj[pix] * image[pix] with respect to
 * (mu_s, mu_a, w_0..w_{n_w-1}) at w = 1, where the phase function is
 * p_w(mu) = p(mu) h_w(mu) / Z(w), h_w = sum_k w_k phi_k. Score-function
 * (likelihood-ratio) terms for every sampled flight and polar angle plus
 * direct terms of each camera contribution; roulette factors are held
 * fixed. Same photons, random numbers and tallies as oracle_walk.
 * grad[2 + n_w], grad_sq[2 + n_w] (sums of per-photon squares) and
 * *value (the functional itself, from the replayed paths) are accumulated
 * (caller zeroes). n_w = 0 skips the phase weights; n_w > 0
 * needs the table phase. Returns 0 or -1. */
int oracle_adjoint(const oracle_walk_cfg *cfg, const double *adj, int n_w, double *grad,
                   double *grad_sq, double *value);

/* oracle_adjoint at phase weights w[n_w] (all > 0; NULL: all 1): the walk's
 * table (cfg) is the phase function p_w = p h_w / Z(w) as tabulated by
 * oracle_phase_table_reweighted from the unweighted table base_omu[n_bins+1]
 * (NULL: cfg's own table, only with w NULL), and the phase-weight scores
 * are d log p_w / dw_k = phi_k / h_w - Z_k / Z(w), Z_k = int p phi_k over
 * the unweighted table. */
int oracle_adjoint_weighted(const oracle_walk_cfg *cfg, const double *adj, int n_w, const double *w,
                            const double *base_omu, double *grad, double *grad_sq, double *value);

/* Gradient of L = sum_pix adj[pix] image[pix] with respect to the voxel
 * densities of c->density (delta-tracking walk), from the oracle walk's own
 * paths; grad[gz*gy*gx] (overwritten), *value = L. max_events: trace room
 * per photon (real events); -1 if a photon needs more. Roulette held fixed. */
int oracle_grid_adjoint(const oracle_walk_cfg *c, const double *adj, int max_events, double *grad,
                        double *value);

/* The same gradient with the flights' transmission scored at the null
 * collisions of delta tracking instead of integrated along each flight:
 * against majorants mubar = majorant_scale x the cell's largest mu_ext
 * (c->majorant_scale > 1, so every voxel has mubar > mu_ext), a null
 * collision at a point of voxel v has probability 1 - mu_ext / mubar, whose
 * derivative with respect to n_v gives the score -k_ext / (mubar - mu_ext);
 * it multiplies the camera terms that follow (B of its flight). Real
 * collisions and camera columns as oracle_grid_adjoint. An unbiased
 * estimate of the same gradient from paths of the walk with those
 * majorants. max_events: trace room per photon (null and real events). */
int oracle_grid_adjoint_nulls(const oracle_walk_cfg *c, const double *adj, int max_events, double *grad,
                              double *value);

#ifdef __cplusplus
}
#endif
#endif
