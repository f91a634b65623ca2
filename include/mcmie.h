/*
 * mcmie.h - C ABI of the GB300 Monte Carlo / Lorenz-Mie photon-transport
 * engine (arXiv 2507.23189, "GPU-Accelerated Monte Carlo Simulation and
 * Experimental Study of Radiative Transfer in Multiple Scattering Media").
 *
 * Conventions for every entry point:
 *  - Every call returns an mc_status and never aborts the process. Invalid
 *    arguments are rejected (MC_ERR_ARG) before anything is launched.
 *  - Lengths are in millimetres, coefficients in mm^-1, particle diameters in
 *    micrometres, wavelengths in nanometres.
 *  - Pointers named d_* are device pointers; all other pointers are host
 *    pointers. All buffers are owned by the caller; the library never frees
 *    or keeps a pointer after a call returns. Device pointers must be 16-byte
 *    aligned (any cudaMalloc / torch allocation is).
 *  - Device calls are asynchronous and ordered on the given stream (0: the
 *    legacy default stream). Device-side problems (event cap reached, a
 *    non-finite value, a table-staging timeout) are recorded as bits in the
 *    caller's error word; mc_check() reads it back and maps it to a status.
 *  - mc_run and mc_trace allocate nothing: scratch memory comes from the
 *    caller's workspace (mc_workspace_bytes()).
 *  - Photons [photon_offset, photon_offset + n_photons) are simulated; photon
 *    p draws event e's random numbers from Philox4x32-10 with key = seed and
 *    counter (p_lo, p_hi, e, 0), so splitting a photon range over calls,
 *    streams or GPUs gives bit-identical integer tallies.
 */
#ifndef MCMIE_H
#define MCMIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MC_NOT_READY = 1,     /* mc_check_within: the stream's work still runs     */
    MC_OK = 0,
    MC_ERR_ARG = -1,      /* invalid argument; nothing was launched            */
    MC_ERR_CUDA = -2,     /* a CUDA runtime call failed                        */
    MC_ERR_NOMEM = -3,    /* workspace too small                               */
    MC_ERR_TIMEOUT = -4,  /* a bounded device wait (table staging) gave up     */
    MC_ERR_OVERFLOW = -5, /* a fixed-point contribution exceeded 2^62, or a
                             tally sum reached 2^63 (wrapped)                  */
    MC_ERR_NUMERIC = -6,  /* a non-finite weight or contribution was seen      */
    MC_ERR_EVENTS = -7,   /* at least one photon hit max_events (truncated)    */
    MC_ERR_TABLE = -8,    /* the device table blob failed its header check     */
    MC_ERR_BOUNDS = -9    /* checked build only: an index check failed         */
} mc_status;

/* Device error-word bits (OR-ed by kernels into *d_error). */
#define MC_EFLAG_EVENTS   0x1u
#define MC_EFLAG_TIMEOUT  0x2u
#define MC_EFLAG_NUMERIC  0x4u
#define MC_EFLAG_OVERFLOW 0x8u  /* a contribution above 2^62, or a non-negative tally
                                    (pixel, radial bin, total) found negative after a
                                    run: its sum passed 2^63 */
#define MC_EFLAG_TABLE    0x10u
#define MC_EFLAG_BOUNDS   0x20u  /* checked build (MC_CHECKED) only: an index fell outside
                                    its array; the access was clamped instead of made */

/* ------------------------------------------------------------------------
 * Phase table (Sec. 2.2 Eq. 3-9, Sec. 2.4 Eq. 12, Sec. 2.5 Eq. 13-14,
 * Sec. 3.1.2): the Mie phase function is computed in double precision,
 * normalised (Eq. 10) and inverted on n_bins equal-probability levels.
 * ------------------------------------------------------------------------ */

typedef struct {
    double diameter_um;    /* sphere diameter d                                 */
    double n_particle_re;  /* particle refractive index n + i k (Eq. 4)         */
    double n_particle_im;  /*   k >= 0 absorbs                                  */
    double n_medium;       /* refractive index of the surrounding medium        */
    double wavelength_nm;  /* vacuum wavelength lambda0                         */
    int n_bins;            /* equal-probability bins; power of two, 64..16384   */
} mie_params;

typedef struct {
    double x;              /* size parameter pi d n_medium / lambda0 (Eq. 3)    */
    double m_re, m_im;     /* relative refractive index m_particle / n_medium   */
    double qext, qsca, qabs;        /* efficiencies (Eq. 13)                    */
    double g;                       /* asymmetry parameter (Eq. 12), series     */
    double g_table;                 /* mean cosine of the tabulated distribution */
    double sigma_ext_mm2, sigma_sca_mm2, sigma_abs_mm2; /* Eq. 14               */
    int nmax;                       /* terms kept in the Mie series             */
} mie_info;

/* Bytes of the packed table blob for n_bins bins (0 for an invalid n_bins). */
size_t mc_table_bytes(int n_bins);

/* Build the Mie phase table on the host.
 *   params   in: particle and wavelength (see mie_params).
 *   info     out: Mie quantities (may be NULL).
 *   table    out: host buffer of mc_table_bytes(n_bins) bytes receiving the
 *            packed single-precision table the kernels stage into shared
 *            memory; copy it to a device buffer for mc_medium.d_table. May be
 *            NULL.
 *   omu64    out: double[n_bins+1], 1 - cos(theta) at the levels i / n_bins
 *            (NULL to skip).
 *   pdf64    out: double[n_bins], density per unit cos(theta) on each bin of
 *            the piecewise-linear inverse CDF (NULL to skip).
 * Returns MC_OK, or MC_ERR_ARG / MC_ERR_NUMERIC. Thread-safe. */
mc_status mie_table_build(const mie_params *params, mie_info *info, void *table,
                          double *omu64, double *pdf64);

/* Phase table of a particle mixture, e.g. the size bins of a polydisperse
 * sample: n_comp particle kinds (params[k], all with the same n_bins) present
 * with number fractions number_frac[k] >= 0 (normalised here). The mixture
 * phase function weights each kind's normalised phase function (Eq. 9-10) by
 * its share f_k sigma_sca,k of the scattering cross section (Eq. 14). info
 * receives the number-averaged cross sections sigma_* (so that Eq. 17 with
 * the total number density gives mu_s, mu_a), efficiencies relative to the
 * mean geometric cross section, the mixture's g, and x, m of params[0].
 * Outputs otherwise as mie_table_build. 1 <= n_comp <= 256. */
mc_status mie_mixture_table_build(const mie_params *params, const double *number_frac, int n_comp,
                                  mie_info *info, void *table, double *omu64, double *pdf64);

/* The paper's own sampling table (Sec. 3.1.2): the phase function at
 * n_theta equally spaced scattering angles theta_i = i pi / (n_theta - 1),
 * its cumulative distribution by the trapezoidal rule on (1/2) P sin(theta),
 * normalised to end at 1; the walk samples it by bisection and linear
 * interpolation in theta (MC_PHASE_PAPER). The paper uses n_theta = 3000.
 * mc_paper_table_bytes: bytes of the packed blob (0 unless 16 <= n_theta <=
 * 16384). mie_paper_table_build:
 *   params   in: particle and wavelength (n_bins is ignored).
 *   info     out (may be NULL): as mie_table_build; g_table is the mean
 *            cosine of the sampled distribution.
 *   table    out (may be NULL): host buffer of mc_paper_table_bytes(n_theta)
 *            bytes; copy it to a 16-byte-aligned device buffer for
 *            mc_medium.d_table.
 *   cdf64    out (may be NULL): double[n_theta], the cumulative distribution.
 * Returns MC_OK, MC_ERR_ARG or MC_ERR_NUMERIC. Thread-safe. */
size_t mc_paper_table_bytes(int n_theta);
mc_status mie_paper_table_build(const mie_params *params, int n_theta, mie_info *info,
                                void *table, double *cdf64);

/* ------------------------------------------------------------------------
 * Transport (Sec. 2.6, Sec. 3.1.3: Eq. 15 free path, Eq. 16 implicit
 * capture, weight threshold; Sec. 4.3: 90-degree side camera).
 * ------------------------------------------------------------------------ */

#define MC_PHASE_TABLE 0   /* sample the staged inverse-CDF table           */
#define MC_PHASE_HG    1   /* Henyey-Greenstein (Eq. 11) with parameter hg_g */
#define MC_PHASE_PAPER 2   /* the paper's CDF table, bisection (Sec. 3.1.2) */

typedef struct {
    double mu_s, mu_a;      /* scattering / absorption coefficients, mm^-1     */
    int phase_kind;         /* MC_PHASE_TABLE, MC_PHASE_HG or MC_PHASE_PAPER   */
    double hg_g;            /* H-G asymmetry, -1 < g < 1 (MC_PHASE_HG only)    */
    const void *d_table;    /* device copy of a mie_table_build() blob, or of
                               a mie_paper_table_build() blob (PAPER)          */
    int n_bins;             /* bins of that blob, or its n_theta for PAPER
                               (checked against the blob's header)             */
} mc_medium;

/* Eq. 17: number density (per mm^3) times the extinction cross section gives
 * mu_ext; mu_s and mu_a follow from the Mie efficiencies, plus an absorption
 * coefficient of the host medium. Writes mu_s and mu_a of *out. */
mc_status mc_medium_from_density(const mie_info *info, double number_density_per_mm3,
                                 double mu_a_medium, mc_medium *out);

/* Eq. 17 solved for the number density: n = tau / (sigma_ext_mm2 length_mm)
 * gives optical depth tau (extinction by the particles) over a path of
 * length_mm; mu_s, mu_a of *out then follow as in mc_medium_from_density
 * (plus mu_a_medium). *number_density_out (may be NULL) receives n in
 * particles per mm^3. tau >= 0, length_mm > 0 and info->sigma_ext_mm2 > 0,
 * all finite, else MC_ERR_ARG. */
mc_status mc_medium_from_optical_depth(const mie_info *info, double tau, double length_mm,
                                       double mu_a_medium, mc_medium *out,
                                       double *number_density_out);

typedef struct {
    double lx, ly, lz;      /* cuvette: x in [0,lx] (beam axis),
                               y in [-ly/2,ly/2], z in [-lz/2,lz/2]            */
    double beam_radius;     /* 0: pencil beam entering at (0,0,0) along +x;
                               > 0: uniform disc of that radius at x = 0       */
} mc_geometry;

typedef struct {
    int nx, nz;             /* side image on the y = +ly/2 face: columns span
                               x in [0,lx], rows span z in [-lz/2,lz/2]        */
    int n_radial;           /* far-face (x = lx) radial profile bins           */
    double r_max;           /* radial profile range [0, r_max)                 */
} mc_camera;
/* Limits: nx, nz in [1, 8192], n_radial in [1, 65536]. The kernels sum the
 * radial profile (8 bytes a bin) and the totals in shared memory next to the
 * phase table (a 4096-bin table takes 41 KB, the largest, 16384 bins, 164 KB;
 * the grid walks add 4 bytes per majorant cell): a combination that does not
 * fit in one CTA's shared memory (227 KB on GB300) is refused with
 * MC_ERR_ARG before anything runs. The image needs no room there: the rows
 * that do not fit are summed in global memory. */

typedef struct {
    uint64_t n_photons;     /* photons to run, at most 2^31 per call (the
                               2^-32-unit weight totals stay below 2^63)       */
    uint64_t photon_offset; /* index of the first photon                       */
    uint64_t seed;          /* Philox key                                      */
    double rr_threshold;    /* weight below which roulette is played           */
    double rr_survival;     /* survival probability (0: plain cut)             */
    uint32_t max_events;    /* free flights per photon before truncation       */
    uint32_t max_scatter;   /* 0: unlimited; else end after that many collisions */
    int image_frac_bits;    /* fixed-point fraction bits of the image (8..48),
                               or 0 with accumulate = 0: mc_auto_frac_bits
                               (n_photons) (the batch: of its largest budget) */
    int accumulate;         /* 0: zero the tallies first; 1: add to them       */
    /* launch tuning; results do not depend on these (0 = automatic) */
    int block_size;         /* threads per CTA: 0 or a multiple of 32, <= 1024 */
    int blocks_per_sm;      /* persistent CTAs per SM: 0 = occupancy maximum   */
    int image_mode;         /* 0 auto, 1 whole image in shared memory (must
                               fit), 2 image atomics straight to global memory,
                               3 the rows around the beam that fit in shared
                               memory there, the other rows global            */
} mc_run_params;

/* Image fraction bits for a photon budget: min(32, 54 - ceil(log2 n)), at
 * least 8 (32 up to 2^22 photons, 27 at 1e8, 24 at 1e9). A pixel's sum then
 * stays a factor 2^9 below 2^63 even if it collected one weight unit per
 * photon. After every run a check flags any image pixel, radial bin or
 * non-negative total that passed 2^63 (MC_EFLAG_OVERFLOW). When tallies
 * accumulate over several calls, pass the F of the whole budget explicitly
 * to each call. */
int mc_auto_frac_bits(uint64_t n_photons);

/* Totals tallied by mc_run, as int64 in the units noted. */
enum {
    MC_TOT_REFLECT = 0,     /* weight leaving x = 0            (2^-32 units)  */
    MC_TOT_FAR = 1,         /* weight leaving x = lx           (2^-32)        */
    MC_TOT_SIDE = 2,        /* weight leaving y/z faces        (2^-32)        */
    MC_TOT_ABSORB = 3,      /* implicitly captured weight      (2^-32)        */
    MC_TOT_ROULETTE = 4,    /* net weight removed by roulette  (2^-32, signed) */
    MC_TOT_TRUNC = 5,       /* weight of truncated photons     (2^-32)        */
    MC_TOT_BALLISTIC = 6,   /* far-face weight, no collision   (2^-32)        */
    MC_TOT_STEPS = 7,       /* sampled free flights (photon-steps), count     */
    MC_N_TOTALS = 8
};
#define MC_WEIGHT_FRAC_BITS 32

typedef struct {
    int64_t *d_image;       /* [nz][nx] camera image, 2^-image_frac_bits units */
    int64_t *d_radial;      /* [n_radial] far-face weight by radius (2^-32)    */
    int64_t *d_totals;      /* [MC_N_TOTALS]                                   */
    uint32_t *d_error;      /* error word (MC_EFLAG_*), OR-ed; zero it first   */
    void *d_work;           /* scratch, >= mc_workspace_bytes() bytes          */
    size_t work_bytes;
} mc_tallies;

/* Scratch bytes mc_run / mc_trace need for this camera. */
size_t mc_workspace_bytes(const mc_camera *camera);

/* Run the photon walk on the GPU (Sec. 3.1.3): every photon of the range
 * enters at x = 0 (on the axis, or uniformly over the beam disc), then
 * repeats free flight (Eq. 15), escape at the first wall crossed, implicit
 * capture (Eq. 16), the side camera's next-event estimate, a scattering
 * angle from the medium's phase function, the rotation and the weight
 * threshold (roulette with run->rr_survival, or the paper's plain cut with
 * 0). Tallies go to *tallies in fixed point: the image [nz][nx], the radial
 * profile of far-face exits, the MC_TOT_* totals. run->accumulate = 0 zeroes
 * them first (on the stream), 1 adds to them. The error word is only OR-ed.
 * Returns at once: MC_ERR_ARG (invalid argument, a phase table and radial
 * profile too large for shared memory together (see mc_camera), or an image
 * tile that image_mode 1 cannot hold there), MC_ERR_NOMEM (workspace too
 * small) or MC_ERR_CUDA (a launch failed) before anything runs on the
 * device, MC_OK when queued. Device-side problems appear in the error word
 * (mc_check). Asynchronous on `stream`; the buffers must stay valid until
 * the stream reaches this work. */
mc_status mc_run(const mc_medium *medium, const mc_geometry *geom,
                 const mc_camera *camera, const mc_run_params *run,
                 const mc_tallies *tallies, void *stream);

/* mc_run for callers that cannot allocate device memory for a workspace (for
 * example a host application that owns all device memory and hands a plug-in
 * only the buffers it reads and writes). The paper has no counterpart: this is
 * an interface convenience. The scratch the walk needs lives in a fixed
 * MC_STATIC_SCRATCH_BYTES device array inside the library, held by every GPU
 * that loads it until exit. Every valid camera needs mc_workspace_bytes() =
 * 256 bytes today, so the MC_ERR_NOMEM rejection of a workspace larger than
 * the array only guards against future growth of the walk's scratch; an
 * invalid camera is MC_ERR_ARG. The array's address is looked up
 * (cudaGetSymbolAddress) by the first call in each CUDA context of a device
 * and cached with the context's id, so a new context (after cudaDeviceReset,
 * say) is looked up again; make the first call in a context before any
 * stream capture. All calls share the array: consecutive calls are
 * independent (the counter is cleared on the stream first), but calls that
 * overlap on the GPU race and must be serialised by the caller. Allocates
 * nothing. Other arguments and errors as for mc_run. */
#define MC_STATIC_SCRATCH_BYTES 4096
mc_status mc_run_static(const mc_medium *medium, const mc_geometry *geom,
                        const mc_camera *camera, const mc_run_params *run,
                        int64_t *d_image, int64_t *d_radial, int64_t *d_totals,
                        uint32_t *d_error, void *stream);

/* Many media in one launch: every CTA goes through the media in order of
 * decreasing estimated cost (photons x (1 + optical depth along x)); its warps
 * take chunks of item_photons photons of the current medium from that
 * medium's counter (0: 128; else 32 .. 2^20), and when the medium's photons
 * are all taken the CTA flushes its tallies into the medium's, stages the
 * next medium's table in shared memory and goes on, so the media follow one
 * another without launch gaps. All instances share geometry, camera and run
 * parameters (run->n_photons, photon_offset and seed are ignored; each
 * instance has its own), and one phase kind and table size. Tallies per
 * instance as for mc_run, bit-identical to running each instance with
 * mc_run. d_work: mc_batch_workspace_bytes(n) bytes (one counter per medium,
 * cleared on the stream by each call). At most 64 media. */
typedef struct {
    mc_medium medium;
    uint64_t n_photons, photon_offset, seed;
    int64_t *d_image, *d_radial, *d_totals;  /* device, [nz][nx], [n_radial], [MC_N_TOTALS] */
} mc_instance;
size_t mc_batch_workspace_bytes(int n_instances);
mc_status mc_run_batch(int n, const mc_instance *inst, const mc_geometry *geom,
                       const mc_camera *camera, const mc_run_params *run,
                       uint64_t item_photons, uint32_t *d_error, void *d_work,
                       size_t work_bytes, void *stream);

/* Phase function with hat-function weights w (n_phase_w of them, device
 * floats, all > 0): p_w(mu) = p(mu) h_w(mu) / Z(w), h_w = sum_k w_k phi_k the
 * linear interpolant of the weights at the nodes mu_k = -1 + 2k/(n_phase_w -
 * 1), p the density of base's table (constant on each bin), Z(w) = int p h_w
 * (Eq. 9-10: the reweighted function is renormalised like the phase
 * function itself). Writes into d_table (table_bytes >= mc_table_bytes(
 * base->n_bins), 16-byte aligned, not base's own blob) the equal-probability
 * table of p_w in the layout of mie_table_build's blob, so that an mc_medium
 * pointing at it makes mc_run sample p_w and use it as the camera density.
 * Built by one CTA in double precision, stream-ordered, nothing copied to
 * the host. Weights that are not all positive and finite (or levels that
 * single precision cannot hold apart) set MC_EFLAG_NUMERIC in *d_error and
 * write an invalid header, so a walk using the blob reports MC_ERR_TABLE.
 * The unweighted table's bin edges are taken in double precision from its
 * bin densities (every bin holds 1/n_bins), and the new densities from the
 * new levels in double precision, as mie_table_build does. 2 <= n_phase_w <=
 * 256; base->phase_kind must be MC_PHASE_TABLE with n_bins <= 8192. The paper
 * has no phase weights; they parametrise the phase function for fitting. */
mc_status mc_phase_table_weighted(const mc_medium *base, int n_phase_w, const float *d_phase_w, void *d_table,
                                  size_t table_bytes, uint32_t *d_error, void *stream);

/* Gradient of L = sum_pix adj[pix] * image[pix] (adj: d_adj_image, float,
 * [nz][nx], in the image's weight units) with respect to mu_s, mu_a and
 * n_phase_w hat-function weights w of the phase function p_w = p h_w / Z(w)
 * (see mc_phase_table_weighted), evaluated at the device weights d_phase_w
 * (all > 0), or at w = 1 when d_phase_w is NULL. medium carries the
 * unweighted table p; with weights, the walk samples p_w through the table
 * mc_phase_table_weighted builds (here into d_work), i.e. the photons mc_run
 * simulates with that table and the same other arguments. Likelihood ratios
 * of every sampled flight (Eq. 15) and polar angle plus the direct terms of
 * each camera contribution (Eq. 16 weight, transport, phase density), on
 * those photons, replayed from their Philox counters (nothing about the
 * paths is stored): the phase-weight scores are phi_k(mu) / h_w(mu) - Z_k /
 * Z(w), Z_k = int p phi_k. Roulette factors are held fixed. d_out[3 +
 * n_phase_w] receives (L, dL/dmu_s, dL/dmu_a, dL/dw_0, ..) in double
 * precision, reduced in a fixed order. n_phase_w: 0 (no phase weights;
 * d_phase_w must be NULL) or 2..256 (MC_PHASE_TABLE only; with d_phase_w,
 * n_bins <= 8192). One pass per
 * photon; with phase weights, photons with more than 8 collisions are
 * replayed once more. MC_PHASE_PAPER is not supported (MC_ERR_ARG).
 * Requires mu_s > 0.
 * d_work: mc_adjoint_workspace_bytes(n_phase_w) bytes. The paper has no
 * gradients; this serves fitting mu_s, mu_a and the phase function. */
size_t mc_adjoint_workspace_bytes(int n_phase_w);
mc_status mc_adjoint(const mc_medium *medium, const mc_geometry *geom,
                     const mc_camera *camera, const mc_run_params *run,
                     const float *d_adj_image, int n_phase_w, const float *d_phase_w,
                     double *d_out, uint32_t *d_error, void *d_work, size_t work_bytes,
                     void *stream);

/* ------------------------------------------------------------------------
 * Heterogeneous media: the number density of the particles on a voxel grid
 * spanning the cuvette (the paper's walls and camera; the complex media its
 * Sec. 6 leaves to future work). In voxel v, mu_ext = k_ext n_v + mu_a and
 * mu_s = k_sca n_v (Eq. 17 per voxel; k_* are the cross sections per
 * particle, e.g. the mixture averages of mie_mixture_table_build). Flights
 * are sampled by delta (Woodcock) tracking against a majorant constant on
 * cells of bx x by x bz voxels; the camera transmittance of a collision is
 * the exact optical depth of its voxel column. Event e of photon p draws
 * Philox (p_lo, p_hi, e, 0) for every tentative collision: u0 optical depth
 * of the flight, u1 polar angle, u2 azimuth, u3 acceptance (real if u3 <
 * mu_ext / majorant), then u3 / (mu_ext / majorant) for roulette.
 * ------------------------------------------------------------------------ */
typedef struct {
    const float *d_density;   /* device, [gz][gy][gx] particles per mm^3 (>= 0, finite) */
    int gx, gy, gz;           /* voxels along x, y, z: 1..4096 each, product <= 2^28 */
    double k_ext, k_sca;      /* mm^2, k_ext >= k_sca >= 0, k_ext > 0 */
    double mu_a;              /* uniform background absorption, mm^-1 (>= 0) */
    int bx, by, bz;           /* majorant cells in voxels (>= 1); at most 16384 cells */
} mc_grid;

/* Device bytes of a prepared grid (per voxel mu_ext and the optical depth
 * above it as two floats, then the cell majorants); 0 if *grid is invalid. */
size_t mc_grid_workspace_bytes(const mc_grid *grid);

/* Prepare d_work (mc_grid_workspace_bytes bytes, 16-byte aligned) from the
 * density: per voxel (mu_ext, optical depth from the voxel's top face to y =
 * +ly/2, summed in double) and per cell the largest mu_ext. Asynchronous on
 * `stream`; redo after the density changes. */
mc_status mc_grid_prepare(const mc_grid *grid, const mc_geometry *geom, void *d_work, size_t work_bytes,
                          void *stream);

/* The walk through a prepared grid. phase: its phase_kind, hg_g, d_table and
 * n_bins give the phase function (a table of the mixture for a polydisperse
 * suspension); its mu_s, mu_a are ignored. max_events bounds the tentative
 * collisions of a photon. d_trace (may be NULL): n_trace * n_events records
 * as mc_trace's, one per real collision and one for the exit. Other
 * arguments and errors as mc_run. */
mc_status mc_run_grid(const mc_grid *grid, const void *d_grid_work, const mc_medium *phase,
                      const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                      const mc_tallies *tallies, void *d_trace, int n_trace, int n_events, void *stream);

/* Gradient of L = sum_pix adj[pix] image[pix] (adj: d_adj_image, float
 * [nz][nx], in the image's weight units) with respect to every voxel density
 * n_v, on the photons mc_run_grid would run with the same arguments. Each
 * photon runs twice on its Philox counters (the first pass sums its camera
 * terms); every real flight i contributes B_i / n_v at its collision voxel
 * (the scattering density k_sca n exp(-int mu_ext)) and -B_i k_ext times its
 * length inside each voxel it crosses, B_i the camera terms from collision i
 * on; every camera term contributes -A k_ext times the length of its column
 * inside each voxel above the collision. Roulette factors are held fixed.
 * d_grad: float [gz][gy][gx], overwritten (terms formed in single precision,
 * summed by double-precision atomics and rounded once; the sums' last bits
 * depend on scheduling); *d_value = L
 * (double, fixed order).
 * d_work: mc_grid_adjoint_workspace_bytes(grid) bytes (three
 * double-precision voxel arrays). The kernel holds the phase table, the
 * majorant cells and 12 KB of per-warp flight queues in shared memory: a
 * table and cell count that do not fit there (the largest table with the
 * most cells does not) are refused with MC_ERR_ARG before anything runs.
 * The paper has no gradients; this serves fitting the density of a
 * heterogeneous medium. */
size_t mc_grid_adjoint_workspace_bytes(const mc_grid *grid);
mc_status mc_grid_adjoint(const mc_grid *grid, const void *d_grid_work, const mc_medium *phase,
                          const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                          const float *d_adj_image, float *d_grad, double *d_value, uint32_t *d_error,
                          void *d_work, size_t work_bytes, void *stream);

/* mc_grid_adjoint with the flights' transmission scored at the null
 * collisions of delta tracking instead of integrated along each flight
 * (same arguments and outputs; d_work: mc_grid_adjoint_nulls_workspace_bytes
 * (grid) bytes: the voxel sum and the column sources, and eight copies of
 * both over the central 32 x 32 voxels of y and z (all x) around the beam
 * axis, over which the CTAs spread their atomics, since many CTAs adding to
 * the same voxels there at once serialise in L2; the copies are summed into
 * the voxels before the fold). The gradient walk uses majorants
 * majorant_scale (1 < scale <= 16) times the cell maxima, so every voxel
 * has mubar > mu_ext; a null collision at a point of voxel v then has
 * probability 1 - mu_ext / mubar, and its derivative with respect to n_v,
 * the score -k_ext / (mubar - mu_ext), times the camera terms that follow
 * its flight is added at v (one atomic per null collision instead of every
 * voxel the flight crosses). Real collisions and camera columns as in
 * mc_grid_adjoint. An unbiased estimate of the same gradient, from paths of
 * the walk with those majorants (so not the photons mc_run_grid runs);
 * max_events counts their tentative collisions. The paper has no
 * gradients; this trades the exact flight integrals for cheaper, noisier
 * per-voxel scores. */
size_t mc_grid_adjoint_nulls_workspace_bytes(const mc_grid *grid);
mc_status mc_grid_adjoint_nulls(const mc_grid *grid, const void *d_grid_work, const mc_medium *phase,
                                const mc_geometry *geom, const mc_camera *camera, const mc_run_params *run,
                                const float *d_adj_image, double majorant_scale, float *d_grad,
                                double *d_value, uint32_t *d_error, void *d_work, size_t work_bytes,
                                void *stream);

/* Image comparison (Sec. 3.1.4: every image normalised the same way, here
 * min-max to [0, 1]; Table 3: RMSE and Pearson r over the pixels; Table 4:
 * radial profiles, i.e. means over n_r equal-width rings about the image
 * centre out to the half-diagonal, compared zone by zone, ring b standing for
 * the angle 180 deg (b + 1/2) / n_r: forward < 30 deg, intermediate 30-120
 * deg, edge > 120 deg). Images: device int64 [nz][nx] (the camera images of
 * mc_run; the unit cancels in the normalisation). d_b may be NULL.
 * d_out: mc_metrics_out_len(n_r) doubles, device:
 *   [0..5]   a vs ref: RMSE, r, zone RMSE (forward, intermediate, edge),
 *            correlation of the radial profiles
 *   [6..11]  the same for b (zeros without b)
 *   [12]     share of rings where a's profile is closer to ref's than b's
 *   [13 ..]  the radial profiles of ref, a and b (n_r each)
 * Rings that hold no pixel are left out of the profile statistics. Sums are
 * double precision in a fixed order (bit-reproducible). 1 <= n_r <= 4096,
 * nx, nz >= 1, nx * nz <= 2^26. d_work: mc_metrics_workspace_bytes(n_r). */
int mc_metrics_out_len(int n_r);
size_t mc_metrics_workspace_bytes(int n_r);
mc_status mc_image_metrics(const int64_t *d_ref, const int64_t *d_a, const int64_t *d_b,
                           int nx, int nz, int n_r, double *d_out, void *d_work,
                           size_t work_bytes, void *stream);

/* Host-buffer form of mc_run, for callers whose inputs and outputs live in
 * host memory. The table blob (mc_table_bytes(n_bins) bytes, or NULL for
 * MC_PHASE_HG) is copied to the device, the walk runs, and image, radial
 * profile and totals are copied back; the call returns when they are in
 * host memory. d_work must hold mc_host_workspace_bytes() bytes of device
 * memory (table, tallies and scratch are carved from it). */
size_t mc_host_workspace_bytes(const mc_medium *medium, const mc_camera *camera);
mc_status mc_run_host(const mc_medium *medium, const void *table,
                      const mc_geometry *geom, const mc_camera *camera,
                      const mc_run_params *run, int64_t *image, int64_t *radial,
                      int64_t *totals, uint32_t *error, void *d_work,
                      size_t work_bytes, void *stream);

/* Per-event trace of the first n_trace photons of the range, first
 * n_events events each (same arithmetic as mc_run, tallies included).
 * d_trace receives n_trace * n_events records of 12 32-bit words:
 *   [0] status (int32): -1 unused, 0 collided, 1 left x = 0, 2 left x = lx,
 *       3 left a side face, 4 ended by roulette, 5 ended by max_scatter,
 *       6 ended by max_events
 *   [1..3] position after the flight (float), [4..6] direction after the
 *   event (float), [7] weight after the event (float), [8] camera
 *   contribution (float), [9] pixel (int32, -1 none), [10] table bin of the
 *   camera density (int32, -1 none), [11] radial bin (int32, -1 none). */
mc_status mc_trace(const mc_medium *medium, const mc_geometry *geom,
                   const mc_camera *camera, const mc_run_params *run,
                   const mc_tallies *tallies, void *d_trace, int n_trace,
                   int n_events, void *stream);

/* Synchronise `stream`, read *d_error and map its bits to a status
 * (MC_OK when zero). */
mc_status mc_check(const uint32_t *d_error, void *stream);

/* mc_check with a host-side watchdog: polls the stream (cudaStreamQuery)
 * for at most timeout_ms milliseconds. MC_NOT_READY when the work is still
 * running then (it goes on; call again or mc_check later); otherwise as
 * mc_check. timeout_ms >= 0, d_error non-NULL, else MC_ERR_ARG. */
mc_status mc_check_within(const uint32_t *d_error, void *stream, double timeout_ms);

/* Self-test of the kernels' bounded waits: one CTA waits on an mbarrier
 * phase that can never complete (it expects bytes no copy delivers), gives
 * up after `tries` polls (1 .. 2^22) and sets MC_EFLAG_TIMEOUT in *d_error,
 * so that mc_check then returns MC_ERR_TIMEOUT and the context stays
 * usable. The same wait guards every table staging. */
mc_status mc_wait_selftest(uint32_t *d_error, uint32_t tries, void *stream);

/* Philox4x32-10 on the device: out[4i..4i+3] = Philox(key = seed,
 * counter = ctr[4i..4i+3]) for i < n. For testing the generator. */
mc_status mc_philox(const uint32_t *d_ctr, uint64_t n, uint64_t seed,
                    uint32_t *d_out, void *stream);

/* Short description of a status code (static string). */
const char *mc_status_string(mc_status s);

#ifdef __cplusplus
}
#endif
#endif /* MCMIE_H */
