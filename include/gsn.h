/*
 * gsn.h -- C ABI of the GB300 binned spectral-fit likelihood engine.
 *
 * The library evaluates, at each minimiser step, the binned Poisson negative
 * log-likelihood of a multi-species spectral model and its gradient
 * (GooStats, arXiv:1812.05686, section 4.1, Eq. (LL)):
 *
 *   NLL(theta) = sum_d sum_{j in window_d} [ mu_dj - n_dj + n_dj ln(n_dj / mu_dj) ]
 *                + 1/2 sum_p ((theta_p - c_p) / sigma_p)^2
 *
 *   mu_dj = eps_d [ sum_{s smeared} f_ds r_s sum_k R_jk(theta) S'_sk
 *                   + sum_{s peak} f_ds r_s int_{bin j} N(x; m_s, w_s) dx
 *                   + sum_{s template} f_ds r_s T_dsj ]
 *
 * with R_jk the bin integral of the analytic detector response of fine
 * true-energy column k (section 2.3): visible mean mu_k = LY * E_q(E_k; kB)
 * (Birks quenching with stopping power S(E) = s0 + s1/E), variance
 * sigma_k^2 = a + b mu_k + c mu_k^2, and either a Gaussian or the
 * moment-matched gamma ("generalized gamma") resolution.  f_ds (default 1)
 * and fixed multipliers of the response parameters of each dataset describe
 * the slices of a multivariate fit (section 2.4, gsn_set_dataset_factors).
 * n = 0 bins
 * contribute mu.  The data-only constant of -ln L is dropped, so NLL = 0 for
 * data equal to the model and an increase of 0.5 is one standard deviation.
 *
 * Conventions
 *  - All calls return 0 (GSN_OK) or a negative GSN_ERR_* code; the message
 *    of the last failure is available from gsn_last_error().
 *  - Pointers are host pointers unless the name ends in _dev (device
 *    pointers, valid on the context's device).
 *  - The library copies every input of gsn_set_* to device memory; the caller
 *    keeps ownership of its buffers.  Outputs are caller-allocated.
 *  - A context is bound to one device and one CUDA stream and is not
 *    thread-safe; use one context per host thread.
 *  - Arrays indexed [a][b] are dense row-major.
 */
#ifndef GSN_H
#define GSN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes -- */
#define GSN_OK                    0
#define GSN_ERR_ARG              -1  /* invalid argument or inconsistent sizes */
#define GSN_ERR_CUDA             -2  /* a CUDA runtime call failed */
#define GSN_ERR_NONPOSITIVE_MU   -3  /* mu <= 0 in a bin with n > 0: NLL set to +inf */
#define GSN_ERR_NONFINITE        -4  /* a parameter, mu or the NLL is not finite */
#define GSN_ERR_STATE            -5  /* set_data / set_species / set_params missing */
#define GSN_ERR_NOMEM            -6  /* device allocation failed */
#define GSN_ERR_TIMEOUT          -7  /* a bounded wait inside a kernel gave up (results not written) */

/* precision of the response build and contraction (the deviance and the
 * NLL reduction are FP64 in both modes) */
#define GSN_FP64                  0
#define GSN_MIXED                 1  /* FP32 response + contraction, FP64 deviance */

/* resolution shape (section 2.3) */
#define GSN_RES_GAUSS             0
#define GSN_RES_GAMMA             1  /* gamma density with mean mu_k, variance sigma_k^2 */
#define GSN_RES_GGAMMA            2  /* generalized gamma of free power p (Stacy's density
                                        p x^(d-1) exp(-(x/s)^p) / (s^d Gamma(d/p)), the
                                        generalized-gamma line shape cited in section 2.3) with
                                        (d, s) moment-matched to mu_k and sigma_k^2; p is the
                                        fit parameter in the power slot; p = 1 is GSN_RES_GAMMA */

/* species kinds (section 4.3) */
#define GSN_ANA                   0  /* fine spectrum smeared by the response */
#define GSN_ANA_SHIFT             1  /* fine spectrum shifted up in true energy, then smeared */
#define GSN_ANA_PEAK              2  /* Gaussian peak in p.e. with free position m and width w */
#define GSN_MC_TEMPLATE           3  /* Monte Carlo template: a histogram in each dataset's visible
                                        bins (section 3.2 template fit, gsn_set_template) */

/* per-dataset parameter slots: gsn_n_slots(S) = 3 S + 6
 *   [0, S)              rate r_s of species s (counts per unit exposure)
 *   S + 0 .. S + 4      LY [p.e./MeV], kB [cm/MeV], a [p.e.^2], b [p.e.], c
 *   S + 5 + 2 s         peak position m_s [p.e.]   (AnaPeak species only)
 *   S + 5 + 2 s + 1     peak width w_s [p.e.]      (AnaPeak species only)
 *   3 S + 5             power p > 0 of the generalized gamma (GSN_RES_GGAMMA only) */
#define GSN_SLOT_LY(S)    ((S) + 0)
#define GSN_SLOT_KB(S)    ((S) + 1)
#define GSN_SLOT_A(S)     ((S) + 2)
#define GSN_SLOT_B(S)     ((S) + 3)
#define GSN_SLOT_C(S)     ((S) + 4)
#define GSN_SLOT_M(S, s)  ((S) + 5 + 2 * (s))
#define GSN_SLOT_W(S, s)  ((S) + 6 + 2 * (s))
#define GSN_SLOT_P(S)     (3 * (S) + 5)

#define GSN_MAX_DATASETS  512  /* histograms, or slices of histograms (section 2.4) */
#define GSN_MAX_SPECIES   64
#define GSN_MAX_GROUPS    256  /* distinct (edges, response slots, response multipliers);
                                  at most 4 datasets share one response evaluation */

typedef struct gsn_ctx gsn_ctx;

typedef struct gsn_options {
    int    precision;      /* GSN_FP64 or GSN_MIXED */
    int    resolution;     /* GSN_RES_GAUSS, GSN_RES_GAMMA or GSN_RES_GGAMMA */
    double band_cut;       /* response band: a column is evaluated only where its
                              density exceeds exp(-band_cut) times its value at
                              the mean (<= 0: 34.5 for FP64, 20.7 for mixed) */
    double birks_s0;       /* stopping power S(E) = s0 + s1/E, MeV/cm (<= 0: 1.55) */
    double birks_s1;       /* MeV^2/cm (< 0: 0.155) */
    int    device;         /* CUDA device ordinal */
    void*  stream;         /* cudaStream_t for all work of the context; NULL = a
                              stream created and owned by the context */
    int    max_toys_per_launch; /* batch chunk bounding scratch memory (<= 0: 4096) */
    int    use_graphs;     /* 1: gsn_eval_grad and the batch calls record their kernel
                              launches into a CUDA graph on first use and replay it when a
                              call repeats with the same sizes and buffers; 0: plain launches.
                              Skipped while tracing is on or while the stream is being
                              captured by the caller. */
    int    autotune;       /* 1: on the first launch of each toy count whose occupancy
                              heuristic splits the work (small batches, single points),
                              time candidate work decompositions on the call's own inputs
                              and keep the fastest for the context; 0: the heuristic plan.
                              Decompositions sum the same terms in another fixed order, so
                              mixed-precision results may differ between contexts in the
                              last FP32 bits; with 0 they are bitwise reproducible. */
} gsn_options;

/* Fill *opt with the defaults described above (FP64, Gaussian, device 0,
 * graphs and autotuning on). */
int gsn_default_options(gsn_options* opt);

/* Create a context.  Errors: GSN_ERR_ARG (bad option), GSN_ERR_CUDA. */
int gsn_create(gsn_ctx** out, const gsn_options* opt);

/* Release the context and every device buffer it owns (NULL is a no-op). */
void gsn_destroy(gsn_ctx* ctx);

/* Message of the last failure on this context ("" if none; static string if ctx is NULL). */
const char* gsn_last_error(const gsn_ctx* ctx);

/* Number of per-dataset slots for n_species species (3 n_species + 6). */
int gsn_n_slots(int n_species);

/* Observed histograms (section 4.1 inputs: histogram, exposure).
 *   n_datasets    1 .. GSN_MAX_DATASETS
 *   n_bins[d]     >= 1
 *   bin_edges[d]  n_bins[d] + 1 strictly ascending edges in p.e., >= 0 for the
 *                 gamma resolution
 *   counts[d]     n_bins[d] observed counts (>= 0; integer values expected)
 *   exposures[d]  > 0
 *   win_lo/hi[d]  default fit window [lo, hi), 0 <= lo <= hi <= n_bins[d]
 * Datasets with identical edges and identical response slots share one
 * response evaluation. */
int gsn_set_data(gsn_ctx* ctx, int n_datasets, const int* n_bins, const double* const* bin_edges,
                 const double* const* counts, const double* exposures,
                 const int* win_lo, const int* win_hi);

/* Species (section 4.3).
 *   fine_centres   n_fine ascending true energies [MeV] (> 0); uniformly spaced
 *                  when an AnaShift species is present
 *   spectra        [n_species][n_fine] non-negative unnormalised shapes; the
 *                  library normalises each row to unit sum (rows of AnaPeak
 *                  species are ignored)
 *   kind           [n_species] GSN_ANA, GSN_ANA_SHIFT or GSN_ANA_PEAK
 *   shift          [n_species] AnaShift offset [MeV], rounded to whole fine
 *                  bins (NULL = no shifts)
 *   dataset_mask   [n_species][n_datasets] 1 where the species contributes
 *                  (at most 8 AnaPeak species per dataset)
 * Requires gsn_set_data first (for n_datasets). */
int gsn_set_species(gsn_ctx* ctx, int n_species, int n_fine, const double* fine_centres,
                    const double* spectra, const int* kind, const double* shift,
                    const unsigned char* dataset_mask);

/* Parameter map (section 2.2 parameter synchronisation) and pull terms (Eq. LL).
 *   slot_map   [n_datasets][gsn_n_slots(n_species)] global parameter index of
 *              each slot, or -1 for an unused slot (rates of absent species,
 *              peak slots of non-peak species).  A parameter referenced by
 *              several datasets is synchronised; its gradient is the sum.
 *   pull_*     n_pulls Gaussian constraints 1/2 ((theta_p - c)/sigma)^2
 * Requires gsn_set_species first. */
int gsn_set_params(gsn_ctx* ctx, int n_params, const int* slot_map, int n_pulls,
                   const int* pull_param, const double* pull_centre, const double* pull_width);

/* Fixed per-dataset factors of a multivariate fit (section 2.4): a second
 * observable (radial position, pulse shape, ...) splits each histogram into
 * slices, passed to gsn_set_data as datasets of their own; every slice scales
 * the response parameters and takes a fraction of each species' rate.
 *   resp_scale   [n_datasets][5] multipliers of (LY, kB, a, b, c): dataset d
 *                evaluates its response at resp_scale[d][i] * (slot value); > 0,
 *                finite.  NULL: all 1.
 *   rate_factor  [n_datasets][n_species] f_ds >= 0, finite: species s enters
 *                dataset d as eps_d f_ds r_s (on top of the species mask).
 *                NULL: all 1.
 * Call after gsn_set_data and gsn_set_species; n_datasets and n_species must
 * match them.  The factors stay until a later gsn_set_data or gsn_set_species
 * changes the number of datasets or species (then they return to 1).  The
 * gradient is with respect to the unscaled global parameters.
 * Errors: GSN_ERR_ARG (sizes, values), GSN_ERR_STATE (data or species missing). */
int gsn_set_dataset_factors(gsn_ctx* ctx, int n_datasets, int n_species, const double* resp_scale,
                            const double* rate_factor);

/* Monte Carlo template of species s in dataset d (section 3.2: the template
 * fit, where a species' expected visible spectrum comes from simulation rather
 * than from the analytic response).  hist holds n_bins[d] values >= 0 with a
 * positive sum; the library normalises it to unit sum, so r_s counts per unit
 * exposure as for the other kinds.  Species s must be of kind GSN_MC_TEMPLATE;
 * a template species without a histogram in a dataset contributes nothing
 * there; hist = NULL removes it.  Datasets whose species are all templates or
 * peaks need no response slots (slot_map -1), and a fit of templates only runs
 * no response kernel.  Call after gsn_set_species (which clears the templates).
 * Errors: GSN_ERR_ARG, GSN_ERR_STATE. */
int gsn_set_template(gsn_ctx* ctx, int species, int dataset, const double* hist);

/* Secondary observable of a dataset (section 2.4 multivariate fit: the extra
 * likelihood pieces of a second observable, e.g. a pulse-shape or radial
 * variable).  The dataset's energy bins form n_slices contiguous slices; each
 * slice carries a histogram of the second observable in n_sec bins.  Species s
 * contributes to slice q its expected counts N_sq (the sum of its expected
 * energy-bin counts over the slice), spread over the secondary bins by the
 * fixed shape P_sqm; every slice lying inside the dataset's fit window adds
 *     sum_m [mu_qm - n_qm + n_qm ln(n_qm / mu_qm)],  mu_qm = sum_s N_sq P_sqm
 * to the NLL (its events also populate the energy histogram: the pieces are
 * added, not conditioned).
 *   slice_start  [n_slices + 1] ascending energy-bin boundaries in [0, n_bins[d]]:
 *                slice q = bins [slice_start[q], slice_start[q+1])
 *   shapes       [n_species][n_slices][n_sec] >= 0; the library normalises every
 *                (s, q) row to unit sum (a zero row: no contribution); NULL removes
 *                the dataset's secondary observable
 *   counts       [n_slices][n_sec] observed counts for single-point calls (NULL: 0)
 * A toy's counts row (the batch calls and the minimiser) then holds gsn_n_counts
 * values: the energy bins of every dataset, then the secondary bins of every
 * dataset that has them (datasets, slices and secondary bins in ascending order).
 * Call after gsn_set_data and gsn_set_species (which clear it).  Not taken by
 * gsn_eval_grad_noalloc.  Errors: GSN_ERR_ARG, GSN_ERR_STATE. */
int gsn_set_secondary(gsn_ctx* ctx, int dataset, int n_slices, const int* slice_start, int n_sec,
                      const double* shapes, const double* counts);

/* Values in a toy's counts row: sum_d n_bins[d] plus every secondary histogram. */
int gsn_n_counts(gsn_ctx* ctx);

/* NLL at params[n_params] with the counts and windows of gsn_set_data.
 * Keeps the per-species shapes of every response group (section 2.5 value
 * cache, shared with gsn_expected) and recomputes them only when a response
 * parameter (LY, kB, a, b, c, p) changes; rate-only steps skip the response.
 * Errors: GSN_ERR_NONPOSITIVE_MU (nll = +inf), GSN_ERR_NONFINITE. */
int gsn_eval(gsn_ctx* ctx, const double* params, double* nll);

/* NLL and gradient grad[n_params] (hand-written adjoint). */
int gsn_eval_grad(gsn_ctx* ctx, const double* params, double* nll, double* grad);

/* Batched pseudo-experiments: each toy has its own parameters, counts and windows.
 *   params      [n_toys][n_params]
 *   toy_counts  [n_toys][gsn_n_counts(ctx)]: energy bins (datasets concatenated), then any secondary bins
 *   toy_win     [n_toys][n_datasets][2] window [lo, hi) per toy and dataset
 *   nll         [n_toys]
 *   grad        [n_toys][n_params], or NULL for the NLL only
 * Host buffers; the call copies them to the device and back, synchronously.
 * n_toys = 0 is a no-op.  The first failing toy's status is returned; the
 * other toys' results are still written. */
int gsn_eval_grad_batch(gsn_ctx* ctx, int n_toys, const double* params, const double* toy_counts,
                        const int* toy_win, double* nll, double* grad);

/* Same as gsn_eval_grad_batch with device-resident inputs and outputs,
 * enqueued on the context's stream.  status_dev (may be NULL) receives one
 * int per toy (0 or a GSN_ERR_* code).  Asynchronous: the results are ready
 * once the stream is synchronised; argument errors are reported at once. */
int gsn_eval_grad_batch_dev(gsn_ctx* ctx, int n_toys, const double* params_dev,
                            const double* toy_counts_dev, const int* toy_win_dev,
                            double* nll_dev, double* grad_dev, int* status_dev);

/* Batched minimisation of the NLL of every toy (the profile likelihood of
 * section 4.2; the toy Monte Carlo discovery test takes two calls, with the
 * signal rate free and fixed at 0, and q0 = 2 (NLL_fixed - NLL_free)).  Each
 * toy runs its own projected L-BFGS (FP64 state, history of 16 pairs,
 * backtracking Armijo line search) in scaled variables u = x / scale; every
 * iteration is one batched NLL + gradient evaluation (as in
 * gsn_eval_grad_batch_dev, with the context's precision) and one update.
 *   params_dev   [n_toys][n_params] device: start points in, minima out
 *   toy_counts_dev, toy_win_dev   as in gsn_eval_grad_batch_dev
 *   free_mask    [n_params] host: 1 = minimised over, 0 = held at its start value
 *   lo, hi       [n_params] host bounds (NULL: unbounded); rates usually lo = 0
 *   scale        [n_params] host, > 0 (NULL: 1); near 1/sqrt(Fisher) conditions best
 *   max_evals    evaluations per toy (<= 0: 200); gtol: largest projected
 *                scaled gradient component at convergence (< 0: 1e-6 for FP64,
 *                1e-4 for the mixed path, whose NLL carries FP32 rounding); ftol:
 *                relative NLL decrease of an accepted step at convergence (< 0: 1e-10)
 *   nll_dev      [n_toys] device: NLL at the minimum
 *   evals_dev    [n_toys] device or NULL: evaluations used
 *   status_dev   [n_toys] device or NULL: 0 converged, 1 evaluation limit,
 *                2 line search failed (the point returned is the best found),
 *                -4 non-finite NLL at the start point
 * Synchronous.  At most 64 parameters.  The paper has no batched minimiser: it
 * fits toys one after another with MINUIT. */
int gsn_minimize_batch_dev(gsn_ctx* ctx, int n_toys, double* params_dev, const double* toy_counts_dev,
                           const int* toy_win_dev, const unsigned char* free_mask, const double* lo,
                           const double* hi, const double* scale, int max_evals, double gtol, double ftol,
                           double* nll_dev, int* evals_dev, int* status_dev);

/* gsn_minimize_batch_dev with per-toy scales and an optional distance-to-minimum stopping rule.
 *   scale_dev  [n_toys][n_params] device (every free parameter's scale finite and > 0, else that
 *              toy ends with status -1); gsn_window_scales_dev makes such scales for toys fitted
 *              in windows of their own
 *   edm        a toy also converges (status 0) once its estimated distance to the minimum,
 *              -g.d / 2 with d = -H^-1 g the L-BFGS step (the stopping rule of MINUIT's MIGRAD,
 *              the minimiser the paper's fits use), falls below edm (NLL units; <= 0: not used)
 * Otherwise as gsn_minimize_batch_dev. */
int gsn_minimize_batch_scaled_dev(gsn_ctx* ctx, int n_toys, double* params_dev, const double* toy_counts_dev,
                                  const int* toy_win_dev, const unsigned char* free_mask, const double* lo,
                                  const double* hi, const double* scale_dev, int max_evals, double gtol, double ftol,
                                  double edm, double* nll_dev, int* evals_dev, int* status_dev);

/* Batched profile-likelihood fits over rates only (section 4.2: the discovery test fits rates
 * with the detector response held).  With the response parameters fixed, every species' expected
 * counts are a fixed shape times its rate, so a toy's expected counts are linear in the free rates
 * and its NLL is convex in them; each toy is minimised by projected Newton iterations with the
 * exact Hessian sum_i n_i B_i B_i^T / mu_i^2 (B_i the free rates' shapes in bin i, pulls added),
 * backtracking on the exact NLL change, until the Newton decrement g.H^-1.g / 2 (the estimated
 * distance to the minimum) is below tol.  Strongly correlated rates, which slow the L-BFGS of
 * gsn_minimize_batch_dev, cost Newton nothing.  The shapes are computed once per call at the toys'
 * start points (the response parameters and the held rates are taken from params_dev).
 * A free rate whose expected counts inside the toy's window are at most 1e3 exp(-band_cut) of its
 * expected counts over the whole histograms (1e-6 with the mixed default band, 1e-12 with FP64)
 * stays at its start value: it reaches the window only through response tails that the band
 * truncates, and its rate is not determined by the data there.
 *   params_dev   [n_toys][n_params] device: start points in, minima out
 *   toy_counts_dev, toy_win_dev   as in gsn_eval_grad_batch_dev
 *   free_mask    [n_params] host: 1 = minimised over; every free parameter must fill rate slots
 *                only (else GSN_ERR_ARG); at most 48 free rates
 *   lo, hi       [n_params] host bounds (NULL: unbounded); rates usually lo = 0
 *   max_iter     Newton iterations per toy (<= 0: 200: a rate that the window barely constrains
 *                may have to grow by orders of magnitude, about a factor 2 per iteration); tol:
 *                decrement at convergence, NLL units
 *                (<= 0: 1e-8)
 *   nll_dev      [n_toys] device: NLL at the minimum (FP64 sums of the context's expected counts)
 *   iters_dev    [n_toys] device or NULL: iterations used
 *   status_dev   [n_toys] device or NULL: 0 converged, 1 iteration limit, 2 no acceptable step
 *                (the point returned is the best found), -4 non-finite NLL
 * Synchronous.  Contexts with secondary observables are not taken (GSN_ERR_ARG).  The paper fits
 * toys one after another with MINUIT. */
int gsn_fit_rates_batch_dev(gsn_ctx* ctx, int n_toys, double* params_dev, const double* toy_counts_dev,
                            const int* toy_win_dev, const unsigned char* free_mask, const double* lo,
                            const double* hi, int max_iter, double tol, double* nll_dev, int* iters_dev,
                            int* status_dev);

/* Per-toy minimiser scales for fits in windows of the toys' own (section 4.2 toy Monte Carlo with
 * uneven fit ranges).  A toy's window holds part of each species' spectrum, and the rate of a
 * species that lies mostly outside it is less constrained than scales taken from the whole
 * histograms (1/sqrt of the Fisher diagonal at theta0, say) assume; a minimiser conditioned with
 * those reaches its evaluation limit on such toys.  For every toy t:
 *     scale_dev[t][i] = scale[i] * min(max(sqrt(N_i,whole / N_i,window), 1), max_factor)
 * for every parameter i that fills only rate slots, with N_i the expected counts of its species at
 * the toy's parameters (params_dev [n_toys][n_params]) over the whole histograms and inside the
 * toy's windows (toy_win_dev [n_toys][n_datasets][2]); scale_dev[t][i] = scale[i] for the other
 * parameters.  The counts of smeared species use a Gaussian response of each column's mean and
 * variance (a scale needs no better); peaks and templates use their own shapes.
 *   scale       [n_params] host, > 0 (NULL: 1)
 *   max_factor  largest factor (<= 0: 100; otherwise >= 1)
 *   scale_dev   [n_toys][n_params] device output
 * Synchronous.  Not in the paper, whose fits run one toy at a time with MINUIT.
 * Errors: GSN_ERR_ARG, GSN_ERR_STATE, GSN_ERR_CUDA. */
int gsn_window_scales_dev(gsn_ctx* ctx, int n_toys, const double* params_dev, const int* toy_win_dev,
                          const double* scale, double max_factor, double* scale_dev);

/* Expected counts per bin and species of one dataset (the validation quantity
 * of section 3.1): mu_per_species[n_bins[d]][n_species]; columns of species
 * absent from the dataset are zero.  Uses the value cache of gsn_eval, so the
 * datasets of one parameter point cost one response evaluation. */
int gsn_expected(gsn_ctx* ctx, const double* params, int dataset, double* mu_per_species);

/* Stream of the context (cudaStream_t), e.g. to order caller work after it. */
void* gsn_stream(gsn_ctx* ctx);

/* NLL and gradient at one parameter point without allocating device memory.
 * The paper has no counterpart: this entry point serves callers that must not
 * call cudaMalloc while they run -- code inside a stream-ordered region that
 * forbids allocation (a step being captured into a CUDA graph, a real-time
 * loop with a pre-reserved memory budget, an allocator that owns the device).
 * The intermediate buffers of the step (column records, band summaries,
 * partial sums of mu, w = 1 - n/mu, partial gradients) live in one static
 * device array of GSN_NOALLOC_SCRATCH_BYTES that the library reserves on
 * every GPU it is loaded on, until the process exits.
 *   params_dev  [n_params] device pointer
 *   nll_dev     [1] device output; grad_dev [n_params] device output
 *   status_dev  [1] device output (0 or a GSN_ERR_* code of the step), or NULL
 * Counts and windows are those of gsn_set_data.  The context's problem must
 * already be on the device: call gsn_eval or gsn_eval_grad once during set-up
 * (else GSN_ERR_STATE), and the context's device must be the current device
 * (else GSN_ERR_STATE; the call does not switch devices).  The work is split
 * by the untuned occupancy plan, so in the mixed-precision mode the result may
 * differ from gsn_eval_grad's (which may use an autotuned plan) in the last
 * FP32 bits of its partial sums.  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  Problems
 * needing more scratch than the array holds are rejected with GSN_ERR_ARG and
 * a message giving the size needed.  Enqueued on the context's stream without
 * synchronising.  Every call, from any context, uses the same array: calls
 * whose kernels overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  Nothing in the array needs to start
 * at zero; each call overwrites what it reads. */
#define GSN_NOALLOC_SCRATCH_BYTES (16u << 20)
int gsn_eval_grad_noalloc(gsn_ctx* ctx, const double* params_dev, double* nll_dev, double* grad_dev,
                          int* status_dev);

/* Work decomposition of a launch of n_toys toys (n_toys >= 1; grad 0/1: without / with the
 * adjoint): the autotuner's choice once it has run for this (n_toys, grad), else the occupancy
 * heuristic.  out[0] fine-column splits of the forward, out[1] warps per adjoint block,
 * out[2] bin splits of the adjoint, out[3] deviance blocks per toy, out[4] 1 if tuned.
 * Puts the problem on the device if needed.  Errors: GSN_ERR_ARG, GSN_ERR_STATE. */
int gsn_plan_info(gsn_ctx* ctx, int n_toys, int grad, int* out5);

/* ----------------------------------------------------------- tracing ----
 * Per-kernel statistics.  While enabled, each kernel launch of the context is
 * bracketed by CUDA events recorded on the context's stream, and the response
 * kernels count the (bin, fine column) pairs they evaluate.  Not part of the
 * paper's method: measurement support for the roofline of each kernel. */
#define GSN_K_COLUMNS    0   /* column prologue: means, resolution, band, T_dk */
#define GSN_K_FORWARD    1   /* response build + contraction -> mu */
#define GSN_K_DEVIANCE   2   /* FP64 deviance over bin ranges, w = 1 - n/mu */
#define GSN_K_BACKWARD   3   /* adjoint over the band */
#define GSN_K_GRADFINAL  4   /* partial-gradient reduction and slot-map scatter */
#define GSN_K_SPECIES    5   /* per-species contraction (gsn_eval, gsn_expected) */
#define GSN_K_MU         6   /* rate-weighted sum of cached per-species shapes */
#define GSN_K_DEVFINAL   7   /* NLL reduction of the deviance partials, pulls, AnaPeak gradient */
#define GSN_K_COUNT      8

/* enable = 1 resets the statistics and starts recording; 0 stops. */
int gsn_profile(gsn_ctx* ctx, int enable);

/* Statistics of one kernel (GSN_K_*) since the last reset: summed event time
 * [ms], number of launches, evaluated (bin, column) pairs (response kernels;
 * 0 otherwise).  Synchronises the context's stream.  Any output may be NULL. */
int gsn_profile_read(gsn_ctx* ctx, int kernel, double* total_ms, long long* launches,
                     unsigned long long* units);

/* Name of a GSN_K_* kernel class ("" when out of range). */
const char* gsn_kernel_name(int kernel);

/* Throughput probe: a synthetic loop of one instruction class on every SM of
 * `device`, timed with CUDA events; returns operations per second.
 *   GSN_PROBE_FFMA  FP32 fused multiply-adds
 *   GSN_PROBE_EX2   SFU base-2 exponentials
 *   GSN_PROBE_DFMA  FP64 fused multiply-adds
 *   GSN_PROBE_NODE  one mixed-precision quadrature node: 2 FFMA + EX2 + FFMA
 *   GSN_PROBE_EX2_BIAS  not a rate: the mean relative error of the SFU exponential over
 *                   the exponents of a Gaussian profile, weighted by the profile (the
 *                   bias the mixed-precision column normalisation divides out) */
#define GSN_PROBE_FFMA 0
#define GSN_PROBE_EX2  1
#define GSN_PROBE_DFMA 2
#define GSN_PROBE_NODE 3
#define GSN_PROBE_EX2_BIAS 4
int gsn_peak_probe(int device, int which, double* ops_per_second);

#ifdef __cplusplus
}
#endif
#endif /* GSN_H */
