// Internal definitions shared by the host API and the kernels of libgsn.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsn {

constexpr int MAXD = 512;    // datasets (histograms, or slices of histograms along a second observable)
constexpr int MAXS = 64;     // species
constexpr int MAXG = 256;    // response groups
constexpr int MAXGDS = 4;    // datasets sharing one response group

// Gauss-Legendre nodes per bin.  Mixed: 3 linear nodes, 6 log-spaced nodes for
// bins whose lower edge lies below XLOG_F.  FP64: 5 linear, 10 log-spaced below XLOG_D.
constexpr int NGM_F = 6, NG_LIN_F = 3, NG_LOG_F = 6;
constexpr int NGM_D = 10, NG_LIN_D = 5, NG_LOG_D = 10;
constexpr double XLOG_F = 8.0, XLOG_D = 16.0;

// bin classes of the node table
constexpr unsigned char BIN_LIN = 0, BIN_LOG = 1, BIN_ZERO = 2;

constexpr int COLBLK = 256;  // columns per column-kernel block and per band summary
constexpr int NFP = 16;      // fields per column record

// Column record fields.
//  mixed gamma : MUH/MUL double-float mean, A = 1/mu, B = d, C = -1/s,
//                KAPPA = ln d - psi(d), XM = log2 f(mode)/f(mu) (0 for d <= 1), N = density
//                at the mode: the response kernels evaluate log2 f(x)/f(mu) - XM, whose
//                maximum is 0, as the SFU exponential's calibration (a profile peaking at 0)
//                assumes
//  mixed gauss : MUH/MUL, A = 1/sigma, N = 1/(sigma sqrt(2 pi))
//  fp64 gamma  : MUH = mu, A = -d ln s - lgamma(d), B = d-1, C = 1/s,
//                KAPPA = ln s + psi(d), N = 1
//  fp64 gauss  : MUH = mu, A = 1/sigma, N = 1
//  mixed ggamma: MUH/MUL, A = 1/mu, B = L2E A_p, C = L2E kappa_1, KAPPA = p,
//                N = density at the mean, with A_p = (mu/s)^p, kappa_1 = d - 1 - p A_p
//                (log f(x)/f(mu) = kappa_1 L - A_p (e^(pL) - 1 - pL), L = ln(x/mu))
//  fp64 ggamma : MUH = mu, A = ln p - d ln s - lgamma(d/p), B = d-1, C = ln s,
//                KAPPA = p, N = 1
//  all         : DEQ = d E_q / d kB, XMIN/XMAX = band in p.e.,
//                TN0.. = N_k * T_dk of each dataset of the group
enum { F_MUH = 0, F_MUL, F_A, F_B, F_C, F_N, F_KAPPA, F_DEQ, F_XMIN, F_XMAX, F_TN0 };
constexpr int F_XM = F_TN0 + MAXGDS;
static_assert(F_XM < NFP, "column record too small");
// Bin-at-zero record of a column (gamma-family responses, NFZ values, zerobuf): P0 = content of the
// bin starting at 0 over N; P0D/P0S its derivatives (gamma): fp64 dP/dd and s^2 dP/ds, mixed
// (mu/d) dP/dmu|var / N and s^2 dP/dvar|mu / N.  Kept out of the column record, which the response
// kernels stream for every bin, so that the record holds a T_dk for up to MAXGDS datasets.
constexpr int NFZ = 4;
enum { Z_P0 = 0, Z_P0D, Z_P0S };

// Adjoint coefficients of a generalized-gamma column (second record, NFG doubles): the adjoint
// accumulates over the band U = (sum W rho, sum W S1, sum W S2, sum W S3, W at the bin at zero),
// with the node sums S1..S3 of the precision (fp64: f l, f y, f y l with l = ln(x/s), y = (x/s)^p;
// mixed: f L, f Q, f E1 L with L = ln(x/mu), E1 = e^(pL) - 1, Q = E1 - pL), and maps them to the derivatives
// of the NLL with respect to the column's mean, variance and the power: rows G_MU, G_VAR, G_P of
// five coefficients each.
constexpr int NFG = 16;
enum { FG_MU = 0, FG_VAR = 5, FG_P = 10 };

constexpr int NRESP = 6;  // LY, kB, a, b, c, p (the power of the generalized gamma)

// Problem tables, in device memory (uploaded once per problem, read by every kernel).
struct Tables {
    int ds_bins[MAXD], ds_off[MAXD], ds_group[MAXD], ds_in_group[MAXD];
    int ds_npk[MAXD];           // AnaPeak species present in the dataset
    int ds_ntpl[MAXD], ds_tpl0[MAXD];  // Monte Carlo templates of the dataset: count, first global index
    int ds_resp[MAXD];          // the dataset has smeared species (its mu includes the response)
    int g_nds[MAXG], g_ds[MAXG][MAXGDS], g_bins[MAXG], g_edge_off[MAXG], g_node_off[MAXG];
    int g_resp[MAXG][NRESP];    // global parameter of each response slot
    int g_zero[MAXG];           // first edge of the group is 0 (gamma bin-at-zero)
    int g_jlin[MAXG];           // first bin of the group from which every bin is linear
    int g_active[MAXG];         // some dataset of the group has smeared species
    double g_rscale[MAXG][NRESP];  // fixed multipliers of the response parameters (section 2.4 slices)
    int sp_kind[MAXS];
};

// Copy of the first FASTG groups and FASTD datasets of Tables, carried in the kernel parameters
// (constant bank): the prologues of the response kernels read these values before their first
// memory access, and problems of up to 8 datasets then need no device-table round trip.
constexpr int FASTG = 8, FASTD = 8;
struct FastTables {
    int g_nds[FASTG], g_ds[FASTG][MAXGDS], g_bins[FASTG], g_edge_off[FASTG], g_node_off[FASTG];
    int g_jlin[FASTG], g_zero[FASTG], g_active[FASTG], g_resp[FASTG][NRESP];
    double g_rscale[FASTG][NRESP];
    int ds_off[FASTD], ds_bins[FASTD], ds_group[FASTD], ds_resp[FASTD];
    int sp_kind[MAXS];          // complete (the species count is at most MAXS)
};

struct KArgs {
    // problem
    int T, D, S, K, P, NSLOT, G, total_bins, nsplit, n_pulls;
    int res;          // 0 gauss, 1 gamma, 2 generalized gamma with a free power
    int precision;    // 0 fp64, 1 mixed
    double cut;       // band cut on the log-density
    // mixed column normalisation: the SFU exponential's mean relative error b over a response
    // profile is measured on the context's device when the context is created; every mixed value
    // is N_k times a sum of such exponentials, so N_k carries the factor 1 / (1 + b)
    float norm_hi, norm_lo;     // 1 / (sqrt(2 pi) (1 + b)) as an FP32 pair (fmaf(x, hi, x * lo))
    double ex2_scale;           // 1 / (1 + b)
    double s0, s1;    // stopping power model
    int max_nds;                // most datasets in one response group
    int fast;                   // every group and dataset is in the kernel-parameter copy ft
    int response;               // some species passes through the response (else columns, forward
                                // and adjoint are skipped: a pure template fit)
    int ntpl;                   // Monte Carlo templates over all datasets
    const int* tpl_s;           // [ntpl] species of each template (datasets in order)
    const long long* tpl_off;   // [ntpl] offset of its normalised histogram in tpl
    const double* tpl;          // concatenated histograms, n_bins of the template's dataset each
    FastTables ft;
    // device-resident problem arrays
    const Tables* tb;
    const double* rfac;         // [D][S] rate coefficient eps_d f_ds of species s in dataset d (0: absent)
    const double* edges;        // per group, J_g + 1 edges, concatenated
    const float* ntab_f;        // [bin][3][NGM_F]: offset from centre, ln(x/xc), weight
    const float* xc_f;          // [bin] bin centre
    const unsigned char* bclass;// [bin] BIN_LIN / BIN_LOG / BIN_ZERO
    const double* ntab_d;       // [bin][3][NGM_D]: x, ln x, weight
    const float* btab_f;        // [bin][8] linear bins, symmetric 3-node rule: xc, offset, ln(1+offset/xc),
                                // ln(1-offset/xc), centre weight, side weight, -, -
    const double* E;            // fine centres [K]
    const float* E_hi;          // double-float split of E
    const float* E_lo;
    const float* Sf;            // normalised shifted spectra [S][K]
    const float* Sf_lo;         // their FP32 residuals S' - Sf (mixed): a piecewise-constant spectrum
                                // would otherwise carry one rounding error over its whole range
    const double* Sd;
    const int* slot_map;        // [D][NSLOT]
    const int* pull_param;
    const double* pull_c;
    const double* pull_w;
    // per launch
    const double* params;  long long params_stride;   // [T][P]
    const double* counts;  long long counts_stride;   // [T][total_bins]
    const int* win;        long long win_stride;      // [T][D][2]
    // scratch
    void* colbuf;          // [T][G][K][NFP] of Real
    void* zerobuf;         // [T][G][K][NFZ] of Real: bin-at-zero values (gamma-family responses)
    double* colbuf2;       // [T][G][K][NFG]: adjoint coefficients (generalized gamma only)
    void* blkbuf;          // [T][G][nblk][2] of Real: min xmin, max xmax
    double* mubuf;         // [T][nsplit][total_bins]
    void* wbuf;            // [T][total_bins] of Real
    double* partbuf;       // [T][G][nbtask][NPART]
    double* gdirect;       // [T][P]
    int nblk;
    int nbtask, bw_warps, bw_bsplit, NPART;
    int ntile;             // forward tiles per group (max over groups)
    int* segoff;           // [T*G + 1] gamma forward: exclusive prefix of the 64-bin segments of every
                           // (toy, group) window (written by the forward launcher)
    int dev_chunks;        // deviance blocks per toy
    double* devpart;       // [T][dev_chunks][2 + ntpl]: partial deviance sum, status flags,
                           // partial sum_j w_j T_j of every template
    // outputs
    double* nll;
    double* grad;
    int* status;
    int want_grad;
    // per-species path (eval with response cache, expected counts)
    double* Mbuf;          // [T][G][S][J_g max] (toy stride mstride)
    long long mstride;
    int Jmax;
    int sp_first, sp_count;
    double* out_species;   // [J][S] for gsn_expected
    int out_dataset, out_bins;
    // secondary observable (section 2.4 multivariate pieces); nsec = 0: none
    int nsec;              // datasets with a secondary observable
    int Qtot;              // their slices
    int nsecb;             // their secondary bins: a toy's counts row holds total_bins + nsecb values
    const int* sec_ds;     // [nsec] dataset
    const int* sec_nq;     // [nsec] slices
    const int* sec_M;      // [nsec] secondary bins per slice
    const int* sec_q0;     // [nsec] first global slice
    const int* sec_coff;   // [nsec] offset of its secondary counts after the energy bins
    const long long* sec_poff;  // [nsec] offset of its normalised shapes [S][Q][M] in sec_P
    const double* sec_P;
    const int* sq_lo;      // [Qtot] energy-bin range [lo, hi) of every slice in its dataset
    const int* sq_hi;
    const int* sq_sec;     // [Qtot] secondary dataset index of the slice
    const int* sec_slice;  // [total_bins] global slice of every energy bin, -1 outside the slices
    const int* sec_segend; // [group bins, node-table order] first slice edge of any dataset of the
                           // group above the bin (or the group's bin count): batches of the tuned
                           // kernels end there, so a batch lies in one slice of every dataset
    double* secN;          // [T][Qtot][S] unscaled per-species slice sums
    double* secV;          // [T][Qtot][S] dNLL / dN_sq per unit rate coefficient
    double* secW;          // [T][nsecb] 1 - n/mu of every secondary bin
    double* secpart;       // [T][nsec][2 + NSLOT] NLL piece, flags, slot gradient
    void* secU;            // [T][Qtot][K] of Real: adjoint weight of the secondary pieces
    void* secRq;           // [T][Qtot][K] of Real: N_k sum_{j in q} R_jk (NULL: slice sums from Mbuf)
    // statistics: evaluated (bin, column) pairs per kernel class (NULL = off)
    unsigned long long* work;
    // tensor-core per-species contraction
    int tc_nsplit;         // column ranges per bin tile
    double* tc_part;       // [tc_nsplit][G][S][Jmax] partial sums
    int* tc_error;         // set to 1 by a CTA whose bounded wait timed out
};

// batched projected L-BFGS (gsn_fit.cu): per toy t, parameters [t][P]
struct FitArgs {
    int T, P, max_evals;
    double gtol, ftol;          // projected gradient (scaled units), relative NLL decrease
    double edm;                 // estimated distance to the minimum at convergence (<= 0: not used)
    double fnoise;              // relative rounding of the NLL tolerated by the line search
    const unsigned char* free;  // [P] 1 = minimised over
    const double* lo;           // [P] bounds
    const double* hi;
    const double* scale;        // [T][P] (scale_stride = P) or [P] shared (scale_stride = 0): u = x / scale
    long long scale_stride;
    const double* nll;          // evaluation of the trial points XT
    const double* grad;
    const int* estatus;
    double* X;                  // accepted point, its gradient, search direction (scaled), trial point
    double* G;
    double* D;
    double* XT;
    double* S;                  // [T][M][P] curvature pairs (scaled), [T][M] 1 / (s . y)
    double* Y;
    double* RHO;
    double* dstate;             // [T][4]: NLL at X, step, directional derivative
    int* istate;                // [T][8]: state, pairs, newest slot, evaluations, status, restarts,
                                // consecutive small decreases
    int* active;                // toys still running after the update
};
cudaError_t launch_lbfgs(const FitArgs& f, cudaStream_t st);

// Newton fits over rates only (gsn_ratefit.cu); per toy t, bins i of all datasets
constexpr int RF_NFMAX = 48;    // free rates at most
struct RateArgs {
    int nf, max_iter;
    double tol;                 // Newton decrement / 2 at convergence (NLL units)
    double fnoise;              // relative rounding allowance of the Armijo test
    double share_min;           // a free rate with window share at most this stays at its start
    const int* fidx;            // [nf] global index of each free rate
    const int* pfree;           // [P] free index of a parameter, -1 if held
    const double* lo;           // [nf] bounds
    const double* hi;
    double* params;             // [T][P]: start points in, minima out
    double* B;                  // [T][total_bins][nf] summed shapes of the free rates (whole histograms)
    double* C;                  // [T][total_bins] expected counts of the held species
    double* N;                  // [T][total_bins] counts, -1 outside the window
    double* mu;                 // [T][total_bins]
    double* dmu;                // [T][total_bins]
    double* nll;                // [T]
    int* iters;                 // [T] or NULL
    int* status;                // [T] or NULL
};
cudaError_t launch_rate_fit(const KArgs& a, const RateArgs& r, cudaStream_t st);
// per-toy minimiser scales: scale [P] (device) times sqrt(N_whole / N_window) for rate parameters;
// nwin, nfull: [T][D][S] scratch; out [T][P]
cudaError_t launch_window_scales(const KArgs& a, double* nwin, double* nfull, const double* scale, double max_factor,
                                 double* out, cudaStream_t st);
constexpr int FIT_HISTORY = 16;

// launchers (gsn_kernels.cu); return cudaError_t of the launches
cudaError_t launch_columns(const KArgs& a, cudaStream_t st);
cudaError_t launch_forward(const KArgs& a, cudaStream_t st);
cudaError_t launch_deviance(const KArgs& a, cudaStream_t st);
cudaError_t launch_devfinal(const KArgs& a, cudaStream_t st);
cudaError_t launch_backward(const KArgs& a, cudaStream_t st);
cudaError_t launch_gradfinal(const KArgs& a, cudaStream_t st);
cudaError_t launch_species(const KArgs& a, cudaStream_t st);
cudaError_t launch_mu_from_species(const KArgs& a, cudaStream_t st);
cudaError_t launch_expected_out(const KArgs& a, cudaStream_t st);
cudaError_t run_probe(int which, int nsm, double* ops_per_second);
cudaError_t launch_forward_mixed(const KArgs& a, cudaStream_t st);
size_t species_tc_smem_bytes();
cudaError_t launch_species_tc(const KArgs& a, const void* tm_hi, const void* tm_lo, cudaStream_t st);
int make_species_tensor_map(void* out, const float* dev, int rows, int cols_pad);
cudaError_t launch_backward_mixed(const KArgs& a, cudaStream_t st);
cudaError_t launch_secondary(const KArgs& a, cudaStream_t st);
cudaError_t launch_secondary_weights(const KArgs& a, cudaStream_t st);
cudaError_t launch_slice_sums(const KArgs& a, cudaStream_t st);
cudaError_t launch_slice_sums_mixed(const KArgs& a, cudaStream_t st);

constexpr int K_COLUMNS = 0, K_FORWARD = 1, K_DEVIANCE = 2, K_BACKWARD = 3, K_GRADFINAL = 4,
              K_SPECIES = 5, K_MU = 6, K_DEVFINAL = 7, K_COUNT = 8;

}  // namespace gsn
