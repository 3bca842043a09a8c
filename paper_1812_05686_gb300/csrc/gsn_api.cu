// Host side of the C ABI declared in include/gsn.h.
#include "../../include/gsn.h"
#include "gsn_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace gsn;

namespace {

struct Buf {
    void* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct gsn_ctx {
    gsn_options opt{};
    int dev = 0;
    double ex2_bias = 0.0;   // measured mean relative error of the SFU exponential on this device
    Buf wscale_b;            // gsn_window_scales_dev: [T][D][S] counts in the window and whole, scales [P]
    Buf rfit_cfg, rfit_ws;   // gsn_fit_rates_batch_dev: bounds and indices; design rows, mu
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nsm = 1;
    std::string err;
    // problem, host copies
    int D = 0;
    std::vector<int> nb;
    std::vector<std::vector<double>> edges, counts;
    std::vector<double> eps;
    std::vector<int> wlo, whi;
    int S = 0, K = 0;
    std::vector<double> E, Sn;        // fine centres, normalised shifted spectra [S][K]
    std::vector<int> kind;
    std::vector<unsigned char> mask;  // [S][D]
    int P = 0;
    std::vector<int> slot_map;
    std::vector<double> rscale;       // [D][NRESP] response multipliers of each dataset (section 2.4 slices;
                                      // the power of the generalized gamma is not scaled)
    std::vector<double> rfrac;        // [D][S] rate fraction of each species in each dataset
    std::map<std::pair<int, int>, std::vector<double>> tpl;  // (dataset, species) -> normalised template
    // secondary observable per dataset (section 2.4 multivariate pieces)
    struct Sec { std::vector<int> start; int Q = 0, M = 0; std::vector<double> P, counts; };
    std::map<int, Sec> sec;
    std::vector<int> pull_p;
    std::vector<double> pull_c, pull_w;
    bool have_data = false, have_species = false, have_params = false, ready = false;
    // derived
    int G = 0, total_bins = 0, Jmax = 0;
    int n_counts = 0;                 // values per toy counts row: energy bins, then secondary bins
    KArgs base{};
    Tables tab{};                     // host copy of the device problem tables
    // persistent device buffers
    std::vector<Buf> owned;
    // scratch
    Buf secRq_b, secN_b, secV_b, secW_b, secpart_b, secU_b;  // per-toy buffers of the secondary pieces
    Buf segbuf;              // forward segment prefix [T*G + 1]
    Buf zerobuf;             // bin-at-zero records [T][G][K][NFZ] (gamma-family responses)
    Buf colbuf, colbuf2, blkbuf, mubuf, wbuf, partbuf, gdirect, devbuf, params, counts_b, win_b, nll_b, grad_b, status_b, Mbuf,
        outbuf;
    unsigned long long scratch_gen = 0;  // bumped whenever a buffer is (re)allocated
    // launch plans chosen by the autotuner, per (toys in a launch, gradient wanted)
    struct PlanRec { int nsplit, ntile, bw_warps, bw_bsplit, nbtask, dev_chunks; };
    std::map<std::pair<int, int>, PlanRec> tuned;
    // CUDA graphs of recent launch sequences, replayed when the same sequence repeats
    struct GraphRec { std::vector<long long> key; cudaGraphExec_t exec; };
    std::vector<GraphRec> graphs;
    // response cache of gsn_eval (section 2.5: values are reused while the response parameters do not change)
    std::vector<double> cache_key;
    bool cache_valid = false;
    // tracing: events around each launch, summed per kernel class
    bool prof = false;
    struct Pending { int kernel; cudaEvent_t e0, e1; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double prof_ms[K_COUNT] = {0};
    long long prof_n[K_COUNT] = {0};
    Buf work;  // unsigned long long[K_COUNT] on the device
    // tensor-core per-species contraction (mixed): TF32 hi / lo split of S' and their TMA maps
    Buf s_hi, s_lo, tc_part, tc_err;
    // batched minimiser: workspace, configuration, evaluation outputs
    Buf fit_ws, fit_cfg, fit_eval, fit_ist;
    alignas(64) unsigned char tm_hi[128], tm_lo[128];
    bool tc_ready = false;
};

namespace {

int fail(gsn_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define CUDA_TRY(ctx, expr)                                                                    \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(ctx, GSN_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int ensure(gsn_ctx* c, Buf& b, size_t bytes) {
    if (b.n >= bytes && b.p) return GSN_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr; b.n = 0;
    if (bytes == 0) return GSN_OK;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GSN_ERR_NOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    b.n = bytes;
    ++c->scratch_gen;
    return GSN_OK;
}

template <class T>
int upload(gsn_ctx* c, const std::vector<T>& v, const T** out) {
    Buf b;
    int rc = ensure(c, b, std::max<size_t>(v.size(), 1) * sizeof(T));
    if (rc) return rc;
    if (!v.empty()) CUDA_TRY(c, cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    c->owned.push_back(b);
    *out = static_cast<const T*>(b.p);
    return GSN_OK;
}

void free_owned(gsn_ctx* c) {
    for (auto& b : c->owned) cudaFree(b.p);
    c->owned.clear();
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton iteration on P_n)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0); w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2; p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

using Plan = gsn_ctx::PlanRec;

// per-dataset slot of response parameter i (LY, kB, a, b, c, then the generalized-gamma power)
int resp_slot(int S, int i) { return i < 5 ? S + i : GSN_SLOT_P(S); }

// Work decomposition of one launch of T toys.  nsplit: fine-column ranges per forward tile
// (partial mu rows, summed by the deviance); bw_warps x 32: columns per adjoint block;
// bw_bsplit: bin ranges per adjoint column block; dev_chunks: deviance blocks per toy.
Plan plan_with(const gsn_ctx* c, int T, int nsplit, int bw_warps, int bsplit) {
    Plan p{};
    const bool e64g = c->opt.precision == GSN_FP64 && c->opt.resolution == GSN_RES_GAUSS;
    const int bins_per_tile = 8 * (e64g ? 31 : 32);
    p.ntile = (c->Jmax + bins_per_tile - 1) / bins_per_tile;
    p.nsplit = std::max(1, std::min(nsplit, std::max(1, c->K / 256)));
    p.bw_warps = bw_warps;
    p.bw_bsplit = std::max(1, std::min(bsplit, 16));
    const int ncb = (c->K + p.bw_warps * 32 - 1) / (p.bw_warps * 32);
    p.nbtask = ncb * p.bw_bsplit;
    const long long dc = (2LL * c->nsm + T - 1) / T;
    p.dev_chunks = (int)std::max<long long>(1, std::min<long long>(dc, (c->total_bins + 127) / 128));
    return p;
}

// occupancy heuristic: about 4 blocks per SM in the forward and the adjoint
Plan heuristic_plan(const gsn_ctx* c, int T) {
    const long long target = 4LL * c->nsm;
    const Plan p0 = plan_with(c, T, 1, 8, 1);
    const long long fw = (long long)T * c->G * p0.ntile;
    const int nsplit = (int)std::min<long long>((target + fw - 1) / fw, 1 << 20);
    const long long bw = (long long)T * c->G * p0.nbtask;
    const int bsplit = (int)std::min<long long>((target + bw - 1) / bw, 16);
    return plan_with(c, T, nsplit, 8, bsplit);
}

Plan make_plan(const gsn_ctx* c, int T) { return heuristic_plan(c, T); }

void drop_graphs(gsn_ctx* c) {
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

constexpr double INV_SQRT2PI_H = 0.39894228040143267794;  // 1 / sqrt(2 pi)

// Mean relative error of the SFU exponential over a Gaussian profile on device dev (the bias the
// mixed column normalisation divides out), measured once per device and process.  Rounded to
// 1e-13 absolute so that the order of the probe's floating-point atomics cannot change it.
cudaError_t device_ex2_bias(int dev, double& out) {
    static std::mutex mu;
    static double bias[64];
    static bool have[64] = {false};
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!have[dev]) {
        double b = 0.0;
        const cudaError_t e = run_probe(4, 1, &b);
        if (e != cudaSuccess) return e;
        bias[dev] = std::nearbyint(b * 1e13) * 1e-13;
        have[dev] = true;
    }
    out = bias[dev];
    return cudaSuccess;
}

int finalize(gsn_ctx* c) {
    if (c->ready) return GSN_OK;
    if (!c->have_data || !c->have_species || !c->have_params)
        return fail(c, GSN_ERR_STATE, "gsn_set_data, gsn_set_species and gsn_set_params must all be called");
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    c->tuned.clear();
    free_owned(c);
    c->cache_valid = false;
    c->tc_ready = false;
    const bool mixed = c->opt.precision == GSN_MIXED;
    // gamma-family responses (gamma, generalized gamma): support x > 0, the bin at zero and
    // log-spaced nodes for the lowest bins
    const bool gamma = c->opt.resolution != GSN_RES_GAUSS;
    const int NSLOT = gsn_n_slots(c->S);
    KArgs& a = c->base;
    a = KArgs{};
    a.D = c->D; a.S = c->S; a.K = c->K; a.P = c->P; a.NSLOT = NSLOT;
    a.res = c->opt.resolution;
    a.precision = mixed ? 1 : 0;
    a.cut = c->opt.band_cut;
    a.s0 = c->opt.birks_s0; a.s1 = c->opt.birks_s1;
    {
        const double norm = INV_SQRT2PI_H / (1.0 + c->ex2_bias);
        a.norm_hi = (float)norm;
        a.norm_lo = (float)(norm - (double)a.norm_hi);
        a.ex2_scale = 1.0 / (1.0 + c->ex2_bias);
    }
    a.n_pulls = (int)c->pull_p.size();
    if (c->rscale.size() != (size_t)c->D * NRESP) c->rscale.assign((size_t)c->D * NRESP, 1.0);
    if (c->rfrac.size() != (size_t)c->D * c->S) c->rfrac.assign((size_t)c->D * c->S, 1.0);
    Tables& tb = c->tab;
    tb = Tables{};
    // species; rate coefficient eps_d f_ds of every (dataset, species), 0 where absent
    for (int s = 0; s < c->S; ++s) tb.sp_kind[s] = c->kind[s];
    std::vector<double> rfac((size_t)c->D * c->S, 0.0);
    for (int d = 0; d < c->D; ++d)
        for (int s = 0; s < c->S; ++s) {
            if (!c->mask[s * c->D + d]) continue;
            rfac[(size_t)d * c->S + s] = c->eps[d] * c->rfrac[(size_t)d * c->S + s];
            if (c->kind[s] == GSN_ANA_PEAK && rfac[(size_t)d * c->S + s] != 0.0) ++tb.ds_npk[d];
            if (c->kind[s] < GSN_ANA_PEAK && rfac[(size_t)d * c->S + s] != 0.0) tb.ds_resp[d] = 1;
        }
    // Monte Carlo templates, datasets in order: species, offset, normalised histogram
    std::vector<int> tpl_s;
    std::vector<long long> tpl_off;
    std::vector<double> tpl_h;
    for (int d = 0; d < c->D; ++d) {
        tb.ds_tpl0[d] = (int)tpl_s.size();
        for (int s = 0; s < c->S; ++s) {
            const auto it = c->tpl.find(std::make_pair(d, s));
            if (it == c->tpl.end() || rfac[(size_t)d * c->S + s] == 0.0) continue;
            tpl_s.push_back(s);
            tpl_off.push_back((long long)tpl_h.size());
            tpl_h.insert(tpl_h.end(), it->second.begin(), it->second.end());
        }
        tb.ds_ntpl[d] = (int)tpl_s.size() - tb.ds_tpl0[d];
    }
    a.ntpl = (int)tpl_s.size();
    // response groups: identical edges, response slots and response multipliers (at most MAXGDS each)
    c->G = 0;
    int off = 0;
    a.max_nds = 1;
    for (int d = 0; d < c->D; ++d) {
        tb.ds_bins[d] = c->nb[d]; tb.ds_off[d] = off;
        off += c->nb[d];
        int gsel = -1;
        for (int g = 0; g < c->G && gsel < 0; ++g) {
            const int d0 = tb.g_ds[g][0];
            if (tb.g_nds[g] >= MAXGDS || c->edges[d0] != c->edges[d]) continue;
            bool same = true;
            for (int i = 0; i < NRESP; ++i)
                same = same && c->slot_map[d0 * NSLOT + resp_slot(c->S, i)] == c->slot_map[d * NSLOT + resp_slot(c->S, i)] &&
                       c->rscale[d0 * NRESP + i] == c->rscale[d * NRESP + i];
            if (same) gsel = g;
        }
        if (gsel < 0) {
            if (c->G >= MAXG)
                return fail(c, GSN_ERR_ARG, "more than " + std::to_string(MAXG) + " distinct response groups");
            gsel = c->G++;
            tb.g_nds[gsel] = 0;
            for (int i = 0; i < NRESP; ++i) {
                tb.g_resp[gsel][i] = c->slot_map[d * NSLOT + resp_slot(c->S, i)];
                tb.g_rscale[gsel][i] = c->rscale[d * NRESP + i];
            }
        }
        tb.ds_group[d] = gsel;
        tb.ds_in_group[d] = tb.g_nds[gsel];
        tb.g_ds[gsel][tb.g_nds[gsel]++] = d;
        a.max_nds = std::max(a.max_nds, tb.g_nds[gsel]);
    }
    c->total_bins = off;
    a.total_bins = off;
    a.G = c->G;
    a.response = 0;
    for (int g = 0; g < c->G; ++g) {
        for (int i = 0; i < tb.g_nds[g]; ++i) tb.g_active[g] |= tb.ds_resp[tb.g_ds[g][i]];
        a.response |= tb.g_active[g];
    }
    // edges and node tables per group
    std::vector<double> edges_all, ntab_d;
    std::vector<float> ntab_f, xc_f, btab_f;
    std::vector<unsigned char> bcls;
    std::vector<double> gx_lin, gw_lin, gx_log, gw_log;
    const int ng_lin = mixed ? NG_LIN_F : NG_LIN_D, ng_log = mixed ? NG_LOG_F : NG_LOG_D;
    const int NGM = mixed ? NGM_F : NGM_D;
    const double xlog = mixed ? XLOG_F : XLOG_D;
    gauss_legendre(ng_lin, gx_lin, gw_lin);
    gauss_legendre(ng_log, gx_log, gw_log);
    c->Jmax = 0;
    int noff = 0;
    for (int g = 0; g < c->G; ++g) {
        const std::vector<double>& x = c->edges[tb.g_ds[g][0]];
        const int J = (int)x.size() - 1;
        tb.g_bins[g] = J;
        tb.g_edge_off[g] = (int)edges_all.size();
        tb.g_node_off[g] = noff;
        tb.g_zero[g] = (gamma && x[0] == 0.0) ? 1 : 0;
        tb.g_jlin[g] = 0;
        if (gamma)
            while (tb.g_jlin[g] < J && !(x[tb.g_jlin[g]] >= xlog && x[tb.g_jlin[g]] > 0.0)) ++tb.g_jlin[g];
        c->Jmax = std::max(c->Jmax, J);
        edges_all.insert(edges_all.end(), x.begin(), x.end());
        for (int j = 0; j < J; ++j) {
            const double lo = x[j], hi = x[j + 1], xc = 0.5 * (lo + hi);
            double nx[NGM_D] = {0}, nw[NGM_D] = {0};
            unsigned char cls = BIN_LIN;
            int ng = ng_lin;
            if (gamma && lo == 0.0) {
                cls = BIN_ZERO; ng = 0;
            } else if (gamma && lo < xlog) {
                cls = BIN_LOG; ng = ng_log;
                const double ul = std::log(lo), uh = std::log(hi);
                for (int n = 0; n < ng; ++n) {
                    nx[n] = std::exp(0.5 * (ul + uh) + 0.5 * (uh - ul) * gx_log[n]);
                    nw[n] = 0.5 * (uh - ul) * gw_log[n] * nx[n];
                }
            } else {
                for (int n = 0; n < ng; ++n) {
                    nx[n] = xc + 0.5 * (hi - lo) * gx_lin[n];
                    nw[n] = 0.5 * (hi - lo) * gw_lin[n];
                }
            }
            bcls.push_back(cls);
            if (mixed) {
                // symmetric 3-node rule of linear bins: centre and +-offset
                const float xcf = (float)xc;
                const double off = 0.5 * (hi - lo) * std::sqrt(0.6);
                // weights 4/9 h and 5/18 h rounded so that centre + 2 sides = h: independent roundings
                // would bias every bin integral of every column by the same ~3e-8
                const float wside = (float)(0.5 * (hi - lo) * 5.0 / 9.0);
                const float wcen = (float)((hi - lo) - 2.0 * (double)wside);
                float bt[8] = {xcf, (float)(xc + off - (double)xcf), (float)std::log1p(off / xc),
                               (float)std::log1p(-off / xc), wcen, wside, 0.f, 0.f};
                if (cls != BIN_LIN) for (int q = 1; q < 8; ++q) bt[q] = 0.f;
                btab_f.insert(btab_f.end(), bt, bt + 8);
            }
            if (mixed) {
                const float xcf = (float)xc;
                xc_f.push_back(xcf);
                float t[3 * NGM_F] = {0};
                double wsum = 0.0, fsum = 0.0;
                int nmax = 0;
                for (int n = 0; n < ng; ++n) {
                    t[n] = (float)(nx[n] - (double)xcf);
                    t[NGM_F + n] = (float)(nx[n] > 0 ? std::log(nx[n] / (double)xcf) : 0.0);
                    t[2 * NGM_F + n] = (float)nw[n];
                    wsum += nw[n];
                    fsum += (double)t[2 * NGM_F + n];
                    if (nw[n] > nw[nmax]) nmax = n;
                }
                // the largest weight absorbs the rounding residual of the others, so that the FP32
                // weights of a bin sum to its rule's total (independent roundings bias every column)
                if (ng > 0) {
                    const double others = fsum - (double)t[2 * NGM_F + nmax];
                    t[2 * NGM_F + nmax] = (float)(wsum - others);
                }
                ntab_f.insert(ntab_f.end(), t, t + 3 * NGM_F);
            } else {
                double t[3 * NGM_D] = {0};
                for (int n = 0; n < ng; ++n) {
                    t[n] = nx[n];
                    t[NGM_D + n] = nx[n] > 0 ? std::log(nx[n]) : 0.0;
                    t[2 * NGM_D + n] = nw[n];
                }
                ntab_d.insert(ntab_d.end(), t, t + 3 * NGM_D);
            }
            (void)NGM;
        }
        noff += J;
    }
    a.Jmax = c->Jmax;
    // kernel-parameter copy of the first groups and datasets
    a.fast = (c->G <= FASTG && c->D <= FASTD) ? 1 : 0;
    for (int g = 0; g < std::min(c->G, FASTG); ++g) {
        a.ft.g_nds[g] = tb.g_nds[g];
        for (int i = 0; i < MAXGDS; ++i) a.ft.g_ds[g][i] = tb.g_ds[g][i];
        a.ft.g_bins[g] = tb.g_bins[g]; a.ft.g_edge_off[g] = tb.g_edge_off[g]; a.ft.g_node_off[g] = tb.g_node_off[g];
        a.ft.g_jlin[g] = tb.g_jlin[g]; a.ft.g_zero[g] = tb.g_zero[g]; a.ft.g_active[g] = tb.g_active[g];
        for (int i = 0; i < NRESP; ++i) { a.ft.g_resp[g][i] = tb.g_resp[g][i]; a.ft.g_rscale[g][i] = tb.g_rscale[g][i]; }
    }
    for (int s = 0; s < c->S; ++s) a.ft.sp_kind[s] = tb.sp_kind[s];
    for (int d = 0; d < std::min(c->D, FASTD); ++d) {
        a.ft.ds_off[d] = tb.ds_off[d]; a.ft.ds_bins[d] = tb.ds_bins[d]; a.ft.ds_group[d] = tb.ds_group[d];
        a.ft.ds_resp[d] = tb.ds_resp[d];
    }
    int rc;
    {
        const std::vector<Tables> tv(1, tb);
        if ((rc = upload(c, tv, &a.tb))) return rc;
    }
    if ((rc = upload(c, rfac, &a.rfac))) return rc;
    if ((rc = upload(c, tpl_s, &a.tpl_s))) return rc;
    if ((rc = upload(c, tpl_off, &a.tpl_off))) return rc;
    if ((rc = upload(c, tpl_h, &a.tpl))) return rc;
    if ((rc = upload(c, edges_all, &a.edges))) return rc;
    if ((rc = upload(c, bcls, &a.bclass))) return rc;
    if (mixed) {
        if ((rc = upload(c, ntab_f, &a.ntab_f))) return rc;
        if ((rc = upload(c, btab_f, &a.btab_f))) return rc;
        if ((rc = upload(c, xc_f, &a.xc_f))) return rc;
    } else {
        if ((rc = upload(c, ntab_d, &a.ntab_d))) return rc;
    }
    // fine centres and spectra
    std::vector<float> Ehi(c->K), Elo(c->K), Sf(c->Sn.size()), Sflo(c->Sn.size());
    for (int k = 0; k < c->K; ++k) { Ehi[k] = (float)c->E[k]; Elo[k] = (float)(c->E[k] - (double)Ehi[k]); }
    for (size_t i = 0; i < Sf.size(); ++i) { Sf[i] = (float)c->Sn[i]; Sflo[i] = (float)(c->Sn[i] - (double)Sf[i]); }
    if ((rc = upload(c, c->E, &a.E))) return rc;
    if ((rc = upload(c, Ehi, &a.E_hi))) return rc;
    if ((rc = upload(c, Elo, &a.E_lo))) return rc;
    if (mixed) {
        if ((rc = upload(c, Sf, &a.Sf))) return rc;
        if ((rc = upload(c, Sflo, &a.Sf_lo))) return rc;
    }
    else       { if ((rc = upload(c, c->Sn, &a.Sd))) return rc; }
    if ((rc = upload(c, c->slot_map, &a.slot_map))) return rc;
    if ((rc = upload(c, c->pull_p, &a.pull_param))) return rc;
    if ((rc = upload(c, c->pull_c, &a.pull_c))) return rc;
    if ((rc = upload(c, c->pull_w, &a.pull_w))) return rc;
    // default counts and windows (single-point calls)
    // secondary observables: per-dataset and per-slice tables, bin -> slice map
    {
        std::vector<int> sds, snq, sM, sq0, scoff, sqlo, sqhi, sqsec, sslice(c->total_bins, -1);
        std::vector<long long> spoff;
        std::vector<double> sP;
        int Qtot = 0, nb = 0;
        for (const auto& kv : c->sec) {
            const int d = kv.first;
            const gsn_ctx::Sec& x = kv.second;
            const int i = (int)sds.size();
            sds.push_back(d); snq.push_back(x.Q); sM.push_back(x.M); sq0.push_back(Qtot); scoff.push_back(nb);
            spoff.push_back((long long)sP.size());
            sP.insert(sP.end(), x.P.begin(), x.P.end());
            for (int q = 0; q < x.Q; ++q) {
                sqlo.push_back(x.start[q]); sqhi.push_back(x.start[q + 1]); sqsec.push_back(i);
                for (int j = x.start[q]; j < x.start[q + 1]; ++j) sslice[tb.ds_off[d] + j] = Qtot + q;
            }
            Qtot += x.Q;
            nb += x.Q * x.M;
        }
        a.nsec = (int)sds.size(); a.Qtot = Qtot; a.nsecb = nb;
        c->n_counts = c->total_bins + nb;
        if (a.nsec) {
            if ((rc = upload(c, sds, &a.sec_ds))) return rc;
            if ((rc = upload(c, snq, &a.sec_nq))) return rc;
            if ((rc = upload(c, sM, &a.sec_M))) return rc;
            if ((rc = upload(c, sq0, &a.sec_q0))) return rc;
            if ((rc = upload(c, scoff, &a.sec_coff))) return rc;
            if ((rc = upload(c, spoff, &a.sec_poff))) return rc;
            if ((rc = upload(c, sP, &a.sec_P))) return rc;
            if ((rc = upload(c, sqlo, &a.sq_lo))) return rc;
            if ((rc = upload(c, sqhi, &a.sq_hi))) return rc;
            if ((rc = upload(c, sqsec, &a.sq_sec))) return rc;
            if ((rc = upload(c, sslice, &a.sec_slice))) return rc;
            // per group: the next slice edge above every bin (node-table order)
            int nnodes = 0;
            for (int g = 0; g < c->G; ++g) nnodes = std::max(nnodes, tb.g_node_off[g] + tb.g_bins[g]);
            std::vector<int> segend(nnodes, 0);
            for (int g = 0; g < c->G; ++g) {
                const int Jg = tb.g_bins[g];
                std::vector<char> edge(Jg + 1, 0);
                edge[Jg] = 1;
                for (int dd = 0; dd < tb.g_nds[g]; ++dd) {
                    const auto it = c->sec.find(tb.g_ds[g][dd]);
                    if (it == c->sec.end()) continue;
                    for (int e : it->second.start) if (e >= 0 && e <= Jg) edge[e] = 1;
                }
                int nxt = Jg;
                for (int j = Jg - 1; j >= 0; --j) {
                    if (edge[j + 1]) nxt = j + 1;
                    segend[tb.g_node_off[g] + j] = nxt;
                }
            }
            if ((rc = upload(c, segend, &a.sec_segend))) return rc;
        }
    }
    std::vector<double> cnt;
    std::vector<int> win;
    for (int d = 0; d < c->D; ++d) {
        cnt.insert(cnt.end(), c->counts[d].begin(), c->counts[d].end());
        win.push_back(c->wlo[d]); win.push_back(c->whi[d]);
    }
    for (const auto& kv : c->sec) cnt.insert(cnt.end(), kv.second.counts.begin(), kv.second.counts.end());
    const double* dc; const int* dw;
    if ((rc = upload(c, cnt, &dc))) return rc;
    if ((rc = upload(c, win, &dw))) return rc;
    a.counts = dc; a.win = dw;
    a.nblk = (c->K + COLBLK - 1) / COLBLK;
    a.NPART = NRESP + MAXGDS * c->S;
    c->ready = true;
    return GSN_OK;
}

// allocate (or grow) the scratch buffers for T toys under plan p
int reserve(gsn_ctx* c, int T, const Plan& p) {
    const size_t rs = c->opt.precision == GSN_MIXED ? sizeof(float) : sizeof(double);
    const int nblk = (c->K + COLBLK - 1) / COLBLK;
    const int npart = NRESP + MAXGDS * c->S;
    int rc;
    if ((rc = ensure(c, c->colbuf, (size_t)T * c->G * c->K * NFP * rs))) return rc;
    if (c->opt.resolution != GSN_RES_GAUSS &&
        (rc = ensure(c, c->zerobuf, (size_t)T * c->G * c->K * NFZ * rs))) return rc;
    if (c->opt.resolution == GSN_RES_GGAMMA &&
        (rc = ensure(c, c->colbuf2, (size_t)T * c->G * c->K * NFG * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->blkbuf, (size_t)T * c->G * nblk * 2 * rs))) return rc;
    if ((rc = ensure(c, c->segbuf, ((size_t)T * c->G + 1) * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->mubuf, (size_t)T * p.nsplit * c->total_bins * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->wbuf, (size_t)T * c->total_bins * rs))) return rc;
    if ((rc = ensure(c, c->partbuf, (size_t)T * c->G * p.nbtask * npart * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->gdirect, (size_t)T * c->P * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->devbuf, (size_t)T * p.dev_chunks * (2 + c->base.ntpl) * sizeof(double)))) return rc;
    const KArgs& b = c->base;
    if (b.nsec) {
        if ((rc = ensure(c, c->secRq_b, (size_t)T * b.Qtot * c->K * rs))) return rc;
        if ((rc = ensure(c, c->secN_b, (size_t)T * b.Qtot * c->S * sizeof(double)))) return rc;
        if ((rc = ensure(c, c->secV_b, (size_t)T * b.Qtot * c->S * sizeof(double)))) return rc;
        if ((rc = ensure(c, c->secW_b, (size_t)T * b.nsecb * sizeof(double)))) return rc;
        if ((rc = ensure(c, c->secpart_b, (size_t)T * b.nsec * (2 + b.NSLOT) * sizeof(double)))) return rc;
        if ((rc = ensure(c, c->secU_b, (size_t)T * b.Qtot * c->K * rs))) return rc;
    }
    return GSN_OK;
}

// fill the plan and scratch fields of a (buffers reserved for at least T toys under p)
void fill(gsn_ctx* c, int T, const Plan& p, KArgs& a) {
    a.work = nullptr;
    a.T = T;
    a.nsplit = p.nsplit; a.ntile = p.ntile;
    a.bw_warps = p.bw_warps; a.bw_bsplit = p.bw_bsplit; a.nbtask = p.nbtask;
    a.dev_chunks = p.dev_chunks;
    a.colbuf = c->colbuf.p; a.colbuf2 = (double*)c->colbuf2.p; a.blkbuf = c->blkbuf.p; a.mubuf = (double*)c->mubuf.p;
    a.segoff = (int*)c->segbuf.p;
    a.zerobuf = c->opt.resolution != GSN_RES_GAUSS ? c->zerobuf.p : nullptr;
    a.wbuf = c->wbuf.p; a.partbuf = (double*)c->partbuf.p; a.gdirect = (double*)c->gdirect.p;
    a.devpart = (double*)c->devbuf.p;
    if (a.nsec) {
        a.secRq = c->secRq_b.p;
        a.secN = (double*)c->secN_b.p; a.secV = (double*)c->secV_b.p; a.secW = (double*)c->secW_b.p;
        a.secpart = (double*)c->secpart_b.p; a.secU = c->secU_b.p;
        a.sp_first = 0; a.sp_count = c->S;
    }
}

int prepare(gsn_ctx* c, int T, const Plan& p, KArgs& a) {
    int rc;
    if ((rc = reserve(c, T, p))) return rc;
    fill(c, T, p, a);
    return GSN_OK;
}

cudaEvent_t take_event(gsn_ctx* c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// resolve recorded event pairs into the per-kernel sums (synchronises the stream)
int drain_profile(gsn_ctx* c) {
    if (c->pending.empty()) return GSN_OK;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, p.e0, p.e1);
        c->prof_ms[p.kernel] += ms;
        c->prof_n[p.kernel] += 1;
        c->event_pool.push_back(p.e0);
        c->event_pool.push_back(p.e1);
    }
    c->pending.clear();
    return GSN_OK;
}

// launch one kernel class, bracketed by events while tracing is on
template <class F>
int launch(gsn_ctx* c, int kernel, KArgs& a, F fn) {
    a.work = c->prof ? (unsigned long long*)c->work.p : nullptr;
    if (!c->prof) {
        CUDA_TRY(c, fn(a, c->stream));
        return GSN_OK;
    }
    gsn_ctx::Pending p{kernel, take_event(c), take_event(c)};
    CUDA_TRY(c, cudaEventRecord(p.e0, c->stream));
    CUDA_TRY(c, fn(a, c->stream));
    CUDA_TRY(c, cudaEventRecord(p.e1, c->stream));
    c->pending.push_back(p);
    if (c->pending.size() > 4096) return drain_profile(c);
    return GSN_OK;
}

int run_step(gsn_ctx* c, KArgs& a, bool grad) {
    int rc;
    if (a.nsec) {
        // secondary observable: the regular forward for mu, the response's slice sums for the
        // extra pieces, the pieces, then the energy deviance; the adjoint adds the pieces' weights
        if (a.response) {
            if ((rc = launch(c, K_COLUMNS, a, launch_columns))) return rc;
            if ((rc = launch(c, K_FORWARD, a, launch_forward))) return rc;
            if ((rc = launch(c, K_MU, a, launch_slice_sums))) return rc;
        }
        if ((rc = launch(c, K_SPECIES, a, launch_secondary))) return rc;
        if ((rc = launch(c, K_DEVIANCE, a, launch_deviance))) return rc;
        if ((rc = launch(c, K_DEVFINAL, a, launch_devfinal))) return rc;
        if (grad) {
            if (a.response) {
                if ((rc = launch(c, K_BACKWARD, a, launch_secondary_weights))) return rc;
                if ((rc = launch(c, K_BACKWARD, a, launch_backward))) return rc;
            }
            if ((rc = launch(c, K_GRADFINAL, a, launch_gradfinal))) return rc;
        }
        return GSN_OK;
    }
    if (a.response) {  // a fit of templates and peaks only has no response to build
        if ((rc = launch(c, K_COLUMNS, a, launch_columns))) return rc;
        if ((rc = launch(c, K_FORWARD, a, launch_forward))) return rc;
    }
    if ((rc = launch(c, K_DEVIANCE, a, launch_deviance))) return rc;
    if ((rc = launch(c, K_DEVFINAL, a, launch_devfinal))) return rc;
    if (grad) {
        if (a.response && (rc = launch(c, K_BACKWARD, a, launch_backward))) return rc;
        if ((rc = launch(c, K_GRADFINAL, a, launch_gradfinal))) return rc;
    }
    return GSN_OK;
}

bool stream_capturing(gsn_ctx* c) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) { cudaGetLastError(); return false; }
    return cs != cudaStreamCaptureStatusNone;
}

// best of `reps` runs of a launch sequence on the context's stream [ms]
template <class F>
int time_best(gsn_ctx* c, int reps, F body, float& best) {
    cudaEvent_t e0 = take_event(c), e1 = take_event(c);
    cudaError_t e = cudaSuccess;
    best = 3.0e38f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaEventRecord(e0, c->stream);
        if (e == cudaSuccess) e = body();
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) best = std::min(best, ms);
    }
    c->event_pool.push_back(e0);
    c->event_pool.push_back(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GSN_ERR_CUDA, std::string("autotuner: ") + cudaGetErrorString(e));
    }
    return GSN_OK;
}

// Plan of a launch of T toys.  With autotuning on, the first launch of each (T, gradient) pair
// whose heuristic plan splits the work times candidate decompositions on the caller's own
// inputs (a holds them and the outputs) and keeps the fastest.  The candidates differ only in
// how the sums are split, so each computes the same quantities in another fixed order.
int choose_plan(gsn_ctx* c, int T, KArgs a, bool grad, Plan& out) {
    const auto key = std::make_pair(T, grad ? 1 : 0);
    const auto it = c->tuned.find(key);
    if (it != c->tuned.end()) { out = it->second; return GSN_OK; }
    const Plan h = heuristic_plan(c, T);
    out = h;
    if (stream_capturing(c)) return GSN_OK;  // no timing inside a caller's capture
    if (!c->opt.autotune || !c->base.response || (h.nsplit == 1 && h.bw_bsplit == 1)) { c->tuned[key] = h; return GSN_OK; }
    const cudaStream_t st = c->stream;
    int rc;
    if ((rc = prepare(c, T, h, a))) return rc;
    CUDA_TRY(c, launch_columns(a, st));  // the column prologue does not depend on the plan
    auto fwd = [&]() {
        cudaError_t e = launch_forward(a, st);
        if (e == cudaSuccess) e = launch_deviance(a, st);
        if (e == cudaSuccess) e = launch_devfinal(a, st);
        return e;
    };
    Plan best = h;
    float tbest = 3.0e38f;
    int last = -1;
    for (int ns : {1, h.nsplit / 4, h.nsplit / 2, h.nsplit, 2 * h.nsplit}) {
        const Plan p = plan_with(c, T, std::max(ns, 1), h.bw_warps, h.bw_bsplit);
        if (p.nsplit == last) continue;
        last = p.nsplit;
        if ((rc = prepare(c, T, p, a))) return rc;
        float ms;
        if ((rc = time_best(c, 3, fwd, ms))) return rc;
        if (ms < tbest) { tbest = ms; best = p; }
    }
    if (grad) {
        if ((rc = prepare(c, T, best, a))) return rc;
        CUDA_TRY(c, fwd());  // mu and w for the adjoint candidates
        auto bwd = [&]() {
            cudaError_t e = launch_backward(a, st);
            if (e == cudaSuccess) e = launch_gradfinal(a, st);
            return e;
        };
        const Plan f = best;
        tbest = 3.0e38f;
        for (int wp : {4, 8})
            for (int bs : {1, 2, 4, 8, 16}) {
                const Plan p = plan_with(c, T, f.nsplit, wp, bs);
                if ((rc = prepare(c, T, p, a))) return rc;
                float ms;
                if ((rc = time_best(c, 3, bwd, ms))) return rc;
                if (ms < tbest) { tbest = ms; best = p; }
            }
    }
    c->tuned[key] = best;
    out = best;
    return GSN_OK;
}

// Run a launch sequence, through a CUDA graph when graphs are on: the first call with a given
// key captures the sequence, later calls with the same key replay it.  The key holds every
// pointer and size the sequence bakes in, plus the scratch generation (a reallocation changes it).
template <class F>
int replay(gsn_ctx* c, std::vector<long long> key, F body) {
    if (!c->opt.use_graphs || c->prof || stream_capturing(c)) return body();
    key.push_back((long long)c->scratch_gen);
    for (auto& g : c->graphs)
        if (g.key == key) {
            CUDA_TRY(c, cudaGraphLaunch(g.exec, c->stream));
            return GSN_OK;
        }
    CUDA_TRY(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int rc = body();
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc ? rc : fail(c, GSN_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GSN_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
    }
    if (c->graphs.size() >= 8) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({key, exec});
    CUDA_TRY(c, cudaGraphLaunch(exec, c->stream));
    return GSN_OK;
}

int status_message(gsn_ctx* c, int st, int toy) {
    if (st == 0) return GSN_OK;
    char buf[160];
    if (st == GSN_ERR_NONPOSITIVE_MU)
        snprintf(buf, sizeof buf, "toy %d: expected counts <= 0 in a bin with observed counts", toy);
    else
        snprintf(buf, sizeof buf, "toy %d: non-finite expected counts, NLL or gradient", toy);
    return fail(c, st, buf);
}

int check_params_host(gsn_ctx* c, const double* params) {
    if (!params) return fail(c, GSN_ERR_ARG, "params is NULL");
    for (int p = 0; p < c->P; ++p)
        if (!std::isfinite(params[p])) return fail(c, GSN_ERR_NONFINITE, "parameter " + std::to_string(p) + " is not finite");
    return GSN_OK;
}

// batched step on device pointers; T toys, chunked by max_toys_per_launch
int batch_device(gsn_ctx* c, int n_toys, const double* params, const double* counts, const int* win,
                 double* nll, double* grad, int* status) {
    int rc;
    if ((rc = finalize(c))) return rc;
    // toys per launch: the option, the grid limit of the forward (toys x groups <= 65535) and a
    // 32 GiB bound on the column records (16 words per toy, group and fine column)
    const size_t rec = (size_t)c->G * c->K * NFP * (c->opt.precision == GSN_MIXED ? sizeof(float) : sizeof(double));
    const long long mem_cap = std::max<long long>(1, (long long)((size_t)32 << 30) / (long long)std::max<size_t>(rec, 1));
    const int chunk = (int)std::max<long long>(1, std::min<long long>({(long long)c->opt.max_toys_per_launch,
                                                                        65535LL / std::max(1, c->G), mem_cap}));
    const bool g = grad != nullptr;
    std::vector<KArgs> args;
    std::vector<Plan> plans;
    std::vector<int> Ts;
    for (int t0 = 0; t0 < n_toys; t0 += chunk) {
        const int T = std::min(chunk, n_toys - t0);
        KArgs a = c->base;
        a.params = params + (size_t)t0 * c->P; a.params_stride = c->P;
        a.counts = counts + (size_t)t0 * c->n_counts; a.counts_stride = c->n_counts;
        a.win = win + (size_t)t0 * c->D * 2; a.win_stride = 2 * c->D;
        a.nll = nll + t0;
        a.grad = grad ? grad + (size_t)t0 * c->P : nullptr;
        a.status = status ? status + t0 : nullptr;
        a.want_grad = g ? 1 : 0;
        Plan p;
        if ((rc = choose_plan(c, T, a, g, p))) return rc;
        args.push_back(a); plans.push_back(p); Ts.push_back(T);
    }
    // every buffer is sized before any launch is recorded, so a captured graph sees final pointers
    for (size_t i = 0; i < args.size(); ++i)
        if ((rc = reserve(c, Ts[i], plans[i]))) return rc;
    std::vector<long long> key = {1, n_toys, chunk, g ? 1 : 0, (long long)params, (long long)counts, (long long)win,
                                  (long long)nll, (long long)grad, (long long)status};
    for (size_t i = 0; i < args.size(); ++i) {
        fill(c, Ts[i], plans[i], args[i]);
        key.insert(key.end(), {plans[i].nsplit, plans[i].bw_warps, plans[i].bw_bsplit, plans[i].dev_chunks});
    }
    return replay(c, key, [&]() {
        for (auto& a : args) {
            const int r = run_step(c, a, g);
            if (r) return r;
        }
        return (int)GSN_OK;
    });
}

}  // namespace

// ======================================================================= API
extern "C" {

int gsn_default_options(gsn_options* o) {
    if (!o) return GSN_ERR_ARG;
    std::memset(o, 0, sizeof *o);
    o->precision = GSN_FP64;
    o->resolution = GSN_RES_GAUSS;
    o->band_cut = 0.0;
    o->birks_s0 = 1.55;
    o->birks_s1 = 0.155;
    o->device = 0;
    o->stream = nullptr;
    o->max_toys_per_launch = 4096;
    o->use_graphs = 1;
    o->autotune = 1;
    return GSN_OK;
}

int gsn_n_slots(int n_species) { return 3 * n_species + 6; }

int gsn_create(gsn_ctx** out, const gsn_options* opt) {
    if (!out) return GSN_ERR_ARG;
    *out = nullptr;
    gsn_ctx* c = new gsn_ctx();
    if (opt) c->opt = *opt; else gsn_default_options(&c->opt);
    gsn_options& o = c->opt;
    if (o.precision != GSN_FP64 && o.precision != GSN_MIXED) { delete c; return GSN_ERR_ARG; }
    if (o.resolution != GSN_RES_GAUSS && o.resolution != GSN_RES_GAMMA && o.resolution != GSN_RES_GGAMMA) {
        delete c;
        return GSN_ERR_ARG;
    }
    if (!(o.band_cut > 0)) o.band_cut = o.precision == GSN_FP64 ? 34.5 : 20.7;
    if (!(o.birks_s0 > 0)) o.birks_s0 = 1.55;
    if (o.birks_s1 < 0) o.birks_s1 = 0.155;
    if (o.max_toys_per_launch <= 0) o.max_toys_per_launch = 4096;
    o.max_toys_per_launch = std::min(o.max_toys_per_launch, 65535);
    c->dev = o.device;
    if (cudaSetDevice(c->dev) != cudaSuccess) { cudaGetLastError(); delete c; return GSN_ERR_CUDA; }
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return GSN_ERR_CUDA; }
        c->own_stream = true;
    }
    cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev);
    if (c->nsm <= 0) c->nsm = 1;
    if (o.precision == GSN_MIXED && device_ex2_bias(c->dev, c->ex2_bias) != cudaSuccess) {
        cudaGetLastError();
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return GSN_ERR_CUDA;
    }
    *out = c;
    return GSN_OK;
}

void gsn_destroy(gsn_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    free_owned(c);
    for (Buf* b : {&c->fit_ws, &c->fit_cfg, &c->fit_eval, &c->fit_ist, &c->wscale_b, &c->rfit_cfg, &c->rfit_ws})
        if (b->p) cudaFree(b->p);
    for (Buf* b : {&c->secRq_b, &c->secN_b, &c->secV_b, &c->secW_b, &c->secpart_b, &c->secU_b,
                   &c->segbuf, &c->zerobuf, &c->colbuf, &c->colbuf2, &c->blkbuf, &c->mubuf, &c->wbuf, &c->partbuf, &c->gdirect, &c->devbuf, &c->params, &c->counts_b,
                   &c->win_b, &c->nll_b, &c->grad_b, &c->status_b, &c->Mbuf, &c->outbuf, &c->s_hi, &c->s_lo,
                   &c->tc_part, &c->tc_err})
        if (b->p) cudaFree(b->p);
    if (c->work.p) cudaFree(c->work.p);
    for (auto& p : c->pending) { c->event_pool.push_back(p.e0); c->event_pool.push_back(p.e1); }
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int gsn_profile(gsn_ctx* c, int enable) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = drain_profile(c))) return rc;
    if (enable) {
        if ((rc = ensure(c, c->work, K_COUNT * sizeof(unsigned long long)))) return rc;
        CUDA_TRY(c, cudaMemsetAsync(c->work.p, 0, K_COUNT * sizeof(unsigned long long), c->stream));
        for (int i = 0; i < K_COUNT; ++i) { c->prof_ms[i] = 0.0; c->prof_n[i] = 0; }
    }
    c->prof = enable != 0;
    return GSN_OK;
}

int gsn_profile_read(gsn_ctx* c, int kernel, double* total_ms, long long* launches, unsigned long long* units) {
    if (!c || kernel < 0 || kernel >= K_COUNT) return GSN_ERR_ARG;
    int rc;
    if ((rc = drain_profile(c))) return rc;
    unsigned long long w[K_COUNT] = {0};
    if (c->work.p) {
        CUDA_TRY(c, cudaMemcpyAsync(w, c->work.p, sizeof w, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    if (total_ms) *total_ms = c->prof_ms[kernel];
    if (launches) *launches = c->prof_n[kernel];
    if (units) *units = w[kernel];
    return GSN_OK;
}

int gsn_plan_info(gsn_ctx* c, int n_toys, int grad, int* out) {
    if (!c) return GSN_ERR_ARG;
    if (n_toys < 1 || !out) return fail(c, GSN_ERR_ARG, "n_toys must be >= 1 and out non-NULL");
    int rc;
    if ((rc = finalize(c))) return rc;
    const auto it = c->tuned.find(std::make_pair(n_toys, grad ? 1 : 0));
    const bool tuned = it != c->tuned.end();
    const Plan p = tuned ? it->second : heuristic_plan(c, n_toys);
    out[0] = p.nsplit; out[1] = p.bw_warps; out[2] = p.bw_bsplit; out[3] = p.dev_chunks;
    out[4] = tuned && c->opt.autotune ? 1 : 0;
    return GSN_OK;
}

const char* gsn_kernel_name(int kernel) {
    static const char* names[K_COUNT] = {"columns", "forward", "deviance", "backward", "gradfinal", "species", "mu",
                                         "devfinal"};
    return (kernel >= 0 && kernel < K_COUNT) ? names[kernel] : "";
}

int gsn_peak_probe(int device, int which, double* ops) {
    if (!ops || which < 0 || which > 4) return GSN_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return GSN_ERR_CUDA; }
    int nsm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    if (run_probe(which, nsm, ops) != cudaSuccess) { cudaGetLastError(); return GSN_ERR_CUDA; }
    return GSN_OK;
}

const char* gsn_last_error(const gsn_ctx* c) {
    if (!c) return "no context";
    return c->err.c_str();
}

void* gsn_stream(gsn_ctx* c) { return c ? (void*)c->stream : nullptr; }

int gsn_set_data(gsn_ctx* c, int n_datasets, const int* n_bins, const double* const* bin_edges,
                 const double* const* counts, const double* exposures, const int* win_lo, const int* win_hi) {
    if (!c) return GSN_ERR_ARG;
    if (n_datasets < 1 || n_datasets > GSN_MAX_DATASETS)
        return fail(c, GSN_ERR_ARG, "n_datasets must be in 1.." + std::to_string(GSN_MAX_DATASETS));
    if (!n_bins || !bin_edges || !counts || !exposures || !win_lo || !win_hi) return fail(c, GSN_ERR_ARG, "NULL argument");
    std::vector<int> nb(n_datasets);
    std::vector<std::vector<double>> ed(n_datasets), cn(n_datasets);
    std::vector<double> ex(n_datasets);
    std::vector<int> lo(n_datasets), hi(n_datasets);
    for (int d = 0; d < n_datasets; ++d) {
        if (n_bins[d] < 1) return fail(c, GSN_ERR_ARG, "n_bins must be >= 1");
        if (!bin_edges[d] || !counts[d]) return fail(c, GSN_ERR_ARG, "NULL edges or counts");
        nb[d] = n_bins[d];
        ed[d].assign(bin_edges[d], bin_edges[d] + n_bins[d] + 1);
        cn[d].assign(counts[d], counts[d] + n_bins[d]);
        for (int j = 0; j < n_bins[d]; ++j) {
            if (!(ed[d][j + 1] > ed[d][j]) || !std::isfinite(ed[d][j + 1]) || !std::isfinite(ed[d][j]))
                return fail(c, GSN_ERR_ARG, "bin edges must be finite and strictly ascending");
            if (!(cn[d][j] >= 0.0) || !std::isfinite(cn[d][j])) return fail(c, GSN_ERR_ARG, "counts must be finite and >= 0");
        }
        if (!(exposures[d] > 0.0) || !std::isfinite(exposures[d])) return fail(c, GSN_ERR_ARG, "exposures must be > 0");
        ex[d] = exposures[d];
        if (win_lo[d] < 0 || win_hi[d] > n_bins[d] || win_lo[d] > win_hi[d])
            return fail(c, GSN_ERR_ARG, "window must satisfy 0 <= lo <= hi <= n_bins");
        lo[d] = win_lo[d]; hi[d] = win_hi[d];
    }
    if (c->have_species && n_datasets != c->D) c->have_species = c->have_params = false;
    if (n_datasets != c->D) { c->rscale.clear(); c->rfrac.clear(); }
    if (n_datasets != c->D || nb != c->nb) { c->tpl.clear(); c->sec.clear(); }
    c->D = n_datasets; c->nb = nb; c->edges = ed; c->counts = cn; c->eps = ex; c->wlo = lo; c->whi = hi;
    c->have_data = true;
    c->ready = false;
    return GSN_OK;
}

int gsn_set_species(gsn_ctx* c, int n_species, int n_fine, const double* fine_centres, const double* spectra,
                    const int* kind, const double* shift, const unsigned char* dataset_mask) {
    if (!c) return GSN_ERR_ARG;
    if (!c->have_data) return fail(c, GSN_ERR_STATE, "gsn_set_data must come first");
    if (n_species < 1 || n_species > GSN_MAX_SPECIES) return fail(c, GSN_ERR_ARG, "n_species must be in 1..64");
    if (n_fine < 2) return fail(c, GSN_ERR_ARG, "n_fine must be >= 2");
    if (!fine_centres || !spectra || !kind || !dataset_mask) return fail(c, GSN_ERR_ARG, "NULL argument");
    std::vector<double> E(fine_centres, fine_centres + n_fine);
    for (int k = 0; k < n_fine; ++k) {
        if (!(E[k] > 0.0) || !std::isfinite(E[k])) return fail(c, GSN_ERR_ARG, "fine centres must be finite and > 0");
        if (k && !(E[k] > E[k - 1])) return fail(c, GSN_ERR_ARG, "fine centres must be strictly ascending");
    }
    const double dE = (E[n_fine - 1] - E[0]) / (n_fine - 1);
    std::vector<double> Sn((size_t)n_species * n_fine, 0.0);
    std::vector<int> kd(kind, kind + n_species);
    for (int s = 0; s < n_species; ++s) {
        if (kd[s] < GSN_ANA || kd[s] > GSN_MC_TEMPLATE) return fail(c, GSN_ERR_ARG, "unknown species kind");
        if (kd[s] == GSN_ANA_PEAK || kd[s] == GSN_MC_TEMPLATE) continue;  // rows not used
        double tot = 0.0;
        for (int k = 0; k < n_fine; ++k) {
            const double v = spectra[(size_t)s * n_fine + k];
            if (!(v >= 0.0) || !std::isfinite(v)) return fail(c, GSN_ERR_ARG, "spectra must be finite and >= 0");
            tot += v;
        }
        long n = 0;
        if (kd[s] == GSN_ANA_SHIFT && shift) {
            for (int k = 1; k < n_fine; ++k)
                if (std::fabs((E[k] - E[k - 1]) - dE) > 1e-9 * dE)
                    return fail(c, GSN_ERR_ARG, "AnaShift needs uniformly spaced fine centres");
            n = (long)std::floor(shift[s] / dE + 0.5);
        }
        if (tot <= 0.0) continue;
        for (int k = 0; k < n_fine; ++k) {
            const long src = (long)k - n;
            if (src >= 0 && src < n_fine) Sn[(size_t)s * n_fine + k] = spectra[(size_t)s * n_fine + src] / tot;
        }
    }
    for (int d = 0; d < c->D; ++d) {
        int np = 0;
        for (int s = 0; s < n_species; ++s) np += (kd[s] == GSN_ANA_PEAK && dataset_mask[(size_t)s * c->D + d]) ? 1 : 0;
        if (np > 8) return fail(c, GSN_ERR_ARG, "at most 8 AnaPeak species per dataset");
    }
    if (n_species != c->S) c->rfrac.clear();
    c->tpl.clear();
    c->sec.clear();
    c->S = n_species; c->K = n_fine; c->E = E; c->Sn = Sn; c->kind = kd;
    c->mask.assign(dataset_mask, dataset_mask + (size_t)n_species * c->D);
    c->have_species = true;
    c->have_params = false;
    c->ready = false;
    return GSN_OK;
}

int gsn_set_params(gsn_ctx* c, int n_params, const int* slot_map, int n_pulls, const int* pull_param,
                   const double* pull_centre, const double* pull_width) {
    if (!c) return GSN_ERR_ARG;
    if (!c->have_species) return fail(c, GSN_ERR_STATE, "gsn_set_species must come first");
    if (n_params < 1 || !slot_map) return fail(c, GSN_ERR_ARG, "n_params must be >= 1 and slot_map non-NULL");
    const int NS = gsn_n_slots(c->S);
    std::vector<int> sm(slot_map, slot_map + (size_t)c->D * NS);
    for (int d = 0; d < c->D; ++d) {
        for (int i = 0; i < NS; ++i)
            if (sm[d * NS + i] < -1 || sm[d * NS + i] >= n_params) return fail(c, GSN_ERR_ARG, "slot_map entry out of range");
        bool smeared = false;
        for (int s = 0; s < c->S; ++s) smeared = smeared || (c->kind[s] < GSN_ANA_PEAK && c->mask[s * c->D + d]);
        for (int i = 0; i < 5 && smeared; ++i)
            if (sm[d * NS + c->S + i] < 0)
                return fail(c, GSN_ERR_ARG, "response slots (LY, kB, a, b, c) of datasets with smeared species must be mapped");
        if (smeared && c->opt.resolution == GSN_RES_GGAMMA && sm[d * NS + GSN_SLOT_P(c->S)] < 0)
            return fail(c, GSN_ERR_ARG, "the power slot of datasets with smeared species must be mapped (generalized gamma)");
        for (int s = 0; s < c->S; ++s)
            if (c->kind[s] == GSN_ANA_PEAK && c->mask[s * c->D + d] &&
                (sm[d * NS + GSN_SLOT_M(c->S, s)] < 0 || sm[d * NS + GSN_SLOT_W(c->S, s)] < 0))
                return fail(c, GSN_ERR_ARG, "AnaPeak species need mapped position and width slots");
    }
    if (n_pulls < 0 || (n_pulls > 0 && (!pull_param || !pull_centre || !pull_width)))
        return fail(c, GSN_ERR_ARG, "bad pull arguments");
    std::vector<int> pp(pull_param, pull_param + n_pulls);
    std::vector<double> pc(pull_centre, pull_centre + n_pulls), pw(pull_width, pull_width + n_pulls);
    for (int i = 0; i < n_pulls; ++i)
        if (pp[i] < 0 || pp[i] >= n_params || !(pw[i] > 0)) return fail(c, GSN_ERR_ARG, "bad pull term");
    c->P = n_params; c->slot_map = sm; c->pull_p = pp; c->pull_c = pc; c->pull_w = pw;
    c->have_params = true;
    c->ready = false;
    return GSN_OK;
}

int gsn_set_secondary(gsn_ctx* c, int dataset, int n_slices, const int* slice_start, int n_sec,
                      const double* shapes, const double* counts) {
    if (!c) return GSN_ERR_ARG;
    if (!c->have_data || !c->have_species)
        return fail(c, GSN_ERR_STATE, "gsn_set_data and gsn_set_species must come before a secondary observable");
    if (dataset < 0 || dataset >= c->D) return fail(c, GSN_ERR_ARG, "dataset out of range");
    c->ready = false;
    if (!shapes) { c->sec.erase(dataset); return GSN_OK; }
    if (n_slices < 1 || n_sec < 1 || !slice_start) return fail(c, GSN_ERR_ARG, "n_slices and n_sec must be >= 1");
    gsn_ctx::Sec x;
    x.Q = n_slices; x.M = n_sec;
    x.start.assign(slice_start, slice_start + n_slices + 1);
    for (int q = 0; q <= n_slices; ++q)
        if (x.start[q] < 0 || x.start[q] > c->nb[dataset] || (q && x.start[q] < x.start[q - 1]))
            return fail(c, GSN_ERR_ARG, "slice_start must ascend within the dataset's bins");
    const size_t nP = (size_t)c->S * n_slices * n_sec;
    x.P.assign(shapes, shapes + nP);
    for (int sp = 0; sp < c->S; ++sp)
        for (int q = 0; q < n_slices; ++q) {
            double* row = x.P.data() + ((size_t)sp * n_slices + q) * n_sec;
            double tot = 0.0;
            for (int m = 0; m < n_sec; ++m) {
                if (!(row[m] >= 0.0) || !std::isfinite(row[m])) return fail(c, GSN_ERR_ARG, "shapes must be finite and >= 0");
                tot += row[m];
            }
            for (int m = 0; m < n_sec; ++m) row[m] = tot > 0.0 ? row[m] / tot : 0.0;
        }
    x.counts.assign((size_t)n_slices * n_sec, 0.0);
    if (counts)
        for (size_t i = 0; i < x.counts.size(); ++i) {
            if (!(counts[i] >= 0.0) || !std::isfinite(counts[i])) return fail(c, GSN_ERR_ARG, "counts must be finite and >= 0");
            x.counts[i] = counts[i];
        }
    c->sec[dataset] = x;
    return GSN_OK;
}

int gsn_n_counts(gsn_ctx* c) {
    if (!c) return GSN_ERR_ARG;
    int n = 0;
    for (int d = 0; d < c->D; ++d) n += c->nb[d];
    for (const auto& kv : c->sec) n += kv.second.Q * kv.second.M;
    return n;
}

int gsn_set_template(gsn_ctx* c, int species, int dataset, const double* hist) {
    if (!c) return GSN_ERR_ARG;
    if (!c->have_data || !c->have_species)
        return fail(c, GSN_ERR_STATE, "gsn_set_data and gsn_set_species must come before the templates");
    if (species < 0 || species >= c->S || dataset < 0 || dataset >= c->D)
        return fail(c, GSN_ERR_ARG, "species or dataset out of range");
    if (c->kind[species] != GSN_MC_TEMPLATE) return fail(c, GSN_ERR_ARG, "the species is not of kind GSN_MC_TEMPLATE");
    const auto key = std::make_pair(dataset, species);
    c->ready = false;
    if (!hist) { c->tpl.erase(key); return GSN_OK; }
    const int J = c->nb[dataset];
    std::vector<double> h(hist, hist + J);
    double tot = 0.0;
    for (double v : h) {
        if (!(v >= 0.0) || !std::isfinite(v)) return fail(c, GSN_ERR_ARG, "template values must be finite and >= 0");
        tot += v;
    }
    if (!(tot > 0.0)) return fail(c, GSN_ERR_ARG, "a template must have a positive sum");
    for (double& v : h) v /= tot;
    c->tpl[key] = h;
    return GSN_OK;
}

int gsn_set_dataset_factors(gsn_ctx* c, int n_datasets, int n_species, const double* resp_scale,
                            const double* rate_factor) {
    if (!c) return GSN_ERR_ARG;
    if (!c->have_data || !c->have_species)
        return fail(c, GSN_ERR_STATE, "gsn_set_data and gsn_set_species must come before the dataset factors");
    if (n_datasets != c->D || n_species != c->S)
        return fail(c, GSN_ERR_ARG, "n_datasets / n_species differ from gsn_set_data / gsn_set_species");
    // the caller's [D][5] multipliers of (LY, kB, a, b, c); the power slot keeps 1
    std::vector<double> rs((size_t)c->D * NRESP, 1.0), rf((size_t)c->D * c->S, 1.0);
    if (resp_scale) {
        for (int d = 0; d < c->D; ++d)
            for (int i = 0; i < 5; ++i) {
                const double v = resp_scale[(size_t)d * 5 + i];
                if (!(v > 0.0) || !std::isfinite(v)) return fail(c, GSN_ERR_ARG, "resp_scale must be finite and > 0");
                rs[(size_t)d * NRESP + i] = v;
            }
    }
    if (rate_factor) {
        rf.assign(rate_factor, rate_factor + rf.size());
        for (double v : rf)
            if (!(v >= 0.0) || !std::isfinite(v)) return fail(c, GSN_ERR_ARG, "rate_factor must be finite and >= 0");
    }
    c->rscale = rs;
    c->rfrac = rf;
    c->ready = false;
    return GSN_OK;
}

int gsn_eval_grad(gsn_ctx* c, const double* params, double* nll, double* grad) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (!nll) return fail(c, GSN_ERR_ARG, "nll is NULL");
    if ((rc = check_params_host(c, params))) return rc;
    if ((rc = ensure(c, c->params, c->P * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->nll_b, sizeof(double)))) return rc;
    if ((rc = ensure(c, c->grad_b, c->P * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->status_b, sizeof(int)))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->params.p, params, c->P * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    KArgs a = c->base;
    a.params = (const double*)c->params.p; a.params_stride = c->P;
    a.counts_stride = 0; a.win_stride = 0;
    a.nll = (double*)c->nll_b.p; a.grad = grad ? (double*)c->grad_b.p : nullptr; a.status = (int*)c->status_b.p;
    a.want_grad = grad ? 1 : 0;
    Plan p;
    if ((rc = choose_plan(c, 1, a, grad != nullptr, p))) return rc;
    if ((rc = prepare(c, 1, p, a))) return rc;
    const std::vector<long long> key = {2, grad ? 1 : 0, p.nsplit, p.bw_warps, p.bw_bsplit, p.dev_chunks};
    if ((rc = replay(c, key, [&]() { return run_step(c, a, grad != nullptr); }))) return rc;
    int st = 0;
    CUDA_TRY(c, cudaMemcpyAsync(nll, c->nll_b.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad) CUDA_TRY(c, cudaMemcpyAsync(grad, c->grad_b.p, c->P * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&st, c->status_b.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return status_message(c, st, 0);
}

// round to the nearest TF32 value (10 explicit mantissa bits, ties to even)
static float tf32_round(float x) {
    uint32_t b;
    std::memcpy(&b, &x, 4);
    b = (b + 0xFFFu + ((b >> 13) & 1u)) & ~0x1FFFu;
    float y;
    std::memcpy(&y, &b, 4);
    return y;
}

// TF32 hi / lo split of S' (rows padded to 16 species, columns to 32) and the TMA maps over them
static int prepare_tensor_core(gsn_ctx* c) {
    if (c->tc_ready) return GSN_OK;
    const int Spad = (c->S + 15) / 16 * 16, Kpad = (c->K + 31) / 32 * 32;
    std::vector<float> hi((size_t)Spad * Kpad, 0.f), lo((size_t)Spad * Kpad, 0.f);
    for (int s = 0; s < c->S; ++s)
        for (int k = 0; k < c->K; ++k) {
            const float v = (float)c->Sn[(size_t)s * c->K + k];
            const float h = tf32_round(v);
            hi[(size_t)s * Kpad + k] = h;
            lo[(size_t)s * Kpad + k] = v - h;
        }
    int rc;
    if ((rc = ensure(c, c->s_hi, hi.size() * sizeof(float)))) return rc;
    if ((rc = ensure(c, c->s_lo, lo.size() * sizeof(float)))) return rc;
    CUDA_TRY(c, cudaMemcpy(c->s_hi.p, hi.data(), hi.size() * sizeof(float), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->s_lo.p, lo.data(), lo.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (make_species_tensor_map(c->tm_hi, (const float*)c->s_hi.p, Spad, Kpad) ||
        make_species_tensor_map(c->tm_lo, (const float*)c->s_lo.p, Spad, Kpad))
        return fail(c, GSN_ERR_CUDA, "cuTensorMapEncodeTiled failed for the species tiles");
    if ((rc = ensure(c, c->tc_err, sizeof(int)))) return rc;
    c->tc_ready = true;
    return GSN_OK;
}

// per-species expected shapes M[g][s][j] at the response parameters of params (T = 1)
static int compute_species(gsn_ctx* c, const double* params_dev) {
    int rc;
    KArgs a = c->base;
    const Plan p = make_plan(c, 1);
    if ((rc = prepare(c, 1, p, a))) return rc;
    if ((rc = ensure(c, c->Mbuf, (size_t)c->G * c->S * c->Jmax * sizeof(double)))) return rc;
    a.params = params_dev; a.params_stride = c->P;
    a.counts_stride = 0; a.win_stride = 0;
    a.Mbuf = (double*)c->Mbuf.p;
    a.sp_first = 0; a.sp_count = c->S;
    if (!a.response) return GSN_OK;  // templates and peaks only: no per-species response shapes
    if ((rc = launch(c, K_COLUMNS, a, launch_columns))) return rc;
    if (c->opt.precision == GSN_MIXED && c->opt.resolution != GSN_RES_GGAMMA) {
        if ((rc = prepare_tensor_core(c))) return rc;
        const int tiles = (c->Jmax + 127) / 128 * c->G * ((c->S + 15) / 16);
        a.tc_nsplit = std::max(1, std::min(64, (3 * c->nsm + tiles - 1) / tiles));
        if ((rc = ensure(c, c->tc_part, (size_t)a.tc_nsplit * c->G * c->S * c->Jmax * sizeof(double)))) return rc;
        a.tc_part = (double*)c->tc_part.p;
        a.tc_error = (int*)c->tc_err.p;
        CUDA_TRY(c, cudaMemsetAsync(c->tc_err.p, 0, sizeof(int), c->stream));
        auto fn = [c](const KArgs& x, cudaStream_t st) { return launch_species_tc(x, c->tm_hi, c->tm_lo, st); };
        if ((rc = launch(c, K_SPECIES, a, fn))) return rc;
    } else {
        if ((rc = launch(c, K_SPECIES, a, launch_species))) return rc;
    }
    return GSN_OK;
}

// GSN_ERR_TIMEOUT if a tensor-core CTA gave up waiting (call after the stream is synchronised)
static int species_status(gsn_ctx* c) {
    if (c->opt.precision != GSN_MIXED || !c->tc_err.p) return GSN_OK;
    int e = 0;
    CUDA_TRY(c, cudaMemcpy(&e, c->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
        c->cache_valid = false;
        return fail(c, GSN_ERR_TIMEOUT, "a tensor-core wait timed out in the per-species contraction");
    }
    return GSN_OK;
}

// Per-species shapes M[g][s][j] at the response parameters of params (already on the device in
// c->params): recomputed only when a response parameter differs bit for bit from the cached
// point -- the value cache of section 2.5, shared by gsn_eval and gsn_expected.
static int species_cached(gsn_ctx* c, const double* params, bool& hit) {
    std::vector<double> key;
    for (int g = 0; g < c->G; ++g)
        for (int i = 0; i < NRESP; ++i) key.push_back(c->tab.g_resp[g][i] >= 0 ? params[c->tab.g_resp[g][i]] : 0.0);
    hit = c->cache_valid && key.size() == c->cache_key.size() &&
          std::memcmp(key.data(), c->cache_key.data(), key.size() * sizeof(double)) == 0;
    if (hit) return GSN_OK;
    int rc;
    if ((rc = compute_species(c, (const double*)c->params.p))) return rc;
    c->cache_key = key;
    c->cache_valid = true;
    return GSN_OK;
}

int gsn_eval(gsn_ctx* c, const double* params, double* nll) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (!nll) return fail(c, GSN_ERR_ARG, "nll is NULL");
    if ((rc = check_params_host(c, params))) return rc;
    if ((rc = ensure(c, c->params, c->P * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->nll_b, sizeof(double)))) return rc;
    if ((rc = ensure(c, c->status_b, sizeof(int)))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->params.p, params, c->P * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    bool hit = false;
    if ((rc = species_cached(c, params, hit))) return rc;
    KArgs a = c->base;
    Plan p = make_plan(c, 1);
    p.nsplit = 1;
    if ((rc = prepare(c, 1, p, a))) return rc;
    a.params = (const double*)c->params.p; a.params_stride = c->P;
    a.counts_stride = 0; a.win_stride = 0;
    a.Mbuf = (double*)c->Mbuf.p;
    a.nll = (double*)c->nll_b.p; a.grad = nullptr; a.status = (int*)c->status_b.p;
    a.want_grad = 0;
    a.Mbuf = (double*)c->Mbuf.p;  // the cached shapes (one parameter point)
    a.secRq = nullptr;            // the secondary pieces take their slice sums from them
    if ((rc = launch(c, K_MU, a, launch_mu_from_species))) return rc;
    if (a.nsec && (rc = launch(c, K_SPECIES, a, launch_secondary))) return rc;
    if ((rc = launch(c, K_DEVIANCE, a, launch_deviance))) return rc;
    if ((rc = launch(c, K_DEVFINAL, a, launch_devfinal))) return rc;
    int st = 0;
    CUDA_TRY(c, cudaMemcpyAsync(nll, c->nll_b.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(&st, c->status_b.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (!hit && (rc = species_status(c))) return rc;
    return status_message(c, st, 0);
}

int gsn_expected(gsn_ctx* c, const double* params, int dataset, double* mu_per_species) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (dataset < 0 || dataset >= c->D || !mu_per_species) return fail(c, GSN_ERR_ARG, "bad dataset or NULL output");
    if ((rc = check_params_host(c, params))) return rc;
    if ((rc = ensure(c, c->params, c->P * sizeof(double)))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->params.p, params, c->P * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    bool hit = false;
    if ((rc = species_cached(c, params, hit))) return rc;
    const size_t n = (size_t)c->nb[dataset] * c->S;
    if ((rc = ensure(c, c->outbuf, n * sizeof(double)))) return rc;
    KArgs a = c->base;
    a.T = 1;
    a.params = (const double*)c->params.p;
    a.Mbuf = (double*)c->Mbuf.p;
    a.out_species = (double*)c->outbuf.p;
    a.out_dataset = dataset;
    a.out_bins = c->nb[dataset];
    if ((rc = launch(c, K_SPECIES, a, launch_expected_out))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(mu_per_species, c->outbuf.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return hit ? GSN_OK : species_status(c);
}

int gsn_eval_grad_batch_dev(gsn_ctx* c, int n_toys, const double* params_dev, const double* toy_counts_dev,
                            const int* toy_win_dev, double* nll_dev, double* grad_dev, int* status_dev) {
    if (!c) return GSN_ERR_ARG;
    if (n_toys < 0) return fail(c, GSN_ERR_ARG, "n_toys must be >= 0");
    if (n_toys == 0) return GSN_OK;
    if (!params_dev || !toy_counts_dev || !toy_win_dev || !nll_dev) return fail(c, GSN_ERR_ARG, "NULL argument");
    return batch_device(c, n_toys, params_dev, toy_counts_dev, toy_win_dev, nll_dev, grad_dev, status_dev);
}

}  // extern "C"

namespace {

// the batched minimiser; scale_dev: per-toy scales [T][P] on the device, or NULL for the shared
// host scales `scale` ([P], NULL: 1)
int minimize_batch(gsn_ctx* c, int n_toys, double* params_dev, const double* toy_counts_dev, const int* toy_win_dev,
                   const unsigned char* free_mask, const double* lo, const double* hi, const double* scale,
                   const double* scale_dev, int max_evals, double gtol, double ftol, double edm, double* nll_dev,
                   int* evals_dev, int* status_dev) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (n_toys < 0) return fail(c, GSN_ERR_ARG, "n_toys must be >= 0");
    if (n_toys == 0) return GSN_OK;
    if (!params_dev || !toy_counts_dev || !toy_win_dev || !nll_dev || !free_mask)
        return fail(c, GSN_ERR_ARG, "NULL argument");
    if (c->P > 64) return fail(c, GSN_ERR_ARG, "the minimiser handles at most 64 parameters");
    if (max_evals < 1) max_evals = 200;
    // the mixed NLL carries FP32 rounding (~1e-7 relative): its gradient cannot resolve 1e-6 sigma
    if (!(gtol >= 0.0)) gtol = c->opt.precision == GSN_MIXED ? 1e-4 : 1e-6;
    if (!(ftol >= 0.0)) ftol = 1e-10;
    const int T = n_toys, P = c->P, M = FIT_HISTORY;
    // configuration: free mask, bounds, scales
    std::vector<double> cfg((size_t)3 * P);
    std::vector<unsigned char> fr(free_mask, free_mask + P);
    for (int i = 0; i < P; ++i) {
        cfg[i] = lo ? lo[i] : -INFINITY;
        cfg[P + i] = hi ? hi[i] : INFINITY;
        cfg[2 * P + i] = scale ? scale[i] : 1.0;
        if (!(cfg[2 * P + i] > 0.0) || !std::isfinite(cfg[2 * P + i]) || cfg[i] > cfg[P + i] || std::isnan(cfg[i]) ||
            std::isnan(cfg[P + i]))
            return fail(c, GSN_ERR_ARG, "bad bound or scale of parameter " + std::to_string(i));
    }
    const size_t ws_doubles = (size_t)T * P * 4 + (size_t)T * M * P * 2 + (size_t)T * M + (size_t)T * 4;
    if ((rc = ensure(c, c->fit_ws, ws_doubles * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->fit_cfg, cfg.size() * sizeof(double) + 64 + P))) return rc;
    if ((rc = ensure(c, c->fit_eval, ((size_t)T * (P + 1)) * sizeof(double) + (size_t)T * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->fit_ist, ((size_t)T * 8 + 1) * sizeof(int)))) return rc;
    double* ws = (double*)c->fit_ws.p;
    FitArgs f{};
    f.T = T; f.P = P; f.max_evals = max_evals; f.gtol = gtol; f.ftol = ftol; f.edm = edm;
    f.fnoise = c->opt.precision == GSN_MIXED ? 1e-7 : 1e-13;
    f.X = ws; f.G = ws + (size_t)T * P; f.D = ws + (size_t)2 * T * P; f.XT = ws + (size_t)3 * T * P;
    f.S = ws + (size_t)4 * T * P; f.Y = f.S + (size_t)T * M * P; f.RHO = f.Y + (size_t)T * M * P;
    f.dstate = f.RHO + (size_t)T * M;
    double* cf = (double*)c->fit_cfg.p;
    f.lo = cf; f.hi = cf + P;
    if (scale_dev) { f.scale = scale_dev; f.scale_stride = P; }
    else { f.scale = cf + 2 * P; f.scale_stride = 0; }
    f.free = (const unsigned char*)(cf + 3 * P);
    double* ev = (double*)c->fit_eval.p;
    f.nll = ev; f.grad = ev + T;
    f.estatus = (const int*)(ev + (size_t)T * (P + 1));
    f.istate = (int*)c->fit_ist.p;
    f.active = f.istate + (size_t)T * 8;
    CUDA_TRY(c, cudaMemcpyAsync(cf, cfg.data(), cfg.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync((void*)f.free, fr.data(), P, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(f.XT, params_dev, (size_t)T * P * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(f.istate, 0, (size_t)T * 8 * sizeof(int), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(f.dstate, 0, (size_t)T * 4 * sizeof(double), c->stream));
    for (int it = 0; it < max_evals; ++it) {
        if ((rc = batch_device(c, T, f.XT, toy_counts_dev, toy_win_dev, ev, ev + T, (int*)f.estatus))) return rc;
        CUDA_TRY(c, cudaMemsetAsync(f.active, 0, sizeof(int), c->stream));
        CUDA_TRY(c, launch_lbfgs(f, c->stream));
        if ((it & 3) == 3 || it + 1 == max_evals) {
            int active = 0;
            CUDA_TRY(c, cudaMemcpyAsync(&active, f.active, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            if (active == 0) break;
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(params_dev, f.X, (size_t)T * P * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpy2DAsync(nll_dev, sizeof(double), f.dstate, 4 * sizeof(double), sizeof(double), T,
                                  cudaMemcpyDeviceToDevice, c->stream));
    if (evals_dev)
        CUDA_TRY(c, cudaMemcpy2DAsync(evals_dev, sizeof(int), f.istate + 3, 8 * sizeof(int), sizeof(int), T,
                                      cudaMemcpyDeviceToDevice, c->stream));
    if (status_dev)
        CUDA_TRY(c, cudaMemcpy2DAsync(status_dev, sizeof(int), f.istate + 4, 8 * sizeof(int), sizeof(int), T,
                                      cudaMemcpyDeviceToDevice, c->stream));
    return GSN_OK;
}

}  // namespace

extern "C" {

int gsn_minimize_batch_dev(gsn_ctx* c, int n_toys, double* params_dev, const double* toy_counts_dev,
                           const int* toy_win_dev, const unsigned char* free_mask, const double* lo, const double* hi,
                           const double* scale, int max_evals, double gtol, double ftol, double* nll_dev,
                           int* evals_dev, int* status_dev) {
    return minimize_batch(c, n_toys, params_dev, toy_counts_dev, toy_win_dev, free_mask, lo, hi, scale, nullptr,
                          max_evals, gtol, ftol, 0.0, nll_dev, evals_dev, status_dev);
}

int gsn_minimize_batch_scaled_dev(gsn_ctx* c, int n_toys, double* params_dev, const double* toy_counts_dev,
                                  const int* toy_win_dev, const unsigned char* free_mask, const double* lo,
                                  const double* hi, const double* scale_dev, int max_evals, double gtol, double ftol,
                                  double edm, double* nll_dev, int* evals_dev, int* status_dev) {
    if (!c) return GSN_ERR_ARG;
    if (!scale_dev) return fail(c, GSN_ERR_ARG, "scale_dev is NULL");
    if (std::isnan(edm)) return fail(c, GSN_ERR_ARG, "edm is NaN");
    return minimize_batch(c, n_toys, params_dev, toy_counts_dev, toy_win_dev, free_mask, lo, hi, nullptr, scale_dev,
                          max_evals, gtol, ftol, edm, nll_dev, evals_dev, status_dev);
}

int gsn_fit_rates_batch_dev(gsn_ctx* c, int n_toys, double* params_dev, const double* toy_counts_dev,
                            const int* toy_win_dev, const unsigned char* free_mask, const double* lo, const double* hi,
                            int max_iter, double tol, double* nll_dev, int* iters_dev, int* status_dev) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (n_toys < 0) return fail(c, GSN_ERR_ARG, "n_toys must be >= 0");
    if (n_toys == 0) return GSN_OK;
    if (!params_dev || !toy_counts_dev || !toy_win_dev || !nll_dev || !free_mask)
        return fail(c, GSN_ERR_ARG, "NULL argument");
    if (c->base.nsec) return fail(c, GSN_ERR_ARG, "rate fits do not take secondary observables");
    if (max_iter < 1) max_iter = 200;
    if (!(tol > 0.0)) tol = 1e-8;
    const int P = c->P, S = c->S, NSLOT = gsn_n_slots(S);
    // free parameters: each must fill rate slots only
    std::vector<int> fidx, pfree(P, -1);
    std::vector<double> flo, fhi;
    for (int p = 0; p < P; ++p) {
        if (!free_mask[p]) continue;
        bool rate = false;
        for (int d = 0; d < c->D; ++d)
            for (int sl = 0; sl < NSLOT; ++sl)
                if (c->slot_map[(size_t)d * NSLOT + sl] == p) {
                    if (sl >= S) return fail(c, GSN_ERR_ARG, "free parameter " + std::to_string(p) + " is not a rate");
                    rate = true;
                }
        if (!rate) return fail(c, GSN_ERR_ARG, "free parameter " + std::to_string(p) + " fills no rate slot");
        const double l = lo ? lo[p] : -INFINITY, h = hi ? hi[p] : INFINITY;
        if (std::isnan(l) || std::isnan(h) || l > h) return fail(c, GSN_ERR_ARG, "bad bounds of parameter " + std::to_string(p));
        pfree[p] = (int)fidx.size();
        fidx.push_back(p); flo.push_back(l); fhi.push_back(h);
    }
    const int nf = (int)fidx.size();
    if (nf > RF_NFMAX) return fail(c, GSN_ERR_ARG, "at most " + std::to_string(RF_NFMAX) + " free rates");
    // toys per pass: per-species shapes and the design rows within 4 GiB
    const size_t per_toy = (size_t)c->G * S * c->Jmax * sizeof(double) +
                           (size_t)c->total_bins * ((size_t)nf + 4) * sizeof(double);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>({(size_t)c->opt.max_toys_per_launch,
                                                                 (size_t)65535 / std::max(1, c->G),
                                                                 ((size_t)4 << 30) / std::max<size_t>(per_toy, 1)}));
    const int T0 = std::min(chunk, n_toys);
    std::vector<double> cfg((size_t)2 * std::max(nf, 1));
    for (int f = 0; f < nf; ++f) { cfg[f] = flo[f]; cfg[nf + f] = fhi[f]; }
    std::vector<int> icfg(fidx);
    icfg.insert(icfg.end(), pfree.begin(), pfree.end());
    if ((rc = ensure(c, c->rfit_cfg, cfg.size() * sizeof(double) + icfg.size() * sizeof(int)))) return rc;
    const size_t nb = (size_t)T0 * c->total_bins;
    if ((rc = ensure(c, c->rfit_ws, nb * ((size_t)std::max(nf, 1) + 4) * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->Mbuf, (size_t)T0 * c->G * S * c->Jmax * sizeof(double)))) return rc;
    double* cf = (double*)c->rfit_cfg.p;
    int* ic = (int*)(cf + cfg.size());
    CUDA_TRY(c, cudaMemcpyAsync(cf, cfg.data(), cfg.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(ic, icfg.data(), icfg.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    for (int t0 = 0; t0 < n_toys; t0 += chunk) {
        const int T = std::min(chunk, n_toys - t0);
        KArgs a = c->base;
        const Plan p = make_plan(c, T);
        if ((rc = prepare(c, T, p, a))) return rc;
        a.params = params_dev + (size_t)t0 * P; a.params_stride = P;
        a.counts = toy_counts_dev + (size_t)t0 * c->n_counts; a.counts_stride = c->n_counts;
        a.win = toy_win_dev + (size_t)t0 * c->D * 2; a.win_stride = 2 * c->D;
        a.Mbuf = (double*)c->Mbuf.p; a.mstride = (long long)c->G * S * c->Jmax;
        a.sp_first = 0; a.sp_count = S;
        a.want_grad = 0;
        if (a.response) {
            CUDA_TRY(c, cudaMemsetAsync(c->Mbuf.p, 0, (size_t)T * c->G * S * c->Jmax * sizeof(double), c->stream));
            if ((rc = launch(c, K_COLUMNS, a, launch_columns))) return rc;
            if ((rc = launch(c, K_SPECIES, a, launch_species))) return rc;
        }
        RateArgs r{};
        r.nf = nf; r.max_iter = max_iter; r.tol = tol; r.fnoise = 1e-12;
        r.share_min = 1e3 * std::exp(-c->opt.band_cut);
        r.fidx = ic; r.pfree = ic + nf; r.lo = cf; r.hi = cf + nf;
        r.params = params_dev + (size_t)t0 * P;
        double* ws = (double*)c->rfit_ws.p;
        const size_t nbT = (size_t)T * c->total_bins;
        r.B = ws; r.C = ws + nbT * std::max(nf, 1); r.N = r.C + nbT; r.mu = r.N + nbT;
        r.dmu = r.mu + nbT;
        r.nll = nll_dev + t0;
        r.iters = iters_dev ? iters_dev + t0 : nullptr;
        r.status = status_dev ? status_dev + t0 : nullptr;
        CUDA_TRY(c, launch_rate_fit(a, r, c->stream));
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // the host configuration must outlive its copies
    return GSN_OK;
}

int gsn_window_scales_dev(gsn_ctx* c, int n_toys, const double* params_dev, const int* toy_win_dev,
                          const double* scale, double max_factor, double* scale_dev) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (n_toys < 0) return fail(c, GSN_ERR_ARG, "n_toys must be >= 0");
    if (n_toys == 0) return GSN_OK;
    if (!params_dev || !toy_win_dev || !scale_dev) return fail(c, GSN_ERR_ARG, "NULL argument");
    if (!(max_factor > 0.0)) max_factor = 100.0;
    if (max_factor < 1.0 || !std::isfinite(max_factor)) return fail(c, GSN_ERR_ARG, "max_factor must be >= 1 and finite");
    const int T = n_toys, P = c->P;
    std::vector<double> sc(P, 1.0);
    for (int i = 0; i < P && scale; ++i) {
        if (!(scale[i] > 0.0) || !std::isfinite(scale[i]))
            return fail(c, GSN_ERR_ARG, "bad scale of parameter " + std::to_string(i));
        sc[i] = scale[i];
    }
    const size_t nds = (size_t)T * c->D * c->S;
    if ((rc = ensure(c, c->wscale_b, (2 * nds + P) * sizeof(double)))) return rc;
    double* nwin = (double*)c->wscale_b.p;
    double* nfull = nwin + nds;
    double* scd = nfull + nds;
    CUDA_TRY(c, cudaMemcpyAsync(scd, sc.data(), P * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    KArgs a = c->base;
    a.T = T;
    a.params = params_dev; a.params_stride = P;
    a.win = toy_win_dev; a.win_stride = 2 * c->D;
    CUDA_TRY(c, launch_window_scales(a, nwin, nfull, scd, max_factor, scale_dev, c->stream));
    // the host buffer sc must outlive the copy
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return GSN_OK;
}

int gsn_eval_grad_batch(gsn_ctx* c, int n_toys, const double* params, const double* toy_counts, const int* toy_win,
                        double* nll, double* grad) {
    if (!c) return GSN_ERR_ARG;
    int rc;
    if ((rc = finalize(c))) return rc;
    if (n_toys < 0) return fail(c, GSN_ERR_ARG, "n_toys must be >= 0");
    if (n_toys == 0) return GSN_OK;
    if (!params || !toy_counts || !toy_win || !nll) return fail(c, GSN_ERR_ARG, "NULL argument");
    for (long long i = 0; i < (long long)n_toys * c->P; ++i)
        if (!std::isfinite(params[i])) return fail(c, GSN_ERR_NONFINITE, "toy parameter not finite");
    for (long long i = 0; i < (long long)n_toys * c->D; ++i) {
        const int d = (int)(i % c->D);
        const int lo = toy_win[2 * i], hi = toy_win[2 * i + 1];
        if (lo < 0 || hi > c->nb[d] || lo > hi) return fail(c, GSN_ERR_ARG, "toy window out of range");
    }
    const size_t TB = (size_t)n_toys;
    if ((rc = ensure(c, c->params, TB * c->P * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->counts_b, TB * c->n_counts * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->win_b, TB * c->D * 2 * sizeof(int)))) return rc;
    if ((rc = ensure(c, c->nll_b, TB * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->grad_b, TB * c->P * sizeof(double)))) return rc;
    if ((rc = ensure(c, c->status_b, TB * sizeof(int)))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->params.p, params, TB * c->P * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->counts_b.p, toy_counts, TB * c->n_counts * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(c->win_b.p, toy_win, TB * c->D * 2 * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if ((rc = batch_device(c, n_toys, (const double*)c->params.p, (const double*)c->counts_b.p, (const int*)c->win_b.p,
                           (double*)c->nll_b.p, grad ? (double*)c->grad_b.p : nullptr, (int*)c->status_b.p)))
        return rc;
    std::vector<int> st(n_toys);
    CUDA_TRY(c, cudaMemcpyAsync(nll, c->nll_b.p, TB * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (grad) CUDA_TRY(c, cudaMemcpyAsync(grad, c->grad_b.p, TB * c->P * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(st.data(), c->status_b.p, TB * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int t = 0; t < n_toys; ++t)
        if (st[t]) return status_message(c, st[t], t);
    return GSN_OK;
}


}  // extern "C"

// ============================================================ no-allocation
// One static device array holds the intermediate buffers of
// gsn_eval_grad_noalloc; its device address is looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GSN_NOALLOC_SCRATCH_BYTES];

namespace {

void* noalloc_address(int dev, std::string& err) {
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) { err = "device ordinal out of range"; return nullptr; }
    std::lock_guard<std::mutex> lock(mu);
    if (addr[dev]) return addr[dev];
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) { cudaGetLastError(); err = "cudaSetDevice failed"; return nullptr; }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur >= 0 && cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        err = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
        return nullptr;
    }
    addr[dev] = p;
    return p;
}

}  // namespace

extern "C" int gsn_eval_grad_noalloc(gsn_ctx* c, const double* params_dev, double* nll_dev, double* grad_dev,
                                     int* status_dev) {
    if (!c) return GSN_ERR_ARG;
    if (!params_dev || !nll_dev || !grad_dev) return fail(c, GSN_ERR_ARG, "NULL device pointer");
    if (!c->ready)
        return fail(c, GSN_ERR_STATE, "the problem is not on the device yet: call gsn_eval or gsn_eval_grad once first");
    if (c->base.nsec)
        return fail(c, GSN_ERR_ARG, "the no-allocation entry point does not take secondary observables");
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != c->dev) {
        cudaGetLastError();
        return fail(c, GSN_ERR_STATE, "the context's device (" + std::to_string(c->dev) + ") must be the current "
                    "device (" + std::to_string(cur) + ") when gsn_eval_grad_noalloc is called");
    }
    std::string err;
    unsigned char* base = static_cast<unsigned char*>(noalloc_address(c->dev, err));
    if (!base) return fail(c, GSN_ERR_CUDA, err);
    KArgs a = c->base;
    const Plan p = make_plan(c, 1);
    const size_t rs = c->opt.precision == GSN_MIXED ? sizeof(float) : sizeof(double);
    const size_t sizes[10] = {
        (size_t)c->G * c->K * NFP * rs,                         // column records
        (size_t)c->G * a.nblk * 2 * rs,                         // band summaries
        (size_t)p.nsplit * c->total_bins * sizeof(double),      // partial mu
        (size_t)c->total_bins * rs,                             // w
        (size_t)c->G * p.nbtask * a.NPART * sizeof(double),     // partial gradients
        (size_t)c->P * sizeof(double),                          // direct gradient terms
        (size_t)p.dev_chunks * (2 + c->base.ntpl) * sizeof(double),   // deviance and template partials
        c->opt.resolution == GSN_RES_GGAMMA ? (size_t)c->G * c->K * NFG * sizeof(double) : 0,  // adjoint coefficients
        ((size_t)c->G + 1) * sizeof(int),                       // forward segment prefix
        c->opt.resolution != GSN_RES_GAUSS ? (size_t)c->G * c->K * NFZ * rs : 0};  // bin-at-zero records
    size_t off[10], total = 0;
    for (int i = 0; i < 10; ++i) { off[i] = total; total += (sizes[i] + 255) & ~(size_t)255; }
    if (total > GSN_NOALLOC_SCRATCH_BYTES)
        return fail(c, GSN_ERR_ARG, "this problem needs " + std::to_string(total) + " bytes of scratch; the "
                    "no-allocation entry point holds " + std::to_string((size_t)GSN_NOALLOC_SCRATCH_BYTES));
    a.T = 1;
    a.nsplit = p.nsplit; a.ntile = p.ntile;
    a.bw_warps = p.bw_warps; a.bw_bsplit = p.bw_bsplit; a.nbtask = p.nbtask;
    a.colbuf = base + off[0]; a.blkbuf = base + off[1]; a.mubuf = (double*)(base + off[2]);
    a.wbuf = base + off[3]; a.partbuf = (double*)(base + off[4]); a.gdirect = (double*)(base + off[5]);
    a.dev_chunks = p.dev_chunks; a.devpart = (double*)(base + off[6]);
    a.colbuf2 = (double*)(base + off[7]);
    a.segoff = (int*)(base + off[8]);
    a.zerobuf = c->opt.resolution != GSN_RES_GAUSS ? (void*)(base + off[9]) : nullptr;
    a.params = params_dev; a.params_stride = c->P;
    a.counts_stride = 0; a.win_stride = 0;
    a.nll = nll_dev; a.grad = grad_dev; a.status = status_dev;
    a.want_grad = 1;
    a.work = nullptr;
    if (a.response) {
        CUDA_TRY(c, launch_columns(a, c->stream));
        CUDA_TRY(c, launch_forward(a, c->stream));
    }
    CUDA_TRY(c, launch_deviance(a, c->stream));
    CUDA_TRY(c, launch_devfinal(a, c->stream));
    if (a.response) CUDA_TRY(c, launch_backward(a, c->stream));
    CUDA_TRY(c, launch_gradfinal(a, c->stream));
    return GSN_OK;
}

