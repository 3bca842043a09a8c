// Batched minimiser for the profile likelihood (section 4.2: toy Monte Carlo discovery test).
//
// Every toy runs its own projected L-BFGS in FP64 in scaled variables u = x / scale: a history of
// FIT_HISTORY curvature pairs, the two-loop recursion for the direction on the free variables
// that are not held at a bound, and a backtracking Armijo line search (quadratic interpolation of
// the step).  One iteration of the host loop is one batched NLL + gradient evaluation of every
// toy's trial point (the same kernels as gsn_eval_grad_batch) followed by k_lbfgs, which accepts
// or shortens the step of each toy and writes its next trial point.  One warp per toy; the
// parameter vector (P <= 64) is spread over the lanes, two entries each.
#include "gsn_device.cuh"

namespace gsn {

namespace {

constexpr int FIT_M = FIT_HISTORY;
constexpr double C1 = 1e-4;        // Armijo constant
constexpr double STEP_MAX = 1e4;   // largest move of one scaled variable in a step (backtracking does the rest)
enum { ST_INIT = 0, ST_SEARCH = 1, ST_DONE = 2 };

DEV double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
DEV double wmax(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// a variable moves in the next step: free, and not held at a bound by a gradient pushing outwards
DEV bool movable(const FitArgs& f, int i, double x, double g) {
    if (!f.free[i]) return false;
    if (x <= f.lo[i] && g > 0.0) return false;
    if (x >= f.hi[i] && g < 0.0) return false;
    return true;
}
// projected gradient in scaled units (0 for variables that do not move); scl: the toy's scales
DEV double proj_grad(const FitArgs& f, const double* scl, int i, double x, double g) {
    return movable(f, i, x, g) ? g * scl[i] : 0.0;
}

}  // namespace

__global__ void __launch_bounds__(128) k_lbfgs(FitArgs f) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t = blockIdx.x * 4 + warp;
    if (t >= f.T) return;
    const int P = f.P;
    int* ist = f.istate + (long long)t * 8;  // state, nhist, head, evals, status, resets, small steps
    if (ist[0] == ST_DONE) return;
    double* X = f.X + (long long)t * P;
    double* G = f.G + (long long)t * P;
    double* Dd = f.D + (long long)t * P;
    double* XT = f.XT + (long long)t * P;
    double* S = f.S + (long long)t * FIT_M * P;
    double* Y = f.Y + (long long)t * FIT_M * P;
    double* RHO = f.RHO + (long long)t * FIT_M;
    double* sc = f.dstate + (long long)t * 4;  // F, alpha, gd, unused
    const double* scl = f.scale + (long long)t * f.scale_stride;
    const double ft = f.nll[t];
    const double* gt = f.grad + (long long)t * P;
    const int i0 = lane, i1 = lane + 32;
    const bool h0 = i0 < P, h1 = i1 < P;
    const int evals = ist[3] + 1;
    int state = ist[0], nhist = ist[1], head = ist[2], status = ist[4], resets = ist[5], small = ist[6];
    int shortened = ist[7];  // the current step was shortened at least once
    double F = sc[0], alpha = sc[1], gd = sc[2];
    bool set_dir = false, done = false;

    if (state == ST_INIT) {
        if (h0) { X[i0] = XT[i0]; G[i0] = gt[i0]; }
        if (h1) { X[i1] = XT[i1]; G[i1] = gt[i1]; }
        F = ft;
        // every free variable needs a finite positive scale (per-toy scales come from the caller)
        const bool bad = (h0 && f.free[i0] && !(scl[i0] > 0.0 && isfinite(scl[i0]))) ||
                         (h1 && f.free[i1] && !(scl[i1] > 0.0 && isfinite(scl[i1])));
        if (__any_sync(0xffffffffu, bad)) { status = -1; done = true; }
        else if (!isfinite(ft) || f.estatus[t] != 0) { status = -4; done = true; }
        else set_dir = true;
    } else {  // ST_SEARCH: the trial point XT was evaluated
        double st = 0.0;  // predicted change g . (x_t - x) of the projected step
        if (h0) st += G[i0] * (XT[i0] - X[i0]);
        if (h1) st += G[i1] * (XT[i1] - X[i1]);
        st = wsum(st);
        // sufficient decrease, allowing the NLL's own rounding (fnoise relative): near the minimum
        // of a mixed-precision NLL true decreases fall below it, and the gradient decides instead
        const bool ok = isfinite(ft) && f.estatus[t] == 0 && ft <= F + C1 * st + f.fnoise * fabs(F);
        if (ok) {
            // the set of variables held at a bound changed: the curvature pairs describe another
            // subspace, so the history restarts
            const bool b0o = h0 && f.free[i0] && (X[i0] <= f.lo[i0] || X[i0] >= f.hi[i0]);
            const bool b1o = h1 && f.free[i1] && (X[i1] <= f.lo[i1] || X[i1] >= f.hi[i1]);
            const bool b0n = h0 && f.free[i0] && (XT[i0] <= f.lo[i0] || XT[i0] >= f.hi[i0]);
            const bool b1n = h1 && f.free[i1] && (XT[i1] <= f.lo[i1] || XT[i1] >= f.hi[i1]);
            if (__any_sync(0xffffffffu, b0o != b0n || b1o != b1n)) { nhist = 0; head = 0; }
            // curvature pair in scaled units, on the free variables only: the gradient of a held
            // parameter changes too, but belongs to no direction the search can take
            double s0 = 0.0, s1 = 0.0, y0 = 0.0, y1 = 0.0;
            if (h0 && f.free[i0]) { s0 = (XT[i0] - X[i0]) / scl[i0]; y0 = (gt[i0] - G[i0]) * scl[i0]; }
            if (h1 && f.free[i1]) { s1 = (XT[i1] - X[i1]) / scl[i1]; y1 = (gt[i1] - G[i1]) * scl[i1]; }
            const double sy = wsum(s0 * y0 + s1 * y1);
            const double ss = wsum(s0 * s0 + s1 * s1), yy = wsum(y0 * y0 + y1 * y1);
            if (sy > 1e-10 * sqrt(ss * yy)) {
                const int slot = head;
                if (h0) { S[slot * P + i0] = s0; Y[slot * P + i0] = y0; }
                if (h1) { S[slot * P + i1] = s1; Y[slot * P + i1] = y1; }
                if (lane == 0) RHO[slot] = 1.0 / sy;
                head = (head + 1) % FIT_M;
                nhist = min(nhist + 1, FIT_M);
            }
            __syncwarp();  // RHO (written by lane 0) is read by every lane in the recursion below
            const double Fprev = F;
            F = ft;
            if (h0) { X[i0] = XT[i0]; G[i0] = gt[i0]; }
            if (h1) { X[i1] = XT[i1]; G[i1] = gt[i1]; }
            double pg = 0.0;
            if (h0) pg = fmax(pg, fabs(proj_grad(f, scl, i0, X[i0], G[i0])));
            if (h1) pg = fmax(pg, fabs(proj_grad(f, scl, i1, X[i1], G[i1])));
            pg = wmax(pg);
            // converged: projected gradient below gtol, or two full (not shortened) steps in a row
            // that each lowered the NLL by at most ftol relative
            small = (!shortened && Fprev - F <= f.ftol * fmax(1.0, fabs(F))) ? small + 1 : 0;
            if (pg <= f.gtol || small >= 2) { status = 0; done = true; }
            else set_dir = true;
        } else {
            // shorten: minimiser of the quadratic through F, the slope gd and ft, within [0.1, 0.5] alpha
            double an = 0.5 * alpha;
            if (isfinite(ft)) {
                const double den = 2.0 * (ft - F - gd * alpha);
                if (den > 0.0) an = fmin(0.5 * alpha, fmax(0.1 * alpha, -gd * alpha * alpha / den));
            }
            alpha = an;
            shortened = 1;
            if (alpha < 1e-12) {
                if (nhist > 0 && resets < 3) { nhist = 0; head = 0; ++resets; set_dir = true; }  // restart steepest
                else { status = 2; done = true; }
            }
        }
    }
    if (!done && evals >= f.max_evals) { status = 1; done = true; }

    if (set_dir && !done) {
        // two-loop recursion on the projected gradient (scaled units)
        double q0 = 0.0, q1 = 0.0;
        if (h0) q0 = proj_grad(f, scl, i0, X[i0], G[i0]);
        if (h1) q1 = proj_grad(f, scl, i1, X[i1], G[i1]);
        // the recursion runs on the subspace of the variables that move
        const bool m0 = h0 && movable(f, i0, X[i0], G[i0]);
        const bool m1 = h1 && movable(f, i1, X[i1], G[i1]);
        double al[FIT_M];
        for (int k = 0; k < nhist; ++k) {
            const int slot = (head - 1 - k + 2 * FIT_M) % FIT_M;
            const double a = RHO[slot] * wsum((m0 ? S[slot * P + i0] * q0 : 0.0) + (m1 ? S[slot * P + i1] * q1 : 0.0));
            al[k] = a;
            if (m0) q0 -= a * Y[slot * P + i0];
            if (m1) q1 -= a * Y[slot * P + i1];
        }
        double gamma = 1.0;
        if (nhist > 0) {
            const int slot = (head - 1 + FIT_M) % FIT_M;
            const double yy = wsum((h0 ? Y[slot * P + i0] * Y[slot * P + i0] : 0.0) +
                                   (h1 ? Y[slot * P + i1] * Y[slot * P + i1] : 0.0));
            gamma = yy > 0.0 ? 1.0 / (RHO[slot] * yy) : 1.0;
        }
        q0 *= gamma; q1 *= gamma;
        for (int k = nhist - 1; k >= 0; --k) {
            const int slot = (head - 1 - k + 2 * FIT_M) % FIT_M;
            const double b = RHO[slot] * wsum((m0 ? Y[slot * P + i0] * q0 : 0.0) + (m1 ? Y[slot * P + i1] * q1 : 0.0));
            if (m0) q0 += S[slot * P + i0] * (al[k] - b);
            if (m1) q1 += S[slot * P + i1] * (al[k] - b);
        }
        double d0 = m0 ? -q0 : 0.0, d1 = m1 ? -q1 : 0.0;
        const double pg0 = h0 ? proj_grad(f, scl, i0, X[i0], G[i0]) : 0.0, pg1 = h1 ? proj_grad(f, scl, i1, X[i1], G[i1]) : 0.0;
        gd = wsum(d0 * pg0 + d1 * pg1);
        if (!(gd < 0.0)) {  // not a descent direction: steepest descent, history dropped
            d0 = -pg0; d1 = -pg1;
            nhist = 0; head = 0;
            gd = wsum(d0 * pg0 + d1 * pg1);
        }
        const double dmax = wmax(fmax(fabs(d0), fabs(d1)));
        // without curvature pairs the first step moves no scaled variable by more than 1
        alpha = dmax > 0.0 ? fmin(1.0, (nhist > 0 ? STEP_MAX : 1.0) / dmax) : 0.0;
        shortened = 0;
        if (h0) Dd[i0] = d0;
        if (h1) Dd[i1] = d1;
        if (dmax == 0.0) { status = 0; done = true; }  // every free variable held at a bound
        // estimated distance to the minimum, -g.d/2 with d = -H^-1 g the quasi-Newton step (the
        // stopping rule of MINUIT's MIGRAD), once curvature pairs describe H
        if (f.edm > 0.0 && nhist > 0 && -0.5 * gd < f.edm) { status = 0; done = true; }
        state = ST_SEARCH;
    }
    if (done) {
        state = ST_DONE;
        if (h0) XT[i0] = X[i0];
        if (h1) XT[i1] = X[i1];
    } else {
        // next trial point: x + alpha d (scaled), projected onto the bounds
        if (h0) XT[i0] = f.free[i0] ? fmin(fmax(X[i0] + alpha * Dd[i0] * scl[i0], f.lo[i0]), f.hi[i0]) : X[i0];
        if (h1) XT[i1] = f.free[i1] ? fmin(fmax(X[i1] + alpha * Dd[i1] * scl[i1], f.lo[i1]), f.hi[i1]) : X[i1];
    }
    __syncwarp();
    if (lane == 0) {
        ist[0] = state; ist[1] = nhist; ist[2] = head; ist[3] = evals; ist[4] = status; ist[5] = resets;
        ist[6] = small; ist[7] = shortened;
        sc[0] = F; sc[1] = alpha; sc[2] = gd;
        if (state != ST_DONE) atomicAdd(f.active, 1);
    }
}

// ------------------------------------------------------------------------------------------
// Per-toy conditioning of the minimiser.  A toy fitted in a window that holds only part of a
// species' spectrum constrains that species' rate less than the whole histograms do, so a scale
// taken from the whole histograms (the caller's) is too small for it.  k_window_counts adds up,
// at the toy's parameters, every species' expected counts over the whole histogram and inside
// the toy's window of every dataset; the response is taken as a Gaussian of each column's mean
// and variance (a scale needs no better).  k_window_scales multiplies the scale of every
// parameter that fills only rate slots by sqrt(N_whole / N_window) of its species, within
// [1, max_factor].
constexpr int WC_CHUNK = 1024;
constexpr int WC_WARPS = 8;

DEV float gauss_mass(float lo, float hi, float mu, float isg) {
    return hi > lo ? normcdff((hi - mu) * isg) - normcdff((lo - mu) * isg) : 0.0f;
}

__global__ void __launch_bounds__(WC_WARPS * 32) k_window_counts(KArgs a, double* nwin, double* nfull) {
    const int t = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ float sp[2][MAXGDS][WC_CHUNK];     // column mass in the window / whole histogram
    __shared__ double acc[2][MAXGDS][MAXS];
    const double* prm = a.params + (long long)t * a.params_stride;
    const int* win = a.win + (long long)t * a.win_stride;
    for (int g = 0; g < a.G; ++g) {
        if (!tb_g_active(a, g)) continue;
        const int nds = tb_g_nds(a, g), J = tb_g_bins(a, g);
        const double* ed = a.edges + tb_g_edge_off(a, g);
        double rp[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int ri = tb_g_resp(a, g, i);
            rp[i] = ri >= 0 ? prm[ri] * tb_g_rscale(a, g, i) : 0.0;
        }
        const double alpha = 1.0 + rp[1] * a.s0, beta = rp[1] * a.s1;
        float xl[MAXGDS] = {}, xh[MAXGDS] = {};
        for (int dd = 0; dd < nds; ++dd) {
            const int d = tb_g_ds(a, g, dd);
            const int lo = max(win[2 * d], 0), hi = min(win[2 * d + 1], J);
            if (hi > lo) { xl[dd] = (float)ed[lo]; xh[dd] = (float)ed[hi]; }
        }
        const float x0 = (float)ed[0], xJ = (float)ed[J];
        for (int i = threadIdx.x; i < 2 * MAXGDS * MAXS; i += blockDim.x) (&acc[0][0][0])[i] = 0.0;
        for (int k0 = 0; k0 < a.K; k0 += WC_CHUNK) {
            const int nk = min(WC_CHUNK, a.K - k0);
            __syncthreads();  // the previous chunk has been consumed (and acc cleared)
            for (int i = threadIdx.x; i < nk; i += blockDim.x) {
                const double E = a.E[k0 + i];
                const double Eq = beta > 0.0 ? E / alpha - beta / (alpha * alpha) * log1p(alpha * E / beta) : E / alpha;
                const double mu = rp[0] * Eq;
                const double var = rp[2] + mu * (rp[3] + rp[4] * mu);
                const float isg = var > 0.0 ? (float)rsqrt(var) : 0.0f;
                for (int dd = 0; dd < nds; ++dd) {
                    sp[0][dd][i] = gauss_mass(xl[dd], xh[dd], (float)mu, isg);
                    sp[1][dd][i] = gauss_mass(x0, xJ, (float)mu, isg);
                }
            }
            __syncthreads();
            for (int s = warp; s < a.S; s += WC_WARPS) {
                if (a.ft.sp_kind[s] >= 2) continue;  // peaks and templates do not pass the response
                // the spectra are on the device in the context's precision only
                const float* Srf = a.precision == 1 ? a.Sf + (long long)s * a.K + k0 : nullptr;
                const double* Srd = a.precision == 1 ? nullptr : a.Sd + (long long)s * a.K + k0;
                float pw[MAXGDS] = {}, pf[MAXGDS] = {};
                for (int i = lane; i < nk; i += 32) {
                    const float sv = Srf ? Srf[i] : (float)Srd[i];
                    for (int dd = 0; dd < nds; ++dd) {
                        pw[dd] = fmaf(sv, sp[0][dd][i], pw[dd]);
                        pf[dd] = fmaf(sv, sp[1][dd][i], pf[dd]);
                    }
                }
                for (int dd = 0; dd < nds; ++dd) {
                    const float w = warp_sum<float>(pw[dd]), f = warp_sum<float>(pf[dd]);
                    if (lane == 0) { acc[0][dd][s] += w; acc[1][dd][s] += f; }
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nds * a.S; i += blockDim.x) {
            const int dd = i / a.S, s = i % a.S, d = tb_g_ds(a, g, dd);
            if (a.ft.sp_kind[s] >= 2) continue;
            const double rf = a.rfac[d * a.S + s];
            nwin[((long long)t * a.D + d) * a.S + s] = rf * acc[0][dd][s];
            nfull[((long long)t * a.D + d) * a.S + s] = rf * acc[1][dd][s];
        }
        __syncthreads();
    }
    // peaks (a Gaussian in p.e.) and templates (their histograms), every dataset
    for (int i = threadIdx.x; i < a.D * a.S; i += blockDim.x) {
        const int d = i / a.S, s = i % a.S;
        const int kind = a.ft.sp_kind[s];
        const double rf = a.rfac[d * a.S + s];
        if (kind < 2 || rf == 0.0) continue;
        const int J = tb_ds_bins(a, d);
        const double* ed = a.edges + tb_g_edge_off(a, tb_ds_group(a, d));
        const int lo = max(win[2 * d], 0), hi = min(win[2 * d + 1], J);
        double vw = 0.0, vf = 0.0;
        if (kind == 2) {
            const int* sm = a.slot_map + (long long)d * a.NSLOT;
            const int im = sm[a.S + 5 + 2 * s], iw = sm[a.S + 6 + 2 * s];
            const double m = im >= 0 ? prm[im] : 0.0, w = iw >= 0 ? fabs(prm[iw]) : 0.0;
            if (w > 0.0) {
                vf = normcdf((ed[J] - m) / w) - normcdf((ed[0] - m) / w);
                if (hi > lo) vw = normcdf((ed[hi] - m) / w) - normcdf((ed[lo] - m) / w);
            }
        } else {
            for (int q = a.tb->ds_tpl0[d]; q < a.tb->ds_tpl0[d] + a.tb->ds_ntpl[d]; ++q) {
                if (a.tpl_s[q] != s) continue;
                const double* h = a.tpl + a.tpl_off[q];
                for (int j = 0; j < J; ++j) { vf += h[j]; if (j >= lo && j < hi) vw += h[j]; }
            }
        }
        nwin[((long long)t * a.D + d) * a.S + s] = rf * vw;
        nfull[((long long)t * a.D + d) * a.S + s] = rf * vf;
    }
}

__global__ void k_window_scales(KArgs a, const double* nwin, const double* nfull, const double* scale,
                                double max_factor, double* out) {
    const int t = blockIdx.x;
    for (int p = threadIdx.x; p < a.P; p += blockDim.x) {
        double sw = 0.0, sf = 0.0;
        bool rate = false, other = false;
        for (int d = 0; d < a.D; ++d) {
            const int* sm = a.slot_map + (long long)d * a.NSLOT;
            for (int sl = 0; sl < a.NSLOT; ++sl) {
                if (sm[sl] != p) continue;
                if (sl < a.S) {
                    rate = true;
                    sw += nwin[((long long)t * a.D + d) * a.S + sl];
                    sf += nfull[((long long)t * a.D + d) * a.S + sl];
                } else {
                    other = true;
                }
            }
        }
        double f = 1.0;
        if (rate && !other && sf > 0.0) f = sw * max_factor * max_factor > sf ? sqrt(sf / sw) : max_factor;
        out[(long long)t * a.P + p] = scale[p] * fmin(fmax(f, 1.0), max_factor);
    }
}

cudaError_t launch_window_scales(const KArgs& a, double* nwin, double* nfull, const double* scale, double max_factor,
                                 double* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(nwin, 0, sizeof(double) * a.T * a.D * a.S, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(nfull, 0, sizeof(double) * a.T * a.D * a.S, st);
    if (e != cudaSuccess) return e;
    k_window_counts<<<a.T, WC_WARPS * 32, 0, st>>>(a, nwin, nfull);
    k_window_scales<<<a.T, 64, 0, st>>>(a, nwin, nfull, scale, max_factor, out);
    return cudaGetLastError();
}

cudaError_t launch_lbfgs(const FitArgs& f, cudaStream_t st) {
    k_lbfgs<<<(f.T + 3) / 4, 128, 0, st>>>(f);
    return cudaGetLastError();
}

}  // namespace gsn
