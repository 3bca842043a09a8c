// Profile-likelihood fits over rates only (section 4.2, the toy Monte Carlo discovery test).
//
// With the response parameters held, every species' expected counts are a fixed shape times its
// rate, so the expected counts of a toy are linear in the free rates theta:
//     mu_i = C_i + sum_f B_if theta_f        (bins i of the toy's windows, all datasets)
// with B_if the summed shapes of the species whose rate is the free parameter f (eps_d f_ds times
// the smeared shape sum_k R_ik S'_sk, the peak profile or the normalised template) and C_i the
// expected counts of the held species.  The NLL sum_i [mu_i - n_i + n_i ln(n_i / mu_i)] (+ pulls) is
// convex in theta, its Hessian H = sum_i n_i B_i B_i^T / mu_i^2 (+ 1/sigma^2 of pulled rates) is
// exact, and Newton's method converges in a few steps however strongly the rates are correlated.
//   k_rate_design  one thread per (toy, bin): the rows B_i, C_i over the whole histograms and the
//                  counts (n = -1 outside the toy's window); the smeared shapes come from the
//                  per-species kernel (Mbuf)
//   k_rate_newton  one block per toy: projected Newton iterations on the free rates held at their
//                  bounds when the gradient pushes outwards, feasible step length, Armijo
//                  backtracking on the exact NLL change sum_i [a dmu_i - n_i ln(1 + a dmu_i / mu_i)];
//                  stops when the Newton decrement g.H^-1.g / 2 (the estimated distance to the
//                  minimum) is below tol.  A free rate whose window share sum_win B_if / sum_all B_if
//                  is at most share_min stays at its start: its counts in the window come from the
//                  response tails the band truncates, and nothing there determines its rate
// mu, B.delta and the NLL are FP64; the gradient is accumulated in FP32 with compensation and the
// Hessian in FP32 within tiles of 32 bins and in FP64 across them: they steer the iteration, while
// the NLL and mu it reports are FP64 and are recomputed from the rates after every step.
#include "gsn_device.cuh"

namespace gsn {

namespace {

constexpr int RF_TB = 32;       // bins per shared-memory tile of B
constexpr int RF_THREADS = 256;

DEV int dataset_of_bin(const KArgs& a, int i) {
    int lo = 0, hi = a.D - 1;  // last dataset whose first bin is <= i
    while (lo < hi) {
        const int m = (lo + hi + 1) >> 1;
        if (tb_ds_off(a, m) <= i) lo = m; else hi = m - 1;
    }
    return lo;
}

}  // namespace

__global__ void __launch_bounds__(256) k_rate_design(KArgs a, RateArgs r) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, t = blockIdx.y;
    if (i >= a.total_bins) return;
    const int d = dataset_of_bin(a, i);
    const int j = i - tb_ds_off(a, d);
    const double* prm = a.params + (long long)t * a.params_stride;
    double* B = r.B + ((long long)t * a.total_bins + i) * r.nf;
    for (int f = 0; f < r.nf; ++f) B[f] = 0.0;
    double C = 0.0;
    const int lo = max(0, a.win[(long long)t * a.win_stride + 2 * d]);
    const int hi = min(tb_ds_bins(a, d), a.win[(long long)t * a.win_stride + 2 * d + 1]);
    const bool inside = j >= lo && j < hi;
    const int g = tb_ds_group(a, d);
    const double* ed = a.edges + tb_g_edge_off(a, g);
    const int* sm = a.slot_map + (long long)d * a.NSLOT;
    for (int s = 0; s < a.S; ++s) {
        const double fr = a.rfac[d * a.S + s];
        const int p = sm[s];
        if (fr == 0.0 || p < 0) continue;
        const int kind = a.ft.sp_kind[s];
        double shape = 0.0;
        if (kind < 2) {
            shape = a.Mbuf[(long long)t * a.mstride + ((long long)g * a.S + s) * a.Jmax + j];
        } else if (kind == 2) {
            const int pm = sm[a.S + 5 + 2 * s], pw = sm[a.S + 6 + 2 * s];
            if (pm >= 0 && pw >= 0) shape = ncdf_diff((ed[j] - prm[pm]) / prm[pw], (ed[j + 1] - prm[pm]) / prm[pw]);
        } else {
            for (int q = a.tb->ds_tpl0[d]; q < a.tb->ds_tpl0[d] + a.tb->ds_ntpl[d]; ++q)
                if (a.tpl_s[q] == s) shape += a.tpl[a.tpl_off[q] + j];
        }
        const int f = r.pfree[p];
        if (f >= 0) B[f] += fr * shape;
        else C += fr * shape * prm[p];
    }
    r.C[(long long)t * a.total_bins + i] = C;
    r.N[(long long)t * a.total_bins + i] = inside ? a.counts[(long long)t * a.counts_stride + i] : -1.0;
}

__global__ void __launch_bounds__(RF_THREADS) k_rate_newton(KArgs a, RateArgs r) {
    const int t = blockIdx.x, tid = threadIdx.x;
    const int nf = r.nf, NB = a.total_bins;
    constexpr int HPT = (RF_NFMAX * RF_NFMAX + RF_THREADS - 1) / RF_THREADS;  // Hessian entries per thread
    __shared__ double th[RF_NFMAX], dl[RF_NFMAX], gf[RF_NFMAX], sz[RF_NFMAX], red[RF_THREADS / 32];
    __shared__ double Hs[RF_NFMAX * RF_NFMAX];
    __shared__ double L[RF_NFMAX * RF_NFMAX];
    __shared__ float tile[RF_TB][RF_NFMAX];
    __shared__ float tw[RF_TB], tr[RF_TB];
    __shared__ int sact[RF_NFMAX], sok[RF_NFMAX], sheld[RF_NFMAX];
    __shared__ double s_nll, s_alpha, s_dec;
    __shared__ int s_state;  // 0 run, 1 converged, 2 line search failed, 3 non-finite
    double* prm = r.params + (long long)t * a.params_stride;
    const double* B = r.B + (long long)t * NB * nf;
    const double* C = r.C + (long long)t * NB;
    const double* N = r.N + (long long)t * NB;
    double* mu = r.mu + (long long)t * NB;
    double* dmu = r.dmu + (long long)t * NB;
    // pulls at theta + alpha delta: free rates add to the NLL, gradient and Hessian; held
    // parameters a constant
    auto pull_nll = [&](double alpha) {
        double v = 0.0;
        for (int k = 0; k < a.n_pulls; ++k) {
            const int p = a.pull_param[k], f = r.pfree[p];
            const double x = f >= 0 ? th[f] + alpha * dl[f] : prm[p];
            const double z = (x - a.pull_c[k]) / a.pull_w[k];
            v += 0.5 * z * z;
        }
        return v;
    };
    for (int f = tid; f < nf; f += blockDim.x) dl[f] = 0.0;
    for (int f = tid; f < nf; f += blockDim.x) th[f] = fmin(fmax(prm[r.fidx[f]], r.lo[f]), r.hi[f]);
    // window share of every free rate (fixed order: one block reduction per rate)
    for (int f = 0; f < nf; ++f) {
        double sw = 0.0, st = 0.0;
        for (int i = tid; i < NB; i += blockDim.x) {
            const double v = B[(long long)i * nf + f];
            st += v;
            if (N[i] >= 0.0) sw += v;
        }
        sw = block_sum_d(sw, red);
        st = block_sum_d(st, red);
        if (tid == 0) sheld[f] = !(sw > r.share_min * st);
        __syncthreads();
    }
    // mu at the start point (FP64) and the NLL
    double part = 0.0;
    bool bad = false;
    for (int i = tid; i < NB; i += blockDim.x) {
        const double n = N[i];
        if (n < 0.0) { mu[i] = 1.0; continue; }
        double m = C[i];
        for (int f = 0; f < nf; ++f) m = fma(B[(long long)i * nf + f], th[f], m);
        mu[i] = m;
        if (n > 0.0) { if (m > 0.0) part += m - n + n * log(n / m); else bad = true; }
        else part += m;
    }
    const int anybad = __syncthreads_or(bad);
    part = block_sum_d(part, red);
    if (tid == 0) { s_nll = part + pull_nll(0.0); s_state = anybad || !isfinite(s_nll) ? 3 : 0; }
    __syncthreads();
    int it = 0;
    for (; it < r.max_iter && s_state == 0; ++it) {
        // gradient (compensated FP32 per parameter) and Hessian (FP32), tiles of RF_TB bins
        const int ne = nf * nf;
        double hacc[HPT] = {};
        float gs = 0.f, gc = 0.f;
        for (int i0 = 0; i0 < NB; i0 += RF_TB) {
            const int nt = min(RF_TB, NB - i0);
            __syncthreads();
            for (int e = tid; e < nt * nf; e += blockDim.x) {
                const int ii = e / nf, f = e % nf;
                tile[ii][f] = (float)B[(long long)(i0 + ii) * nf + f];
            }
            for (int ii = tid; ii < nt; ii += blockDim.x) {
                const double n = N[i0 + ii], m = mu[i0 + ii];
                tw[ii] = n > 0.0 ? (float)(n / (m * m)) : 0.f;
                tr[ii] = n >= 0.0 ? (float)(1.0 - n / m) : 0.f;
            }
            __syncthreads();
            if (tid < nf) {
                float part32 = 0.f;
                for (int ii = 0; ii < nt; ++ii) part32 = fmaf(tr[ii], tile[ii][tid], part32);
                two_sum_acc(gs, gc, part32);
            }
#pragma unroll
            for (int m = 0; m < HPT; ++m) {
                const int e = tid + m * RF_THREADS;
                if (e < ne) {
                    const int p = e / nf, q = e % nf;
                    float h = 0.f;  // FP32 within a tile, FP64 across tiles
                    for (int ii = 0; ii < nt; ++ii) h = fmaf(tw[ii] * tile[ii][p], tile[ii][q], h);
                    hacc[m] += (double)h;
                }
            }
        }
        __syncthreads();
        if (tid < nf) gf[tid] = (double)gs + (double)gc;
#pragma unroll
        for (int m = 0; m < HPT; ++m) {
            const int e = tid + m * RF_THREADS;
            if (e < ne) Hs[e] = hacc[m];
        }
        __syncthreads();
        if (tid == 0) {
            for (int k = 0; k < a.n_pulls; ++k) {
                const int f = r.pfree[a.pull_param[k]];
                if (f < 0) continue;
                const double s2 = 1.0 / (a.pull_w[k] * a.pull_w[k]);
                gf[f] += (th[f] - a.pull_c[k]) * s2;
                Hs[f * nf + f] += s2;
            }
            // active set: free rates not held at a bound by their gradient, with information
            int na = 0;
            for (int f = 0; f < nf; ++f) {
                const bool held = (th[f] <= r.lo[f] && gf[f] > 0.0) || (th[f] >= r.hi[f] && gf[f] < 0.0);
                if (!held && !sheld[f] && Hs[f * nf + f] > 0.0) sact[na++] = f;
            }
            // Newton step on the active set: Cholesky of H_AA (FP64), pivots that vanish against
            // their diagonal drop the direction (no information along it); a rate at a bound whose
            // step points out of the feasible set leaves the active set and the step is redone
            for (int pass = 0; pass <= nf; ++pass) {
                for (int x = 0; x < na; ++x)
                    for (int y = 0; y <= x; ++y) L[x * na + y] = Hs[sact[x] * nf + sact[y]];
                for (int x = 0; x < na; ++x) {
                    double dgl = L[x * na + x];
                    for (int k = 0; k < x; ++k) if (sok[k]) dgl -= L[x * na + k] * L[x * na + k];
                    sok[x] = dgl > 1e-10 * Hs[sact[x] * nf + sact[x]];
                    const double piv = sok[x] ? sqrt(dgl) : 0.0;
                    L[x * na + x] = piv;
                    for (int y = x + 1; y < na; ++y) {
                        double v = Hs[sact[y] * nf + sact[x]];
                        for (int k = 0; k < x; ++k) if (sok[k]) v -= L[y * na + k] * L[x * na + k];
                        L[y * na + x] = sok[x] ? v / piv : 0.0;
                    }
                }
                for (int x = 0; x < na; ++x) {  // L z = -g
                    double v = -gf[sact[x]];
                    for (int k = 0; k < x; ++k) v -= L[x * na + k] * sz[k];
                    sz[x] = sok[x] ? v / L[x * na + x] : 0.0;
                }
                for (int f = 0; f < nf; ++f) dl[f] = 0.0;
                for (int x = na - 1; x >= 0; --x) {  // L^T delta = z
                    double v = sz[x];
                    for (int k = x + 1; k < na; ++k) v -= L[k * na + x] * dl[sact[k]];
                    dl[sact[x]] = sok[x] ? v / L[x * na + x] : 0.0;
                }
                int drop = -1;
                for (int x = 0; x < na && drop < 0; ++x) {
                    const int f = sact[x];
                    if ((th[f] <= r.lo[f] && dl[f] < 0.0) || (th[f] >= r.hi[f] && dl[f] > 0.0)) drop = x;
                }
                if (drop < 0) break;
                for (int x = drop; x + 1 < na; ++x) sact[x] = sact[x + 1];
                --na;
            }
            double dec = 0.0;
            for (int x = 0; x < na; ++x) dec -= gf[sact[x]] * dl[sact[x]];
            s_dec = dec;
            // longest feasible step along delta (at most 1)
            double amax = 1.0;
            for (int f = 0; f < nf; ++f) {
                if (dl[f] < 0.0 && th[f] + dl[f] < r.lo[f]) amax = fmin(amax, (r.lo[f] - th[f]) / dl[f]);
                if (dl[f] > 0.0 && th[f] + dl[f] > r.hi[f]) amax = fmin(amax, (r.hi[f] - th[f]) / dl[f]);
            }
            s_alpha = fmax(amax, 0.0);
            if (0.5 * dec < r.tol) s_state = 1;
            else if (!(dec > 0.0) || !(s_alpha > 0.0)) s_state = 1;  // no descent left within the bounds
        }
        __syncthreads();
        if (s_state != 0) break;
        // dmu = B delta (FP64: correlated rates take large steps whose terms cancel in B delta)
        for (int i = tid; i < NB; i += blockDim.x) {
            double d = 0.0;
            if (N[i] >= 0.0)
                for (int f = 0; f < nf; ++f) d = fma(B[(long long)i * nf + f], dl[f], d);
            dmu[i] = d;
        }
        __syncthreads();
        // backtracking on the exact NLL change (FP64)
        double alpha = s_alpha, gd = -s_dec;
        bool accepted = false;
        for (int bt = 0; bt < 40; ++bt) {
            double dn = 0.0;
            bool infeas = false;
            for (int i = tid; i < NB; i += blockDim.x) {
                const double n = N[i];
                if (n < 0.0) continue;
                const double d = alpha * dmu[i], m = mu[i];
                if (n > 0.0) {
                    if (m + d <= 0.0) infeas = true;
                    else dn += d - n * log1p(d / m);
                } else {
                    dn += d;
                }
            }
            const int any_inf = __syncthreads_or(infeas);
            dn = block_sum_d(dn, red);
            if (tid == 0) s_dec = dn + (a.n_pulls ? pull_nll(alpha) - pull_nll(0.0) : 0.0);  // the trial step's NLL change
            __syncthreads();
            const double dtot = s_dec;
            __syncthreads();
            if (!any_inf && isfinite(dtot) && dtot <= 1e-4 * alpha * gd + r.fnoise * fabs(s_nll)) {
                accepted = true;
                break;
            }
            alpha *= 0.5;
        }
        if (!accepted) {
            if (tid == 0) s_state = 2;
            __syncthreads();
            break;
        }
        // take the step: rates clamped onto their bounds, then mu recomputed from them (FP64), so
        // that mu and the NLL belong to the rates reported, with no drift over the iterations
        if (tid == 0) {
            for (int f = 0; f < nf; ++f) th[f] = fmin(fmax(th[f] + alpha * dl[f], r.lo[f]), r.hi[f]);
            s_nll += s_dec;
        }
        __syncthreads();
        for (int i = tid; i < NB; i += blockDim.x) {
            if (N[i] < 0.0) continue;
            double m = C[i];
            for (int f = 0; f < nf; ++f) m = fma(B[(long long)i * nf + f], th[f], m);
            mu[i] = m;
        }
        __syncthreads();
    }
    // results: the NLL from mu (FP64), the minimum, iterations and status
    part = 0.0;
    for (int i = tid; i < NB; i += blockDim.x) {
        const double n = N[i], m = mu[i];
        if (n < 0.0) continue;
        part += n > 0.0 ? m - n + n * log(n / m) : m;
    }
    part = block_sum_d(part, red);
    if (tid == 0) {
        for (int f = 0; f < nf; ++f) prm[r.fidx[f]] = th[f];
        const double v = part + pull_nll(0.0);
        r.nll[t] = v;
        if (r.iters) r.iters[t] = it;
        int st = s_state == 1 ? 0 : s_state == 0 ? 1 : s_state == 2 ? 2 : -4;
        if (!isfinite(v)) st = -4;
        if (r.status) r.status[t] = st;
    }
}

cudaError_t launch_rate_fit(const KArgs& a, const RateArgs& r, cudaStream_t st) {
    k_rate_design<<<dim3((a.total_bins + 255) / 256, a.T), 256, 0, st>>>(a, r);
    k_rate_newton<<<a.T, RF_THREADS, 0, st>>>(a, r);
    return cudaGetLastError();
}

}  // namespace gsn
