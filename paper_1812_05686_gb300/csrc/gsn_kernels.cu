// Kernels of the binned spectral-fit likelihood (GooStats, arXiv:1812.05686).
//
// One minimiser step for T parameter points ("toys") runs as
//   k_columns   per fine column k: visible mean mu_k (Birks quenching, section
//               2.3 reading), resolution, response band, rate-weighted spectra
//               T_dk = eps_d sum_s r_s S'_sk of each dataset (section 3.2)
//   k_forward   mu_dj = sum_k R_jk T_dk: the response bin integrals R_jk are
//               generated in registers and contracted at once (the
//               "response mesh" and "smearing convolution" of section 2.5 fused)
//   k_deviance  FP64 Poisson deviance of Eq. (LL) over a range of bins per block
//               (AnaPeak profiles added to mu), w_dj = 1 - n_dj / mu_dj for the adjoint
//   k_devfinal  fixed-order sum of the deviance partials, pulls, status, and the
//               closed-form AnaPeak gradient terms
//   k_backward  adjoint: per column, sums over the band of w-weighted response
//               values and their derivatives, then the chain rule to
//               (LY, kB, a, b, c) and S'^T u for the rates
//   k_gradfinal fixed-order sum of the per-task partial gradients and scatter
//               through the slot map (section 2.2 parameter synchronisation)
// Mixed precision: FP32 response build and contraction with double-float
// column means, FP32 partial sums flushed to FP64 per column block, FP64
// deviance and reductions.  FP64: everything in double.
#include "gsn_device.cuh"
#include "gsn_ggamma.cuh"

namespace gsn {

// ------------------------------------------------------------- columns -----
template <class R, int RES, bool FAST>
__global__ void __launch_bounds__(COLBLK) k_columns(KArgs a) {
    const int t = blockIdx.z, g = blockIdx.y;
    if (!tb_g_active<FAST>(a, g)) return;  // no smeared species in the group
    const int k = blockIdx.x * COLBLK + threadIdx.x;
    __shared__ double sres[NRESP];
    // eps_d r_s as an unevaluated pair (hi + lo): one rounding of eps_d r_s to FP32 would be
    // shared by every column and bin of the toy, a coherent bias of mu that does not average out
    __shared__ R srate[MAXGDS][MAXS], srate_lo[MAXGDS][MAXS];
    __shared__ float sdf[8];      // per-toy double-float constants (mixed)
    __shared__ R sred[2][COLBLK / 32];
    const double* prm = a.params + (long long)t * a.params_stride;
    if (threadIdx.x < NRESP) {
        const int q = tb_g_resp<FAST>(a, g, threadIdx.x);  // the power slot is unmapped unless RES == 2
        sres[threadIdx.x] = q >= 0 ? prm[q] * tb_g_rscale<FAST>(a, g, threadIdx.x) : 1.0;
    }
    for (int i = threadIdx.x; i < MAXGDS * a.S; i += blockDim.x) {
        const int dd = i / a.S, s = i % a.S;
        double v = 0.0;
        if (dd < tb_g_nds<FAST>(a, g)) {
            const int d = tb_g_ds<FAST>(a, g, dd);
            const double f = a.rfac[d * a.S + s];
            if (a.ft.sp_kind[s] < 2 && f != 0.0) {  // smeared species (Ana, AnaShift)
                const int p = a.slot_map[d * a.NSLOT + s];
                if (p >= 0) v = f * prm[p];
            }
        }
        srate[dd][s] = (R)v;
        srate_lo[dd][s] = (R)(v - (double)(R)v);
    }
    __syncthreads();
    const double LY = sres[0], kB = sres[1], ra = sres[2], rb = sres[3], rc = sres[4];
    const double alpha = 1.0 + kB * a.s0, beta = kB * a.s1;
    if (sizeof(R) == 4 && threadIdx.x == 0) {
        const double ia = 1.0 / alpha;
        sdf[0] = (float)ia; sdf[1] = (float)(ia - (double)(float)ia);
        sdf[2] = (float)LY; sdf[3] = (float)(LY - (double)(float)LY);
        sdf[4] = (float)(beta / (alpha * alpha));                 // beta / alpha^2
        sdf[5] = beta > 0 ? (float)(alpha / beta) : 0.0f;         // alpha / beta
        sdf[6] = (float)(a.s0 * beta / alpha);
        sdf[7] = (float)(1.0 / (alpha * alpha));
    }
    __syncthreads();

    R xmin = (R)INFINITY, xmax = (R)-INFINITY;
    if (k < a.K) {
        R* rec = colrec<R>(a, t, g, k);
        R f[NFP], z[NFZ];
#pragma unroll
        for (int i = 0; i < NFP; ++i) f[i] = 0;
#pragma unroll
        for (int i = 0; i < NFZ; ++i) z[i] = 0;
        R Nk = 1;
        if constexpr (RES == 2) {
            // generalized gamma: mean, variance and everything of the column in FP64
            const double E = a.E[k];
            double Eq = E / alpha, L = 0.0, y = 0.0;
            if (beta > 0) {
                y = alpha * E / beta;
                L = log1p(y);
                Eq = y < 1.0 ? -(beta / (alpha * alpha)) * (L - y) : E / alpha - (beta / (alpha * alpha)) * L;
            }
            const double mud = LY * Eq;
            const double vard = fma(mud, fma(rc, mud, rb), ra);
            const double D = L - y, r1 = y / (1.0 + y);
            f[F_DEQ] = (R)(beta > 0 ? (a.s0 * (beta / alpha) * (2.0 * D + y * r1) - a.s1 * (D + y * r1)) / (alpha * alpha) : NAN);
            f[F_MUH] = (R)mud;
            if constexpr (sizeof(R) == 4) f[F_MUL] = (R)(mud - (double)(R)mud);
            double gco[NFG];
            const double x1 = a.edges[tb_g_edge_off<FAST>(a, g) + 1];
            Nk = (R)gg_column<R>(mud, vard, sres[5], a.cut, x1, tb_g_zero<FAST>(a, g) != 0, sizeof(R) == 4, a.ex2_scale, f, z, gco,
                                 xmin, xmax);
            double* g2 = a.colbuf2 + (((long long)t * a.G + g) * a.K + k) * NFG;
#pragma unroll
            for (int i = 0; i < NFG; ++i) g2[i] = gco[i];
        } else {
            R mu, var, deq;
            if constexpr (sizeof(R) == 4) {
                // E_q = E/alpha - (beta/alpha^2) ln(1 + alpha E / beta), mean in double-float
                const float Eh = a.E_hi[k], El = a.E_lo[k];
                float qh, ql;
                df_mul(Eh, El, sdf[0], sdf[1], qh, ql);
                float Dy = 0.f, y = 0.f, Ly = 0.f;
                if (beta > 0) {
                    y = Eh * sdf[5];
                    Dy = log1pmx2_f(y, Ly);
                    if (y < 1.0f) { qh = -sdf[4] * Dy; ql = 0.f; }
                    else df_add(qh, ql, -sdf[4] * Ly, qh, ql);
                }
                float muh, mul;
                df_mul(qh, ql, sdf[2], sdf[3], muh, mul);
                f[F_MUH] = muh; f[F_MUL] = mul;
                mu = muh;
                // dE_q/dkB = (1/alpha^2) [ s0 (beta/alpha) (2 D + y r) - s1 (D + y r) ], r = y/(1+y);
                // for y >= 1 the same terms as 2 ln(1+y) - y (2 - r) and ln(1+y) - r (no cancellation)
                const float r1 = y / (1.0f + y);
                const float ta = y < 1.0f ? fmaf(2.0f, Dy, y * r1) : fmaf(2.0f, Ly, -y * (2.0f - r1));
                const float tb = y < 1.0f ? fmaf(y, r1, Dy) : Ly - r1;
                deq = beta > 0 ? sdf[7] * (sdf[6] * ta - (float)a.s1 * tb) : (float)NAN;
            } else {
                const double E = a.E[k];
                double Eq = E / alpha;
                double L = 0, y = 0;
                if (beta > 0) {
                    y = alpha * E / beta;
                    L = log1p(y);
                    Eq = y < 1.0 ? -(beta / (alpha * alpha)) * (L - y) : E / alpha - (beta / (alpha * alpha)) * L;
                }
                mu = LY * Eq;
                f[F_MUH] = mu;
                const double D = L - y, r1 = y / (1.0 + y);
                deq = beta > 0 ? (a.s0 * (beta / alpha) * (2.0 * D + y * r1) - a.s1 * (D + y * r1)) / (alpha * alpha) : NAN;
            }
            // in FP64 and rounded once: FP32 copies of a, b, c would scale every column's variance alike
            var = (R)fma((double)mu, fma(rc, (double)mu, rb), ra);
            f[F_DEQ] = deq;
            if constexpr (RES == 0) {
                const R sig = sqrt(var), isg = R(1) / sig;
                f[F_A] = isg;
                if constexpr (sizeof(R) == 4) Nk = fmaf(isg, a.norm_hi, isg * a.norm_lo);
                const R zc = sqrt(R(2) * (R)a.cut);
                xmin = mu - zc * sig;
                xmax = mu + zc * sig;
            } else {
                const R d = mu * mu / var, s = var / mu;
                if constexpr (sizeof(R) == 4) {
                    f[F_A] = 1.0f / mu;
                    f[F_B] = d;
                    f[F_C] = -1.0f / s;
                    // exponent offset XM: the log2 density at the mode t = -1/d over that at the
                    // mean, L2E ((d-1) ln(1 - 1/d) + 1) = L2E sum_k u^k / (k (k+1)), u = 1/d, from
                    // the FP32 shape the kernels use; the normalisation takes the factor 2^XM, so
                    // that values are unchanged
                    if (d >= 8.0f) {
                        // density at the mean: exp(-corr(d)) / (sigma sqrt(2 pi)), corr = Stirling remainder
                        const float id = 1.0f / d, id2 = id * id;
                        const float corr = id * (1.0f / 12 - id2 * (1.0f / 360 - id2 * (1.0f / 1260 - id2 * (1.0f / 1680))));
                        float m = fmaf(id, 1.0f / 72, 1.0f / 56);
                        m = fmaf(m, id, 1.0f / 42);
                        m = fmaf(m, id, 1.0f / 30);
                        m = fmaf(m, id, 1.0f / 20);
                        m = fmaf(m, id, 1.0f / 12);
                        m = fmaf(m, id, 1.0f / 6);
                        m = fmaf(m, id, 0.5f);
                        const float xm = mul_l2e(m * id);
                        f[F_XM] = xm;
                        // exp(y), |y| < 0.06, by its Taylor polynomial (remainder below 1e-12), and a
                        // correctly rounded 1/sigma: expf and rsqrtf go through SFU approximations
                        // whose errors vary slowly with the argument, and y and the variance vary
                        // slowly from column to column, so neighbouring columns would share the error
                        const float y = fmaf(xm, 0.69314718f, -corr);
                        float ey = fmaf(y, 1.0f / 720, 1.0f / 120);
                        ey = fmaf(ey, y, 1.0f / 24);
                        ey = fmaf(ey, y, 1.0f / 6);
                        ey = fmaf(ey, y, 0.5f);
                        ey = fmaf(ey, y, 1.0f);
                        ey = fmaf(ey, y, 1.0f);
                        const float nq = ey * (1.0f / sqrtf(var));
                        Nk = fmaf(nq, a.norm_hi, nq * a.norm_lo);
                        f[F_KAPPA] = 0.5f * id + id2 * (1.0f / 12 - id2 * (1.0f / 120 - id2 * (1.0f / 252 - id2 * (1.0f / 240))));
                    } else {
                        const double df = (double)d;
                        const float xm = df > 1.0 ? (float)(1.4426950408889634 * fma(df - 1.0, log1p(-1.0 / df), 1.0)) : 0.0f;
                        f[F_XM] = xm;
                        const double dd = (double)mu * (double)mu / (double)var, sd = (double)var / (double)mu;
                        Nk = (float)(exp((dd - 1.0) * log((double)mu) - (double)mu / sd - dd * log(sd) - lgamma(dd) +
                                         0.69314718055994531 * (double)xm) * a.ex2_scale);
                        f[F_KAPPA] = (float)(log(dd) - digamma_d(dd));
                    }
                } else {
                    f[F_A] = -d * log(s) - lgamma(d);
                    f[F_B] = d - 1.0;
                    f[F_C] = 1.0 / s;
                    f[F_KAPPA] = log(s) + digamma_d(d);
                }
                // conservative band from bounds on h(t) = (d-1) D(t) - t, x = mu (1 + t)
                const R c = (R)a.cut;
                R thi;
                if (d >= R(1)) {
                    const R bq = R(2) - R(2) * c;
                    thi = (-bq + sqrt(bq * bq + R(8) * c * (d + R(1)))) / (R(2) * (d + R(1)));
                } else {
                    thi = c / d;
                }
                // for d > 1, h + cut is concave: Newton steps from these outer bounds stay outside the band
                if (d > R(1)) {
                    for (int it = 0; it < 3; ++it) {
                        const R L1 = log1p(thi);
                        const R h = (d - R(1)) * (L1 - thi) - thi + c;
                        const R hp = -(d - R(1)) * thi / (R(1) + thi) - R(1);
                        thi = thi - h / hp;
                    }
                }
                xmax = mu * (R(1) + thi);
                xmin = 0;
                if (d > R(1)) {
                    R tlo = -(R(1) + sqrt(R(1) + R(2) * c * (d - R(1)))) / (d - R(1));
                    if (tlo > R(-1)) {
                        for (int it = 0; it < 3; ++it) {
                            const R L1 = log1p(tlo);
                            const R h = (d - R(1)) * (L1 - tlo) - tlo + c;
                            const R hp = -(d - R(1)) * tlo / (R(1) + tlo) - R(1);
                            tlo = fmax(tlo - h / hp, tlo);
                        }
                        xmin = mu * (R(1) + tlo);
                    }
                }
                if (tb_g_zero<FAST>(a, g)) {
                    const R x1 = (R)a.edges[tb_g_edge_off<FAST>(a, g) + 1];
                    if (xmin <= x1) {
                        R P, Pd, Ps2;
                        gamma_bin_zero<R>(d, s, x1, P, Pd, Ps2);
                        z[Z_P0] = P / Nk;
                        if constexpr (sizeof(R) == 4) {
                            // mixed adjoint: (mu/d) dP/dmu at fixed variance, s^2 dP/dvar at fixed mean
                            z[Z_P0D] = (R(2) * Pd - Ps2 / mu) / Nk;
                            z[Z_P0S] = (Ps2 / mu - Pd) / Nk;
                        } else {
                            z[Z_P0D] = Pd; z[Z_P0S] = Ps2;
                        }
                    }
                }
            }
        }  // RES 0 / 1
        f[F_N] = Nk;
        f[F_XMIN] = xmin;
        f[F_XMAX] = xmax;
        for (int dd = 0; dd < tb_g_nds<FAST>(a, g); ++dd) {
            if constexpr (sizeof(R) == 4) {
                // T = sum_s rate_s S'_sk as an unevaluated FP32 pair (Th + Tl): the products' and the
                // sums' rounding errors and the rates' and spectra's residuals go to Tl, and T N is
                // rounded once.  Where the spectra are constant over a range of columns (a flat or
                // shoulder species), a rounded T would repeat one rounding error in all of them;
                // the rounding of T N varies with N from column to column.
                float Th = 0.f, Tl = 0.f;
                for (int s = 0; s < a.S; ++s) {
                    const float sv = a.Sf[(long long)s * a.K + k], r = srate[dd][s];
                    const float p = r * sv;
                    Tl = fmaf(r, sv, -p) + Tl;
                    Tl = fmaf(srate_lo[dd][s], sv, Tl);
                    Tl = fmaf(r, a.Sf_lo[(long long)s * a.K + k], Tl);
                    two_sum_acc(Th, Tl, p);
                }
                f[F_TN0 + dd] = fmaf(Th, Nk, Tl * Nk);
            } else {
                R T = 0;
                for (int s = 0; s < a.S; ++s) T = fma(srate[dd][s], a.Sd[(long long)s * a.K + k], T);
                f[F_TN0 + dd] = T * Nk;
            }
        }
#pragma unroll
        for (int i = 0; i < NFP; ++i) rec[i] = f[i];
        if (a.zerobuf) {
            R* zr = zerorec<R>(a, t, g, k);
#pragma unroll
            for (int i = 0; i < NFZ; ++i) zr[i] = z[i];
        }
    }
    // band summary of this column block
    R mn = warp_min<R>(xmin), mx = warp_max<R>(xmax);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sred[0][w] = mn; sred[1][w] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < COLBLK / 32; ++i) { mn = fmin(mn, sred[0][i]); mx = fmax(mx, sred[1][i]); }
        R* b = reinterpret_cast<R*>(a.blkbuf) + (((long long)t * a.G + g) * a.nblk + blockIdx.x) * 2;
        b[0] = mn; b[1] = mx;
    }
}

// ------------------------------------------------------------- forward -----
template <class R, int RES, int NG>
DEV int forward_loop(const KArgs& a, int t, int g, int split, float xlo_w, float xhi_w, bool valid,
                     bool is_zero, const R* nodes, R xc, double* accd) {
    int ncol = 0;
    const int nds = tb_g_nds(a, g);
    const int kchunk = (a.K + a.nsplit - 1) / a.nsplit;
    const int k_beg = split * kchunk, k_end = min(a.K, k_beg + kchunk);
    const R* blk = reinterpret_cast<const R*>(a.blkbuf) + ((long long)t * a.G + g) * a.nblk * 2;
    R del[NG], lam[NG], wt[NG];
    [[maybe_unused]] GGSides sides{};
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            del[n] = nodes[n]; lam[n] = nodes[NGM_F + n]; wt[n] = valid ? nodes[2 * NGM_F + n] : R(0);
        }
        if constexpr (RES == 2 && NG == 3) {
            // the toy's power (the value every column record of the toy carries)
            const int q = tb_g_resp(a, g, 5);
            const float pw = (float)(a.params[(long long)t * a.params_stride + q] * tb_g_rscale(a, g, 5));
            sides = gg_sides(pw, lam);
        }
    } else {
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            del[n] = nodes[n]; lam[n] = nodes[NGM_D + n]; wt[n] = valid ? nodes[2 * NGM_D + n] : R(0);
        }
    }
    for (int b = k_beg / COLBLK; b * COLBLK < k_end; ++b) {
        if (blk[2 * b + 1] < (R)xlo_w || blk[2 * b] > (R)xhi_w) continue;
        // FP32: partial sums of up to 32 columns folded into compensated (s, cs) pairs
        R acc[MAXGDS] = {}, sacc[MAXGDS] = {}, cacc[MAXGDS] = {};
        const int kb = max(b * COLBLK, k_beg), ke = min((b + 1) * COLBLK, k_end);
        for (int k = kb; k < ke; ++k) {
            const R* c = colrec<R>(a, t, g, k);
            if (c[F_XMAX] < (R)xlo_w || c[F_XMIN] > (R)xhi_w) continue;
            ++ncol;
            R v;
            if constexpr (sizeof(R) == 4) {
                if constexpr (RES == 2 && NG == 3) v = gg_bin_value_f3(c, xc, lam, wt, sides);
                else if constexpr (RES == 2) v = gg_bin_value_f<NG>(c, xc, lam, wt);
                else v = bin_value_f<RES, NG>(c, xc, del, lam, wt);
                if (RES >= 1 && is_zero) v = valid ? zerorec<R>(a, t, g, k)[Z_P0] : 0.0f;
            } else {
                if constexpr (RES == 2) v = gg_bin_value_d<NG>(c, lam, wt);
                else v = bin_value_gamma_d<NG>(c, del, lam, wt);
                if (is_zero) v = valid ? zerorec<R>(a, t, g, k)[Z_P0] : 0.0;
            }
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd)
                if (dd < nds) acc[dd] = fma(v, c[F_TN0 + dd], acc[dd]);
            if constexpr (sizeof(R) == 4) {
                if ((k & 31) == 31) {
#pragma unroll
                    for (int dd = 0; dd < MAXGDS; ++dd) { two_sum_acc(sacc[dd], cacc[dd], acc[dd]); acc[dd] = 0; }
                }
            }
        }
#pragma unroll
        for (int dd = 0; dd < MAXGDS; ++dd) {
            if constexpr (sizeof(R) == 4) {
                two_sum_acc(sacc[dd], cacc[dd], acc[dd]);
                accd[dd] += (double)sacc[dd] + (double)cacc[dd];
            } else {
                accd[dd] += (double)acc[dd];
            }
        }
    }
    return ncol;
}

// statistics: (bin, column) pairs evaluated by a warp
DEV void count_work(const KArgs& a, int kind, bool lane_valid, long long n_other) {
    if (!a.work) return;
    const unsigned m = __ballot_sync(0xffffffffu, lane_valid);
    if ((threadIdx.x & 31) == 0 && n_other > 0)
        atomicAdd(&a.work[kind], (unsigned long long)n_other * (unsigned long long)__popc(m));
}

// lanes <-> bins (32 per warp), loop over the columns of the band.  The FP32 generalized gamma is
// held to 64 registers: four resident blocks per SM instead of three
template <class R, int RES>
__global__ void __launch_bounds__(FWD_WARPS * 32, (sizeof(R) == 4 && RES == 2) ? 4 : 1) k_forward(KArgs a) {
    const int tile = blockIdx.x, split = blockIdx.y;
    const int t = blockIdx.z / a.G, g = blockIdx.z % a.G;
    if (!tb_g_active(a, g)) return;  // no smeared species in the group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int wlo, whi;
    toy_window_union(a, t, g, wlo, whi);
    const int j0 = (tile * FWD_WARPS + warp) * 32;
    if (j0 >= whi || j0 + 32 <= wlo) return;
    const int j = j0 + lane;
    const bool valid = j >= wlo && j < whi;
    const int jr = min(max(j, wlo), whi - 1);
    const int nb = tb_g_node_off(a, g) + jr;
    const int jf = max(j0, wlo), jl = min(j0 + 31, whi - 1);
    const float xlo_w = (float)a.edges[tb_g_edge_off(a, g) + jf];
    const float xhi_w = (float)a.edges[tb_g_edge_off(a, g) + jl + 1];
    const unsigned char cls = a.bclass[nb];
    const bool low = __any_sync(0xffffffffu, cls != BIN_LIN);
    double accd[MAXGDS] = {};
    int ncol;
    if constexpr (sizeof(R) == 4) {
        const float* nodes = a.ntab_f + (long long)nb * 3 * NGM_F;
        const float xc = a.xc_f[nb];
        if (low) ncol = forward_loop<float, RES, NG_LOG_F>(a, t, g, split, xlo_w, xhi_w, valid, cls == BIN_ZERO, nodes, xc, accd);
        else     ncol = forward_loop<float, RES, NG_LIN_F>(a, t, g, split, xlo_w, xhi_w, valid, false, nodes, xc, accd);
    } else {
        const double* nodes = a.ntab_d + (long long)nb * 3 * NGM_D;
        if (low) ncol = forward_loop<double, RES, NG_LOG_D>(a, t, g, split, xlo_w, xhi_w, valid, cls == BIN_ZERO, nodes, 0.0, accd);
        else     ncol = forward_loop<double, RES, NG_LIN_D>(a, t, g, split, xlo_w, xhi_w, valid, false, nodes, 0.0, accd);
    }
    count_work(a, K_FORWARD, valid, ncol);
    if (valid) {
        double* out = a.mubuf + ((long long)t * a.nsplit + split) * a.total_bins;
        for (int dd = 0; dd < tb_g_nds(a, g); ++dd) out[tb_ds_off(a, tb_g_ds(a, g, dd)) + j] = accd[dd];
    }
}

// FP64 Gaussian: exact bin integrals from erfc at the edges.  Lanes <-> edges,
// 31 bins per warp; the upper edge of a bin comes from the next lane.
__global__ void __launch_bounds__(FWD_WARPS * 32) k_forward_gauss64(KArgs a) {
    const int tile = blockIdx.x, split = blockIdx.y;
    const int t = blockIdx.z / a.G, g = blockIdx.z % a.G;
    if (!tb_g_active(a, g)) return;  // no smeared species in the group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int wlo, whi;
    toy_window_union(a, t, g, wlo, whi);
    const int j0 = (tile * FWD_WARPS + warp) * 31;
    if (j0 >= whi || j0 + 31 <= wlo) return;
    const int J = tb_g_bins(a, g);
    const int j = j0 + lane;
    const bool valid = lane < 31 && j >= wlo && j < whi;
    const double xe = a.edges[tb_g_edge_off(a, g) + min(j, J)];
    const int jf = max(j0, wlo), jl = min(j0 + 30, whi - 1);
    const double xlo_w = a.edges[tb_g_edge_off(a, g) + jf], xhi_w = a.edges[tb_g_edge_off(a, g) + jl + 1];
    const int nds = tb_g_nds(a, g);
    const int kchunk = (a.K + a.nsplit - 1) / a.nsplit;
    const int k_beg = split * kchunk, k_end = min(a.K, k_beg + kchunk);
    const double* blk = reinterpret_cast<const double*>(a.blkbuf) + ((long long)t * a.G + g) * a.nblk * 2;
    double acc[MAXGDS] = {};
    int ncol = 0;
    for (int b = k_beg / COLBLK; b * COLBLK < k_end; ++b) {
        if (blk[2 * b + 1] < xlo_w || blk[2 * b] > xhi_w) continue;
        const int kb = max(b * COLBLK, k_beg), ke = min((b + 1) * COLBLK, k_end);
        for (int k = kb; k < ke; ++k) {
            const double* c = colrec<double>(a, t, g, k);
            if (c[F_XMAX] < xlo_w || c[F_XMIN] > xhi_w) continue;
            ++ncol;
            const double z = (xe - c[F_MUH]) * c[F_A];
            const bool up = z >= 0.0;
            const double q = 0.5 * erfc(fabs(z) * INV_SQRT2);
            const double q1 = __shfl_down_sync(0xffffffffu, q, 1);
            const bool up1 = __shfl_down_sync(0xffffffffu, (int)up, 1) != 0;
            double v = (up == up1) ? (up ? q - q1 : q1 - q) : 1.0 - q - q1;
            if (!valid) v = 0.0;
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd)
                if (dd < nds) acc[dd] = fma(v, c[F_TN0 + dd], acc[dd]);
        }
    }
    count_work(a, K_FORWARD, valid, ncol);
    if (valid) {
        double* out = a.mubuf + ((long long)t * a.nsplit + split) * a.total_bins;
        for (int dd = 0; dd < nds; ++dd) out[tb_ds_off(a, tb_g_ds(a, g, dd)) + j] = acc[dd];
    }
}

// ------------------------------------------------------------ deviance -----
// bins [lo, hi) of edges ed[0..J] whose content of N(x; m, w) exceeds exp(-cut) of its peak density
DEV void peak_bins(const double* ed, int J, double m, double w, double cut, int& lo, int& hi) {
    const double z = sqrt(2.0 * cut);
    const double xa = m - z * w, xb = m + z * w;
    int l = 0, h = J;
    while (l < h) { const int q = (l + h) >> 1; if (ed[q + 1] <= xa) l = q + 1; else h = q; }
    lo = l;
    l = 0; h = J;
    while (l < h) { const int q = (l + h) >> 1; if (ed[q] < xb) l = q + 1; else h = q; }
    hi = l;
}

// AnaPeak species of one dataset (at most MAXPK), with the bins their profile reaches;
// r holds eps_d f_ds times the rate
constexpr int MAXPK = 8;
struct PeakInfo {
    int s[MAXPK], lo[MAXPK], hi[MAXPK], n;
    double r[MAXPK], m[MAXPK], w[MAXPK];
};

// Called by the whole block with the same d; returns the number of peaks (pk untouched when the
// dataset has none, so no barrier is needed then).
DEV int load_peaks(const KArgs& a, const double* prm, int d, PeakInfo& pk) {
    if (a.tb->ds_npk[d] == 0) return 0;
    __syncthreads();  // earlier readers of pk are done
    if (threadIdx.x == 0) {
        const double* ed = a.edges + tb_g_edge_off(a, tb_ds_group(a, d));
        int np = 0;
        for (int s = 0; s < a.S && np < MAXPK; ++s) {
            const double f = a.rfac[d * a.S + s];
            if (a.ft.sp_kind[s] != 2 || f == 0.0) continue;
            const int pr = a.slot_map[d * a.NSLOT + s];
            pk.s[np] = s;
            pk.r[np] = pr >= 0 ? f * prm[pr] : 0.0;
            pk.m[np] = prm[a.slot_map[d * a.NSLOT + a.S + 5 + 2 * s]];
            pk.w[np] = prm[a.slot_map[d * a.NSLOT + a.S + 6 + 2 * s]];
            int lo, hi;
            peak_bins(ed, tb_ds_bins(a, d), pk.m[np], pk.w[np], a.cut, lo, hi);
            pk.lo[np] = lo; pk.hi[np] = hi;
            ++np;
        }
        pk.n = np;
    }
    __syncthreads();
    return pk.n;
}

// sum of the nsplit partial mu rows of one bin, in a fixed order (four interleaved accumulators)
DEV double sum_splits(const double* p, long long stride, int n) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int i = 0;
    for (; i + 4 <= n; i += 4) {
        s0 += p[i * stride]; s1 += p[(i + 1) * stride];
        s2 += p[(i + 2) * stride]; s3 += p[(i + 3) * stride];
    }
    for (; i < n; ++i) s0 += p[i * stride];
    return (s0 + s1) + (s2 + s3);
}

// Stage 1 of the deviance, grid (T, dev_chunks): every block takes one contiguous range of the
// concatenated bins of a toy, completes mu (split sum + AnaPeak profiles), writes
// w = 1 - n/mu for the adjoint and the block's partial sum of the Eq. (LL) terms and status flags.
template <class R>
__global__ void __launch_bounds__(256) k_deviance(KArgs a) {
    const int t = blockIdx.x, c = blockIdx.y;
    __shared__ double sh[32];
    __shared__ PeakInfo pk;
    __shared__ double tcoef[MAXS];    // eps_d f_ds r_s of the dataset's Monte Carlo templates
    __shared__ long long toff[MAXS];  // and the offsets of their histograms
    const double* prm = a.params + (long long)t * a.params_stride;
    const double* cnt = a.counts + (long long)t * a.counts_stride;
    R* wout = reinterpret_cast<R*>(a.wbuf) + (long long)t * a.total_bins;
    const int pstride = 2 + a.ntpl;
    double* dp = a.devpart + ((long long)t * a.dev_chunks + c) * pstride;
    for (int q = threadIdx.x; q < a.ntpl; q += blockDim.x) dp[2 + q] = 0.0;  // datasets outside the block
    const int chunk = (a.total_bins + a.dev_chunks - 1) / a.dev_chunks;
    const int b0 = c * chunk, b1 = min(a.total_bins, b0 + chunk);
    const long long sstride = a.total_bins;
    const double* mrow = a.mubuf + (long long)t * a.nsplit * a.total_bins;
    double part = 0.0;
    int bad_mu = 0, bad_fin = 0;
    for (int d = 0; d < a.D; ++d) {
        const int J = tb_ds_bins(a, d), off = tb_ds_off(a, d);
        const int j0 = max(0, b0 - off), j1 = min(J, b1 - off);
        if (j0 >= j1) continue;
        int lo = a.win[t * a.win_stride + 2 * d], hi = a.win[t * a.win_stride + 2 * d + 1];
        lo = max(lo, 0); hi = min(hi, J);
        const int npk = load_peaks(a, prm, d, pk);
        const int ntp = a.tb->ds_ntpl[d];
        if (ntp > 0) {
            __syncthreads();  // earlier readers of tcoef / toff are done
            for (int q = threadIdx.x; q < ntp; q += blockDim.x) {
                const int gq = a.tb->ds_tpl0[d] + q, s = a.tpl_s[gq];
                const int p = a.slot_map[d * a.NSLOT + s];
                tcoef[q] = p >= 0 ? a.rfac[d * a.S + s] * prm[p] : 0.0;
                toff[q] = a.tpl_off[gq];
            }
            __syncthreads();
        }
        const double* ed = a.edges + tb_g_edge_off(a, tb_ds_group(a, d));
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            double w = 0.0;
            if (j >= lo && j < hi) {
                double mu = tb_ds_resp(a, d) ? sum_splits(mrow + off + j, sstride, a.nsplit) : 0.0;
                for (int q = 0; q < npk; ++q) {
                    if (j < pk.lo[q] || j >= pk.hi[q]) continue;
                    const double m = pk.m[q], wd = pk.w[q];
                    mu += pk.r[q] * ncdf_diff((ed[j] - m) / wd, (ed[j + 1] - m) / wd);
                }
                for (int q = 0; q < ntp; ++q) mu = fma(tcoef[q], a.tpl[toff[q] + j], mu);
                const double n = cnt[off + j];
                double term;
                if (n > 0.0) {
                    if (!(mu > 0.0)) { bad_mu = 1; term = INFINITY; }
                    else term = mu - n + n * log(n / mu);
                } else {
                    term = mu;
                }
                if (!isfinite(mu)) bad_fin = 1;
                part += term;
                w = mu > 0.0 ? 1.0 - n / mu : 0.0;
            }
            wout[off + j] = (R)w;
        }
        // template rate gradients: this block's share of sum_j w_j T_j (w as the adjoint reads it)
        for (int q = 0; q < ntp; ++q) {
            double gpart = 0.0;
            for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
                const double wj = (double)wout[off + j];  // written above by this thread
                if (wj != 0.0) gpart = fma(wj, a.tpl[toff[q] + j], gpart);
            }
            gpart = block_sum_d(gpart, sh);
            if (threadIdx.x == 0) dp[2 + a.tb->ds_tpl0[d] + q] = gpart;
        }
    }
    const double sum = block_sum_d(part, sh);
    const int any_bad_mu = __syncthreads_or(bad_mu), any_bad_fin = __syncthreads_or(bad_fin);
    if (threadIdx.x == 0) {
        dp[0] = sum;
        dp[1] = (double)(any_bad_mu | (any_bad_fin << 1));
    }
}

// Stage 2, one block per toy: fixed-order sum of the stage-1 partials, pull terms, status, and
// the direct gradient terms (AnaPeak rate / position / width in closed form, pulls).
__global__ void __launch_bounds__(256) k_devfinal(KArgs a) {
    const int t = blockIdx.x;
    __shared__ double sh[32];
    __shared__ PeakInfo pk;
    const double* prm = a.params + (long long)t * a.params_stride;
    double* gdir = a.gdirect + (long long)t * a.P;
    if (a.want_grad)
        for (int p = threadIdx.x; p < a.P; p += blockDim.x) gdir[p] = 0.0;
    __syncthreads();  // gdir zeroed before thread 0 accumulates into it
    if (a.want_grad) {
        const float* wf = reinterpret_cast<const float*>(a.wbuf) + (long long)t * a.total_bins;
        const double* wd64 = reinterpret_cast<const double*>(a.wbuf) + (long long)t * a.total_bins;
        for (int d = 0; d < a.D; ++d) {
            const int npk = load_peaks(a, prm, d, pk);
            const int off = tb_ds_off(a, d);
            const double* ed = a.edges + tb_g_edge_off(a, tb_ds_group(a, d));
            for (int q = 0; q < npk; ++q) {
                const int s = pk.s[q];
                const double f = a.rfac[d * a.S + s];
                const int pr = a.slot_map[d * a.NSLOT + s];
                const int pm = a.slot_map[d * a.NSLOT + a.S + 5 + 2 * s];
                const int pw = a.slot_map[d * a.NSLOT + a.S + 6 + 2 * s];
                const double r = pk.r[q], m = pk.m[q], wd = pk.w[q];  // r = eps_d f_ds rate
                double gr = 0.0, gm = 0.0, gw = 0.0;
                for (int j = pk.lo[q] + threadIdx.x; j < pk.hi[q]; j += blockDim.x) {
                    const double wj = a.precision == 1 ? (double)wf[off + j] : wd64[off + j];
                    if (wj == 0.0) continue;
                    const double z0 = (ed[j] - m) / wd, z1 = (ed[j + 1] - m) / wd;
                    const double p0 = exp(-0.5 * z0 * z0) * INV_SQRT2PI, p1 = exp(-0.5 * z1 * z1) * INV_SQRT2PI;
                    gr += wj * ncdf_diff(z0, z1);
                    gm += wj * (-(p1 - p0) / wd);
                    gw += wj * (-(z1 * p1 - z0 * p0) / wd);
                }
                gr = block_sum_d(gr, sh);
                gm = block_sum_d(gm, sh);
                gw = block_sum_d(gw, sh);
                if (threadIdx.x == 0) {
                    if (pr >= 0) gdir[pr] += f * gr;
                    gdir[pm] += r * gm;
                    gdir[pw] += r * gw;
                }
            }
        }
    }
    if (threadIdx.x == 0) {
        const int pstride = 2 + a.ntpl;
        const double* dp = a.devpart + (long long)t * a.dev_chunks * pstride;
        double nll = 0.0;
        int flags = 0;
        for (int c = 0; c < a.dev_chunks; ++c) { nll += dp[pstride * c]; flags |= (int)dp[pstride * c + 1]; }
        if (a.want_grad && a.ntpl > 0) {
            // Monte Carlo template rates: d mu_dj / d r_s = eps_d f_ds T_dsj
            for (int d = 0; d < a.D; ++d)
                for (int q = 0; q < a.tb->ds_ntpl[d]; ++q) {
                    const int gq = a.tb->ds_tpl0[d] + q, s = a.tpl_s[gq];
                    const int p = a.slot_map[d * a.NSLOT + s];
                    if (p < 0) continue;
                    double g = 0.0;
                    for (int c = 0; c < a.dev_chunks; ++c) g += dp[pstride * c + 2 + gq];
                    gdir[p] += a.rfac[d * a.S + s] * g;
                }
        }
        // secondary-observable pieces (section 2.4): NLL, flags and slot gradients per dataset
        for (int i = 0; i < a.nsec; ++i) {
            const double* sp = a.secpart + ((long long)t * a.nsec + i) * (2 + a.NSLOT);
            nll += sp[0];
            flags |= (int)sp[1];
            if (a.want_grad) {
                const int d = a.sec_ds[i];
                for (int sl = 0; sl < a.NSLOT; ++sl) {
                    const int p = a.slot_map[d * a.NSLOT + sl];
                    if (p >= 0 && sp[2 + sl] != 0.0) gdir[p] += sp[2 + sl];
                }
            }
        }
        for (int i = 0; i < a.n_pulls; ++i) {
            const int p = a.pull_param[i];
            const double z = (prm[p] - a.pull_c[i]) / a.pull_w[i];
            nll += 0.5 * z * z;
            if (a.want_grad) gdir[p] += z / a.pull_w[i];
        }
        int st = 0;
        if (flags & 1) { st = -3; nll = INFINITY; }
        else if ((flags & 2) || !isfinite(nll)) st = -4;
        a.nll[t] = nll;
        if (a.status) a.status[t] = st;
    }
}

// ------------------------------------------------------------ backward -----
// lanes <-> columns; each warp sweeps the bins of its columns' band.  The FP32 generalized gamma is
// held to 64 registers (four resident blocks per SM instead of three)
template <class R, int RES>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && RES == 2) ? 4 : 1) k_backward(KArgs a) {
    const int task = blockIdx.x, g = blockIdx.y, t = blockIdx.z;
    if (!tb_g_active(a, g)) return;  // no smeared species in the group
    const int W = a.bw_warps;
    const int cbw = task / a.bw_bsplit, bsp = task % a.bw_bsplit;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kbase = cbw * W * 32;
    const int k = kbase + warp * 32 + lane;
    const bool kval = k < a.K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* su = reinterpret_cast<R*>(smem_raw);                        // [MAXGDS][W*32]
    double* sresp = reinterpret_cast<double*>(smem_raw + sizeof(R) * MAXGDS * W * 32 + 16);  // [W][NRESP]
    const int nds = tb_g_nds(a, g);
    const int J = tb_g_bins(a, g);
    const double* ed = a.edges + tb_g_edge_off(a, g);
    const double* prm = a.params + (long long)t * a.params_stride;
    const double LY = prm[tb_g_resp(a, g, 0)] * tb_g_rscale(a, g, 0);
    const double rb = prm[tb_g_resp(a, g, 3)] * tb_g_rscale(a, g, 3), rc = prm[tb_g_resp(a, g, 4)] * tb_g_rscale(a, g, 4);
    int wlo, whi;
    toy_window_union(a, t, g, wlo, whi);

    R c[NFP];
    {
        const R* cr = colrec<R>(a, t, g, kval ? k : a.K - 1);
#pragma unroll
        for (int i = 0; i < NFP; ++i) c[i] = cr[i];
    }
    const R xmn = warp_min<R>(kval ? c[F_XMIN] : (R)INFINITY);
    const R xmx = warp_max<R>(kval ? c[F_XMAX] : (R)-INFINITY);
    int ja = 0, jb = -1;
    if (xmx >= xmn) {
        // first bin whose upper edge exceeds xmn, last bin whose lower edge is below xmx
        int lo = 0, hi = J;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (ed[m + 1] <= (double)xmn) lo = m + 1; else hi = m; }
        ja = lo;
        lo = 0; hi = J;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (ed[m] < (double)xmx) lo = m + 1; else hi = m; }
        jb = lo - 1;
        ja = max(ja, wlo); jb = min(jb, whi - 1);
        const int len = jb - ja + 1;
        if (len > 0) {
            const int ch = (len + a.bw_bsplit - 1) / a.bw_bsplit;
            const int na = ja + bsp * ch;
            jb = min(jb, na + ch - 1);
            ja = na;
        }
    }
    const R* wv[MAXGDS];
    for (int dd = 0; dd < MAXGDS; ++dd)
        wv[dd] = reinterpret_cast<const R*>(a.wbuf) + (long long)t * a.total_bins + tb_ds_off(a, tb_g_ds(a, g, dd < nds ? dd : 0));
    // secondary pieces: bin j of slice q adds U_qk N_k to the pair's weight (per dataset of the group)
    const R* secU = a.nsec ? reinterpret_cast<const R*>(a.secU) + (long long)t * a.Qtot * a.K : nullptr;
    auto sec_weight = [&](int j) -> R {
        R u = 0;
        if (secU && kval)
            for (int dd = 0; dd < nds; ++dd) {
                const int q = a.sec_slice[tb_ds_off(a, tb_g_ds(a, g, dd)) + j];
                if (q >= 0) u += secU[(long long)q * a.K + k];
            }
        return u * c[F_N];
    };
    R U0[MAXGDS] = {};
    R U1 = 0, U2 = 0;
    // generalized gamma: W-weighted node sums (rho, S1, S2, S3; compensated in FP32) and the W of
    // the bin at zero, mapped to the mean / variance / power derivatives by the adjoint record
    R Gs[4] = {0, 0, 0, 0}, Gc[4] = {0, 0, 0, 0}, Z0 = 0, U0c[MAXGDS] = {};
    const int nbase = tb_g_node_off(a, g);
    if constexpr (RES == 2) {
        const R p = c[F_KAPPA];
        // FP32, linear bins: side-node terms Q(e), E1(e), e = p ln(x_n/x_c), of the bins of the
        // current 32-bin batch, one bin per lane, handed to every lane by shuffle (the lanes share
        // the toy and so p); the nodes then follow from the centre by the addition formula.  FP32
        // sums run plain within a batch and are folded into the compensated accumulators at its end.
        [[maybe_unused]] float sQ0 = 0.f, sE0 = 0.f, sQ2 = 0.f, sE2 = 0.f;
        [[maybe_unused]] float bG[4] = {0.f, 0.f, 0.f, 0.f}, bU[MAXGDS] = {};
        for (int j = ja; j <= jb; ++j) {
            if constexpr (sizeof(R) == 4) {
                if (((j - ja) & 31) == 0) {
                    const int jj = j + (threadIdx.x & 31);
                    sQ0 = sE0 = sQ2 = sE2 = 0.f;
                    if (jj <= jb && a.bclass[nbase + jj] == BIN_LIN) {
                        const float* ndj = a.ntab_f + (long long)(nbase + jj) * 3 * NGM_F;
                        sQ0 = gg_q2f(p * (ndj[NGM_F] - ndj[NGM_F + 1]), sE0);
                        sQ2 = gg_q2f(p * (ndj[NGM_F + 2] - ndj[NGM_F + 1]), sE2);
                    }
                }
            }
            R wj[MAXGDS];
            R Wj = 0;
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd) {
                wj[dd] = dd < nds ? wv[dd][j] : R(0);
                Wj = fma(wj[dd], c[F_TN0 + dd], Wj);
            }
            if (secU) Wj += sec_weight(j);
            const unsigned char cls = a.bclass[nbase + j];
            R rho = 0;
            if (cls == BIN_ZERO) {
                rho = zerorec<R>(a, t, g, kval ? k : a.K - 1)[Z_P0];
                Z0 += Wj;
            } else {
                R s1 = 0, s2 = 0, s3 = 0;
                if constexpr (sizeof(R) == 4) {
                    const float* nd = a.ntab_f + (long long)(nbase + j) * 3 * NGM_F;
                    const float Dx = (a.xc_f[nbase + j] - c[F_MUH]) - c[F_MUL];
                    float Lc;
                    log1pmx2_f(Dx * c[F_A], Lc);
                    if (cls == BIN_LIN) {
                        const int src = (j - ja) & 31;
                        const float Q0 = __shfl_sync(0xffffffffu, sQ0, src), E0 = __shfl_sync(0xffffffffu, sE0, src);
                        const float Q2 = __shfl_sync(0xffffffffu, sQ2, src), E2 = __shfl_sync(0xffffffffu, sE2, src);
                        const float L1 = Lc + nd[NGM_F + 1];
                        float e1;
                        const float Qc = gg_q2f(p * L1, e1);
                        const float Ln[3] = {L1 + (nd[NGM_F] - nd[NGM_F + 1]), L1, L1 + (nd[NGM_F + 2] - nd[NGM_F + 1])};
                        const float Qn[3] = {fmaf(e1, E0, Qc + Q0), Qc, fmaf(e1, E2, Qc + Q2)};
                        const float En[3] = {fmaf(e1, E0, e1 + E0), e1, fmaf(e1, E2, e1 + E2)};
#pragma unroll
                        for (int n = 0; n < 3; ++n) {
                            const float fw = nd[2 * NGM_F + n] * ex2f(fmaf(-c[F_B], Qn[n], c[F_C] * Ln[n]));
                            rho += fw; s1 = fmaf(fw, Ln[n], s1); s2 = fmaf(fw, Qn[n], s2); s3 = fmaf(fw * En[n], Ln[n], s3);
                        }
                    } else {
                        for (int n = 0; n < NG_LOG_F; ++n) {
                            const float L = Lc + nd[NGM_F + n];
                            float e1;
                            const float Q = gg_q2f(p * L, e1);
                            const float fw = nd[2 * NGM_F + n] * ex2f(fmaf(-c[F_B], Q, c[F_C] * L));
                            rho += fw; s1 = fmaf(fw, L, s1); s2 = fmaf(fw, Q, s2); s3 = fmaf(fw * e1, L, s3);
                        }
                    }
                } else {
                    const double* nd = a.ntab_d + (long long)(nbase + j) * 3 * NGM_D;
                    const int NG = cls == BIN_LOG ? NG_LOG_D : NG_LIN_D;
                    for (int n = 0; n < NG; ++n) {
                        const double l = nd[NGM_D + n] - c[F_C];   // ln(x/s)
                        const double y = exp(p * l);
                        const double fw = nd[2 * NGM_D + n] * exp(fma(c[F_B], nd[NGM_D + n], c[F_A]) - y);
                        rho += fw; s1 = fma(fw, l, s1); s2 = fma(fw, y, s2); s3 = fma(fw * y, l, s3);
                    }
                }
                if constexpr (sizeof(R) == 4) {
                    bG[0] = fmaf(Wj, rho, bG[0]); bG[1] = fmaf(Wj, s1, bG[1]);
                    bG[2] = fmaf(Wj, s2, bG[2]); bG[3] = fmaf(Wj, s3, bG[3]);
                } else {
                    Gs[0] += Wj * rho; Gs[1] += Wj * s1; Gs[2] += Wj * s2; Gs[3] += Wj * s3;
                }
            }
            if constexpr (sizeof(R) == 4) {
#pragma unroll
                for (int dd = 0; dd < MAXGDS; ++dd)
                    if (dd < nds) bU[dd] = fmaf(wj[dd], rho, bU[dd]);
                if (((j - ja) & 31) == 31 || j == jb) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) { two_sum_acc(Gs[i], Gc[i], bG[i]); bG[i] = 0.f; }
#pragma unroll
                    for (int dd = 0; dd < MAXGDS; ++dd) { two_sum_acc(U0[dd], U0c[dd], bU[dd]); bU[dd] = 0.f; }
                }
            } else {
#pragma unroll
                for (int dd = 0; dd < MAXGDS; ++dd) U0[dd] = fma(wj[dd], rho, U0[dd]);
            }
        }
    } else if constexpr (sizeof(R) == 8 && RES == 0) {
        // exact Gaussian bin integrals from the edges, derivatives from the edge densities
        const double mu = c[F_MUH], isg = c[F_A];
        double zp = 0, qp = 0, pp = 0;
        bool upp = false;
        for (int e = ja; e <= jb + 1; ++e) {
            const double z = (ed[e] - mu) * isg;
            const bool up = z >= 0.0;
            const double q = 0.5 * erfc(fabs(z) * INV_SQRT2);
            const double ph = exp(-0.5 * z * z) * INV_SQRT2PI;
            if (e > ja) {
                const int j = e - 1;
                const double Rv = (up == upp) ? (upp ? qp - q : q - qp) : 1.0 - qp - q;
                double Wj = 0.0;
#pragma unroll
                for (int dd = 0; dd < MAXGDS; ++dd)
                    if (dd < nds) { const double w = wv[dd][j]; U0[dd] = fma(w, Rv, U0[dd]); Wj = fma(w, c[F_TN0 + dd], Wj); }
                if (secU) Wj += sec_weight(j);
                // d R / d mu = U1 / sigma, d R / d sigma = U2 / sigma (applied per column below)
                U1 = fma(Wj, -(ph - pp), U1);
                U2 = fma(Wj, -(z * ph - zp * pp), U2);
            }
            zp = z; qp = q; pp = ph; upp = up;
        }
    } else {
        for (int j = ja; j <= jb; ++j) {
            R wj[MAXGDS];
            R Wj = 0;
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd) {
                wj[dd] = dd < nds ? wv[dd][j] : R(0);
                Wj = fma(wj[dd], c[F_TN0 + dd], Wj);
            }
            if (secU) Wj += sec_weight(j);
            const unsigned char cls = a.bclass[nbase + j];
            R rho = 0;
            if (RES == 1 && cls == BIN_ZERO) {
                const R* zr = zerorec<R>(a, t, g, kval ? k : a.K - 1);
                rho = zr[Z_P0];
                U1 = fma(Wj, zr[Z_P0D], U1);
                U2 = fma(Wj, zr[Z_P0S], U2);
            } else if constexpr (sizeof(R) == 4) {
                const float* nd = a.ntab_f + (long long)(nbase + j) * 3 * NGM_F;
                const float Dx = (a.xc_f[nbase + j] - c[F_MUH]) - c[F_MUL];
                const int NG = cls == BIN_LOG ? NG_LOG_F : NG_LIN_F;
                if constexpr (RES == 0) {
                    const float z = Dx * c[F_A];
                    float Z1 = 0.f, Z2 = 0.f;
                    for (int n = 0; n < NG; ++n) {
                        const float zn = fmaf(nd[n], c[F_A], z);
                        const float qn = zn * zn;
                        const float fw = nd[2 * NGM_F + n] * ex2f(-fmaf(0.5f * L2E, qn, qn * HALF_L2E_LO));
                        rho += fw; Z1 = fmaf(fw, zn, Z1); Z2 = fmaf(fw, fmaf(zn, zn, -1.0f), Z2);
                    }
                    U1 = fmaf(Wj, Z1, U1);
                    U2 = fmaf(Wj, Z2, U2);
                } else {
                    // the mixed gamma record (B = d, C = -1/s, KAPPA = ln d - psi(d)): sums of
                    // (mu/d) d ln f/d mu at fixed variance and s^2 d ln f/d var at fixed mean per node
                    const float A = c[F_A];
                    const float tt = Dx * A;
                    float L1;
                    const float Dt = log1pmx2_f(tt, L1);
                    const float P2 = mul_l2e(c[F_B]), Q2 = fmaf(L2E, c[F_B], fmaf(L2E_LO, c[F_B] - 1.0f, -L2E));
                    const float R2 = mul_l2e(c[F_C]);
                    const float Ec = fmaf(P2, Dt, fmaf(-L2E, L1, -c[F_XM]));
                    const float kap = c[F_KAPPA];
                    float u1 = 0.f, u2 = 0.f;
                    for (int n = 0; n < NG; ++n) {
                        const float fw = nd[2 * NGM_F + n] * ex2f(Ec + fmaf(R2, nd[n], Q2 * nd[NGM_F + n]));
                        const float L1n = L1 + nd[NGM_F + n];
                        const float tn = fmaf(nd[n], A, tt);
                        rho += fw;
                        u1 = fmaf(fw, fmaf(2.0f, L1n + kap, -tn), u1);
                        u2 = fmaf(fw, -((L1n - tn) + kap), u2);
                    }
                    U1 = fmaf(Wj, u1, U1);
                    U2 = fmaf(Wj, u2, U2);
                }
            } else {
                // FP64 gamma: f = exp((d-1) ln x - x/s + A); df/dd = f (ln x - ln s - psi(d)); df/ds = f (x - mu)/s^2
                const double* nd = a.ntab_d + (long long)(nbase + j) * 3 * NGM_D;
                const int NG = cls == BIN_LOG ? NG_LOG_D : NG_LIN_D;
                double L = 0.0, X = 0.0;
                for (int n = 0; n < NG; ++n) {
                    const double fw = nd[2 * NGM_D + n] * exp(fma(c[F_B], nd[NGM_D + n], fma(-c[F_C], nd[n], c[F_A])));
                    rho += fw; L = fma(fw, nd[NGM_D + n] - c[F_KAPPA], L); X = fma(fw, nd[n] - c[F_MUH], X);
                }
                U1 = fma(Wj, L, U1);
                U2 = fma(Wj, X, U2);
            }
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd) U0[dd] = fma(wj[dd], rho, U0[dd]);
        }
    }
    count_work(a, K_BACKWARD, kval, (long long)(jb - ja + 1));
    // chain rule per column
    R r[NRESP] = {};
    if (kval) {
        const R mu = sizeof(R) == 4 ? c[F_MUH] + c[F_MUL] : c[F_MUH];
        R g_mu, g_var;
        if constexpr (RES == 2) {
            // FP64 combination of the (compensated) sums with the FP64 coefficients
            const double* g2 = a.colbuf2 + (((long long)t * a.G + g) * a.K + k) * NFG;
            const double U[5] = {(double)Gs[0] + (double)Gc[0], (double)Gs[1] + (double)Gc[1],
                                 (double)Gs[2] + (double)Gc[2], (double)Gs[3] + (double)Gc[3], (double)Z0};
            double gm = 0.0, gv = 0.0, gp = 0.0;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                gm = fma(g2[FG_MU + i], U[i], gm);
                gv = fma(g2[FG_VAR + i], U[i], gv);
                gp = fma(g2[FG_P + i], U[i], gp);
            }
            g_mu = (R)gm; g_var = (R)gv;
            r[5] = (R)gp;
        } else if constexpr (RES == 0) {
            g_mu = U1 * c[F_A];
            g_var = R(0.5) * U2 * c[F_A] * c[F_A];
        } else if constexpr (sizeof(R) == 4) {
            g_mu = U1 * (c[F_B] * c[F_A]);     // (d / mu) U1
            g_var = U2 * (c[F_C] * c[F_C]);    // U2 / s^2
        } else {
            // fp64: C = 1/s, d = mu / s
            const R d = sizeof(R) == 4 ? c[F_B] : mu * c[F_C];
            const R s = sizeof(R) == 4 ? R(-1) / c[F_C] : R(1) / c[F_C];
            const R var = d * s * s;
            const R gd = U1, gs = U2 * c[F_C] * c[F_C];
            g_mu = gd * (R(2) * d / mu) - gs * (s / mu);
            g_var = -gd * (d / var) + gs / mu;
        }
        const R g_mt = g_mu + g_var * ((R)rb + R(2) * (R)rc * mu);
        r[0] = g_mt * (mu / (R)LY);
        r[1] = g_mt * (R)LY * c[F_DEQ];
        r[2] = g_var;
        r[3] = g_var * mu;
        r[4] = g_var * mu * mu;
    }
    // per-column terms of opposite signs cancel in these sums: compensated in FP32
#pragma unroll
    for (int i = 0; i < NRESP; ++i) {
        R v;
        if constexpr (sizeof(R) == 4) v = warp_sum_comp(r[i], 0.f);
        else v = warp_sum<R>(r[i]);
        if (lane == 0) sresp[warp * NRESP + i] = (double)v;
    }
    for (int dd = 0; dd < MAXGDS; ++dd) su[dd * W * 32 + warp * 32 + lane] = kval ? (U0[dd] + U0c[dd]) * c[F_N] : R(0);
    __syncthreads();
    double* part = a.partbuf + (((long long)t * a.G + g) * a.nbtask + task) * a.NPART;
    if (threadIdx.x < NRESP) {
        double s = 0.0;
        for (int w = 0; w < W; ++w) s += sresp[w * NRESP + threadIdx.x];
        part[threadIdx.x] = s;
    }
    const int ncol = min(W * 32, a.K - kbase);
    for (int i = threadIdx.x; i < MAXGDS * a.S; i += blockDim.x) {
        const int dd = i / a.S, s = i % a.S;
        double v = 0.0;
        if (dd < nds && a.ft.sp_kind[s] < 2 && a.rfac[tb_g_ds(a, g, dd) * a.S + s] != 0.0) {
            R acc = 0;
            if constexpr (sizeof(R) == 4) {
                // blocks of 32 columns folded into a compensated sum
                const float* Srow = a.Sf + (long long)s * a.K + kbase;
                float cmp = 0.f, part32 = 0.f;
                for (int cc = 0; cc < ncol; ++cc) {
                    part32 = fmaf(Srow[cc], su[dd * W * 32 + cc], part32);
                    if ((cc & 31) == 31) { two_sum_acc(acc, cmp, part32); part32 = 0.f; }
                }
                two_sum_acc(acc, cmp, part32);
                acc += cmp;
            } else {
                const double* Srow = a.Sd + (long long)s * a.K + kbase;
                for (int cc = 0; cc < ncol; ++cc) acc = fma(Srow[cc], su[dd * W * 32 + cc], acc);
            }
            v = (double)acc;
        }
        part[NRESP + i] = v;
    }
}

// ------------------------------------------------------------ gradfinal ----
__global__ void __launch_bounds__(128) k_gradfinal(KArgs a) {
    const int t = blockIdx.x;
    __shared__ double vals[NRESP + MAXGDS * MAXS];  // one group's reduced partials
    double* gr = a.grad + (long long)t * a.P;
    if (threadIdx.x == 0) {
        const double* gd = a.gdirect + (long long)t * a.P;
        for (int p = 0; p < a.P; ++p) gr[p] = gd[p];
    }
    // group by group (fixed order): sum of the per-task partials, then the slot-map scatter
    for (int g = 0; g < a.G; ++g) {
        if (!tb_g_active(a, g)) continue;  // no adjoint partials for groups without smeared species
        for (int v = threadIdx.x; v < a.NPART; v += blockDim.x) {
            const double* p = a.partbuf + ((long long)t * a.G + g) * a.nbtask * a.NPART + v;
            double s = 0.0;
            for (int task = 0; task < a.nbtask; ++task) s += p[(long long)task * a.NPART];
            vals[v] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            // the slots hold unscaled parameters: d(scale p)/dp = scale
            for (int i = 0; i < NRESP; ++i)
                if (tb_g_resp(a, g, i) >= 0) gr[tb_g_resp(a, g, i)] += vals[i] * tb_g_rscale(a, g, i);
            for (int dd = 0; dd < tb_g_nds(a, g); ++dd) {
                const int d = tb_g_ds(a, g, dd);
                for (int s = 0; s < a.S; ++s) {
                    const double f = a.rfac[d * a.S + s];
                    if (a.ft.sp_kind[s] >= 2 || f == 0.0) continue;
                    const int p = a.slot_map[d * a.NSLOT + s];
                    if (p >= 0) gr[p] += f * vals[NRESP + dd * a.S + s];
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bool fin = true;
        for (int p = 0; p < a.P; ++p) fin = fin && isfinite(gr[p]);
        if (!fin && a.status && a.status[t] == 0) a.status[t] = -4;
    }
}

// ---------------------------------------------------- per-species path -----
// M[g][s][j] = sum_k R_jk S'_sk for species s in [sp_first, sp_first + sp_count)
template <class R, int RES, int NG>
DEV void species_loop(const KArgs& a, int t, int g, float xlo_w, float xhi_w, bool valid, bool is_zero,
                      const R* nodes, R xc, double* accd, int nsp) {
    R del[NG], lam[NG], wt[NG];
    constexpr int NGM = sizeof(R) == 4 ? NGM_F : NGM_D;
#pragma unroll
    for (int n = 0; n < NG; ++n) { del[n] = nodes[n]; lam[n] = nodes[NGM + n]; wt[n] = valid ? nodes[2 * NGM + n] : R(0); }
    const R* blk = reinterpret_cast<const R*>(a.blkbuf) + ((long long)t * a.G + g) * a.nblk * 2;
    for (int b = 0; b < a.nblk; ++b) {
        if (blk[2 * b + 1] < (R)xlo_w || blk[2 * b] > (R)xhi_w) continue;
        R acc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] = 0;
        const int kb = b * COLBLK, ke = min(a.K, kb + COLBLK);
        for (int k = kb; k < ke; ++k) {
            const R* c = colrec<R>(a, t, g, k);
            if (c[F_XMAX] < (R)xlo_w || c[F_XMIN] > (R)xhi_w) continue;
            R v;
            if constexpr (sizeof(R) == 4) {
                if constexpr (RES == 2) v = gg_bin_value_f<NG>(c, xc, lam, wt);
                else v = bin_value_f<RES, NG>(c, xc, del, lam, wt);
                if (RES >= 1 && is_zero) v = valid ? zerorec<R>(a, t, g, k)[Z_P0] : 0.0f;
            } else {
                if constexpr (RES == 2) v = gg_bin_value_d<NG>(c, lam, wt);
                else v = bin_value_gamma_d<NG>(c, del, lam, wt);
                if (is_zero) v = valid ? zerorec<R>(a, t, g, k)[Z_P0] : 0.0;
            }
            v *= c[F_N];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (i < nsp) {
                    const R sv = sizeof(R) == 4 ? (R)a.Sf[(long long)(a.sp_first + i) * a.K + k]
                                                : (R)a.Sd[(long long)(a.sp_first + i) * a.K + k];
                    acc[i] = fma(v, sv, acc[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) accd[i] += (double)acc[i];
    }
}

// grid (bin tiles, groups, toys x species chunks of 16): M[t][g][s][j] (toy stride a.mstride)
template <class R, int RES>
__global__ void __launch_bounds__(FWD_WARPS * 32) k_species(KArgs a) {
    const int tile = blockIdx.x, g = blockIdx.y;
    const int nchunk = (a.sp_count + 15) / 16, t = blockIdx.z / nchunk, chunk = blockIdx.z % nchunk;
    if (!tb_g_active(a, g)) return;  // no smeared species in the group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int J = tb_g_bins(a, g);
    const int j0 = (tile * FWD_WARPS + warp) * 32;
    if (j0 >= J) return;
    const int j = j0 + lane;
    const bool valid = j < J;
    const int jr = min(j, J - 1);
    const int nb = tb_g_node_off(a, g) + jr;
    const int jl = min(j0 + 31, J - 1);
    const float xlo_w = (float)a.edges[tb_g_edge_off(a, g) + j0];
    const float xhi_w = (float)a.edges[tb_g_edge_off(a, g) + jl + 1];
    const unsigned char cls = a.bclass[nb];
    const bool low = __any_sync(0xffffffffu, cls != BIN_LIN);
    const int nsp = min(16, a.sp_count - chunk * 16);
    KArgs b = a;
    b.sp_first = a.sp_first + chunk * 16;
    double accd[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) accd[i] = 0.0;
    if constexpr (sizeof(R) == 4) {
        const float* nodes = a.ntab_f + (long long)nb * 3 * NGM_F;
        const float xc = a.xc_f[nb];
        if (low) species_loop<float, RES, NG_LOG_F>(b, t, g, xlo_w, xhi_w, valid, cls == BIN_ZERO, nodes, xc, accd, nsp);
        else     species_loop<float, RES, NG_LIN_F>(b, t, g, xlo_w, xhi_w, valid, false, nodes, xc, accd, nsp);
    } else {
        const double* nodes = a.ntab_d + (long long)nb * 3 * NGM_D;
        if (low) species_loop<double, RES, NG_LOG_D>(b, t, g, xlo_w, xhi_w, valid, cls == BIN_ZERO, nodes, 0.0, accd, nsp);
        else     species_loop<double, RES, NG_LIN_D>(b, t, g, xlo_w, xhi_w, valid, false, nodes, 0.0, accd, nsp);
    }
    if (valid)
        for (int i = 0; i < nsp; ++i) a.Mbuf[(long long)t * a.mstride + ((long long)g * a.S + b.sp_first + i) * a.Jmax + j] = accd[i];
}

// FP64 Gaussian per-species path: exact erfc bin integrals (lanes <-> edges, 31 bins per warp)
__global__ void __launch_bounds__(FWD_WARPS * 32) k_species_gauss64(KArgs a) {
    const int tile = blockIdx.x, g = blockIdx.y;
    const int nchunk = (a.sp_count + 15) / 16, t = blockIdx.z / nchunk, chunk = blockIdx.z % nchunk;
    if (!tb_g_active(a, g)) return;  // no smeared species in the group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int J = tb_g_bins(a, g);
    const int j0 = (tile * FWD_WARPS + warp) * 31;
    if (j0 >= J) return;
    const int j = j0 + lane;
    const bool valid = lane < 31 && j < J;
    const double xe = a.edges[tb_g_edge_off(a, g) + min(j, J)];
    const int jl = min(j0 + 30, J - 1);
    const double xlo_w = a.edges[tb_g_edge_off(a, g) + j0], xhi_w = a.edges[tb_g_edge_off(a, g) + jl + 1];
    const int sp0 = a.sp_first + chunk * 16;
    const int nsp = min(16, a.sp_count - chunk * 16);
    const double* blk = reinterpret_cast<const double*>(a.blkbuf) + ((long long)t * a.G + g) * a.nblk * 2;
    double acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = 0.0;
    for (int b = 0; b < a.nblk; ++b) {
        if (blk[2 * b + 1] < xlo_w || blk[2 * b] > xhi_w) continue;
        const int kb = b * COLBLK, ke = min(a.K, kb + COLBLK);
        for (int k = kb; k < ke; ++k) {
            const double* c = colrec<double>(a, t, g, k);
            if (c[F_XMAX] < xlo_w || c[F_XMIN] > xhi_w) continue;
            const double z = (xe - c[F_MUH]) * c[F_A];
            const bool up = z >= 0.0;
            const double q = 0.5 * erfc(fabs(z) * INV_SQRT2);
            const double q1 = __shfl_down_sync(0xffffffffu, q, 1);
            const bool up1 = __shfl_down_sync(0xffffffffu, (int)up, 1) != 0;
            double v = (up == up1) ? (up ? q - q1 : q1 - q) : 1.0 - q - q1;
            if (!valid) v = 0.0;
#pragma unroll
            for (int i = 0; i < 16; ++i)
                if (i < nsp) acc[i] = fma(v, a.Sd[(long long)(sp0 + i) * a.K + k], acc[i]);
        }
    }
    if (valid)
        for (int i = 0; i < nsp; ++i) a.Mbuf[(long long)t * a.mstride + ((long long)g * a.S + sp0 + i) * a.Jmax + j] = acc[i];
}

// mu_dj = sum_s eps_d f_ds r_s M[g][s][j] (smeared species; peaks are added by k_deviance)
// grid (bins, toys): mu of toy t from its per-species shapes (one column split)
__global__ void k_mu_from_species(KArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, t = blockIdx.y;
    if (i >= a.total_bins) return;
    int lo = 0, hi = a.D - 1;  // last dataset whose first bin is <= i
    while (lo < hi) { const int m = (lo + hi + 1) >> 1; if (tb_ds_off(a, m) <= i) lo = m; else hi = m - 1; }
    const int d = lo;
    const int j = i - tb_ds_off(a, d);
    const int g = tb_ds_group(a, d);
    const double* prm = a.params + (long long)t * a.params_stride;
    const double* M = a.Mbuf + (long long)t * a.mstride;
    double mu = 0.0;
    for (int s = 0; s < a.S; ++s) {
        const double f = a.rfac[d * a.S + s];
        if (a.ft.sp_kind[s] >= 2 || f == 0.0) continue;
        const int p = a.slot_map[d * a.NSLOT + s];
        if (p < 0) continue;
        mu = fma(f * prm[p], M[((long long)g * a.S + s) * a.Jmax + j], mu);
    }
    a.mubuf[(long long)t * a.total_bins + i] = mu;
}

// expected counts per bin and species of one dataset
__global__ void k_expected_out(KArgs a) {
    const int d = a.out_dataset;
    const int J = tb_ds_bins(a, d);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= J * a.S) return;
    const int j = i / a.S, s = i % a.S;
    const int g = tb_ds_group(a, d);
    const double* prm = a.params;
    double v = 0.0;
    const double f = a.rfac[d * a.S + s];
    if (f != 0.0) {
        const int pr = a.slot_map[d * a.NSLOT + s];
        const double r = pr >= 0 ? prm[pr] : 0.0;
        if (a.ft.sp_kind[s] == 2) {
            const double* ed = a.edges + tb_g_edge_off(a, g);
            const double m = prm[a.slot_map[d * a.NSLOT + a.S + 5 + 2 * s]];
            const double wd = prm[a.slot_map[d * a.NSLOT + a.S + 6 + 2 * s]];
            v = f * r * ncdf_diff((ed[j] - m) / wd, (ed[j + 1] - m) / wd);
        } else if (a.ft.sp_kind[s] == 3) {
            for (int q = 0; q < a.tb->ds_ntpl[d]; ++q) {
                const int gq = a.tb->ds_tpl0[d] + q;
                if (a.tpl_s[gq] == s) v = f * r * a.tpl[a.tpl_off[gq] + j];
            }
        } else {
            v = f * r * a.Mbuf[((long long)g * a.S + s) * a.Jmax + j];
        }
    }
    a.out_species[i] = v;
}


// ------------------------------------------------------------- probes ------
// Synthetic throughput loops: 8 independent chains per thread, every SM busy.
constexpr int PROBE_ITERS = 2048;
template <int WHICH>
__global__ void __launch_bounds__(256) k_probe(float* sink, double* sinkd, float seed) {
    float x[8];
    double y[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) { x[i] = seed * (0.1f + 0.01f * i) + 1e-3f * threadIdx.x; y[i] = (double)x[i]; }
    const float b = 0.999f, c = 1e-4f;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if constexpr (WHICH == 0) x[i] = fmaf(x[i], b, c);
            if constexpr (WHICH == 1) x[i] = ex2f(-x[i]);
            if constexpr (WHICH == 2) y[i] = fma(y[i], 0.999, 1e-4);
            if constexpr (WHICH == 3) x[i] = fmaf(0.7f, ex2f(fmaf(-0.5f, x[i], fmaf(0.25f, x[i], -0.3f))), x[i] * 0.5f);
        }
    }
    float s = 0.f; double sd = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) { s += x[i]; sd += y[i]; }
    if (s == 12345.678f) sink[threadIdx.x] = s;
    if (sd == 12345.678) sinkd[threadIdx.x] = sd;
}

// Mean relative error of ex2f over the exponents of a unit Gaussian profile, -(log2 e / 2) z^2 on
// a uniform grid of z in [-6.5, 6.5], each weighted by the profile value; FP64 exp2 is the reference.
__global__ void __launch_bounds__(256) k_ex2_bias(long long n, double* acc) {
    __shared__ double sh[32];
    double se = 0.0, sw = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double z = -6.5 + 13.0 * (i + 0.5) / n;
        const float x = (float)(-0.72134752044448170 * z * z);
        const double ref = exp2((double)x);
        se += ((double)ex2f(x) - ref);
        sw += ref;
    }
    se = block_sum_d(se, sh);
    sw = block_sum_d(sw, sh);
    if (threadIdx.x == 0) { atomicAdd(acc, se); atomicAdd(acc + 1, sw); }
}

cudaError_t run_ex2_bias(double* bias) {
    double* acc = nullptr;
    cudaError_t err;
    if ((err = cudaMalloc(&acc, 2 * sizeof(double)))) return err;
    double h[2] = {0.0, 0.0};
    err = cudaMemcpy(acc, h, sizeof h, cudaMemcpyHostToDevice);
    if (!err) { k_ex2_bias<<<1024, 256>>>(1LL << 26, acc); err = cudaGetLastError(); }
    if (!err) err = cudaMemcpy(h, acc, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(acc);
    *bias = h[1] > 0 ? h[0] / h[1] : 0.0;
    return err;
}

cudaError_t run_probe(int which, int nsm, double* ops) {
    if (which == 4) return run_ex2_bias(ops);
    float* sink = nullptr;
    double* sinkd = nullptr;
    cudaStream_t st;
    cudaEvent_t e0, e1;
    cudaError_t err;
    if ((err = cudaMalloc(&sink, 256 * sizeof(float)))) return err;
    if ((err = cudaMalloc(&sinkd, 256 * sizeof(double)))) { cudaFree(sink); return err; }
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    cudaEventCreate(&e0); cudaEventCreate(&e1);
    const int blocks = nsm * 8;
    auto launch = [&](void) {
        switch (which) {
            case 0: k_probe<0><<<blocks, 256, 0, st>>>(sink, sinkd, 0.5f); break;
            case 1: k_probe<1><<<blocks, 256, 0, st>>>(sink, sinkd, 0.5f); break;
            case 2: k_probe<2><<<blocks, 256, 0, st>>>(sink, sinkd, 0.5f); break;
            default: k_probe<3><<<blocks, 256, 0, st>>>(sink, sinkd, 0.5f); break;
        }
    };
    launch();  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = fminf(best, ms);
    }
    err = cudaGetLastError();
    *ops = (double)blocks * 256.0 * 8.0 * PROBE_ITERS / (best * 1e-3);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    cudaFree(sink); cudaFree(sinkd);
    return err;
}

// ------------------------------------------------------------ launchers ----
cudaError_t launch_columns(const KArgs& a, cudaStream_t st) {
    dim3 grid(a.nblk, a.G, a.T);
    if (a.precision == 1) {
        if (a.res == 2)  k_columns<float, 2, false><<<grid, COLBLK, 0, st>>>(a);
        else if (a.fast) {
            if (a.res == 0) k_columns<float, 0, true><<<grid, COLBLK, 0, st>>>(a);
            else            k_columns<float, 1, true><<<grid, COLBLK, 0, st>>>(a);
        } else {
            if (a.res == 0) k_columns<float, 0, false><<<grid, COLBLK, 0, st>>>(a);
            else            k_columns<float, 1, false><<<grid, COLBLK, 0, st>>>(a);
        }
    } else {
        if (a.res == 0)      k_columns<double, 0, false><<<grid, COLBLK, 0, st>>>(a);
        else if (a.res == 1) k_columns<double, 1, false><<<grid, COLBLK, 0, st>>>(a);
        else                 k_columns<double, 2, false><<<grid, COLBLK, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_forward(const KArgs& a, cudaStream_t st) {
    dim3 grid(a.ntile, a.nsplit, a.T * a.G);
    if (a.precision == 1) {
        // the generalized gamma of free power runs the general per-node kernel
        if (a.res == 2) k_forward<float, 2><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else return launch_forward_mixed(a, st);
    } else {
        if (a.res == 0)      k_forward_gauss64<<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else if (a.res == 1) k_forward<double, 1><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else                 k_forward<double, 2><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_deviance(const KArgs& a, cudaStream_t st) {
    dim3 grid(a.T, a.dev_chunks);
    if (a.precision == 1) k_deviance<float><<<grid, 256, 0, st>>>(a);
    else                  k_deviance<double><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_devfinal(const KArgs& a, cudaStream_t st) {
    k_devfinal<<<a.T, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_backward(const KArgs& a, cudaStream_t st) {
    // the tuned mixed adjoint serves the Gaussian and gamma responses (with or without secondary observables)
    if (a.precision == 1 && a.res != 2) return launch_backward_mixed(a, st);
    dim3 grid(a.nbtask, a.G, a.T);
    const int threads = a.bw_warps * 32;
    const size_t rs = a.precision == 1 ? sizeof(float) : sizeof(double);
    const size_t sm = rs * MAXGDS * threads + 16 + sizeof(double) * a.bw_warps * NRESP;
    if (a.precision == 1 && a.res == 0)      k_backward<float, 0><<<grid, threads, sm, st>>>(a);
    else if (a.precision == 1 && a.res == 1) k_backward<float, 1><<<grid, threads, sm, st>>>(a);
    else if (a.precision == 1)               k_backward<float, 2><<<grid, threads, sm, st>>>(a);
    else if (a.res == 0)   k_backward<double, 0><<<grid, threads, sm, st>>>(a);
    else if (a.res == 1)   k_backward<double, 1><<<grid, threads, sm, st>>>(a);
    else                   k_backward<double, 2><<<grid, threads, sm, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gradfinal(const KArgs& a, cudaStream_t st) {
    k_gradfinal<<<a.T, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_species(const KArgs& a, cudaStream_t st) {
    const int nchunk = (a.sp_count + 15) / 16;
    if (a.precision == 0 && a.res == 0) {
        dim3 grid((a.Jmax + FWD_WARPS * 31 - 1) / (FWD_WARPS * 31), a.G, nchunk * a.T);
        k_species_gauss64<<<grid, FWD_WARPS * 32, 0, st>>>(a);
        return cudaGetLastError();
    }
    dim3 grid((a.Jmax + FWD_WARPS * 32 - 1) / (FWD_WARPS * 32), a.G, nchunk * a.T);
    if (a.precision == 1) {
        if (a.res == 0)      k_species<float, 0><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else if (a.res == 1) k_species<float, 1><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else                 k_species<float, 2><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    } else {
        if (a.res == 1) k_species<double, 1><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else            k_species<double, 2><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_mu_from_species(const KArgs& a, cudaStream_t st) {
    k_mu_from_species<<<dim3((a.total_bins + 255) / 256, a.T), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_expected_out(const KArgs& a, cudaStream_t st) {
    const int n = a.out_bins * a.S;
    k_expected_out<<<(n + 255) / 256, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gsn
