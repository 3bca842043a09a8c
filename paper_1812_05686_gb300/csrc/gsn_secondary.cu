// Multivariate likelihood: the extra likelihood pieces of a secondary observable (section 2.4).
//
// A dataset's energy bins form slices; each slice carries a histogram of a second observable.
// Species s contributes to slice q its expected counts N_sq = eps f_ds r_s U_sq, where
// U_sq = sum_{j in q} (species shape of bin j) comes from the per-toy, per-species shapes M of the
// response (smeared species), the normalised template (template species) or the peak profile
// integrated over the slice (AnaPeak), and spreads them over the secondary bins with the fixed
// shape P_sqm.  Every slice inside the toy's window adds the Poisson term of
// mu_qm = sum_s N_sq P_sqm to the NLL.
//   k_slice_sums         Rq[t][q][k] = N_k sum_{j in q} R_jk over the bins of every slice inside the
//                        toy's window (lanes <-> columns), so that U_sq = sum_k Rq_qk S'_sk: the
//                        pieces need slice sums only, and mu comes from the regular forward
//   k_secondary          one block per (toy, dataset with a secondary observable): U, the terms,
//                        omega_qm = 1 - n_qm / mu_qm, v_sq = sum_m omega_qm P_sqm and the direct
//                        gradient terms of the rate and peak slots (fixed-order sums)
//   k_secondary_weights  U_qk = sum_s v_sq eps f_ds r_s S'_sk per fine column: the adjoint adds
//                        U_{q(j) k} N_k to the weight of every (bin j, column k) pair of slice q
#include "gsn_device.cuh"
#include "gsn_ggamma.cuh"

namespace gsn {

// toy window of dataset d clipped to its bins
DEV void toy_window(const KArgs& a, int t, int d, int& lo, int& hi) {
    const int J = tb_ds_bins(a, d);
    lo = max(0, a.win[(long long)t * a.win_stride + 2 * d]);
    hi = min(J, a.win[(long long)t * a.win_stride + 2 * d + 1]);
}

__global__ void __launch_bounds__(256) k_secondary(KArgs a) {
    const int t = blockIdx.x, i = blockIdx.y;
    const int d = a.sec_ds[i], Q = a.sec_nq[i], M = a.sec_M[i], q0 = a.sec_q0[i];
    const int S = a.S;
    __shared__ double sh[32];
    __shared__ int sflag;
    if (threadIdx.x == 0) sflag = 0;
    const double* prm = a.params + (long long)t * a.params_stride;
    int lo, hi;
    toy_window(a, t, d, lo, hi);
    const int g = tb_ds_group(a, d);
    const double* Mg = a.Mbuf + (long long)t * a.mstride + (long long)g * S * a.Jmax;
    const double* ed = a.edges + tb_g_edge_off(a, g);
    const double* P = a.sec_P + a.sec_poff[i];                       // [S][Q][M]
    double* U = a.secN + ((long long)t * a.Qtot + q0) * S;           // [Q][S]
    double* V = a.secV + ((long long)t * a.Qtot + q0) * S;           // [Q][S]
    double* om = a.secW + (long long)t * a.nsecb + a.sec_coff[i];    // [Q][M]
    const double* nq = a.counts + (long long)t * a.counts_stride + a.total_bins + a.sec_coff[i];
    auto active = [&](int q) {
        const int jl = a.sq_lo[q0 + q], jh = a.sq_hi[q0 + q];
        return jl >= lo && jh <= hi && jh > jl;
    };
    // 1) unscaled slice sums of every species (0 for slices outside the window)
    for (int e = threadIdx.x; e < Q * S; e += blockDim.x) {
        const int q = e / S, s = e % S;
        double u = 0.0;
        if (active(q) && a.rfac[d * S + s] != 0.0) {
            const int jl = a.sq_lo[q0 + q], jh = a.sq_hi[q0 + q];
            const int kind = a.ft.sp_kind[s];
            if (kind < 2) {
                if (!a.secRq)  // per-species shapes of one point (the value cache of gsn_eval)
                    for (int j = jl; j < jh; ++j) u += Mg[(long long)s * a.Jmax + j];
            } else if (kind == 3) {
                for (int gq = a.tb->ds_tpl0[d]; gq < a.tb->ds_tpl0[d] + a.tb->ds_ntpl[d]; ++gq)
                    if (a.tpl_s[gq] == s)
                        for (int j = jl; j < jh; ++j) u += a.tpl[a.tpl_off[gq] + j];
            } else {
                const int pm = a.slot_map[d * a.NSLOT + S + 5 + 2 * s], pw = a.slot_map[d * a.NSLOT + S + 6 + 2 * s];
                if (pm >= 0 && pw >= 0) {
                    const double m = prm[pm], w = prm[pw];
                    u = ncdf_diff((ed[jl] - m) / w, (ed[jh] - m) / w);
                }
            }
        }
        U[e] = u;
    }
    __syncthreads();
    if (a.secRq) {
        // smeared species from the slice sums: U_sq = sum_k Rq_qk S'_sk, one warp per (q, s), lanes
        // striding over the columns, fixed-order warp sum
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int e = warp; e < Q * S; e += nw) {
            const int q = e / S, s = e % S;
            if (a.ft.sp_kind[s] >= 2 || a.rfac[d * S + s] == 0.0 || !active(q)) continue;
            double u = 0.0;
            if (a.precision == 1) {
                // FP32 products in compensated (TwoSum) lane sums: the FP64 rate would bound this
                const float* Rq = reinterpret_cast<const float*>(a.secRq) + ((long long)t * a.Qtot + q0 + q) * a.K;
                const float* Sr = a.Sf + (long long)s * a.K;
                const float* Srl = a.Sf_lo + (long long)s * a.K;
                float us = 0.f, uc = 0.f;
                for (int k = lane; k < a.K; k += 32) {
                    const float pr = Rq[k] * Sr[k];
                    two_sum_acc(us, uc, pr);
                    uc = fmaf(Rq[k], Srl[k], fmaf(Rq[k], Sr[k], -pr) + uc);   // the product's rounding error, S' residual
                }
                u = (double)us + (double)uc;
            } else {
                const double* Rq = reinterpret_cast<const double*>(a.secRq) + ((long long)t * a.Qtot + q0 + q) * a.K;
                const double* Sr = a.Sd + (long long)s * a.K;
                for (int k = lane; k < a.K; k += 32) u = fma(Rq[k], Sr[k], u);
            }
            u = warp_sum<double>(u);
            if (lane == 0) U[e] = u;
        }
        __syncthreads();
    }
    // 2) expected secondary counts, Poisson terms, omega
    double part = 0.0;
    int flags = 0;
    for (int e = threadIdx.x; e < Q * M; e += blockDim.x) {
        const int q = e / M, m = e % M;
        double w = 0.0;
        if (active(q)) {
            double mu = 0.0;
            for (int s = 0; s < S; ++s) {
                const double u = U[q * S + s];
                const int p = a.slot_map[d * a.NSLOT + s];
                if (u == 0.0 || p < 0) continue;
                mu = fma(a.rfac[d * S + s] * prm[p] * u, P[((long long)s * Q + q) * M + m], mu);
            }
            const double n = nq[e];
            if (n > 0.0) {
                if (mu > 0.0) part += mu - n + n * log(n / mu);
                else flags |= 1;
            } else {
                part += mu;
            }
            if (!isfinite(mu)) flags |= 2;
            w = mu > 0.0 ? 1.0 - n / mu : 0.0;
        }
        om[e] = w;
    }
    if (flags) atomicOr(&sflag, flags);
    part = block_sum_d(part, sh);  // its barriers also publish sflag and omega
    __syncthreads();
    const int fl = sflag;
    // 3) v_sq = sum_m omega_qm P_sqm
    for (int e = threadIdx.x; e < Q * S; e += blockDim.x) {
        const int q = e / S, s = e % S;
        double v = 0.0;
        if (active(q))
            for (int m = 0; m < M; ++m) v = fma(om[q * M + m], P[((long long)s * Q + q) * M + m], v);
        V[e] = v;
    }
    __syncthreads();
    // 4) slot gradient of the dataset: rates (every kind) and peak position / width
    double* out = a.secpart + ((long long)t * a.nsec + i) * (2 + a.NSLOT);
    if (threadIdx.x == 0) { out[0] = part; out[1] = (double)fl; }
    for (int sl = threadIdx.x; sl < a.NSLOT; sl += blockDim.x) out[2 + sl] = 0.0;
    __syncthreads();
    if (a.want_grad) {
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
            const double f = a.rfac[d * S + s];
            if (f == 0.0) continue;
            double gr = 0.0, gm = 0.0, gw = 0.0;
            const bool peak = a.ft.sp_kind[s] == 2;
            const int pm = a.slot_map[d * a.NSLOT + S + 5 + 2 * s], pw = a.slot_map[d * a.NSLOT + S + 6 + 2 * s];
            const bool pk = peak && pm >= 0 && pw >= 0;
            const double m = pk ? prm[pm] : 0.0, wd = pk ? prm[pw] : 1.0;
            for (int q = 0; q < Q; ++q) {
                const double v = V[q * S + s];
                if (v == 0.0) continue;
                gr = fma(v, U[q * S + s], gr);
                if (pk) {
                    const int jl = a.sq_lo[q0 + q], jh = a.sq_hi[q0 + q];
                    const double z0 = (ed[jl] - m) / wd, z1 = (ed[jh] - m) / wd;
                    const double p0 = exp(-0.5 * z0 * z0) * INV_SQRT2PI, p1 = exp(-0.5 * z1 * z1) * INV_SQRT2PI;
                    gm = fma(v, -(p1 - p0) / wd, gm);
                    gw = fma(v, -(z1 * p1 - z0 * p0) / wd, gw);
                }
            }
            out[2 + s] = f * gr;
            if (pk) {
                const int pr = a.slot_map[d * a.NSLOT + s];
                const double r = pr >= 0 ? f * prm[pr] : 0.0;
                out[2 + S + 5 + 2 * s] = r * gm;
                out[2 + S + 6 + 2 * s] = r * gw;
            }
        }
    }
}

// grid (column blocks of 256, groups, toys); lanes <-> columns.  Every warp walks the bins of its
// columns' band (the warp's union) inside each active slice of the group's datasets.
template <class R, int RES>
__global__ void __launch_bounds__(256) k_slice_sums(KArgs a) {
    const int g = blockIdx.y, t = blockIdx.z;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const bool kval = k < a.K;
    if (!tb_g_active(a, g)) return;
    R c[NFP];
    {
        const R* cr = colrec<R>(a, t, g, kval ? k : a.K - 1);
#pragma unroll
        for (int i = 0; i < NFP; ++i) c[i] = cr[i];
    }
    const int J = tb_g_bins(a, g), nbase = tb_g_node_off(a, g);
    const double* ed = a.edges + tb_g_edge_off(a, g);
    const R xmn = warp_min<R>(kval ? c[F_XMIN] : (R)INFINITY);
    const R xmx = warp_max<R>(kval ? c[F_XMAX] : (R)-INFINITY);
    int ja = 0, jb = -1;
    if (xmx >= xmn) {
        int lo = 0, hi = J;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (ed[m + 1] <= (double)xmn) lo = m + 1; else hi = m; }
        ja = lo;
        lo = 0; hi = J;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (ed[m] < (double)xmx) lo = m + 1; else hi = m; }
        jb = lo - 1;
    }
    R* out = reinterpret_cast<R*>(a.secRq) + (long long)t * a.Qtot * a.K;
    for (int dd = 0; dd < tb_g_nds(a, g); ++dd) {
        const int d = tb_g_ds(a, g, dd);
        int i = -1;
        for (int x = 0; x < a.nsec; ++x) if (a.sec_ds[x] == d) i = x;
        if (i < 0) continue;
        int wlo, whi;
        toy_window(a, t, d, wlo, whi);
        for (int q = 0; q < a.sec_nq[i]; ++q) {
            const int qg = a.sec_q0[i] + q, jl = a.sq_lo[qg], jh = a.sq_hi[qg];
            if (!(jl >= wlo && jh <= whi && jh > jl)) continue;
            double sum = 0.0;
            if constexpr (sizeof(R) == 8 && RES == 0) {
                // FP64 Gaussian: the exact integral over the slice
                if (kval) sum = ncdf_diff((ed[jl] - c[F_MUH]) * c[F_A], (ed[jh] - c[F_MUH]) * c[F_A]);
            } else {
                const int j0 = max(jl, ja), j1 = min(jh - 1, jb);
                R acc = 0;
                for (int j = j0; j <= j1; ++j) {
                    const unsigned char cls = a.bclass[nbase + j];
                    R v;
                    if (RES >= 1 && cls == BIN_ZERO) {
                        v = zerorec<R>(a, t, g, kval ? k : a.K - 1)[Z_P0];
                    } else if constexpr (sizeof(R) == 4) {
                        const float* nd = a.ntab_f + (long long)(nbase + j) * 3 * NGM_F;
                        const float xc = a.xc_f[nbase + j];
                        if (cls == BIN_LOG) {
                            if constexpr (RES == 2) v = gg_bin_value_f<NG_LOG_F>(c, xc, nd + NGM_F, nd + 2 * NGM_F);
                            else v = bin_value_f<RES, NG_LOG_F>(c, xc, nd, nd + NGM_F, nd + 2 * NGM_F);
                        } else {
                            if constexpr (RES == 2) v = gg_bin_value_f<NG_LIN_F>(c, xc, nd + NGM_F, nd + 2 * NGM_F);
                            else v = bin_value_f<RES, NG_LIN_F>(c, xc, nd, nd + NGM_F, nd + 2 * NGM_F);
                        }
                    } else {
                        const double* nd = a.ntab_d + (long long)(nbase + j) * 3 * NGM_D;
                        if (cls == BIN_LOG) {
                            if constexpr (RES == 2) v = gg_bin_value_d<NG_LOG_D>(c, nd + NGM_D, nd + 2 * NGM_D);
                            else v = bin_value_gamma_d<NG_LOG_D>(c, nd, nd + NGM_D, nd + 2 * NGM_D);
                        } else {
                            if constexpr (RES == 2) v = gg_bin_value_d<NG_LIN_D>(c, nd + NGM_D, nd + 2 * NGM_D);
                            else v = bin_value_gamma_d<NG_LIN_D>(c, nd, nd + NGM_D, nd + 2 * NGM_D);
                        }
                    }
                    acc += v;
                }
                sum = (double)acc * (double)c[F_N];
            }
            if (kval) out[(long long)qg * a.K + k] = (R)sum;
        }
    }
}

// FP64: grid (column blocks, slices, toys)
__global__ void __launch_bounds__(256) k_secondary_weights(KArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y, t = blockIdx.z;
    if (k >= a.K) return;
    const int i = a.sq_sec[q], d = a.sec_ds[i];
    const double* prm = a.params + (long long)t * a.params_stride;
    const double* V = a.secV + ((long long)t * a.Qtot + q) * a.S;
    double u = 0.0;
    for (int s = 0; s < a.S; ++s) {
        const double v = V[s], f = a.rfac[d * a.S + s];
        const int p = a.slot_map[d * a.NSLOT + s];
        if (v == 0.0 || f == 0.0 || p < 0 || a.ft.sp_kind[s] >= 2) continue;
        u = fma(v * f * prm[p], a.Sd[(long long)s * a.K + k], u);
    }
    reinterpret_cast<double*>(a.secU)[((long long)t * a.Qtot + q) * a.K + k] = u;
}

// Mixed precision: the weight is added to the adjoint's FP32 pair weights, so it is formed in FP32.
// The coefficients c_qs = v_sq eps f_ds r_s of a block of SW_Q slices are built once per block
// (FP64, rounded to FP32) in shared memory; each thread holds one column and reads S'_sk once per
// block of slices.  Grid (column blocks, toys).
constexpr int SW_Q = 16;
__global__ void __launch_bounds__(256) k_secondary_weights_f(KArgs a) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, t = blockIdx.y;
    const int S = a.S;
    extern __shared__ float scoef[];                       // [SW_Q][S]
    int* slist = reinterpret_cast<int*>(scoef + SW_Q * S);  // smeared species
    __shared__ int ns;
    if (threadIdx.x == 0) {
        int n = 0;
        for (int sp = 0; sp < S; ++sp)
            if (a.ft.sp_kind[sp] < 2) slist[n++] = sp;
        ns = n;
    }
    const double* prm = a.params + (long long)t * a.params_stride;
    float* out = reinterpret_cast<float*>(a.secU) + (long long)t * a.Qtot * a.K;
    for (int q0 = 0; q0 < a.Qtot; q0 += SW_Q) {
        const int nq = min(SW_Q, a.Qtot - q0);
        __syncthreads();
        for (int e = threadIdx.x; e < SW_Q * S; e += blockDim.x) {
            const int qq = e / S, sp = e % S;
            float v = 0.f;
            if (qq < nq) {
                const int q = q0 + qq, d = a.sec_ds[a.sq_sec[q]];
                const double vs = a.secV[((long long)t * a.Qtot + q) * S + sp], f = a.rfac[d * S + sp];
                const int pp = a.slot_map[d * a.NSLOT + sp];
                if (vs != 0.0 && f != 0.0 && pp >= 0) v = (float)(vs * f * prm[pp]);
            }
            scoef[qq * S + sp] = v;
        }
        __syncthreads();
        if (k >= a.K) continue;
        float u[SW_Q] = {};
        for (int i = 0; i < ns; ++i) {
            const int sp = slist[i];
            const float sv = a.Sf[(long long)sp * a.K + k];
#pragma unroll
            for (int qq = 0; qq < SW_Q; ++qq) u[qq] = fmaf(scoef[qq * S + sp], sv, u[qq]);
        }
#pragma unroll
        for (int qq = 0; qq < SW_Q; ++qq)
            if (qq < nq) out[(long long)(q0 + qq) * a.K + k] = u[qq];
    }
}

cudaError_t launch_secondary(const KArgs& a, cudaStream_t st) {
    k_secondary<<<dim3(a.T, a.nsec), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_slice_sums(const KArgs& a, cudaStream_t st) {
    // mixed Gaussian and gamma responses: the batched, lanes-on-columns kernel of gsn_mixed.cu
    if (a.precision == 1 && a.res != 2) return launch_slice_sums_mixed(a, st);
    const dim3 grid((a.K + 255) / 256, a.G, a.T);
    if (a.precision == 1) {
        if (a.res == 0)      k_slice_sums<float, 0><<<grid, 256, 0, st>>>(a);
        else if (a.res == 1) k_slice_sums<float, 1><<<grid, 256, 0, st>>>(a);
        else                 k_slice_sums<float, 2><<<grid, 256, 0, st>>>(a);
    } else {
        if (a.res == 0)      k_slice_sums<double, 0><<<grid, 256, 0, st>>>(a);
        else if (a.res == 1) k_slice_sums<double, 1><<<grid, 256, 0, st>>>(a);
        else                 k_slice_sums<double, 2><<<grid, 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_secondary_weights(const KArgs& a, cudaStream_t st) {
    if (a.precision == 1) {
        const size_t sh = (size_t)SW_Q * a.S * sizeof(float) + (size_t)a.S * sizeof(int);
        k_secondary_weights_f<<<dim3((a.K + 255) / 256, a.T), 256, sh, st>>>(a);
    } else {
        k_secondary_weights<<<dim3((a.K + 255) / 256, a.Qtot, a.T), 256, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace gsn
