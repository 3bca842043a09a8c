// Multivariate likelihood: the extra likelihood pieces of a secondary observable (section 2.4).
//
// A dataset's energy bins form slices; each slice carries a histogram of a second observable.
// Species s contributes to slice q its expected counts N_sq = eps f_ds r_s U_sq, where
// U_sq = sum_{j in q} (species shape of bin j) comes from the per-toy, per-species shapes M of the
// response (smeared species), the normalised template (template species) or the peak profile
// integrated over the slice (AnaPeak), and spreads them over the secondary bins with the fixed
// shape P_sqm.  Every slice inside the toy's window adds the Poisson term of
// mu_qm = sum_s N_sq P_sqm to the NLL.
//   k_secondary          one block per (toy, dataset with a secondary observable): U, the terms,
//                        omega_qm = 1 - n_qm / mu_qm, v_sq = sum_m omega_qm P_sqm and the direct
//                        gradient terms of the rate and peak slots (fixed-order sums)
//   k_secondary_weights  U_qk = sum_s v_sq eps f_ds r_s S'_sk per fine column: the adjoint adds
//                        U_{q(j) k} N_k to the weight of every (bin j, column k) pair of slice q
#include "gsn_device.cuh"

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

// grid (column blocks, slices, toys)
template <class R>
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
        const double sv = sizeof(R) == 4 ? (double)a.Sf[(long long)s * a.K + k] : a.Sd[(long long)s * a.K + k];
        u = fma(v * f * prm[p], sv, u);
    }
    reinterpret_cast<R*>(a.secU)[((long long)t * a.Qtot + q) * a.K + k] = (R)u;
}

cudaError_t launch_secondary(const KArgs& a, cudaStream_t st) {
    k_secondary<<<dim3(a.T, a.nsec), 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_secondary_weights(const KArgs& a, cudaStream_t st) {
    const dim3 grid((a.K + 255) / 256, a.Qtot, a.T);
    if (a.precision == 1) k_secondary_weights<float><<<grid, 256, 0, st>>>(a);
    else                  k_secondary_weights<double><<<grid, 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace gsn
