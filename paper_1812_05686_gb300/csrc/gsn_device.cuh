// Device helpers shared by the kernel translation units of libgsn.
#pragma once
#include "gsn_internal.cuh"

#include <math.h>

namespace gsn {

#define DEV __device__ __forceinline__

constexpr float L2E = 1.4426950408889634f;           // log2(e)
constexpr float L2E_LO = (float)(1.4426950408889634 - (double)L2E);
constexpr float HALF_L2E_LO = (float)(0.72134752044448170 - 0.5 * (double)L2E);
constexpr double INV_SQRT2 = 0.70710678118654752440;
constexpr double INV_SQRT2PI = 0.39894228040143267794;
// The mixed column normalisation 1/(sqrt(2 pi) (1 + b)), b the measured mean relative error of the
// SFU exponential ex2.approx.ftz.f32 over a Gaussian profile, is a kernel argument (KArgs::norm_hi,
// norm_lo, ex2_scale): applied as fmaf(x, norm_hi, x * norm_lo), the exact product enters the
// single rounding, so the FP32 rounding of the constant does not scale every column alike.
constexpr int FWD_WARPS = 8;

// problem-table reads: the kernel-parameter copy for the first groups / datasets, else device memory;
// FAST = true (problems of at most FASTG groups and FASTD datasets) reads the copy unconditionally
template <bool FAST = false> DEV int tb_g_nds(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_nds[g] : a.tb->g_nds[g]; }
template <bool FAST = false> DEV int tb_g_ds(const KArgs& a, int g, int i) { return (FAST || g < FASTG) ? a.ft.g_ds[g][i] : a.tb->g_ds[g][i]; }
template <bool FAST = false> DEV int tb_g_bins(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_bins[g] : a.tb->g_bins[g]; }
template <bool FAST = false> DEV int tb_g_edge_off(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_edge_off[g] : a.tb->g_edge_off[g]; }
template <bool FAST = false> DEV int tb_g_node_off(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_node_off[g] : a.tb->g_node_off[g]; }
template <bool FAST = false> DEV int tb_g_jlin(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_jlin[g] : a.tb->g_jlin[g]; }
template <bool FAST = false> DEV int tb_g_zero(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_zero[g] : a.tb->g_zero[g]; }
template <bool FAST = false> DEV int tb_g_resp(const KArgs& a, int g, int i) { return (FAST || g < FASTG) ? a.ft.g_resp[g][i] : a.tb->g_resp[g][i]; }
template <bool FAST = false> DEV double tb_g_rscale(const KArgs& a, int g, int i) { return (FAST || g < FASTG) ? a.ft.g_rscale[g][i] : a.tb->g_rscale[g][i]; }
template <bool FAST = false> DEV int tb_ds_off(const KArgs& a, int d) { return (FAST || d < FASTD) ? a.ft.ds_off[d] : a.tb->ds_off[d]; }
template <bool FAST = false> DEV int tb_ds_bins(const KArgs& a, int d) { return (FAST || d < FASTD) ? a.ft.ds_bins[d] : a.tb->ds_bins[d]; }
template <bool FAST = false> DEV int tb_ds_group(const KArgs& a, int d) { return (FAST || d < FASTD) ? a.ft.ds_group[d] : a.tb->ds_group[d]; }
template <bool FAST = false> DEV int tb_ds_resp(const KArgs& a, int d) { return (FAST || d < FASTD) ? a.ft.ds_resp[d] : a.tb->ds_resp[d]; }
template <bool FAST = false> DEV int tb_g_active(const KArgs& a, int g) { return (FAST || g < FASTG) ? a.ft.g_active[g] : a.tb->g_active[g]; }

// ------------------------------------------------------------------ math --
DEV float ex2f(float x) {  // 2^x on the SFU
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// D(t) = ln(1 + t) - t with relative precision: for t in [-1/2, 1] from the
// series ln(1+t) = 2 atanh(u), u = t/(2+t), rearranged so that no leading
// terms cancel: D = -t u + 2 u^3 (1/3 + u^2/5 + u^4/7 + ...).
DEV float log1pmx_f(float t) {
    if (t >= -0.5f && t <= 1.0f) {
        // 1/(2+t): the SFU reciprocal and one Newton step, which leaves the rounding error only.  The
        // SFU result's mean error over 2+t in [1.6, 1.9] is ~1e-8, and a broad profile (small shape
        // d) spends its weight there: the bias would scale every such column alike
        const float x = 2.0f + t;
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        r = fmaf(fmaf(-x, r, 1.0f), r, r);
        const float u = t * r;
        float v = u * u;
        float p = fmaf(v, 1.0f / 15.0f, 1.0f / 13.0f);
        p = fmaf(p, v, 1.0f / 11.0f);
        p = fmaf(p, v, 1.0f / 9.0f);
        p = fmaf(p, v, 1.0f / 7.0f);
        p = fmaf(p, v, 1.0f / 5.0f);
        p = fmaf(p, v, 1.0f / 3.0f);
        return fmaf(2.0f * u * v, p, -t * u);
    }
    return log1pf(t) - t;
}
// D(t) without the range test, for callers that know |t/(2+t)| <= 1/3 wherever the result
// matters: the same series, evaluated branch-free (2 D = -2 t u + u^3 (2/3 + 2 u^2/5 + ...))
DEV float log1pmx_poly(float t) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(2.0f + t));
    const float u = t * r;
    const float v = u * u;
    float p = fmaf(v, 2.0f / 15.0f, 2.0f / 13.0f);
    p = fmaf(p, v, 2.0f / 11.0f);
    p = fmaf(p, v, 2.0f / 9.0f);
    p = fmaf(p, v, 2.0f / 7.0f);
    p = fmaf(p, v, 2.0f / 5.0f);
    p = fmaf(p, v, 2.0f / 3.0f);
    return fmaf(u * v, p, -t * u);
}

// D(t) and L1 = ln(1 + t) together; L1 directly from log1p where |t| is large
DEV float log1pmx2_f(float t, float& L1) {
    if (t >= -0.5f && t <= 1.0f) {
        const float D = log1pmx_f(t);
        L1 = D + t;
        return D;
    }
    L1 = log1pf(t);
    return L1 - t;
}

// digamma by upward recurrence and the asymptotic series (Abramowitz & Stegun 6.3.18)
DEV double digamma_d(double x) {
    double acc = 0.0;
    while (x < 12.0) { acc -= 1.0 / x; x += 1.0; }
    double ix = 1.0 / x, ix2 = ix * ix;
    double s = ix2 * (1.0 / 12 - ix2 * (1.0 / 120 - ix2 * (1.0 / 252 - ix2 * (1.0 / 240 - ix2 * (1.0 / 132)))));
    return acc + log(x) - 0.5 * ix - s;
}
DEV float digamma_f(float x) {
    float acc = 0.0f;
    while (x < 6.0f) { acc -= 1.0f / x; x += 1.0f; }
    float ix = 1.0f / x, ix2 = ix * ix;
    float s = ix2 * (1.0f / 12 - ix2 * (1.0f / 120 - ix2 * (1.0f / 252 - ix2 * (1.0f / 240))));
    return acc + logf(x) - 0.5f * ix - s;
}

// double-float helpers (error-free products and sums)
DEV void df_mul(float ah, float al, float bh, float bl, float& rh, float& rl) {
    float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, fmaf(al, bh, e));
    rh = p + e;
    rl = e - (rh - p);
}
DEV void df_add(float ah, float al, float b, float& rh, float& rl) {
    float s = ah + b;
    float bb = s - ah;
    float e = (ah - (s - bb)) + (b - bb);
    e += al;
    rh = s + e;
    rl = e - (rh - s);
}

// Phi(z1) - Phi(z0) for z0 <= z1 without cancellation in the tails
DEV double ncdf_diff(double z0, double z1) {
    if (z0 >= 0.0) return 0.5 * (erfc(z0 * INV_SQRT2) - erfc(z1 * INV_SQRT2));
    if (z1 <= 0.0) return 0.5 * (erfc(-z1 * INV_SQRT2) - erfc(-z0 * INV_SQRT2));
    return 1.0 - 0.5 * (erfc(-z0 * INV_SQRT2) + erfc(z1 * INV_SQRT2));
}

template <class R> DEV R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <class R> DEV R warp_min(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class R> DEV R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// fixed-order block sum of one double per thread (result valid in thread 0)
DEV double block_sum_d(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) s += sh[i];
    return s;
}

template <bool FAST = false>
DEV void toy_window_union(const KArgs& a, int t, int g, int& wlo, int& whi) {
    const int J = tb_g_bins<FAST>(a, g);
    wlo = J; whi = 0;
    for (int dd = 0; dd < tb_g_nds<FAST>(a, g); ++dd) {
        const int d = tb_g_ds<FAST>(a, g, dd);
        int lo = a.win[t * a.win_stride + 2 * d], hi = a.win[t * a.win_stride + 2 * d + 1];
        lo = max(lo, 0); hi = min(hi, J);
        if (hi > lo) { wlo = min(wlo, lo); whi = max(whi, hi); }
    }
}

template <class R> DEV R* colrec(const KArgs& a, int t, int g, int k) {
    return reinterpret_cast<R*>(a.colbuf) + (((long long)t * a.G + g) * a.K + k) * NFP;
}
template <class R> DEV R* zerorec(const KArgs& a, int t, int g, int k) {
    return reinterpret_cast<R*>(a.zerobuf) + (((long long)t * a.G + g) * a.K + k) * NFZ;
}

// ------------------------------------------------------- bin-at-zero -------
// P(d, y) = e^-y sum_n y^(d+n) / Gamma(d+n+1), its d-derivative (through
// psi(d+n+1) = psi(d+1) + sum_{m<=n} 1/(d+m)), and s^2 dP/ds = -s y^d e^-y / Gamma(d).
template <class R> DEV void gamma_bin_zero(R d, R s, R x1, R& P, R& Pd, R& Ps2) {
    const R y = x1 / s;
    const R ly = log(y);
    const R pref = exp(d * ly - y - lgamma(d + R(1)));
    R term = 1, sum = 1, H = 0, hsum = 0;
    const int nmax = sizeof(R) == 8 ? 80 : 40;
    for (int n = 1; n < nmax; ++n) {
        term *= y / (d + R(n));
        H += R(1) / (d + R(n));
        sum += term;
        hsum += term * H;
        if (term < R(sizeof(R) == 8 ? 1e-18 : 1e-9) * sum) break;
    }
    P = pref * sum;
    const R psi1 = sizeof(R) == 8 ? (R)digamma_d((double)d + 1.0) : (R)digamma_f((float)d + 1.0f);
    Pd = P * (ly - psi1) - pref * hsum;
    Ps2 = -s * exp(d * ly - y - lgamma(d));
}


// compensated warp sum of (s, c) pairs; result in every lane
DEV float warp_sum_comp(float s, float c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, o);
        const float co = __shfl_xor_sync(0xffffffffu, c, o);
        const float tsum = s + so;
        const float bp = tsum - s;
        c = c + co + ((s - (tsum - bp)) + (so - bp));
        s = tsum;
    }
    return s + c;
}

// compensated (TwoSum) accumulation of x into (s, c)
DEV void two_sum_acc(float& s, float& c, float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
}

// log2(e) x with the exact product inside one rounding: per-column constants made with the FP32
// log2(e) alone would carry its rounding (1.3e-8) into the exponent of every column
DEV float mul_l2e(float x) { return fmaf(L2E, x, x * L2E_LO); }

// --------------------------------------------------- response evaluators ---
// Mixed: unnormalised bin value rho_jk = sum_n w_n exp(E_n) of a column record.
template <int RES, int NG>
DEV float bin_value_f(const float* c, float xc, const float* del, const float* lam, const float* wt) {
    const float Dx = (xc - c[F_MUH]) - c[F_MUL];
    float rho = 0.0f;
    if constexpr (RES == 0) {
        const float z = Dx * c[F_A];
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const float zn = fmaf(del[n], c[F_A], z);
            const float q = zn * zn;
            rho = fmaf(wt[n], ex2f(-fmaf(0.5f * L2E, q, q * HALF_L2E_LO)), rho);
        }
    } else {
        // log f(x) - log f(mu) = (d-1) D(t) - t = d D(t) - ln(1+t), t = x/mu - 1; less XM (log2 units)
        const float t = Dx * c[F_A];
        float L1;
        const float Dt = log1pmx2_f(t, L1);
        const float B2 = fmaf(L2E, c[F_B], fmaf(L2E_LO, c[F_B] - 1.0f, -L2E)), C2 = mul_l2e(c[F_C]);
        const float Ec = fmaf(mul_l2e(c[F_B]), Dt, fmaf(-L2E, L1, -c[F_XM]));
#pragma unroll
        for (int n = 0; n < NG; ++n)
            rho = fmaf(wt[n], ex2f(Ec + fmaf(C2, del[n], B2 * lam[n])), rho);
    }
    return rho;
}

// FP64 gamma: sum_n w_n exp((d-1) ln x_n - x_n/s - d ln s - lgamma(d))
template <int NG>
DEV double bin_value_gamma_d(const double* c, const double* x, const double* lx, const double* wt) {
    double rho = 0.0;
#pragma unroll
    for (int n = 0; n < NG; ++n) rho = fma(wt[n], exp(fma(c[F_B], lx[n], fma(-c[F_C], x[n], c[F_A]))), rho);
    return rho;
}

}  // namespace gsn
