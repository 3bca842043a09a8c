// Generalized-gamma response with a free power p (Stacy's density, the line shape of the
// generalized-gamma response cited in section 2.3):
//   f(x; d, s, p) = p x^(d-1) exp(-(x/s)^p) / (s^d Gamma(d/p)),  x > 0,
// CDF P(d/p, (x/s)^p).  Every column's (d, s) follow from its mean mu and variance var by moment
// matching for the fit parameter p:
//   mu = s Gamma(x + a) / Gamma(x),  mu^2 + var = s^2 Gamma(x + 2a) / Gamma(x),  x = d/p, a = 1/p.
// Eliminating s leaves H(x) = lnGamma(x+2a) + lnGamma(x) - 2 lnGamma(x+a) = ln(1 + var/mu^2).
// H and the other log-gamma / digamma differences are O(1/x) while the log-gammas are O(x ln x),
// so they come from Stirling's series (Abramowitz & Stegun 6.1.40, 6.3.18) with the leading terms
// combined analytically, after the recurrences lnGamma(z+1) = lnGamma(z) + ln z and
// psi(z+1) = psi(z) + 1/z have moved the argument to >= 10.  All column work is FP64.
#pragma once
#include "gsn_device.cuh"

namespace gsn {

constexpr double GG_XSTIR = 10.0;

// Stirling tails at one argument z >= 10, sharing 1/z:
//   lt = lnGamma(z) - [(z - 1/2) ln z - z + ln(2 pi)/2] = sum_n B_2n / (2n (2n-1) z^(2n-1)), n <= 8
//   dt = psi(z) - [ln z - 1/(2z)] = -sum_n B_2n / (2n z^2n), n <= 8
DEV void gg_tails(double z, double& lt, double& dt, double& iz) {
    iz = 1.0 / z;
    const double v = iz * iz;
    double s = fma(v, -3617.0 / 122400, 1.0 / 156);
    s = fma(s, v, -691.0 / 360360);
    s = fma(s, v, 1.0 / 1188);
    s = fma(s, v, -1.0 / 1680);
    s = fma(s, v, 1.0 / 1260);
    s = fma(s, v, -1.0 / 360);
    s = fma(s, v, 1.0 / 12);
    lt = s * iz;
    double u = fma(v, -3617.0 / 8160, 1.0 / 12);
    u = fma(u, v, -691.0 / 32760);
    u = fma(u, v, 1.0 / 132);
    u = fma(u, v, -1.0 / 240);
    u = fma(u, v, 1.0 / 252);
    u = fma(u, v, -1.0 / 120);
    u = fma(u, v, 1.0 / 12);
    dt = -u * v;
}
DEV int gg_shift(double x) { return x >= GG_XSTIR ? 0 : (int)ceil(GG_XSTIR - x); }

// H(x) = ln[Gamma(x + 2a) Gamma(x) / Gamma(x + a)^2] and dH/dx = psi(x + 2a) - 2 psi(x + a) + psi(x),
// evaluated together (the tails at x, x + a, x + 2a and ln(1 - q^2), q = a/(x + a), serve both)
DEV void gg_H_Hx(double x, double a, double& H, double& Hx) {
    const int m = gg_shift(x);
    const double xm = x + m;
    double l0, d0, i0, l1, d1, i1, l2, d2, i2;
    gg_tails(xm, l0, d0, i0);
    gg_tails(xm + a, l1, d1, i1);
    gg_tails(xm + 2.0 * a, l2, d2, i2);
    const double q = a * i1;
    const double lq = log1p(-q * q);
    double h = fma(xm - 0.5, lq, 2.0 * a * log1p(q)) + ((l2 - 2.0 * l1) + l0);
    double hx = lq - a * a * (i0 * i1 * i2) + ((d2 - 2.0 * d1) + d0);
    for (int i = 0; i < m; ++i) {
        const double xi = x + i, ei = a / xi;
        if (ei < 0.5) { const double qi = ei / (1.0 + ei); h -= log1p(-qi * qi); }
        else h -= log(xi) + log(xi + 2.0 * a) - 2.0 * log(xi + a);
        hx -= 2.0 * a * a / (xi * (xi + a) * (xi + 2.0 * a));
    }
    H = h;
    Hx = hx;
}

// x = d/p solving H(x) = r = ln(1 + var/mu^2): Newton's method on ln H against ln x, started from
// the series reversion of the first four terms of H's large-x expansion (Stirling's series with the
// Bernoulli polynomials B_2..B_5; a = 1 gives ln(1 + 1/x)),
//   H(x) = a^2/x + a^2 (1/2 - a)/x^2 + a^2 (7a^2 - 6a + 1)/(6 x^3) - a^3 (6a^2 - 7a + 2)/(4 x^4) + O(x^-5),
// whose relative error is O(x^-4): a column of x >= 100 needs a single step.  Stops once a step is
// below 1e-7 (the error left is its square).  lnx = ln x; hx = dH/dx at the root (the value at the
// last point evaluated, moved to the root with dHx/dx = -2 Hx / x of the leading term).  Returns a
// negative value if it fails.
DEV double gg_solve_shape(double r, double a, double& lnx, double& hx) {
    const double b2 = 0.5 - a, b3 = (1.0 + a * (7.0 * a - 6.0)) / 6.0, b4 = -a * (2.0 + a * (6.0 * a - 7.0)) / 4.0;
    const double y0 = r / (a * a);
    const double y = y0 * (1.0 + y0 * (-b2 + y0 * ((2.0 * b2 * b2 - b3) + y0 * (b2 * (5.0 * b3 - 5.0 * b2 * b2) - b4))));
    double x = 1.0 / y;
    if (!(x > 0.0) || !isfinite(x) || x < 0.5 / y0) x = 1.0 / y0;
    double u = log(x);
    for (int it = 0; it < 60; ++it) {
        double h;
        gg_H_Hx(x, a, h, hx);
        const double step = fmin(5.0, fmax(-5.0, -log(h / r) * h / (x * hx)));
        u += step;
        x = exp(u);
        if (fabs(step) < 1e-7) {
            hx *= exp(-2.0 * step);
            lnx = u;
            return x;
        }
    }
    return -1.0;
}

// At the matched shape x = d/p (lx = ln x): ls = lnGamma(x + a) - lnGamma(x), psi(x), lnGamma(x) and
// da = psi(x + a) - psi(x), evaluated together (the tails at x and x + a and ln(1 + a/x) serve all
// four; below 10 the recurrences move the differences' arguments, and lnGamma / psi come from the
// library / digamma_d)
DEV void gg_at_shape(double x, double lx, double a, double& ls, double& psi, double& lgx, double& da) {
    const int m = gg_shift(x);
    const double xm = x + m;
    double l0, d0, i0, l1, d1, i1;
    gg_tails(xm, l0, d0, i0);
    gg_tails(xm + a, l1, d1, i1);
    const double lq = log1p(a * i0);
    double g = fma(xm - 0.5, lq, a * log(xm + a) - a) + (l1 - l0);
    double dd = lq + 0.5 * a * (i0 * i1) + (d1 - d0);
    for (int i = 0; i < m; ++i) {
        const double xi = x + i;
        g -= log1p(a / xi);
        dd += a / (xi * (xi + a));
    }
    ls = g;
    da = dd;
    if (m == 0) {
        psi = lx - 0.5 * i0 + d0;
        lgx = fma(x - 0.5, lx, -x) + 0.91893853320467274178 + l0;
    } else {
        psi = digamma_d(x);
        lgx = lgamma(x);
    }
}

// ---- FP32 helpers of the mixed path ----
// Q2(q) = e^q - 1 - q with relative precision, and E1 = e^q - 1.  The series
// Q2(h) = h^2 (1/2 + h/6 + ... + h^8/10!) has relative truncation error below 2 |h|^9 / 11! (1e-10
// at |h| = 1/2).  |q| <= 1/2 (the bulk of a band): the series at q.  |q| <= 2: the series at
// h = q/4 and two doublings Q2(2h) = E1(h)^2 + 2 Q2(h), E1(2h) = E1(h)^2 + 2 E1(h), which add
// non-negative terms to Q2.  Beyond, e^q - 1 - q loses at most a factor ~1.7 to cancellation.
DEV float gg_q2_series(float h) {
    float s = fmaf(h, 1.0f / 3628800, 1.0f / 362880);
    s = fmaf(s, h, 1.0f / 40320);
    s = fmaf(s, h, 1.0f / 5040);
    s = fmaf(s, h, 1.0f / 720);
    s = fmaf(s, h, 1.0f / 120);
    s = fmaf(s, h, 1.0f / 24);
    s = fmaf(s, h, 1.0f / 6);
    s = fmaf(s, h, 0.5f);
    return (h * h) * s;
}
DEV float gg_q2f(float q, float& e1) {
    const float aq = fabsf(q);
    if (aq <= 0.5f) {
        const float Q = gg_q2_series(q);
        e1 = q + Q;
        return Q;
    }
    if (aq <= 2.0f) {
        const float h = 0.25f * q;
        float Q = gg_q2_series(h);
        float E = h + Q;
        Q = fmaf(E, E, 2.0f * Q); E = fmaf(E, E, 2.0f * E);
        Q = fmaf(E, E, 2.0f * Q); E = fmaf(E, E, 2.0f * E);
        e1 = E;
        return Q;
    }
    const float e = ex2f(mul_l2e(q)) - 1.0f;
    e1 = e;
    return e - q;
}

// lower regularised incomplete gamma P(a, y) by its power series, with dP/da and y^a e^-y / Gamma(a)
DEV void gg_inc_gamma(double a, double y, double& P, double& Pa, double& py) {
    const double ly = log(y);
    const double pref = exp(a * ly - y - lgamma(a + 1.0));
    double term = 1.0, sum = 1.0, H = 0.0, hsum = 0.0;
    for (int n = 1; n < 200; ++n) {
        term *= y / (a + n);
        H += 1.0 / (a + n);
        sum += term;
        hsum += term * H;
        if (term < 1e-18 * sum) break;
    }
    P = pref * sum;
    Pa = P * (ly - digamma_d(a + 1.0)) - pref * hsum;
    py = exp(a * ly - y - lgamma(a));
}

// Column prologue of the generalized gamma (FP64 for both precisions).  Fills the record fields
// that depend on the response (everything but TN), the band [xmin, xmax] and the adjoint record
// g (NFG values); mu, var: the column's mean and variance, p the power, deq = d E_q / d kB.
// Returns the normalisation N_k that multiplies the T_dk (mixed: the density at the mean times
// ex2_scale = 1 / (1 + b), b the SFU exponentials' measured mean relative error; FP64: 1).
template <class R>
DEV double gg_column(double mu, double var, double p, double cut, double x1, bool zero_bin, bool mixed,
                     double ex2_scale, R* f, R* z, double* gco, R& xmin, R& xmax) {
    const double a = 1.0 / p;
    const double r = log1p(var / (mu * mu));
    double Hx, lxs;                                   // dH/dx at the root, ln(d/p)
    const double xs = gg_solve_shape(r, a, lxs, Hx);  // d/p
    const double d = p * xs;
    double ls, psi, lgx, da;                          // ln(mu/s), psi(d/p), lnGamma(d/p), psi(d/p + a) - psi(d/p)
    gg_at_shape(xs, lxs, a, ls, psi, lgx, da);
    const double lns = log(mu) - ls;                  // ln s
    const double A = exp(p * ls);                     // (mu/s)^p
    const double k1 = (d - 1.0) - p * A;
    // density at the mean: ln f(mu) = ln p - ln mu + d ln(mu/s) - A - lnGamma(d/p)
    const double lfm = log(p) - log(mu) + d * ls - A - lgx;
    double Nk = 1.0;
    if (mixed) {
        Nk = exp(lfm) * ex2_scale;
        f[F_A] = (R)(1.0 / mu);
        f[F_B] = (R)(1.4426950408889634 * A);
        f[F_C] = (R)(1.4426950408889634 * k1);
    } else {
        f[F_A] = (R)(log(p) - d * lns - lgx);
        f[F_B] = (R)(d - 1.0);
        f[F_C] = (R)lns;
    }
    f[F_KAPPA] = (R)p;
    // band [xmin, xmax] where E(L) = log f/f(mu) >= -cut, in FP32 (bounds need only be conservative:
    // the cut is widened by 0.01 against the FP32 rounding of E).  E is concave in L
    // (E'' = -A p^2 e^(pL)), so Newton steps started outside the band stay outside.
    {
        const float k1f = (float)k1, Af = (float)A, pf = (float)p, cf = (float)cut + 0.01f;
        const float Lmax = 80.0f / pf;                // e^(pL) stays finite in FP32
        auto E = [&](float L, float& dE) {
            float e1;
            const float Q = gg_q2f(pf * L, e1);
            dE = fmaf(-Af * pf, e1, k1f);
            return fmaf(-Af, Q, k1f * L);
        };
        const float Ap2 = Af * pf * pf;
        // E <= k1 L - A p^2 L^2 / 2 for L >= 0: the positive root of that bound is outside the band
        float L = fminf((k1f + sqrtf(k1f * k1f + 2.0f * Ap2 * cf)) / Ap2, Lmax);
        for (int it = 0; it < 4 && L < Lmax; ++it) {
            float dE;
            const float e = E(L, dE);
            const float Ln = L - (e + cf) / dE;
            if (isfinite(Ln) && Ln > 0.0f && Ln < L) L = Ln;
        }
        xmax = L >= Lmax ? (R)1e30 : (R)(mu * (double)expf(L));
        xmin = 0;
        if (d > 1.0) {
            float Lo = -sqrtf(2.0f * cf / Ap2), dE;
            int grow = 0;
            while (E(Lo, dE) > -cf && grow < 60 && Lo > -Lmax) { Lo = 1.5f * Lo - 0.5f; ++grow; }
            if (Lo > -Lmax) {
                for (int it = 0; it < 4; ++it) {
                    const float e = E(Lo, dE);
                    const float Ln = Lo - (e + cf) / dE;
                    if (isfinite(Ln) && Ln < 0.0f && Ln > Lo) Lo = Ln;
                }
                xmin = (R)(mu * (double)expf(Lo));
            }
        }
    }
    // bin at zero: P(d/p, (x1/s)^p) and its derivatives at fixed (d, s, p)
    double P0 = 0.0, P0d = 0.0, P0s = 0.0, P0p = 0.0;
    if (zero_bin && (double)xmin <= x1) {
        const double lxs = log(x1) - lns;
        const double y = exp(p * lxs);
        double P, Pa, py;
        gg_inc_gamma(xs, y, P, Pa, py);
        P0 = P; P0d = Pa / p; P0s = -p * py; P0p = -(d / (p * p)) * Pa + py * lxs;
    }
    z[Z_P0] = (R)(P0 / Nk);
    // moment matching H(x, a) = ln rho, ln s = ln mu - G(x, a): implicit derivatives of x and u = ln s
    // dH/da = 2 [psi(x + 2a) - psi(x + a)] = 2 (dH/dx + [psi(x + a) - psi(x)]): no cancellation
    const double Ha = 2.0 * (Hx + da);
    const double Gx = da, Ga = psi + da;              // psi(x + a) = psi(x) + [psi(x + a) - psi(x)]
    const double r_mu = -2.0 * var / (mu * (mu * mu + var)), r_var = 1.0 / (mu * mu + var);
    const double x_mu = r_mu / Hx, x_var = r_var / Hx, x_p = Ha / (p * p * Hx);
    const double J_dmu = p * x_mu, J_dvar = p * x_var, J_dp = xs + p * x_p;
    const double J_umu = 1.0 / mu - Gx * x_mu, J_uvar = -Gx * x_var, J_up = -Gx * x_p + Ga / (p * p);
    // node-sum combinations (see the record comment): g_d = U1 + m0 Ur, s g_s = m1 U2 + m2 Ur,
    // g_p = m3 Ur + m4 U3 + m5 U1 + m6 (s g_s of the nodes)
    double m0, m1, m2, m3, m4, m5, m6;
    if (mixed) {
        const double cd = ls - psi / p;
        m0 = cd; m1 = p * A; m2 = -(1.0 + k1);
        m3 = 1.0 / p - (d / p) * cd; m4 = -A; m5 = -A; m6 = -ls / p;
    } else {
        m0 = -psi / p; m1 = p; m2 = -d;
        m3 = 1.0 / p + d * psi / (p * p); m4 = -1.0; m5 = 0.0; m6 = 0.0;
    }
    const double gd[5] = {m0, 1.0, 0.0, 0.0, P0d / Nk};
    const double gs[5] = {m2, 0.0, m1, 0.0, P0s / Nk};
    const double gp[5] = {m3 + m6 * m2, m5, m6 * m1, m4, P0p / Nk};
    double row[3][5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        row[0][i] = J_dmu * gd[i] + J_umu * gs[i];
        row[1][i] = J_dvar * gd[i] + J_uvar * gs[i];
        row[2][i] = gp[i] + J_dp * gd[i] + J_up * gs[i];
    }
    if (mixed) {
        // the mixed adjoint accumulates f Q with Q = E1 - pL (relative precision) instead of f E1:
        // the first-order parts of the L and E1 sums, which cancel in the variance and power
        // derivatives, then combine here in FP64
        for (int r3 = 0; r3 < 3; ++r3) row[r3][1] += p * row[r3][2];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        gco[FG_MU + i] = row[0][i];
        gco[FG_VAR + i] = row[1][i];
        gco[FG_P + i] = row[2][i];
    }
    gco[15] = 0;
    return Nk;
}

// mixed bin value of a generalized-gamma column relative to its density at the mean:
// sum_n w_n exp(E(L_n)), L_n = ln(x_c/mu) + ln(x_n/x_c)
template <int NG>
DEV float gg_bin_value_f(const float* c, float xc, const float* lam, const float* wt) {
    const float Dx = (xc - c[F_MUH]) - c[F_MUL];
    float Lc;
    log1pmx2_f(Dx * c[F_A], Lc);
    const float p = c[F_KAPPA], Ap = c[F_B], Kp = c[F_C];
    float rho = 0.0f;
#pragma unroll
    for (int n = 0; n < NG; ++n) {
        const float L = Lc + lam[n];
        float e1;
        const float Q = gg_q2f(p * L, e1);
        rho = fmaf(wt[n], ex2f(fmaf(-Ap, Q, Kp * L)), rho);   // the large term A Q rounded once
    }
    return rho;
}

// Linear bins, 3-node rule (nodes left, centre, right): the side nodes from the centre node by
// Q(q + e) = Q(q) + Q(e) + E1(q) E1(e), E1 = e^q - 1 (exact), with e = p ln(x_n / x_c) fixed per
// bin and toy.  The terms are O(q^2, e^2, q e): where they cancel (a side node at the mean) the
// result is O(e^2) with an absolute error of a few ulp of it, far below the exponent's rounding.
struct GGSides { float dlam0, dlam2, Q0, Q2, E0, E2; };
DEV GGSides gg_sides(float p, const float* lam) {
    GGSides g;
    g.dlam0 = lam[0] - lam[1];
    g.dlam2 = lam[2] - lam[1];
    g.Q0 = gg_q2f(p * g.dlam0, g.E0);
    g.Q2 = gg_q2f(p * g.dlam2, g.E2);
    return g;
}
DEV float gg_bin_value_f3(const float* c, float xc, const float* lam, const float* wt, const GGSides& sd) {
    const float Dx = (xc - c[F_MUH]) - c[F_MUL];
    float Lc;
    log1pmx2_f(Dx * c[F_A], Lc);
    const float p = c[F_KAPPA], Ap = c[F_B], Kp = c[F_C];
    const float L1 = Lc + lam[1];
    float e1;
    const float Q = gg_q2f(p * L1, e1);
    const float Ql = fmaf(e1, sd.E0, Q + sd.Q0), Qr = fmaf(e1, sd.E2, Q + sd.Q2);
    const float vl = ex2f(fmaf(-Ap, Ql, Kp * (L1 + sd.dlam0)));
    const float vc = ex2f(fmaf(-Ap, Q, Kp * L1));
    const float vr = ex2f(fmaf(-Ap, Qr, Kp * (L1 + sd.dlam2)));
    return fmaf(wt[0], vl, fmaf(wt[1], vc, wt[2] * vr));
}

// FP64 bin value: sum_n w_n exp(ln p - d ln s - lnGamma(d/p) + (d-1) ln x_n - (x_n/s)^p)
template <int NG>
DEV double gg_bin_value_d(const double* c, const double* lx, const double* wt) {
    double rho = 0.0;
#pragma unroll
    for (int n = 0; n < NG; ++n) {
        const double y = exp(c[F_KAPPA] * (lx[n] - c[F_C]));
        rho = fma(wt[n], exp(fma(c[F_B], lx[n], c[F_A]) - y), rho);
    }
    return rho;
}

}  // namespace gsn
