// Mixed-precision response kernels (FP32 response build and contraction).
//
// k_forward_m   lanes <-> 32 bins of one toy; the warp streams the column
//               records of its band in batches of 32: each lane prefetches one
//               record into registers while the warp evaluates the previous
//               batch from a per-warp shared-memory copy, so record loads stay
//               off the critical path.  A ballot over the batch skips columns
//               whose band misses the warp's bins.
// k_backward_m  lanes <-> 32 columns; the warp streams the per-bin data of its
//               band (node offsets, weights, w_dj) the same way.  The adjoint
//               accumulates dNLL/dmu_k at fixed variance and dNLL/dsigma_k^2 at
//               fixed mean directly (no chain rule through shape and scale).
//               Its common case (gamma columns of shape >= D_POLY) evaluates two
//               bins per instruction with the packed FP32 operations of sm_100+
//               (fma / add / mul .rn.f32x2): the adjoint is FP32-issue bound, and
//               the packed form halves its instruction count.  (The forward stays
//               scalar: its chains are short between SFU operations, and packing
//               two columns into one chain left it latency bound and slower.)
// Both use the symmetric 3-point Gauss-Legendre rule of linear bins (centre
// node without offset terms); bins below the log-spaced threshold and the bin
// at zero take the general node table.  FP32 partial sums are folded per batch
// into compensated (TwoSum) accumulators.
#include "gsn_device.cuh"

namespace gsn {

constexpr float SQ_HALF_L2E = 0.84932180028801904f;   // sqrt(log2(e) / 2)
constexpr float SQ_HALF_L2E_LO = (float)(0.84932180028801904 - (double)SQ_HALF_L2E);
// Columns of shape d >= D_POLY take a branch-free series for ln(1+t) - t, through u^11
// (u = t/(2+t)): inside their band |u| <= 0.5 (d = 50, the far left tail; 0.35 at d = 100), and
// the omitted terms, 2 u^13/13 + ..., change a column's mass over its band by at most 4e-10
// (d = 50; 6e-12 at d = 100, 1e-14 at d = 300), below the FP32 roundings of its constants.
constexpr float D_POLY = 50.0f;

// record fields after the per-warp transformation of the forward kernel
//   q0 = (mu_hi, mu_lo, A, P)   q1 = (Q, R, -XM, -L2E A)   q2 = (TN0, TN1, TN2, TN3)
//   gamma: A = 1/mu, P = L2E d, Q = L2E (d-1), R = L2E C (C = -1/s)
//   gauss: A = sqrt(L2E/2)/sigma
struct RecF {
    float4 q0, q1, q2;
};
// the two-bin forward's record: P = L2E d of the general (scalar) path sits in the TN3 slot when
// the group has at most three datasets (48 bytes), in a fourth vector otherwise (64 bytes)
template <bool WIDE> struct RecG;
template <> struct RecG<false> {
    float4 q0, q1, q2;
    DEV float P() const { return q2.w; }
};
template <> struct RecG<true> {
    float4 q0, q1, q2, q3;
    DEV float P() const { return q3.x; }
};

template <int RES>
DEV RecF transform_record(const float4 r0, const float4 r1, const float4 r2, const float4 r3) {
    RecF o;
    if (RES == 1) {
        o.q0 = make_float4(r0.x, r0.y, r0.z, mul_l2e(r0.w));
        o.q1 = make_float4(fmaf(L2E, r0.w, fmaf(L2E_LO, r0.w - 1.0f, -L2E)), mul_l2e(r1.x), -r3.z, -mul_l2e(r0.z));
    } else {
        o.q0 = make_float4(r0.x, r0.y, fmaf(SQ_HALF_L2E, r0.z, r0.z * SQ_HALF_L2E_LO), 0.f);
        o.q1 = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    o.q2 = make_float4(r2.z, r2.w, r3.x, r3.y);  // TN0..TN3 (record fields F_TN0..F_TN0 + 3)
    return o;
}

// ---- packed FP32 (two lanes of work per instruction: fma / add / mul .rn.f32x2 on sm_100+) ----
DEV float2 f2(float x) { return make_float2(x, x); }
DEV float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
DEV float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
DEV float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
DEV float2 ex2f2(float2 x) { return make_float2(ex2f(x.x), ex2f(x.y)); }
DEV float2 rcp2(float2 x) {
    float2 r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(x.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(x.y));
    return r;
}
// D(t) = ln(1 + t) - t of log1pmx_poly for two arguments; nt = -t
DEV float2 log1pmx_poly2(float2 t, float2 nt) {
    const float2 u = mul2(t, rcp2(add2(t, f2(2.0f))));
    const float2 v = mul2(u, u);
    float2 p = fma2(v, f2(2.0f / 11.0f), f2(2.0f / 9.0f));
    p = fma2(p, v, f2(2.0f / 7.0f));
    p = fma2(p, v, f2(2.0f / 5.0f));
    p = fma2(p, v, f2(2.0f / 3.0f));
    return mul2(u, fma2(v, p, nt));  // u (v p - t)
}

// value of one linear bin for a column of shape d >= D_POLY:
// log2 f(x)/f(mu) - XM = L2E ((d-1) D(t) - t) - XM, t = x/mu - 1
DEV float pair_value_poly(const RecF& c, float xc, float dl, float lp, float lm, float w0, float w1) {
    const float Dx = (xc - c.q0.x) - c.q0.y;
    const float tt = Dx * c.q0.z;
    const float Ec = fmaf(c.q1.x, log1pmx_poly(tt), fmaf(Dx, c.q1.w, c.q1.z));
    const float cd = c.q1.y * dl;
    const float ap = fmaf(c.q1.x, lp, Ec) + cd;
    const float am = fmaf(c.q1.x, lm, Ec) - cd;
    return fmaf(w1, ex2f(ap) + ex2f(am), w0 * ex2f(Ec));
}

// value of one linear bin (symmetric 3-node rule) for one column
template <int RES>
DEV float pair_value(const RecF& c, float xc, float dl, float lp, float lm, float w0, float w1) {
    const float Dx = (xc - c.q0.x) - c.q0.y;
    if (RES == 1) {
        const float tt = Dx * c.q0.z;
        float L1;
        const float Dt = log1pmx2_f(tt, L1);
        const float Ec = fmaf(c.q0.w, Dt, fmaf(-L2E, L1, c.q1.z));
        const float cd = c.q1.y * dl;
        const float ap = fmaf(c.q1.x, lp, Ec) + cd;
        const float am = fmaf(c.q1.x, lm, Ec) - cd;
        return fmaf(w1, ex2f(ap) + ex2f(am), w0 * ex2f(Ec));
    } else {
        const float z = Dx * c.q0.z;
        const float dz = dl * c.q0.z;
        const float zp = z + dz, zm = z - dz;
        return fmaf(w1, ex2f(-zp * zp) + ex2f(-zm * zm), w0 * ex2f(-z * z));
    }
}

// ------------------------------------------------------------- forward -----
template <int RES, int NDS, bool FAST>
__global__ void __launch_bounds__(FWD_WARPS * 32) k_forward_m(KArgs a) {
    const int tile = blockIdx.x, split = blockIdx.y;
    const int t = blockIdx.z / a.G, g = blockIdx.z % a.G;
    if (!tb_g_active<FAST>(a, g)) return;  // no smeared species in the group
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ RecF srec[FWD_WARPS][32];
    int wlo, whi;
    toy_window_union<FAST>(a, t, g, wlo, whi);
    // warps tile the toy's window from its first bin, so no warp starts outside it
    const int j0 = wlo + (tile * FWD_WARPS + warp) * 32;
    if (j0 >= whi) return;
    const int j = j0 + lane;
    const bool valid = j < whi;
    const int jr = min(j, whi - 1);
    const int nb = tb_g_node_off<FAST>(a, g) + jr;
    const int jf = j0, jl = min(j0 + 31, whi - 1);
    const float xlo_w = (float)a.edges[tb_g_edge_off<FAST>(a, g) + jf];
    const float xhi_w = (float)a.edges[tb_g_edge_off<FAST>(a, g) + jl + 1];
    const int nds = tb_g_nds<FAST>(a, g);
    const int kchunk = (a.K + a.nsplit - 1) / a.nsplit;
    const int k_beg = split * kchunk, k_end = min(a.K, k_beg + kchunk);
    const float* blk = reinterpret_cast<const float*>(a.blkbuf) + ((long long)t * a.G + g) * a.nblk * 2;

    // column range of the band: first and last 256-column block that overlaps
    int kfirst = k_end, klast = k_beg;
    for (int b = k_beg / COLBLK; b * COLBLK < k_end; ++b) {
        if (blk[2 * b + 1] < xlo_w || blk[2 * b] > xhi_w) continue;
        kfirst = min(kfirst, max(b * COLBLK, k_beg));
        klast = max(klast, min((b + 1) * COLBLK, k_end));
    }

    double accd[MAXGDS] = {};
    int ncol = 0;
    if (j0 < tb_g_jlin<FAST>(a, g)) {  // the warp holds bins below the first linear bin
        // warp holds bins of the general node table (log-spaced or the bin at zero)
        const unsigned char cls = a.bclass[nb];
        const float* nodes = a.ntab_f + (long long)nb * 3 * NGM_F;
        const float xc = a.xc_f[nb];
        float del[NG_LOG_F], lam[NG_LOG_F], wt[NG_LOG_F];
#pragma unroll
        for (int n = 0; n < NG_LOG_F; ++n) {
            del[n] = nodes[n]; lam[n] = nodes[NGM_F + n]; wt[n] = valid ? nodes[2 * NGM_F + n] : 0.f;
        }
        for (int k = kfirst; k < klast; ++k) {
            const float* c = colrec<float>(a, t, g, k);
            if (c[F_XMAX] < xlo_w || c[F_XMIN] > xhi_w) continue;
            ++ncol;
            float v = bin_value_f<RES, NG_LOG_F>(c, xc, del, lam, wt);
            if (RES == 1 && cls == BIN_ZERO) v = valid ? zerorec<float>(a, t, g, k)[Z_P0] : 0.0f;
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd)
                if (dd < nds) accd[dd] += (double)(v * c[F_TN0 + dd]);
        }
    } else {
        const float4 b0 = reinterpret_cast<const float4*>(a.btab_f)[2 * nb];
        const float4 b1 = reinterpret_cast<const float4*>(a.btab_f)[2 * nb + 1];
        const float xc = b0.x, dl = b0.y, lp = b0.z, lm = b0.w;
        const float w0 = valid ? b1.x : 0.f, w1 = valid ? b1.y : 0.f;
        float s[MAXGDS] = {}, cc[MAXGDS] = {};
        const float4* rec = reinterpret_cast<const float4*>(colrec<float>(a, t, g, 0));
        float4 r0 = make_float4(0, 0, 0, 0), r1 = r0, r2 = r0, r3 = r0;
        auto load = [&](int k) {
            if (k < klast) {
                const float4* p = rec + (long long)k * 4;
                r0 = p[0]; r1 = p[1]; r2 = p[2]; r3 = p[3];
            } else {
                r2 = make_float4(INFINITY, -INFINITY, 0.f, 0.f);
            }
        };
        load(kfirst + lane);
        for (int kb = kfirst; kb < klast; kb += 32) {
            const bool hit = !(r2.y < xlo_w || r2.x > xhi_w);  // (XMIN, XMAX) of column kb + lane
            unsigned m = __ballot_sync(0xffffffffu, hit);
            // every column of the batch has shape >= D_POLY (or is not evaluated)
            const bool poly = RES == 1 && __all_sync(0xffffffffu, !hit || r0.w >= D_POLY);
            srec[warp][lane] = transform_record<RES>(r0, r1, r2, r3);
            __syncwarp();
            load(kb + 32 + lane);
            ncol += __popc(m);
            float acc[MAXGDS] = {};
            auto one = [&](int cidx) {
                const RecF c = srec[warp][cidx];
                const float v = pair_value<RES>(c, xc, dl, lp, lm, w0, w1);
                acc[0] = fmaf(v, c.q2.x, acc[0]);
                if (NDS > 1) acc[1] = fmaf(v, c.q2.y, acc[1]);
                if (NDS > 2) acc[2] = fmaf(v, c.q2.z, acc[2]);
                if (NDS > 3) acc[3] = fmaf(v, c.q2.w, acc[3]);
            };
            if (m == 0xffffffffu && poly) {
                // dense batch of wide columns: branch-free evaluation, several chains in flight
#pragma unroll 4
                for (int cidx = 0; cidx < 32; ++cidx) {
                    const RecF c = srec[warp][cidx];
                    const float v = pair_value_poly(c, xc, dl, lp, lm, w0, w1);
                    acc[0] = fmaf(v, c.q2.x, acc[0]);
                    if (NDS > 1) acc[1] = fmaf(v, c.q2.y, acc[1]);
                    if (NDS > 2) acc[2] = fmaf(v, c.q2.z, acc[2]);
                    if (NDS > 3) acc[3] = fmaf(v, c.q2.w, acc[3]);
                }
            } else if (m == 0xffffffffu) {
                // every column of the batch reaches the warp's bins: fixed trip count, two chains in flight
#pragma unroll 2
                for (int cidx = 0; cidx < 32; ++cidx) one(cidx);
            } else {
                while (m) {
                    const int cidx = __ffs(m) - 1;
                    m &= m - 1;
                    one(cidx);
                }
            }
#pragma unroll
            for (int dd = 0; dd < NDS; ++dd) two_sum_acc(s[dd], cc[dd], acc[dd]);
            __syncwarp();
        }
#pragma unroll
        for (int dd = 0; dd < MAXGDS; ++dd) accd[dd] = (double)s[dd] + (double)cc[dd];
    }
    if (a.work) {
        const unsigned m = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) atomicAdd(&a.work[K_FORWARD], (unsigned long long)ncol * __popc(m));
    }
    if (valid) {
        double* out = a.mubuf + ((long long)t * a.nsplit + split) * a.total_bins;
#pragma unroll
        for (int dd = 0; dd < MAXGDS; ++dd)
            if (dd < nds) out[tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, dd)) + j] = accd[dd];
    }
}

// ------------------------------------------------- forward, gamma, 2 bins per lane -----
// Record fields of the two-bin forward after the per-warp transformation (negated copies let the
// packed operations form differences without an extra negation; all negations are exact):
//   q0 = (-mu_hi, -mu_lo, A, -A)   q1 = (Q, R, -XM, -L2E A)   q2 = (TN0, TN1, TN2, TN3 | P)   [q3 = (P, -, -, -)]
//   A = 1/mu, P = L2E d, Q = L2E (d-1), R = L2E C (C = -1/s), XM the column's exponent offset
template <bool WIDE>
DEV RecG<WIDE> transform_record_g2(const float4 r0, const float4 r1, const float4 r2, const float4 r3) {
    RecG<WIDE> o;
    const float R = mul_l2e(r1.x);
    o.q0 = make_float4(-r0.x, -r0.y, r0.z, -r0.z);
    o.q1 = make_float4(fmaf(L2E, r0.w, fmaf(L2E_LO, r0.w - 1.0f, -L2E)), R, -r3.z, -mul_l2e(r0.z));
    if constexpr (WIDE) {
        o.q2 = make_float4(r2.z, r2.w, r3.x, r3.y);
        o.q3 = make_float4(mul_l2e(r0.w), 0.f, 0.f, 0.f);
    } else {
        o.q2 = make_float4(r2.z, r2.w, r3.x, mul_l2e(r0.w));
    }
    return o;
}

// two linear bins of one column (shape d >= D_POLY), packed: the scalar pair_value_poly per lane half;
// ndl = -dl, so that each side node's exponent is two fused operations
template <class Rec>
DEV float2 pair_value_poly2(const Rec& c, float2 xc, float2 dl, float2 ndl, float2 lp, float2 lm, float2 w0, float2 w1) {
    const float2 Dx = add2(add2(xc, f2(c.q0.x)), f2(c.q0.y));
    const float2 D = log1pmx_poly2(mul2(Dx, f2(c.q0.z)), mul2(Dx, f2(c.q0.w)));
    const float2 Ec = fma2(f2(c.q1.x), D, fma2(Dx, f2(c.q1.w), f2(c.q1.z)));
    const float2 ap = fma2(f2(c.q1.y), dl, fma2(f2(c.q1.x), lp, Ec));
    const float2 am = fma2(f2(c.q1.y), ndl, fma2(f2(c.q1.x), lm, Ec));
    return fma2(w1, add2(ex2f2(ap), ex2f2(am)), mul2(w0, ex2f2(Ec)));
}

// one linear bin of one column, any shape (the scalar pair_value<1> on the two-bin record layout)
template <class Rec>
DEV float pair_value_g2(const Rec& c, float xc, float dl, float lp, float lm, float w0, float w1) {
    const float Dx = (xc + c.q0.x) + c.q0.y;
    float L1;
    const float Dt = log1pmx2_f(Dx * c.q0.z, L1);
    const float Ec = fmaf(c.P(), Dt, fmaf(-L2E, L1, c.q1.z));
    const float cd = c.q1.y * dl;
    const float ap = fmaf(c.q1.x, lp, Ec) + cd;
    const float am = fmaf(c.q1.x, lm, Ec) - cd;
    return fmaf(w1, ex2f(ap) + ex2f(am), w0 * ex2f(Ec));
}

// Gamma response, lanes <-> bins j0 + lane and j0 + 32 + lane (64 bins per warp): the column record of
// a batch is read once from shared memory for both bins, and the common case (every column of the
// batch reaches the warp and has shape >= D_POLY) evaluates the two bins with packed FP32 operations.
// Otherwise as k_forward_m.
// 64-bin segments of every (toy, group) window, as an exclusive prefix: warp w of the forward takes
// segment w - segoff[i] of the (toy, group) i with segoff[i] <= w < segoff[i + 1], so the blocks of
// the forward hold only warps with work (a block whose warps had left early would keep its
// registers until its last warp finished).  One block; T G <= 65535.
template <bool FAST>
__global__ void __launch_bounds__(1024) k_fwd_segments(KArgs a) {
    __shared__ int part[1024];
    const int n = a.T * a.G;
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
    auto nseg = [&](int i) {
        const int t = i / a.G, g = i % a.G;
        if (!tb_g_active<FAST>(a, g)) return 0;
        int wlo, whi;
        toy_window_union<FAST>(a, t, g, wlo, whi);
        return whi > wlo ? (whi - wlo + 63) / 64 : 0;
    };
    int sum = 0;
    for (int i = i0; i < i1; ++i) sum += nseg(i);
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {  // inclusive scan of the per-thread sums
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = part[threadIdx.x] - sum;
    for (int i = i0; i < i1; ++i) { a.segoff[i] = run; run += nseg(i); }
    if (threadIdx.x == blockDim.x - 1) a.segoff[n] = part[threadIdx.x];
}

// resident 256-thread blocks per SM the two-bin forward's register budget is sized for
#ifndef GSN_FWD_MINBLOCKS
#define GSN_FWD_MINBLOCKS 3
#endif

template <int NDS, bool FAST>
__global__ void __launch_bounds__(FWD_WARPS * 32, GSN_FWD_MINBLOCKS) k_forward_m2(KArgs a) {
    const int split = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this warp's (toy, group) and segment: the last i with segoff[i] <= gw (a warp-uniform search)
    const int gw = blockIdx.x * FWD_WARPS + warp;
    const int n = a.T * a.G;
    if (gw >= a.segoff[n]) return;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (a.segoff[mid] <= gw) lo = mid; else hi = mid;
    }
    const int t = lo / a.G, g = lo % a.G;
    constexpr bool WIDE = NDS > 3;
    __shared__ RecG<WIDE> srec[FWD_WARPS][32];
    int wlo, whi;
    toy_window_union<FAST>(a, t, g, wlo, whi);
    const int j0 = wlo + (gw - a.segoff[lo]) * 64;
    const int jj[2] = {j0 + lane, j0 + 32 + lane};
    const bool valid[2] = {jj[0] < whi, jj[1] < whi};
    const int nb[2] = {tb_g_node_off<FAST>(a, g) + min(jj[0], whi - 1), tb_g_node_off<FAST>(a, g) + min(jj[1], whi - 1)};
    const int jl = min(j0 + 63, whi - 1);
    const float xlo_w = (float)a.edges[tb_g_edge_off<FAST>(a, g) + j0];
    const float xhi_w = (float)a.edges[tb_g_edge_off<FAST>(a, g) + jl + 1];
    const int nds = tb_g_nds<FAST>(a, g);
    const int kchunk = (a.K + a.nsplit - 1) / a.nsplit;
    const int k_beg = split * kchunk, k_end = min(a.K, k_beg + kchunk);
    const float* blk = reinterpret_cast<const float*>(a.blkbuf) + ((long long)t * a.G + g) * a.nblk * 2;

    // column range of the band: first and last 256-column block that overlaps
    int kfirst = k_end, klast = k_beg;
    for (int b = k_beg / COLBLK; b * COLBLK < k_end; ++b) {
        if (blk[2 * b + 1] < xlo_w || blk[2 * b] > xhi_w) continue;
        kfirst = min(kfirst, max(b * COLBLK, k_beg));
        klast = max(klast, min((b + 1) * COLBLK, k_end));
    }

    double accd[2][MAXGDS] = {};
    int ncol = 0;
    if (j0 < tb_g_jlin<FAST>(a, g)) {
        // the warp holds bins below the first linear bin: general node table, one half at a time
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned char cls = a.bclass[nb[h]];
            const float* nodes = a.ntab_f + (long long)nb[h] * 3 * NGM_F;
            const float xc = a.xc_f[nb[h]];
            float del[NG_LOG_F], lam[NG_LOG_F], wt[NG_LOG_F];
#pragma unroll
            for (int n = 0; n < NG_LOG_F; ++n) {
                del[n] = nodes[n]; lam[n] = nodes[NGM_F + n]; wt[n] = valid[h] ? nodes[2 * NGM_F + n] : 0.f;
            }
            int nc = 0;
            for (int k = kfirst; k < klast; ++k) {
                const float* c = colrec<float>(a, t, g, k);
                if (c[F_XMAX] < xlo_w || c[F_XMIN] > xhi_w) continue;
                ++nc;
                float v = bin_value_f<1, NG_LOG_F>(c, xc, del, lam, wt);
                if (cls == BIN_ZERO) v = valid[h] ? zerorec<float>(a, t, g, k)[Z_P0] : 0.0f;
#pragma unroll
                for (int dd = 0; dd < MAXGDS; ++dd)
                    if (dd < nds) accd[h][dd] += (double)(v * c[F_TN0 + dd]);
            }
            ncol = nc;
        }
    } else {
        const float4 a0 = reinterpret_cast<const float4*>(a.btab_f)[2 * nb[0]];
        const float4 a1 = reinterpret_cast<const float4*>(a.btab_f)[2 * nb[0] + 1];
        const float4 b0 = reinterpret_cast<const float4*>(a.btab_f)[2 * nb[1]];
        const float4 b1 = reinterpret_cast<const float4*>(a.btab_f)[2 * nb[1] + 1];
        const float2 xc = make_float2(a0.x, b0.x), dl = make_float2(a0.y, b0.y), ndl = make_float2(-a0.y, -b0.y);
        const float2 lp = make_float2(a0.z, b0.z), lm = make_float2(a0.w, b0.w);
        const float2 w0 = make_float2(valid[0] ? a1.x : 0.f, valid[1] ? b1.x : 0.f);
        const float2 w1 = make_float2(valid[0] ? a1.y : 0.f, valid[1] ? b1.y : 0.f);
        float s[2][MAXGDS] = {}, cc[2][MAXGDS] = {};
        const float4* rec = reinterpret_cast<const float4*>(colrec<float>(a, t, g, 0));
        float4 r0 = make_float4(0, 0, 0, 0), r1 = r0, r2 = r0, r3 = r0;
        auto load = [&](int k) {
            if (k < klast) {
                const float4* p = rec + (long long)k * 4;
                r0 = p[0]; r1 = p[1]; r2 = p[2]; r3 = p[3];
            } else {
                r2 = make_float4(INFINITY, -INFINITY, 0.f, 0.f);
            }
        };
        load(kfirst + lane);
        for (int kb = kfirst; kb < klast; kb += 32) {
            const bool hit = !(r2.y < xlo_w || r2.x > xhi_w);  // (XMIN, XMAX) of column kb + lane
            unsigned m = __ballot_sync(0xffffffffu, hit);
            // every column of the batch has shape >= D_POLY (or is not evaluated)
            const bool poly = __all_sync(0xffffffffu, !hit || r0.w >= D_POLY);
            srec[warp][lane] = transform_record_g2<WIDE>(r0, r1, r2, r3);
            __syncwarp();
            load(kb + 32 + lane);
            ncol += __popc(m);
            float2 acc[MAXGDS] = {};
            if (m == 0xffffffffu && poly) {
                // dense batch of wide columns: both bins per instruction, four columns in flight
#pragma unroll 4
                for (int cidx = 0; cidx < 32; ++cidx) {
                    const RecG<WIDE> c = srec[warp][cidx];
                    const float2 v = pair_value_poly2(c, xc, dl, ndl, lp, lm, w0, w1);
                    acc[0] = fma2(v, f2(c.q2.x), acc[0]);
                    if (NDS > 1) acc[1] = fma2(v, f2(c.q2.y), acc[1]);
                    if (NDS > 2) acc[2] = fma2(v, f2(c.q2.z), acc[2]);
                    if (NDS > 3) acc[3] = fma2(v, f2(c.q2.w), acc[3]);
                }
            } else {
                while (m) {
                    const int cidx = __ffs(m) - 1;
                    m &= m - 1;
                    const RecG<WIDE> c = srec[warp][cidx];
                    const float va = pair_value_g2(c, xc.x, dl.x, lp.x, lm.x, w0.x, w1.x);
                    const float vb = pair_value_g2(c, xc.y, dl.y, lp.y, lm.y, w0.y, w1.y);
                    const float tn[MAXGDS] = {c.q2.x, c.q2.y, c.q2.z, WIDE ? c.q2.w : 0.f};
#pragma unroll
                    for (int dd = 0; dd < NDS; ++dd) {
                        acc[dd].x = fmaf(va, tn[dd], acc[dd].x);
                        acc[dd].y = fmaf(vb, tn[dd], acc[dd].y);
                    }
                }
            }
#pragma unroll
            for (int dd = 0; dd < NDS; ++dd) {
                two_sum_acc(s[0][dd], cc[0][dd], acc[dd].x);
                two_sum_acc(s[1][dd], cc[1][dd], acc[dd].y);
            }
            __syncwarp();
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int dd = 0; dd < MAXGDS; ++dd) accd[h][dd] = (double)s[h][dd] + (double)cc[h][dd];
    }
    if (a.work) {
        const unsigned bins = __popc(__ballot_sync(0xffffffffu, valid[0])) + __popc(__ballot_sync(0xffffffffu, valid[1]));
        if (lane == 0) atomicAdd(&a.work[K_FORWARD], (unsigned long long)ncol * bins);
    }
    double* out = a.mubuf + ((long long)t * a.nsplit + split) * a.total_bins;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!valid[h]) continue;
#pragma unroll
        for (int dd = 0; dd < MAXGDS; ++dd)
            if (dd < nds) out[tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, dd)) + jj[h]] = accd[h][dd];
    }
}

// ------------------------------------------------------------ backward -----

// resident 256-thread blocks per SM the adjoint's register budget is sized for
#ifndef GSN_BW_MINBLOCKS
#define GSN_BW_MINBLOCKS 4
#endif

// SEC: the context has secondary observables (section 2.4): every pair of a bin j that lies in an
// active slice q of a dataset of the group adds U_qk N_k to its weight (k_secondary_weights); the
// batches of linear bins then end at the slices' edges, so the added weight is one per-column value
// per batch.
// Groups of three or four datasets keep twice as many accumulators: their adjoint gets the register
// budget of three resident blocks (80 registers; at 64 it spilled ~300 bytes per thread).
template <int RES, int NDS, bool FAST, bool SEC>
__global__ void __launch_bounds__(256, NDS > 2 ? 3 : GSN_BW_MINBLOCKS) k_backward_m(KArgs a) {
    const int task = blockIdx.x, g = blockIdx.y, t = blockIdx.z;
    if (!tb_g_active<FAST>(a, g)) return;  // no smeared species in the group
    const int W = a.bw_warps;
    const int cbw = task / a.bw_bsplit, bsp = task % a.bw_bsplit;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int kbase = cbw * W * 32;
    const int k = kbase + warp * 32 + lane;
    const bool kval = k < a.K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* sbin = reinterpret_cast<float4*>(smem_raw);                      // per warp 384 floats of bin data
    float* su = reinterpret_cast<float*>(smem_raw + sizeof(float4) * 3 * 32 * W);   // [MAXGDS][W*32]
    double* sresp = reinterpret_cast<double*>(smem_raw + sizeof(float4) * 3 * 32 * W + sizeof(float) * MAXGDS * W * 32);
    const int nds = tb_g_nds<FAST>(a, g);
    const int J = tb_g_bins<FAST>(a, g);
    const double* ed = a.edges + tb_g_edge_off<FAST>(a, g);
    const double* prm = a.params + (long long)t * a.params_stride;
    const double LY = prm[tb_g_resp<FAST>(a, g, 0)] * tb_g_rscale<FAST>(a, g, 0);
    const double rb = prm[tb_g_resp<FAST>(a, g, 3)] * tb_g_rscale<FAST>(a, g, 3), rc = prm[tb_g_resp<FAST>(a, g, 4)] * tb_g_rscale<FAST>(a, g, 4);
    int wlo, whi;
    toy_window_union<FAST>(a, t, g, wlo, whi);

    float c[NFP];
    {
        const float4* cr = reinterpret_cast<const float4*>(colrec<float>(a, t, g, kval ? k : a.K - 1));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 v = cr[i];
            c[4 * i] = v.x; c[4 * i + 1] = v.y; c[4 * i + 2] = v.z; c[4 * i + 3] = v.w;
        }
    }
    const float xmn = warp_min<float>(kval ? c[F_XMIN] : INFINITY);
    const float xmx = warp_max<float>(kval ? c[F_XMAX] : -INFINITY);
    int ja = 0, jb = -1;
    if (xmx >= xmn) {
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
    const float* wrow = reinterpret_cast<const float*>(a.wbuf) + (long long)t * a.total_bins;
    const float* wv0 = wrow + tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, 0));
    const float* wv1 = wrow + tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, nds > 1 ? 1 : 0));
    const float* wv2 = wrow + tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, nds > 2 ? 2 : 0));
    const float* wv3 = wrow + tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, nds > 3 ? 3 : 0));
    const float TN0 = c[F_TN0], TN1 = NDS > 1 ? c[F_TN0 + 1] : 0.f, TN2 = NDS > 2 ? c[F_TN0 + 2] : 0.f,
                TN3 = NDS > 3 ? c[F_TN0 + 3] : 0.f;
    // accumulators: U0 per dataset (rates) in [0, MAXGDS), then U1, U2 (gamma: d/dmu at fixed
    // variance, d/dvar at fixed mean, scaled by mu/d and s^2; gauss: z- and (z^2-1)-weighted sums)
    constexpr int IU1 = MAXGDS, IU2 = MAXGDS + 1;
    float sU[MAXGDS + 2] = {}, cU[MAXGDS + 2] = {};
    const float A = c[F_A];
    const float P2 = mul_l2e(c[F_B]), Q2 = fmaf(L2E, c[F_B], fmaf(L2E_LO, c[F_B] - 1.0f, -L2E)),
                R2 = mul_l2e(c[F_C]);
    const float kap = c[F_KAPPA];
    const float Ag = fmaf(SQ_HALF_L2E, A, A * SQ_HALF_L2E_LO);
    const float mL2EA = -mul_l2e(A), nXM = -c[F_XM];
    const bool wpoly = RES == 1 && __all_sync(0xffffffffu, !kval || c[F_B] >= D_POLY);
    const int jlin = tb_g_jlin<FAST>(a, g);
    const int nbase = tb_g_node_off<FAST>(a, g);
    // secondary pieces: U_qk N_k of the slices that contain bin j, summed over the group's datasets
    const float* secU = SEC ? reinterpret_cast<const float*>(a.secU) + (long long)t * a.Qtot * a.K : nullptr;
    auto sec_weight = [&](int j) -> float {
        float u = 0.f;
        if (SEC && kval)
            for (int dd = 0; dd < nds; ++dd) {
                const int q = a.sec_slice[tb_ds_off<FAST>(a, tb_g_ds<FAST>(a, g, dd)) + j];
                if (q >= 0) u += secU[(long long)q * a.K + k];
            }
        return u * c[F_N];
    };

    // bins of the general node table, one at a time
    for (int j = ja; j <= min(jb, jlin - 1); ++j) {
        const float w[MAXGDS] = {wv0[j], NDS > 1 ? wv1[j] : 0.f, NDS > 2 ? wv2[j] : 0.f, NDS > 3 ? wv3[j] : 0.f};
        float Wj = fmaf(w[0], TN0, fmaf(w[1], TN1, fmaf(w[2], TN2, w[3] * TN3)));
        if (SEC) Wj += sec_weight(j);
        const unsigned char cls = a.bclass[nbase + j];
        float rho = 0.f, u1 = 0.f, u2 = 0.f;
        if (RES == 1 && cls == BIN_ZERO) {
            const float* zr = zerorec<float>(a, t, g, kval ? k : a.K - 1);
            rho = zr[Z_P0]; u1 = zr[Z_P0D]; u2 = zr[Z_P0S];
        } else {
            const float* nd = a.ntab_f + (long long)(nbase + j) * 3 * NGM_F;
            const float Dx = (a.xc_f[nbase + j] - c[F_MUH]) - c[F_MUL];
            const int NG = cls == BIN_LOG ? NG_LOG_F : NG_LIN_F;
            if (RES == 1) {
                const float tt = Dx * A;
                float L1;
                const float Dt = log1pmx2_f(tt, L1);
                const float Ec = fmaf(P2, Dt, fmaf(-L2E, L1, nXM));
                for (int n = 0; n < NG; ++n) {
                    const float fw = nd[2 * NGM_F + n] * ex2f(Ec + fmaf(R2, nd[n], Q2 * nd[NGM_F + n]));
                    const float L1n = L1 + nd[NGM_F + n];
                    const float tn = fmaf(nd[n], A, tt);
                    rho += fw;
                    u1 = fmaf(fw, fmaf(2.0f, L1n + kap, -tn), u1);
                    u2 = fmaf(fw, -((L1n - tn) + kap), u2);
                }
            } else {
                const float z = Dx * A;
                for (int n = 0; n < NG; ++n) {
                    const float zn = fmaf(nd[n], A, z);
                    const float q = zn * zn;
                    const float fw = nd[2 * NGM_F + n] * ex2f(-fmaf(0.5f * L2E, q, q * HALF_L2E_LO));
                    rho += fw; u1 = fmaf(fw, zn, u1); u2 = fmaf(fw, fmaf(zn, zn, -1.0f), u2);
                }
            }
        }
        two_sum_acc(sU[IU1], cU[IU1], Wj * u1);
        two_sum_acc(sU[IU2], cU[IU2], Wj * u2);
#pragma unroll
        for (int dd = 0; dd < MAXGDS; ++dd) two_sum_acc(sU[dd], cU[dd], w[dd] * rho);
    }

    // linear bins in batches of 32, staged per warp as interleaved pairs (bins 2p, 2p+1): each float4
    // holds one quantity of both bins, so the packed FP32 path reads its float2 operands directly.
    //   pair p: (xc, xc', dl, dl') (lp, lp', lm, lm') (w0, w0', w1, w1') (wd0, wd0', wd1, wd1') (wd2, wd2', wd3, wd3')
    const int jstart = max(ja, jlin);
    if (jstart <= jb) {
        float4 b0 = make_float4(0, 0, 0, 0), b1 = b0;
        float bw2 = 0.f, bw3 = 0.f;
        // bins of a batch: up to 32, to jb, and (SEC) to the next slice edge
        auto blen = [&](int j) {
            const int n = min(32, jb - j + 1);
            return SEC ? min(n, a.sec_segend[nbase + j] - j) : n;
        };
        auto load = [&](int jj, int lim) {
            // bins at or past lim pad the last pair: the geometry of bin lim - 1 with zero weights
            const float4* bt = reinterpret_cast<const float4*>(a.btab_f) + 2 * (long long)(nbase + min(jj, lim - 1));
            b0 = bt[0];
            if (jj < lim) {
                const float4 x = bt[1];
                b1 = make_float4(x.x, x.y, wv0[jj], NDS > 1 ? wv1[jj] : 0.f);
                bw2 = NDS > 2 ? wv2[jj] : 0.f;
                bw3 = NDS > 3 ? wv3[jj] : 0.f;
            } else {
                b1 = make_float4(0.f, 0.f, 0.f, 0.f);
                bw2 = 0.f;
                bw3 = 0.f;
            }
        };
        int nbat = blen(jstart);
        load(jstart + lane, jstart + nbat);
        float* my = reinterpret_cast<float*>(sbin) + (long long)warp * 32 * 12;   // 16 pairs x 20 floats
        const float4* P = reinterpret_cast<const float4*>(my);
        // per-column constants of the packed path
        const float2 Av = f2(A), nAv = f2(-A), nmuhv = f2(-c[F_MUH]), nmulv = f2(-c[F_MUL]);
        const float2 Q2v = f2(Q2), R2v = f2(R2), nR2v = f2(-R2), mL2EAv = f2(mL2EA), nXMv = f2(nXM);
        const float2 kapv = f2(kap);
        const float2 TN0v = f2(TN0), TN1v = f2(TN1), TN2v = f2(TN2), TN3v = f2(TN3);
        for (int jj0 = jstart; jj0 <= jb;) {
            {
                float* q = my + (lane >> 1) * 20 + (lane & 1);
                q[0] = b0.x; q[2] = b0.y; q[4] = b0.z; q[6] = b0.w;
                q[8] = b1.x; q[10] = b1.y; q[12] = b1.z; q[14] = b1.w;
                if (NDS > 2) q[16] = bw2;
                if (NDS > 3) q[18] = bw3;
            }
            __syncwarp();
            const int jn = jj0 + nbat;
            const int nnext = jn <= jb ? blen(jn) : 0;
            load(jn + lane, min(jn + nnext, jb + 1));  // past jb: no loads beyond the band's last bin
            const int npair = (nbat + 1) >> 1;
            const float useg = SEC ? sec_weight(jj0) : 0.f;  // the batch's secondary weight
            // a4 accumulates -u2
            float2 a0 = f2(0.f), a1 = a0, a2 = a0, a3 = a0, a4 = a0, a5 = a0;  // a5: the fourth dataset
            if (RES == 1 && wpoly) {
                // shape >= D_POLY: branch-free series, exponent (d-1) D - t; two bins per instruction
#pragma unroll 2
                for (int p = 0; p < npair; ++p) {
                    const float4 X0 = P[p * 5], X1 = P[p * 5 + 1], X2 = P[p * 5 + 2], X3 = P[p * 5 + 3];
                    const float2 xc = make_float2(X0.x, X0.y), dl = make_float2(X0.z, X0.w);
                    const float2 lp = make_float2(X1.x, X1.y), lm = make_float2(X1.z, X1.w);
                    const float2 w0 = make_float2(X2.x, X2.y), w1 = make_float2(X2.z, X2.w);
                    const float2 wd0 = make_float2(X3.x, X3.y), wd1 = make_float2(X3.z, X3.w);
                    float2 wd2 = f2(0.f), wd3 = f2(0.f);
                    float2 Wj = mul2(wd0, TN0v);
                    if (NDS > 1) Wj = fma2(wd1, TN1v, Wj);
                    if (NDS > 2) {
                        const float4 X4 = P[p * 5 + 4];
                        wd2 = make_float2(X4.x, X4.y);
                        wd3 = make_float2(X4.z, X4.w);
                        Wj = fma2(wd2, TN2v, Wj);
                        if (NDS > 3) Wj = fma2(wd3, TN3v, Wj);
                    }
                    if (SEC) Wj = add2(Wj, f2(useg));  // pad bins have zero value and derivatives
                    const float2 Dx = add2(add2(xc, nmuhv), nmulv);
                    const float2 tt = mul2(Dx, Av);
                    const float2 Dt = log1pmx_poly2(tt, mul2(Dx, nAv));
                    const float2 Ec = fma2(Q2v, Dt, fma2(Dx, mL2EAv, nXMv));
                    const float2 ap = fma2(R2v, dl, fma2(Q2v, lp, Ec));
                    const float2 am = fma2(nR2v, dl, fma2(Q2v, lm, Ec));
                    const float2 e0 = mul2(w0, ex2f2(Ec));
                    const float2 ep = mul2(w1, ex2f2(ap));
                    const float2 em = mul2(w1, ex2f2(am));
                    const float2 rho = add2(add2(e0, ep), em);
                    const float2 Ls = fma2(ep, lp, mul2(em, lm));                  // sum w f ln(x_n / x_c)
                    const float2 XAn = mul2(fma2(ep, f2(-1.f), em), mul2(dl, Av));  // -sum w f (x_n - x_c) / mu
                    const float2 gk = add2(Dt, kapv);                               // D + kappa
                    const float2 cmu = fma2(f2(2.f), gk, tt);                       // 2 (ln(1+t) + kappa) - t
                    const float2 u1 = fma2(cmu, rho, fma2(f2(2.f), Ls, XAn));
                    const float2 nu2 = fma2(gk, rho, add2(XAn, Ls));
                    a0 = fma2(wd0, rho, a0);
                    if (NDS > 1) a1 = fma2(wd1, rho, a1);
                    if (NDS > 2) a2 = fma2(wd2, rho, a2);
                    if (NDS > 3) a5 = fma2(wd3, rho, a5);
                    a3 = fma2(Wj, u1, a3);
                    a4 = fma2(Wj, nu2, a4);
                }
            } else {
                for (int i = 0; i < nbat; ++i) {
                    const float* Q = my + (i >> 1) * 20 + (i & 1);
                    const float xc = Q[0], dl = Q[2], lp = Q[4], lm = Q[6];
                    const float w0 = Q[8], w1 = Q[10], wd0 = Q[12], wd1 = Q[14];
                    const float wd2 = NDS > 2 ? Q[16] : 0.f, wd3 = NDS > 3 ? Q[18] : 0.f;
                    const float Wj = fmaf(wd0, TN0, fmaf(wd1, TN1, fmaf(wd2, TN2, wd3 * TN3))) + useg;
                    const float Dx = (xc - c[F_MUH]) - c[F_MUL];
                    float rho, u1, u2;
                    if (RES == 1) {
                        const float tt = Dx * A;
                        float L1;
                        const float Dt = log1pmx2_f(tt, L1);
                        const float Ec = fmaf(P2, Dt, fmaf(-L2E, L1, nXM));
                        const float cd = R2 * dl;
                        const float e0 = w0 * ex2f(Ec);
                        const float ep = w1 * ex2f(fmaf(Q2, lp, Ec) + cd);
                        const float em = w1 * ex2f(fmaf(Q2, lm, Ec) - cd);
                        rho = e0 + ep + em;
                        const float Ls = fmaf(ep, lp, em * lm);           // sum w f ln(x_n / x_c)
                        const float XA = (ep - em) * (dl * A);             // sum w f (x_n - x_c) / mu
                        const float cmu = fmaf(2.0f, L1 + kap, -tt);
                        u1 = fmaf(cmu, rho, fmaf(2.0f, Ls, -XA));
                        u2 = fmaf(-(Dt + kap), rho, XA - Ls);
                    } else {
                        const float z = Dx * A;
                        const float dz = dl * A;
                        const float zp = z + dz, zm = z - dz;
                        const float zg = Dx * Ag, dzg = dl * Ag;
                        const float zgp = zg + dzg, zgm = zg - dzg;
                        const float e0 = w0 * ex2f(-zg * zg);
                        const float ep = w1 * ex2f(-zgp * zgp);
                        const float em = w1 * ex2f(-zgm * zgm);
                        rho = e0 + ep + em;
                        u1 = fmaf(e0, z, fmaf(ep, zp, em * zm));
                        u2 = fmaf(e0, fmaf(z, z, -1.0f), fmaf(ep, fmaf(zp, zp, -1.0f), em * fmaf(zm, zm, -1.0f)));
                    }
                    a0.x = fmaf(wd0, rho, a0.x);
                    if (NDS > 1) a1.x = fmaf(wd1, rho, a1.x);
                    if (NDS > 2) a2.x = fmaf(wd2, rho, a2.x);
                    if (NDS > 3) a5.x = fmaf(wd3, rho, a5.x);
                    a3.x = fmaf(Wj, u1, a3.x);
                    a4.x = fmaf(Wj, -u2, a4.x);
                }
            }
            two_sum_acc(sU[0], cU[0], a0.x + a0.y);
            if (NDS > 1) two_sum_acc(sU[1], cU[1], a1.x + a1.y);
            if (NDS > 2) two_sum_acc(sU[2], cU[2], a2.x + a2.y);
            if (NDS > 3) two_sum_acc(sU[3], cU[3], a5.x + a5.y);
            two_sum_acc(sU[IU1], cU[IU1], a3.x + a3.y);
            two_sum_acc(sU[IU2], cU[IU2], -(a4.x + a4.y));
            __syncwarp();
            jj0 = jn;
            nbat = nnext;
        }
    }
    if (a.work) {
        const unsigned m = __ballot_sync(0xffffffffu, kval);
        if (lane == 0 && jb >= ja) atomicAdd(&a.work[K_BACKWARD], (unsigned long long)(jb - ja + 1) * __popc(m));
    }
    // chain rule per column: mean and variance derivatives to (LY, kB, a, b, c); the record is read
    // again (an L2 hit) rather than kept in registers through the bin loops
    {
        const float4* cr = reinterpret_cast<const float4*>(colrec<float>(a, t, g, kval ? k : a.K - 1));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 v = cr[i];
            c[4 * i] = v.x; c[4 * i + 1] = v.y; c[4 * i + 2] = v.z; c[4 * i + 3] = v.w;
        }
    }
    float r[NRESP] = {0, 0, 0, 0, 0}, rc_[NRESP] = {0, 0, 0, 0, 0};
    if (kval) {
        const float U1 = sU[IU1] + cU[IU1], U2 = sU[IU2] + cU[IU2];
        const float mu = c[F_MUH] + c[F_MUL];
        float g_mu, g_var;
        if (RES == 1) {
            g_mu = U1 * (c[F_B] * A);          // (d / mu) U1
            g_var = U2 * (c[F_C] * c[F_C]);    // U2 / s^2
        } else {
            g_mu = U1 * A;
            g_var = 0.5f * U2 * A * A;
        }
        const float g_mt = fmaf(g_var, (float)rb + 2.0f * (float)rc * mu, g_mu);
        r[0] = g_mt * (mu / (float)LY);
        r[1] = g_mt * (float)LY * c[F_DEQ];
        r[2] = g_var;
        r[3] = g_var * mu;
        r[4] = g_var * mu * mu;
    }
#pragma unroll
    for (int i = 0; i < NRESP; ++i) {
        const float v = warp_sum_comp(r[i], rc_[i]);
        if (lane == 0) sresp[warp * NRESP + i] = (double)v;
    }
    for (int dd = 0; dd < MAXGDS; ++dd)
        su[dd * W * 32 + warp * 32 + lane] = kval ? (sU[dd] + cU[dd]) * c[F_N] : 0.f;
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
        if (dd < nds && a.ft.sp_kind[s] < 2 && a.rfac[tb_g_ds<FAST>(a, g, dd) * a.S + s] != 0.0) {
            const float* Srow = a.Sf + (long long)s * a.K + kbase;
            float acc = 0.f, cmp = 0.f, part32 = 0.f;
            for (int cc = 0; cc < ncol; ++cc) {
                part32 = fmaf(Srow[cc], su[dd * W * 32 + cc], part32);
                if ((cc & 31) == 31) { two_sum_acc(acc, cmp, part32); part32 = 0.f; }
            }
            two_sum_acc(acc, cmp, part32);
            v = (double)acc + (double)cmp;
        }
        part[NRESP + i] = v;
    }
}

// ------------------------------------------------ slice sums (secondary pieces) -----
// Rq[t][q][k] = N_k sum_{j in q} R_jk for the active slices q of the group's datasets, mixed
// Gaussian / gamma responses: lanes <-> columns as in the adjoint, the bins of each column's band
// inside the toy's window in batches that end at the slices' edges (sec_segend), staged per warp;
// a batch's value sum goes to the slice of every dataset that holds the batch.  Rq is cleared
// before the launch; a column belongs to one lane of one block, so its entries are only
// read-modified-written by that lane.  Grid (columns / 256, groups, toys).
template <int RES, bool FAST>
__global__ void __launch_bounds__(256) k_slice_sums_m(KArgs a) {
    const int g = blockIdx.y, t = blockIdx.z;
    if (!tb_g_active<FAST>(a, g)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = blockIdx.x * 256 + threadIdx.x;
    const bool kval = k < a.K;
    __shared__ float4 sbin[8][32 * 3];   // per warp: 16 pairs x 20 floats of bin geometry
    const int nds = tb_g_nds<FAST>(a, g);
    const int J = tb_g_bins<FAST>(a, g);
    const double* ed = a.edges + tb_g_edge_off<FAST>(a, g);
    int wlo, whi;
    toy_window_union<FAST>(a, t, g, wlo, whi);
    float c[NFP];
    {
        const float4* cr = reinterpret_cast<const float4*>(colrec<float>(a, t, g, kval ? k : a.K - 1));
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 v = cr[i];
            c[4 * i] = v.x; c[4 * i + 1] = v.y; c[4 * i + 2] = v.z; c[4 * i + 3] = v.w;
        }
    }
    const float xmn = warp_min<float>(kval ? c[F_XMIN] : INFINITY);
    const float xmx = warp_max<float>(kval ? c[F_XMAX] : -INFINITY);
    int ja = 0, jb = -1;
    if (xmx >= xmn) {
        int lo = 0, hi = J;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (ed[m + 1] <= (double)xmn) lo = m + 1; else hi = m; }
        ja = lo;
        lo = 0; hi = J;
        while (lo < hi) { const int m = (lo + hi) >> 1; if (ed[m] < (double)xmx) lo = m + 1; else hi = m; }
        jb = lo - 1;
        ja = max(ja, wlo); jb = min(jb, whi - 1);
    }
    // the dataset windows and the slice of dataset dd holding bin j if it is active (inside the window)
    int dlo[MAXGDS], dhi[MAXGDS], doff[MAXGDS];
    for (int dd = 0; dd < MAXGDS; ++dd) {
        const int d = tb_g_ds<FAST>(a, g, dd < nds ? dd : 0);
        doff[dd] = tb_ds_off<FAST>(a, d);
        dlo[dd] = max(0, a.win[(long long)t * a.win_stride + 2 * d]);
        dhi[dd] = min(J, a.win[(long long)t * a.win_stride + 2 * d + 1]);
    }
    auto active_slice = [&](int dd, int j) {
        const int q = a.sec_slice[doff[dd] + j];
        return (q >= 0 && a.sq_lo[q] >= dlo[dd] && a.sq_hi[q] <= dhi[dd]) ? q : -1;
    };
    float* Rq = reinterpret_cast<float*>(a.secRq) + (long long)t * a.Qtot * a.K;
    const float Nk = c[F_N];
    auto add_to_slices = [&](int j, float v) {
        for (int dd = 0; dd < nds; ++dd) {
            const int q = active_slice(dd, j);
            if (q >= 0 && kval) Rq[(long long)q * a.K + k] += v * Nk;
        }
    };
    const int jlin = tb_g_jlin<FAST>(a, g);
    const int nbase = tb_g_node_off<FAST>(a, g);
    // bins of the general node table, one at a time
    for (int j = ja; j <= min(jb, jlin - 1); ++j) {
        const unsigned char cls = a.bclass[nbase + j];
        float v;
        if (RES == 1 && cls == BIN_ZERO) {
            v = zerorec<float>(a, t, g, kval ? k : a.K - 1)[Z_P0];
        } else {
            const float* nd = a.ntab_f + (long long)(nbase + j) * 3 * NGM_F;
            const float xc = a.xc_f[nbase + j];
            v = cls == BIN_LOG ? bin_value_f<RES, NG_LOG_F>(c, xc, nd, nd + NGM_F, nd + 2 * NGM_F)
                               : bin_value_f<RES, NG_LIN_F>(c, xc, nd, nd + NGM_F, nd + 2 * NGM_F);
        }
        add_to_slices(j, v);
    }
    // linear bins: batches ending at slice edges, two bins per instruction for wide gamma columns
    const int jstart = max(ja, jlin);
    if (jstart > jb) return;
    const float A = c[F_A];
    const float P2 = mul_l2e(c[F_B]), Q2 = fmaf(L2E, c[F_B], fmaf(L2E_LO, c[F_B] - 1.0f, -L2E));
    const float R2 = mul_l2e(c[F_C]);
    const float Ag = fmaf(SQ_HALF_L2E, A, A * SQ_HALF_L2E_LO);
    const float mL2EA = -mul_l2e(A), nXM = -c[F_XM];
    const bool wpoly = RES == 1 && __all_sync(0xffffffffu, !kval || c[F_B] >= D_POLY);
    float* my = reinterpret_cast<float*>(sbin[warp]);
    const float4* P = reinterpret_cast<const float4*>(my);
    auto blen = [&](int j) { return min(min(32, jb - j + 1), a.sec_segend[nbase + j] - j); };
    float4 b0 = make_float4(0, 0, 0, 0), b1 = b0;
    auto load = [&](int jj, int lim) {
        const float4* bt = reinterpret_cast<const float4*>(a.btab_f) + 2 * (long long)(nbase + min(jj, lim - 1));
        b0 = bt[0];
        const float4 x = bt[1];
        b1 = jj < lim ? make_float4(x.x, x.y, 0.f, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    int nbat = blen(jstart);
    load(jstart + lane, jstart + nbat);
    const float2 Av = f2(A), nAv = f2(-A), nmuhv = f2(-c[F_MUH]), nmulv = f2(-c[F_MUL]);
    const float2 Q2v = f2(Q2), R2v = f2(R2), nR2v = f2(-R2), mL2EAv = f2(mL2EA), nXMv = f2(nXM);
    for (int jj0 = jstart; jj0 <= jb;) {
        {
            float* q = my + (lane >> 1) * 20 + (lane & 1);
            q[0] = b0.x; q[2] = b0.y; q[4] = b0.z; q[6] = b0.w;
            q[8] = b1.x; q[10] = b1.y;
        }
        __syncwarp();
        const int jn = jj0 + nbat;
        const int nnext = jn <= jb ? blen(jn) : 0;
        load(jn + lane, min(jn + nnext, jb + 1));
        bool want = false;  // some dataset of the group holds this batch in an active slice
        for (int dd = 0; dd < nds; ++dd) want |= active_slice(dd, jj0) >= 0;
        if (want) {
            float2 acc = f2(0.f);
            if (wpoly) {
                const int npair = (nbat + 1) >> 1;
#pragma unroll 2
                for (int p = 0; p < npair; ++p) {
                    const float4 X0 = P[p * 5], X1 = P[p * 5 + 1], X2 = P[p * 5 + 2];
                    const float2 xc = make_float2(X0.x, X0.y), dl = make_float2(X0.z, X0.w);
                    const float2 lp = make_float2(X1.x, X1.y), lm = make_float2(X1.z, X1.w);
                    const float2 w0 = make_float2(X2.x, X2.y), w1 = make_float2(X2.z, X2.w);
                    const float2 Dx = add2(add2(xc, nmuhv), nmulv);
                    const float2 Dt = log1pmx_poly2(mul2(Dx, Av), mul2(Dx, nAv));
                    const float2 Ec = fma2(Q2v, Dt, fma2(Dx, mL2EAv, nXMv));
                    const float2 ap = fma2(R2v, dl, fma2(Q2v, lp, Ec));
                    const float2 am = fma2(nR2v, dl, fma2(Q2v, lm, Ec));
                    acc = fma2(w1, add2(ex2f2(ap), ex2f2(am)), fma2(w0, ex2f2(Ec), acc));
                }
            } else {
                for (int i = 0; i < nbat; ++i) {
                    const float* Q = my + (i >> 1) * 20 + (i & 1);
                    const float xc = Q[0], dl = Q[2], lp = Q[4], lm = Q[6], w0 = Q[8], w1 = Q[10];
                    const float Dx = (xc - c[F_MUH]) - c[F_MUL];
                    float v;
                    if (RES == 1) {
                        const float tt = Dx * A;
                        float L1;
                        const float Dt = log1pmx2_f(tt, L1);
                        const float Ec = fmaf(P2, Dt, fmaf(-L2E, L1, nXM));
                        const float cd = R2 * dl;
                        v = fmaf(w1, ex2f(fmaf(Q2, lp, Ec) + cd) + ex2f(fmaf(Q2, lm, Ec) - cd), w0 * ex2f(Ec));
                    } else {
                        const float zg = Dx * Ag, dzg = dl * Ag;
                        const float zgp = zg + dzg, zgm = zg - dzg;
                        v = fmaf(w1, ex2f(-zgp * zgp) + ex2f(-zgm * zgm), w0 * ex2f(-zg * zg));
                    }
                    acc.x += v;
                }
            }
            add_to_slices(jj0, acc.x + acc.y);
        }
        __syncwarp();
        jj0 = jn;
        nbat = nnext;
    }
}

cudaError_t launch_slice_sums_mixed(const KArgs& a, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(a.secRq, 0, sizeof(float) * (size_t)a.T * a.Qtot * a.K, st);
    if (e != cudaSuccess) return e;
    const dim3 grid((a.K + 255) / 256, a.G, a.T);
    if (a.fast) { if (a.res == 0) k_slice_sums_m<0, true><<<grid, 256, 0, st>>>(a); else k_slice_sums_m<1, true><<<grid, 256, 0, st>>>(a); }
    else        { if (a.res == 0) k_slice_sums_m<0, false><<<grid, 256, 0, st>>>(a); else k_slice_sums_m<1, false><<<grid, 256, 0, st>>>(a); }
    return cudaGetLastError();
}

// (toy, group) pairs from which the gamma forward takes two bins per lane: below, a launch (a single
// point, a few toys) has too few 64-bin segments to fill the GPU, and one bin per lane is faster
constexpr int FWD2_MIN_PAIRS = 32;

template <int RES, bool FAST>
static cudaError_t launch_fwd(const KArgs& a, cudaStream_t st, int nds) {
    if (RES == 1 && a.T * a.G >= FWD2_MIN_PAIRS) {
        // 64 bins per warp; the grid covers every (toy, group) with the most segments a window can
        // have (a.ntile * 32 FWD_WARPS >= Jmax bins), and blocks past the last segment return at once
        k_fwd_segments<FAST><<<1, 1024, 0, st>>>(a);
        const long long nseg_max = (long long)a.T * a.G * ((a.ntile * FWD_WARPS * 32 + 63) / 64);
        dim3 grid((unsigned)((nseg_max + FWD_WARPS - 1) / FWD_WARPS), a.nsplit, 1);
        if (nds == 1) k_forward_m2<1, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else if (nds == 2) k_forward_m2<2, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else if (nds == 3) k_forward_m2<3, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        else k_forward_m2<4, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
        return cudaGetLastError();
    }
    dim3 grid(a.ntile, a.nsplit, a.T * a.G);
    if (nds == 1) k_forward_m<RES, 1, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    else if (nds == 2) k_forward_m<RES, 2, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    else if (nds == 3) k_forward_m<RES, 3, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    else k_forward_m<RES, 4, FAST><<<grid, FWD_WARPS * 32, 0, st>>>(a);
    return cudaGetLastError();
}

template <int RES, bool FAST, bool SEC>
static cudaError_t launch_bwd_sec(const KArgs& a, cudaStream_t st, int nds) {
    dim3 grid(a.nbtask, a.G, a.T);
    const int threads = a.bw_warps * 32;
    const size_t sm = sizeof(float4) * 3 * threads + sizeof(float) * MAXGDS * threads + sizeof(double) * a.bw_warps * NRESP;
    if (nds == 1) k_backward_m<RES, 1, FAST, SEC><<<grid, threads, sm, st>>>(a);
    else if (nds == 2) k_backward_m<RES, 2, FAST, SEC><<<grid, threads, sm, st>>>(a);
    else if (nds == 3) k_backward_m<RES, 3, FAST, SEC><<<grid, threads, sm, st>>>(a);
    else k_backward_m<RES, 4, FAST, SEC><<<grid, threads, sm, st>>>(a);
    return cudaGetLastError();
}

template <int RES, bool FAST>
static cudaError_t launch_bwd(const KArgs& a, cudaStream_t st, int nds) {
    return a.nsec ? launch_bwd_sec<RES, FAST, true>(a, st, nds) : launch_bwd_sec<RES, FAST, false>(a, st, nds);
}

static int max_group_datasets(const KArgs& a) { return a.max_nds > 1 ? a.max_nds : 1; }

cudaError_t launch_forward_mixed(const KArgs& a, cudaStream_t st) {
    const int nds = max_group_datasets(a);
    if (a.fast) return a.res == 0 ? launch_fwd<0, true>(a, st, nds) : launch_fwd<1, true>(a, st, nds);
    return a.res == 0 ? launch_fwd<0, false>(a, st, nds) : launch_fwd<1, false>(a, st, nds);
}

cudaError_t launch_backward_mixed(const KArgs& a, cudaStream_t st) {
    const int nds = max_group_datasets(a);
    if (a.fast) return a.res == 0 ? launch_bwd<0, true>(a, st, nds) : launch_bwd<1, true>(a, st, nds);
    return a.res == 0 ? launch_bwd<0, false>(a, st, nds) : launch_bwd<1, false>(a, st, nds);
}

}  // namespace gsn
