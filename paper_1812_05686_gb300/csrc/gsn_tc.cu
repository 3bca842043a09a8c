// Per-species contraction M[g][s][j] = sum_k R_jk S'_sk on the 5th-generation
// tensor cores (tcgen05, sm_103a), mixed precision.
//
// A CTA owns 128 bins (one TMEM lane each) x one column range x 16 species.
// For every chunk of 32 fine columns:
//   - the 128 threads generate their bin's response values R_jk (FP32, the
//     same bin quadrature as the other mixed kernels), split them into TF32
//     hi + lo parts and store both tiles in shared memory in the K-major
//     core-matrix layout (8 rows x 16 bytes per core matrix, no swizzle);
//   - one thread loads the matching S' tiles (pre-split hi / lo, 16 species x
//     32 columns) with TMA (128-byte swizzle) onto an mbarrier;
//   - the same thread issues, per k-step of 8 columns, the three products
//     A_hi B_hi + A_hi B_lo + A_lo B_hi (tcgen05.mma kind::tf32, M = 128,
//     N = 16) into FP32 accumulators in tensor memory and commits them to a
//     second mbarrier.
// The tensor-core accumulation does not round to nearest: every accumulating
// MMA loses a fraction of an ulp of its accumulator, always the same way, which
// adds up to a coherent bias of the contraction.  So the A_hi B_hi products of
// each pair of k-steps get an accumulator of their own (two per chunk), the
// small cross terms a third, and all three are read back (tcgen05.ld) after
// every chunk of 32 columns and folded into compensated FP32 sums; the partial
// sums of each column range are written in FP64 and reduced over the ranges in
// a fixed order.
// Every wait is bounded: a CTA that times out sets an error flag, waits
// (bounded) for its own operations in flight, frees its tensor memory and
// returns.
#include "gsn_device.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace gsn {

namespace {

constexpr int TC_ROWS = 128;     // bins per CTA = MMA M = TMEM lanes
constexpr int TC_N = 16;         // species per CTA = MMA N
constexpr int TC_KC = 32;        // columns per chunk (one 128-byte swizzle row of S')
constexpr uint32_t TC_TMEM_COLS = 64;  // accumulators: hi*hi of k-steps 0-1 | 2-3 | cross terms
constexpr long long WAIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

DEV void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
DEV void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
DEV bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}
// bounded wait on an mbarrier phase; false on timeout
DEV bool mbar_wait(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > WAIT_CYCLES) return false;
    return true;
}
DEV void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tm), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// shared-memory matrix descriptor: start, leading / stride byte offsets, sm100 version, layout
DEV uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(layout & 7u) << 61;
    return d;
}

// instruction descriptor: D f32, A/B tf32, K-major, M = 128, N = 16
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_ROWS >> 4) << 24);

DEV void umma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accum)
        : "memory");
}
DEV void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
DEV void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
DEV uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

struct __align__(1024) TcSmem {
    float bhi[TC_N * TC_KC];         // S'_hi tile, 16 x 128 B, 128-byte swizzle (TMA)
    float blo[TC_N * TC_KC];         // S'_lo tile
    float ahi[TC_ROWS * TC_KC];      // R_hi tile, core-matrix layout
    float alo[TC_ROWS * TC_KC];      // R_lo tile
    float4 rec[TC_KC * 4];           // column records of the chunk
    unsigned long long bar_tma, bar_mma;
    uint32_t tmem_base;
};

// offset (floats) of element (row r, column k) of a 128 x 32 K-major tile of core matrices:
// core (r/8, k/4) at 128 bytes x (8 (r/8) + k/4), row r%8 at 16 bytes, element k%4
DEV int core_off(int r, int k) { return ((r >> 3) * 8 + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3); }

template <int RES>
__global__ void __launch_bounds__(TC_ROWS) k_species_tc(const __grid_constant__ CUtensorMap tm_hi,
                                                        const __grid_constant__ CUtensorMap tm_lo, KArgs a) {
    extern __shared__ unsigned char smem_dyn[];
    TcSmem& sm = *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~(uintptr_t)1023);
    const int tile = blockIdx.x, g = blockIdx.y;
    const int split = blockIdx.z % a.tc_nsplit, sp0 = (blockIdx.z / a.tc_nsplit) * TC_N;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int J = tb_g_bins(a, g);
    const int j0 = tile * TC_ROWS;
    if (j0 >= J || !tb_g_active(a, g)) return;  // whole CTA exits before any allocation
    const int j = j0 + tid;
    const bool valid = j < J;
    const int jr = min(j, J - 1);
    const int nb = tb_g_node_off(a, g) + jr;
    const int jl = min(j0 + TC_ROWS - 1, J - 1);
    const float xlo_w = (float)a.edges[tb_g_edge_off(a, g) + j0];
    const float xhi_w = (float)a.edges[tb_g_edge_off(a, g) + jl + 1];

    // column range: this split's share of the band of the 128 bins, in whole chunks
    const float* blk = reinterpret_cast<const float*>(a.blkbuf) + (long long)g * a.nblk * 2;
    int kfirst = a.K, klast = 0;
    for (int b = 0; b < a.nblk; ++b) {
        if (blk[2 * b + 1] < xlo_w || blk[2 * b] > xhi_w) continue;
        kfirst = min(kfirst, b * COLBLK);
        klast = max(klast, min((b + 1) * COLBLK, a.K));
    }
    const int nchunk_all = klast > kfirst ? (klast - kfirst + TC_KC - 1) / TC_KC : 0;
    const int per = (nchunk_all + a.tc_nsplit - 1) / a.tc_nsplit;
    const int c_beg = split * per, c_end = min(nchunk_all, c_beg + per);

    // node table of this thread's bin (general rule: log-spaced / zero bins included)
    const unsigned char cls = a.bclass[nb];
    const float* nodes = a.ntab_f + (long long)nb * 3 * NGM_F;
    const float xc = a.xc_f[nb];
    float del[NG_LOG_F], lam[NG_LOG_F], wt[NG_LOG_F];
#pragma unroll
    for (int n = 0; n < NG_LOG_F; ++n) {
        del[n] = nodes[n]; lam[n] = nodes[NGM_F + n]; wt[n] = valid ? nodes[2 * NGM_F + n] : 0.f;
    }
    const bool low = __syncthreads_or(cls != BIN_LIN) != 0;

    const uint32_t bar_tma = smem_u32(&sm.bar_tma), bar_mma = smem_u32(&sm.bar_mma);
    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sm.tmem_base)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem_base;
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);

    float accs[TC_N], accc[TC_N];
#pragma unroll
    for (int i = 0; i < TC_N; ++i) { accs[i] = 0.f; accc[i] = 0.f; }
    uint32_t ph_tma = 0, ph_mma = 0;
    bool ok = true, tma_pending = false, mma_pending = false;
    const uint32_t sa_hi = smem_u32(sm.ahi), sa_lo = smem_u32(sm.alo);
    const uint32_t sb_hi = smem_u32(sm.bhi), sb_lo = smem_u32(sm.blo);

    for (int cc = c_beg; cc < c_end && ok; ++cc) {
        const int k0 = kfirst + cc * TC_KC;
        // column records of the chunk (one float4 per thread)
        {
            const int col = tid >> 2, part = tid & 3;
            const int k = k0 + col;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < a.K) v = reinterpret_cast<const float4*>(colrec<float>(a, 0, g, k))[part];
            else if (part == 2) v = make_float4(INFINITY, -INFINITY, 0.f, 0.f);
            sm.rec[tid] = v;
        }
        if (tid == 0) {
            mbar_expect_tx(bar_tma, 2u * TC_N * TC_KC * sizeof(float));
            tma_load_2d(sb_hi, &tm_hi, k0, sp0, bar_tma);
            tma_load_2d(sb_lo, &tm_lo, k0, sp0, bar_tma);
        }
        __syncthreads();
        // response values of this thread's bin for the 32 columns, split into TF32 hi + lo
        for (int q = 0; q < TC_KC; q += 4) {
            float hi4[4], lo4[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float* c = reinterpret_cast<const float*>(&sm.rec[(q + e) * 4]);
                float v = 0.f;
                if (!(c[F_XMAX] < xlo_w || c[F_XMIN] > xhi_w)) {
                    v = low ? bin_value_f<RES, NG_LOG_F>(c, xc, del, lam, wt) : bin_value_f<RES, NG_LIN_F>(c, xc, del, lam, wt);
                    if (RES == 1 && cls == BIN_ZERO) v = valid ? zerorec<float>(a, 0, g, k0 + q + e)[Z_P0] : 0.f;
                    v *= c[F_N];
                }
                const uint32_t h = tf32_rna(v);
                hi4[e] = __uint_as_float(h);
                lo4[e] = v - hi4[e];
            }
            *reinterpret_cast<float4*>(&sm.ahi[core_off(tid, q)]) = make_float4(hi4[0], hi4[1], hi4[2], hi4[3]);
            *reinterpret_cast<float4*>(&sm.alo[core_off(tid, q)]) = make_float4(lo4[0], lo4[1], lo4[2], lo4[3]);
        }
        fence_proxy_async();
        __syncthreads();
        // the outcome of a bounded wait is made uniform over the CTA before anyone leaves the loop
        if (__syncthreads_or(!mbar_wait(bar_tma, ph_tma))) { ok = false; tma_pending = true; break; }
        ph_tma ^= 1u;
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int s = 0; s < TC_KC / 8; ++s) {
                const uint64_t ah = smem_desc(sa_hi + 256u * s, 128, 1024, 0);
                const uint64_t al = smem_desc(sa_lo + 256u * s, 128, 1024, 0);
                const uint64_t bh = smem_desc(sb_hi + 32u * s, 16, 1024, 2);
                const uint64_t bl = smem_desc(sb_lo + 32u * s, 16, 1024, 2);
                umma_tf32(tmem + (uint32_t)(TC_N * (s >> 1)), ah, bh, (uint32_t)(s & 1));
                umma_tf32(tmem + 2u * TC_N, ah, bl, s > 0 ? 1u : 0u);
                umma_tf32(tmem + 2u * TC_N, al, bh, 1u);
            }
            umma_commit(bar_mma);
        }
        if (__syncthreads_or(!mbar_wait(bar_mma, ph_mma))) { ok = false; mma_pending = true; break; }
        ph_mma ^= 1u;
        tc_fence_after();
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            float v[16];
            tmem_ld16(taddr + (uint32_t)(TC_N * r), v);
#pragma unroll
            for (int i = 0; i < TC_N; ++i) two_sum_acc(accs[i], accc[i], v[i]);
        }
        tc_fence_before();
        __syncthreads();
    }
    if (!ok) {
        // timed out: record it, let this CTA's operations in flight finish (bounded), free TMEM
        if (tid == 0) atomicExch(a.tc_error, 1);
        if (tma_pending) mbar_wait(bar_tma, ph_tma);
        if (mma_pending) mbar_wait(bar_mma, ph_mma);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    if (a.work && tid == 0 && c_end > c_beg)
        atomicAdd(&a.work[K_SPECIES], (unsigned long long)min(TC_ROWS, J - j0) * (unsigned long long)(c_end - c_beg) * TC_KC);
    if (valid && ok) {
        double* out = a.tc_part + ((long long)split * a.G + g) * (long long)a.S * a.Jmax;
        for (int i = 0; i < TC_N && sp0 + i < a.S; ++i)
            out[(long long)(sp0 + i) * a.Jmax + j] = (double)accs[i] + (double)accc[i];
    }
}

// M[g][s][j] = fixed-order sum over the column ranges
__global__ void k_species_tc_reduce(KArgs a) {
    const long long n = (long long)a.G * a.S * a.Jmax;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int p = 0; p < a.tc_nsplit; ++p) s += a.tc_part[(long long)p * n + i];
    a.Mbuf[i] = s;
}

}  // namespace

size_t species_tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

cudaError_t launch_species_tc(const KArgs& a, const void* tm_hi, const void* tm_lo, cudaStream_t st) {
    const int nchunk = (a.S + TC_N - 1) / TC_N;
    dim3 grid((a.Jmax + TC_ROWS - 1) / TC_ROWS, a.G, a.tc_nsplit * nchunk);
    const size_t sm = species_tc_smem_bytes();
    const CUtensorMap& h = *static_cast<const CUtensorMap*>(tm_hi);
    const CUtensorMap& l = *static_cast<const CUtensorMap*>(tm_lo);
    cudaError_t e;
    if (a.res == 0) {
        e = cudaFuncSetAttribute(k_species_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_species_tc<0><<<grid, TC_ROWS, sm, st>>>(h, l, a);
    } else {
        e = cudaFuncSetAttribute(k_species_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_species_tc<1><<<grid, TC_ROWS, sm, st>>>(h, l, a);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)a.G * a.S * a.Jmax;
    k_species_tc_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// 2-D tensor map over a [rows][cols] FP32 array (row pitch cols_pad floats), box 32 x 16, 128-byte swizzle
int make_species_tensor_map(void* out, const float* dev, int rows, int cols_pad) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t gdim[2] = {(cuuint64_t)cols_pad, (cuuint64_t)rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)cols_pad * sizeof(float)};
    const cuuint32_t box[2] = {TC_KC, TC_N};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult r = encode(static_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)dev, gdim, gstride,
                              box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace gsn
