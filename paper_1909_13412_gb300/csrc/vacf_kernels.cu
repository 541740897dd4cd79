// vacf_kernels.cu -- velocity autocorrelation and mean squared displacement
// accumulators of liblbp (sm_103a).
//
// C(k) = sum_i sum_{t0} V_i(t0).V_i(t0 + k) over all time origins (the VACF of
// Section 3 / Fig. 2) and M(k) = sum_i sum_{t0} |X_i(t0 + k) - X_i(t0)|^2,
// the mean squared displacement of the same particles (X the unwrapped
// position, X(t) - X(t - 1) = V(t) by Eq. 2).  The particle kernel writes
// every step's velocities (FP32) into a ring of K + 2B samples.  Every B = 64
// samples the correlator forms, for the B new samples t and every lag k <= K,
//     G(t, k) = sum_j V_j(t) V_j(t - k)          (j over the 3 n_p components)
// -- a dense contraction -- and both observables follow from G exactly:
//   C(k) += sum_t G(t, k);
//   the squared displacement over the window (e - k, e], summed over the
//   particles, W(e, k) = sum_i |sum_{s=e-k+1}^{e} V_i(s)|^2, obeys
//     W(e, k) = W(e - 1, k - 1) + H(e, k),
//     H(e, k) = G(e, 0) + 2 sum_{m=1}^{k-1} G(e, m),
//   (|w + v|^2 = |w|^2 + 2 v.w + |v|^2 with w the window sum up to e - 1), and
//   M(k) += W(e, k) for every new sample e >= k (an origin t0 = e - k >= 0).
// So the MSD needs no positions and no per-particle state: between blocks
// only W(last sample, k), k <= K, is kept (FP64).
//
// k_vacf_mma    : CTA = 128 lags x 256 components: the products of the 64 new
//                 samples with the 191 window samples as a matrix product on
//                 the tensor cores (TF32 in three terms, FP32 accuracy); its
//                 band is G restricted to the CTA's components, written as FP32
//                 partials part[chunk][t][k].
// k_corr_gsum   : G(t, k) = sum over chunks of the partials, in chunk order, FP64.
// k_msd_scan    : H(t, k), a prefix sum over k of each G row (FP64).
// k_msd_diag    : W along the diagonals e - k = const through the block.
// k_corr_acc    : C(k) += sum_t G(t, k), M(k) += sum_e W(e, k), pair counts;
//                 the last block marks the samples done.
#include <cuda.h>
#include <cuda_runtime.h>

#include "lbp_async.cuh"
#include "lbp_internal.cuh"

namespace lbp {

using namespace async;

constexpr int VB = 64;  // samples per correlation block

// ---------------------------------------------------------------------------
// k_vacf_tc: the block correlation on the 5th-generation tensor cores.
//
// The ring keeps every sample as two fp16 planes, hi = fp16(4096 V) and
// lo = fp16(4096 V - hi): 22 significant bits (the scale keeps the tail lo in
// fp16's normal range for |V| >= 2^-12, and |V| < 16 is checked by the
// particle kernel).  The product of two samples is formed in three terms,
// a.b = a_hi b_hi + a_hi b_lo + a_lo b_hi (the dropped a_lo b_lo is below
// 2^-22 of it), so kind::f16 MMAs give FP32-level accuracy at twice the TF32
// rate and half its operand bytes.
//
// A CTA covers TC_LT = 192 lags [k0, k0 + 192) and TC_JCH = 1024 components.
// With the window rows s = s_lo + r, s_lo = tb - k0 - 191, r in [0, 256) (255
// used) as the MMA's A operand (two M = 128 tiles) and the block's 64 new
// samples as B (N = 64), the accumulator D[r][t] = sum_j V_j(s) V_j(tb + t)
// holds G(t, k0 + kk) on the band kk = t + 191 - r in [0, 192).  Per
// sub-chunk of 64 components (one 128-byte row of fp16, the width of the
// 128-byte swizzle):
//   warp 8 (one thread) loads the four operand tiles (window hi/lo, new
//          hi/lo) with TMA straight into the swizzled K-major layout the MMA
//          reads, two stages deep;
//   warp 9 (one thread) issues 2 M tiles x 4 K steps x 3 terms = 24
//          tcgen05.mma (M 128, N 64, K 16) into a fresh TMEM accumulator set
//          (two sets of 128 columns, alternating), then commits them to the
//          stage's "empty" barrier and the set's "full" barrier;
//   warps 0-7 move the set from TMEM to registers (tcgen05.ld, one row per
//          thread: warp w reads lanes 32 (w % 4).. of M tile w / 4) and add it,
//          rounded to nearest, to FP32 running sums, then release the set.
// A fresh accumulator per sub-chunk keeps the tensor core's own FP32
// accumulation to 12 products per entry.  At the end each thread writes its
// row's band entries as FP32 partials part[chunk][t][k] (scaled back by
// 2^-24), coalesced along the lags.  Every mbarrier wait is bounded; a wait
// that runs out sets ERR_TIMEOUT and a CTA abort flag, the producer then
// waits for the copies it issued and the MMA thread for the MMAs it issued,
// and TMEM is freed before the CTA leaves.
//
// Ring rows: sample m is kept at row m % cap and, for the first TC_ROWS rows,
// again at row cap + m % cap, so every window of TC_ROWS rows is contiguous
// for TMA.  With cap >= K + 320 a window that starts before sample 0 (read at
// negative row coordinates, which TMA fills with zeros) has not wrapped yet.
// ---------------------------------------------------------------------------
constexpr int TC_LT = 192;                 // lags per CTA
constexpr int TC_ROWS = 256;               // window rows: TC_LT + VB - 1 = 255, one spare
constexpr int TC_KC = 64;                  // components per sub-chunk (128 bytes of fp16)
constexpr int TC_JCH = 1024;               // components per CTA
constexpr int TC_STAGES = 2;
constexpr int TC_A_BYTES = TC_ROWS * 128;  // one plane of window rows
constexpr int TC_B_BYTES = VB * 128;       // one plane of new-sample rows
constexpr int TC_STAGE_BYTES = 2 * TC_A_BYTES + 2 * TC_B_BYTES;  // 80 KB
constexpr int TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;        // + 1024-byte alignment slack
constexpr int TC_TMEM_COLS = 256;          // two accumulator sets of 2 x 64 columns
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 2);  // + TMA warp + MMA warp

int vacf_block_samples() { return VB; }
int vacf_chunk_components() { return TC_JCH; }
int vacf_ring_dup_rows() { return TC_ROWS; }

struct VacfArgs {
    const float *ring;  // FP32 ring of the per-particle VACF, [cap][3 n_p]
    int cap;     // ring samples
    int ncomp;   // 3 n_p
    int K;
    long long *d_vacf;  // [0] t0, [1] samples done, [2] samples written, [3] block counter,
                        // [4] parity of the MSD state
    int flush;
    float *part;        // [nchunks][VB][K+1] partial G of each component chunk
    int nchunks;
    double *G, *H, *W;  // [VB][K+1] each
    double *wstate;     // [2][K+1] W(last sample, k), by parity
    double *sum;        // [K+1] VACF sums
    double *msd;        // [K+1] MSD sums
    long long *cnt;     // [K+1]
    int np;
    unsigned int *done; // block counter of the last kernel of the chain
    int *err;
    long long wait_cycles;
};

__device__ __forceinline__ bool vacf_range(const VacfArgs &A, long long &tb, long long &te) {
    tb = A.d_vacf[1];
    te = A.d_vacf[2];
    if (te - tb > VB) te = tb + VB;
    if (A.flush) return te > tb;
    return te - tb == VB;
}

// shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart
__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr) {
    return (unsigned long long)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((unsigned long long)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// D[tmem] (+)= A * B^T, fp16 operands from shared memory, FP32 accumulator
__device__ __forceinline__ void umma_f16(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on an mbarrier once every MMA issued so far by this thread completes
__device__ __forceinline__ void umma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of this thread's lane, waited for
__device__ __forceinline__ void tmem_ld16(unsigned taddr, unsigned (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_vacf_tc(const VacfArgs A, const __grid_constant__ CUtensorMap tm_win, const __grid_constant__ CUtensorMap tm_new) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    extern __shared__ unsigned char tc_smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) unsigned long long bar_full[TC_STAGES], bar_empty[TC_STAGES], bar_accf[2],
        bar_acce[2];
    __shared__ unsigned s_tmem;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int k0 = blockIdx.x * TC_LT;
    const int j0 = blockIdx.y * TC_JCH;
    const int nj = A.ncomp - j0 < TC_JCH ? A.ncomp - j0 : TC_JCH;
    const int nsub = (nj + TC_KC - 1) / TC_KC;
    const long long s_lo = tb - k0 - (TC_LT - 1);  // sample of window row 0

    if (tid == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(smem_addr(&bar_full[i]), 1);
            mbar_init(smem_addr(&bar_empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_addr(&bar_accf[i]), 1);
            mbar_init(smem_addr(&bar_acce[i]), TC_EPI_WARPS);
        }
        s_abort = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;

    if (warp == TC_EPI_WARPS) {
        // ---- TMA producer
        if (lane == 0) {
            const int zw = s_lo < 0 ? (int)s_lo : (int)(s_lo % A.cap);
            const int zn = (int)(tb % A.cap);
            int c = 0;
            for (; c < nsub; ++c) {
                const int st = c % TC_STAGES;
                if (s_abort) break;
                if (c >= TC_STAGES &&
                    !mbar_wait(smem_addr(&bar_empty[st]), ((c / TC_STAGES) - 1) & 1, A.wait_cycles, &s_abort)) {
                    atomicOr(A.err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                unsigned char *base = sm + st * TC_STAGE_BYTES;
                const unsigned bar = smem_addr(&bar_full[st]);
                mbar_expect_tx(bar, TC_STAGE_BYTES);
                const int x = j0 + c * TC_KC;
                tma_load_3d(smem_addr(base), &tm_win, x, 0, zw, bar);
                tma_load_3d(smem_addr(base + TC_A_BYTES), &tm_win, x, 1, zw, bar);
                tma_load_3d(smem_addr(base + 2 * TC_A_BYTES), &tm_new, x, 0, zn, bar);
                tma_load_3d(smem_addr(base + 2 * TC_A_BYTES + TC_B_BYTES), &tm_new, x, 1, zn, bar);
            }
            // the last copies into each stage have landed before this thread leaves
            for (int j = c > TC_STAGES ? c - TC_STAGES : 0; j < c; ++j)
                mbar_wait(smem_addr(&bar_full[j % TC_STAGES]), (j / TC_STAGES) & 1, DRAIN_CYCLES, nullptr);
        }
    } else if (warp == TC_EPI_WARPS + 1) {
        // ---- MMA issuer
        if (lane == 0) {
            // kind::f16 instruction descriptor: FP32 D, fp16 A and B, both
            // K-major, N = 64, M = 128
            const unsigned idesc = (1u << 4) | ((unsigned)(VB >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
            int c = 0;
            for (; c < nsub; ++c) {
                const int st = c % TC_STAGES, set = c & 1;
                if (!mbar_wait(smem_addr(&bar_full[st]), (c / TC_STAGES) & 1, A.wait_cycles, &s_abort) ||
                    (c >= 2 && !mbar_wait(smem_addr(&bar_acce[set]), ((c >> 1) - 1) & 1, A.wait_cycles, &s_abort))) {
                    atomicOr(A.err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                tc_fence_after();
                const unsigned base = smem_addr(sm + st * TC_STAGE_BYTES);
                const unsigned a_hi = base, a_lo = base + TC_A_BYTES;
                const unsigned b_hi = base + 2 * TC_A_BYTES, b_lo = b_hi + TC_B_BYTES;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    const unsigned d = tmem + (unsigned)(set * 128 + m * 64);
#pragma unroll
                    for (int ks = 0; ks < TC_KC / 16; ++ks) {
                        const unsigned ao = (unsigned)(m * (TC_A_BYTES / 2) + ks * 32), bo = (unsigned)(ks * 32);
                        umma_f16(d, umma_desc(a_hi + ao), umma_desc(b_hi + bo), idesc, ks > 0 ? 1u : 0u);
                        umma_f16(d, umma_desc(a_hi + ao), umma_desc(b_lo + bo), idesc, 1u);
                        umma_f16(d, umma_desc(a_lo + ao), umma_desc(b_hi + bo), idesc, 1u);
                    }
                }
                umma_commit(smem_addr(&bar_empty[st]));
                umma_commit(smem_addr(&bar_accf[set]));
            }
            // every MMA issued has completed before TMEM is freed
            if (c > 0)
                mbar_wait(smem_addr(&bar_accf[(c - 1) & 1]), ((c - 1) >> 1) & 1, DRAIN_CYCLES, nullptr);
        }
    } else {
        // ---- epilogue: window row r of M tile mt
        const int mt = warp >> 2, q = warp & 3;
        const int r = 128 * mt + 32 * q + lane;
        float acc[VB];
#pragma unroll
        for (int i = 0; i < VB; ++i) acc[i] = 0.f;
        for (int c = 0; c < nsub; ++c) {
            const int set = c & 1;
            if (!mbar_wait(smem_addr(&bar_accf[set]), (c >> 1) & 1, A.wait_cycles, &s_abort)) {
                atomicOr(A.err, ERR_TIMEOUT);
                s_abort = 1;
                break;
            }
            tc_fence_after();
            const unsigned taddr = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(set * 128 + mt * 64);
#pragma unroll
            for (int g = 0; g < VB / 16; ++g) {
                unsigned v[16];
                tmem_ld16(taddr + 16 * g, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[16 * g + i] = __fadd_rn(acc[16 * g + i], __uint_as_float(v[i]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&bar_acce[set]));
        }
        if (!s_abort) {
            // band entries of this row: G(t, k0 + kk) with kk = t + 191 - r,
            // back in V^2 units (the ring holds 4096 V)
            const int K1 = A.K + 1;
            float *out = A.part + (long long)blockIdx.y * VB * K1 + k0;
#pragma unroll
            for (int t = 0; t < VB; ++t) {
                const int kk = t + TC_LT - 1 - r;
                if (t < nb && kk >= 0 && kk < TC_LT && k0 + kk < K1)
                    out[(long long)t * K1 + kk] = acc[t] * 5.9604644775390625e-08f;  // 2^-24
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

cudaError_t prepare_vacf_kernels() {
    return cudaFuncSetAttribute(k_vacf_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
}

// Tensor maps of the fp16 hi/lo ring ([rows][2][ld] halves, rows = cap +
// TC_ROWS): window boxes of 64 components x 1 plane x TC_ROWS samples and
// new-sample boxes of 64 x 1 x VB, in the 128-byte swizzle.  Encoded once per
// ring by the driver's cuTensorMapEncodeTiled (found through the runtime).
cudaError_t encode_vacf_tensor_maps(Sim &s) {
    using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)(3ll * s.np), 2, (cuuint64_t)(s.vacf_cap + TC_ROWS)};
    const cuuint64_t strides[2] = {(cuuint64_t)s.ring_ld * 2, (cuuint64_t)s.ring_ld * 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t box_w[3] = {TC_KC, 1, TC_ROWS}, box_n[3] = {TC_KC, 1, VB};
    CUtensorMap *maps = reinterpret_cast<CUtensorMap *>(s.tmaps);
    for (int i = 0; i < 2; ++i) {
        const CUresult r = encode(&maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, s.ring16, dims, strides,
                                  i == 0 ? box_w : box_n, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

// G(t, k) for the block's samples: the chunk partials summed in chunk order
// (FP64), one thread per (t, k).
__global__ void __launch_bounds__(256) k_corr_gsum(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int t = blockIdx.y;
    if (t >= (int)(te - tb)) return;
    const int K1 = A.K + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K1) return;
    const long long stride = (long long)VB * K1;
    const float *p = A.part + (long long)t * K1 + k;
    double g = 0.0;
#pragma unroll 8
    for (int c = 0; c < A.nchunks; ++c) g += (double)p[c * stride];
    A.G[(long long)t * K1 + k] = g;
}

// H(t, k) = G(t, 0) + 2 sum_{m=1}^{k-1} G(t, m) for k = 1..K, one CTA per sample
// row: each thread sums a run of consecutive m, the runs' totals are scanned
// across the CTA (warp shuffles, then the warps' totals in order), and each
// thread writes its run's prefix sums -- a fixed order (FP64).  H(t, 0) = 0.
constexpr int SCAN_T = 256;
__global__ void __launch_bounds__(SCAN_T) k_msd_scan(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int t = blockIdx.x;
    if (t >= (int)(te - tb)) return;
    const int K1 = A.K + 1;
    const double *g = A.G + (long long)t * K1;
    double *h = A.H + (long long)t * K1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nm = A.K - 1;  // terms m = 1 .. K - 1
    const int per = nm > 0 ? (nm + SCAN_T - 1) / SCAN_T : 0;
    const int m0 = 1 + threadIdx.x * per;
    double run = 0.0;
    for (int i = 0; i < per; ++i)
        if (m0 + i <= nm) run += 2.0 * g[m0 + i];
    double x = run;  // inclusive scan within the warp
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __shared__ double wsum[SCAN_T / 32];
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    double pre = x - run;  // the terms before this thread's run
    for (int w = 0; w < warp; ++w) pre += wsum[w];
    const double g0 = g[0];
    if (threadIdx.x == 0) {
        h[0] = 0.0;
        if (A.K >= 1) h[1] = g0;
    }
    for (int i = 0; i < per; ++i) {
        const int m = m0 + i;
        if (m <= nm) {
            pre += 2.0 * g[m];
            h[m + 1] = g0 + pre;
        }
    }
}

// W(e, k) along the diagonals: thread d walks the block's samples e = tb + j
// with k = d - (nb - 1) + j, W(e, k) = W(e - 1, k - 1) + H(e, k) (W(., 0) = 0),
// starting from the kept W(tb - 1, .) and leaving W(te - 1, d) for the next
// block.  Writes W[j][k] for 1 <= k <= K.
constexpr int DIAG_T = 64;  // small blocks: the walk is latency-bound, so spread it over SMs
__global__ void __launch_bounds__(DIAG_T) k_msd_diag(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    const int K1 = A.K + 1;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;  // k at the block's last sample
    if (d < 1 || d > A.K + nb - 1) return;
    const int par = (int)(A.d_vacf[4] & 1);
    const double *prev = A.wstate + (long long)par * K1;
    double *next = A.wstate + (long long)(par ^ 1) * K1;
    const int k0 = d - nb;  // k at sample tb - 1
    double w = k0 >= 1 ? prev[k0] : 0.0;
    // the walk's loads are independent of one another: 16 at a time in flight
    for (int j0 = 0; j0 < nb; j0 += 16) {
        double hv[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = j0 + i, k = k0 + 1 + j;
            hv[i] = (j < nb && k >= 1 && k < K1) ? A.H[(long long)j * K1 + k] : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int j = j0 + i, k = k0 + 1 + j;
            if (j < nb && k >= 1 && k < K1) {
                w += hv[i];
                A.W[(long long)j * K1 + k] = w;
            }
        }
    }
    if (d < K1) next[d] = w;
}

// C(k) += sum_t G(t, k); M(k) += sum_{e >= k} W(e, k); pair counts (the same
// origins for both).  The last block marks the samples done and flips the
// parity of the kept W.
constexpr int ACC_T = 64;
__global__ void __launch_bounds__(ACC_T) k_corr_acc(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    const int K1 = A.K + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K1) {
        double c = 0.0, m = 0.0;
        for (int j0 = 0; j0 < nb; j0 += 16) {
            double gv[16], wv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int j = j0 + i;
                gv[i] = j < nb ? A.G[(long long)j * K1 + k] : 0.0;
                wv[i] = (j < nb && k >= 1 && tb + j >= k) ? A.W[(long long)j * K1 + k] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                c += gv[i];
                m += wv[i];
            }
        }
        A.sum[k] += c;
        A.msd[k] += m;
        const long long first = tb > k ? tb : (long long)k;
        if (te > first) A.cnt[k] += (long long)A.np * (te - first);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int dn = atomicAdd(A.done, 1u);
        if (dn == gridDim.x - 1) {
            A.d_vacf[1] = te;
            A.d_vacf[4] += 1;
            *A.done = 0u;
            __threadfence();
        }
    }
}

// Per-particle sums: csum[i][k] += sum_{t in block} V_i(t).V_i(t - k), one
// thread per (lag, particle), products FP32, block sum FP32 (at most 192
// terms), running sums FP64.  The last block advances the samples done.
__global__ void __launch_bounds__(256) k_vacf_pp(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int i = blockIdx.y;
    const int np = A.np;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= A.K; k += gridDim.x * blockDim.x) {
        float acc = 0.f;
        const long long t1 = tb > k ? tb : k;
        int sa = (int)(t1 % A.cap), sb = (int)((t1 - k) % A.cap);
        for (long long t = t1; t < te; ++t) {
            const float *a = A.ring + (long long)sa * 3 * np;
            const float *b = A.ring + (long long)sb * 3 * np;
#pragma unroll
            for (int c = 0; c < 3; ++c) acc = fmaf(a[c * np + i], b[c * np + i], acc);
            if (++sa == A.cap) sa = 0;
            if (++sb == A.cap) sb = 0;
        }
        A.sum[(long long)i * (A.K + 1) + k] += (double)acc;
        if (i == 0) {
            const long long first = tb > k ? tb : (long long)k;
            if (te > first) A.cnt[k] += te - first;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int d = atomicAdd(A.done, 1u);
        if (d == gridDim.x * gridDim.y - 1) {
            A.d_vacf[1] = te;
            *A.done = 0u;
            __threadfence();
        }
    }
}

cudaError_t launch_vacf_block(Sim &s, bool flush, cudaStream_t st) {
    if (s.vacf_lag < 0 || s.np == 0) return cudaSuccess;
    if (s.vacf_pp) {
        VacfArgs A;
        A.ring = s.ring;
        A.cap = s.vacf_cap;
        A.ncomp = 3 * s.np;
        A.K = s.vacf_lag;
        A.d_vacf = s.d_vacf;
        A.flush = flush ? 1 : 0;
        A.part = nullptr;
        A.sum = s.vacf_sum;
        A.cnt = s.vacf_cnt;
        A.np = s.np;
        A.done = reinterpret_cast<unsigned int *>(s.d_vacf + 3);
        dim3 g((s.vacf_lag + 1 + 255) / 256, s.np);
        k_vacf_pp<<<g, 256, 0, st>>>(A);
        return cudaGetLastError();
    }
    VacfArgs A;
    A.ring = s.ring;
    A.cap = s.vacf_cap;
    A.ncomp = 3 * s.np;
    A.K = s.vacf_lag;
    A.d_vacf = s.d_vacf;
    A.flush = flush ? 1 : 0;
    A.part = s.vacf_part;
    A.nchunks = s.vacf_nchunks;
    A.G = s.corr_g;
    A.H = s.corr_h;
    A.W = s.corr_w;
    A.wstate = s.msd_state;
    A.sum = s.vacf_sum;
    A.msd = s.msd_sum;
    A.cnt = s.vacf_cnt;
    A.np = s.np;
    A.done = reinterpret_cast<unsigned int *>(s.d_vacf + 3);
    A.err = s.d_err;
    A.wait_cycles = s.wait_cycles;
    const int K1 = s.vacf_lag + 1;
    const CUtensorMap *maps = reinterpret_cast<const CUtensorMap *>(s.tmaps);
    dim3 g1((s.vacf_lag + TC_LT) / TC_LT, s.vacf_nchunks);
    k_vacf_tc<<<g1, TC_THREADS, TC_SMEM, st>>>(A, maps[0], maps[1]);
    k_corr_gsum<<<dim3((K1 + 255) / 256, VB), 256, 0, st>>>(A);
    k_msd_scan<<<VB, SCAN_T, 0, st>>>(A);
    k_msd_diag<<<(K1 + VB + DIAG_T - 1) / DIAG_T, DIAG_T, 0, st>>>(A);
    k_corr_acc<<<(K1 + ACC_T - 1) / ACC_T, ACC_T, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace lbp
