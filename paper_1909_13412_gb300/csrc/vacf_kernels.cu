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
#include <cuda_runtime.h>

#include "lbp_internal.cuh"

namespace lbp {

constexpr int VB = 64;        // samples per correlation block
constexpr int VKT = 128;      // lags per CTA
constexpr int VJCH = 256;     // components per CTA (short CTAs interleave with the lattice pass)
constexpr int VWIN = VB + VKT - 1;

int vacf_block_samples() { return VB; }
int vacf_chunk_components() { return VJCH; }

struct VacfArgs {
    const float *ring;
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
};

__device__ __forceinline__ bool vacf_range(const VacfArgs &A, long long &tb, long long &te) {
    tb = A.d_vacf[1];
    te = A.d_vacf[2];
    if (te - tb > VB) te = tb + VB;
    if (A.flush) return te > tb;
    return te - tb == VB;
}

// ---------------------------------------------------------------------------
// k_vacf_mma: the block correlation on the tensor cores.  For the CTA's 128
// lags and 256 components the products of the B = 64 new samples t with
// the 191 window samples s form a matrix product
//     P[t][s] = sum_j V_j(t) V_j(s)       (64 x 192, inner dimension 256),
// and lag k0 + kk collects the band s = t + 127 - kk:  C(k) = sum_t P[t][.].
// The product runs as mma.sync m16n8k8 with TF32 operands in three terms,
// a.b = a_hi b_hi + a_hi b_lo + a_lo b_hi (a_hi = a rounded to TF32, a_lo =
// the rest rounded to TF32), which keeps FP32 accuracy (the dropped a_lo b_lo
// is below 2^-22 of the product); accumulation is FP32 in the tensor core.
// Eight warps: warp w takes the 16 samples of M tile w/2 and 9 of the 18 N
// tiles of 8 window rows that meet its band (the rest of the 24 are zero
// contributions).  The band of P goes through shared memory and each of 128
// threads sums its lag over t in FP64, in sample order, into the chunk's
// partial (the reduce kernel adds the chunks in chunk order): the result does
// not depend on scheduling.
// ---------------------------------------------------------------------------
constexpr int MJ = 32;           // components per staged sub-chunk
constexpr int MLD = MJ + 4;      // staged row stride (floats): conflict-free fragment loads
constexpr int MWR = 192;         // window rows staged (VWIN = 191, one zero row)
constexpr int MWRA = MWR + 8;    // rows allocated: the fragment loads of a warp's last
                                 // N tile pair read one 8-row tile past the staged rows
constexpr int MPLD = MWR + 4;    // row stride of the P tile in the epilogue
constexpr int MMA_SMEM = 2 * (VB + MWRA) * MLD * 4;  // hi and lo copies: 76,032 bytes
static_assert(VB * MPLD * 4 <= MMA_SMEM, "the P tile reuses the staging space");

__device__ __forceinline__ unsigned tf32_rna(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float d[4], const unsigned a[4], const unsigned b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// value v split into its TF32 head and tail, stored at index i of hi / lo
__device__ __forceinline__ void stage_split(unsigned *hi, unsigned *lo, int i, float v) {
    const unsigned h = tf32_rna(v);
    hi[i] = h;
    lo[i] = tf32_rna(v - __uint_as_float(h));
}

// four 8 x 4 blocks of 32-bit values (8 x 8 of 16-bit) from shared memory,
// one register each; thread i gives the address of row i % 8 of block i / 8
__device__ __forceinline__ void ldsm_x4(unsigned r[4], const unsigned *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__global__ void __launch_bounds__(256) k_vacf_mma(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    extern __shared__ float vsm[];
    unsigned *hA = reinterpret_cast<unsigned *>(vsm);
    unsigned *lA = hA + VB * MLD;
    unsigned *hW = lA + VB * MLD;
    unsigned *lW = hW + MWRA * MLD;
    __shared__ long long s_row[VB + MWR];  // ring offset of each staged row, -1: zero row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = blockIdx.x * VKT;
    const int jc0 = blockIdx.y * VJCH;
    const long long s_lo = tb - k0 - (VKT - 1);  // sample of window row 0
    const int mt = warp >> 1;                   // M tile: samples 16 mt .. 16 mt + 15
    const int nt0 = 2 * mt + 9 * (warp & 1);    // first of the warp's 9 N tiles
    const int cap = A.cap;

    // ring rows of the 64 new samples and the 192 window rows, once per CTA
    for (int rr = threadIdx.x; rr < VB + MWR; rr += blockDim.x) {
        long long off = -1;
        if (rr < VB) {
            if (rr < nb) off = (long long)((tb + rr) % cap) * A.ncomp;
        } else {
            const int sr = rr - VB;
            const long long smp = s_lo + sr;
            // rows older than te - cap were overwritten; they only meet lags > K
            if (sr < VWIN && smp >= 0 && smp >= te - cap && smp < te) off = (long long)(smp % cap) * A.ncomp;
        }
        s_row[rr] = off;
    }

    float acc[9][4];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;

    // ldmatrix row addresses: A fragment of M tile mt (rows g and g + 8, columns
    // c and c + 4 of the 8-column step) and B fragments of N tile pairs
    const int mrow = lane & 7, mblk = lane >> 3;
    const int a_off = (16 * mt + mrow + 8 * (mblk & 1)) * MLD + 4 * (mblk >> 1);
    const int b_off = (8 * (nt0 + (mblk >> 1)) + mrow) * MLD + 4 * (mblk & 1);

    // staging: warp w holds rows w, w + 8, ..., w + 248 of a sub-chunk (lane =
    // component) in registers; the next sub-chunk's loads are issued before
    // the current one's products, so they are in flight during them
    float v[32];
    auto load_rows = [&](int jb) {
        const bool colok = jb + lane < A.ncomp;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const long long off = s_row[warp + 8 * i];
            v[i] = (off >= 0 && colok) ? __ldg(A.ring + off + jb + lane) : 0.f;
        }
    };
    __syncthreads();  // s_row
    load_rows(jc0);
    for (int js = 0; js < VJCH; js += MJ) {
        const int jb = jc0 + js;
        if (jb >= A.ncomp) break;
        __syncthreads();  // the previous products are done with the staged tiles
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int rr = warp + 8 * i;  // rows 0..63: new samples (i < 8); then the window
            if (i < 8)
                stage_split(hA, lA, rr * MLD + lane, v[i]);
            else
                stage_split(hW, lW, (rr - VB) * MLD + lane, v[i]);
        }
        __syncthreads();
        if (js + MJ < VJCH && jb + MJ < A.ncomp) load_rows(jb + MJ);
        // the tensor core adds into its FP32 accumulator with truncation, which
        // biases long chains of additions; each sub-chunk's 12 products per
        // entry go to a fresh accumulator that is then added, rounded to
        // nearest, to the running sum
        float pacc[9][4];
#pragma unroll
        for (int q = 0; q < 9; ++q) pacc[q][0] = pacc[q][1] = pacc[q][2] = pacc[q][3] = 0.f;
#pragma unroll
        for (int k8 = 0; k8 < MJ; k8 += 8) {
            unsigned ah[4], al[4];
            ldsm_x4(ah, hA + a_off + k8);
            ldsm_x4(al, lA + a_off + k8);
#pragma unroll
            for (int q = 0; q < 9; q += 2) {
                // N tiles nt0 + q and nt0 + q + 1 (the last pair also loads the tile
                // after the warp's nine -- rows up to 199, inside the allocation --
                // and does not use it)
                unsigned bh[4], bl[4];
                ldsm_x4(bh, hW + b_off + 8 * q * MLD + k8);
                ldsm_x4(bl, lW + b_off + 8 * q * MLD + k8);
                mma_tf32(pacc[q], al, bh);
                mma_tf32(pacc[q], ah, bl);
                mma_tf32(pacc[q], ah, bh);
                if (q + 1 < 9) {
                    mma_tf32(pacc[q + 1], al, bh + 2);
                    mma_tf32(pacc[q + 1], ah, bl + 2);
                    mma_tf32(pacc[q + 1], ah, bh + 2);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[q][r] = __fadd_rn(acc[q][r], pacc[q][r]);
    }
    __syncthreads();
    // the tile P[t][s] (only the band is read back) and the lag sums over t
    float *sP = vsm;
    const int g = lane >> 2, c = lane & 3;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int t = 16 * mt + g, sr = 8 * (nt0 + q) + 2 * c;
        sP[t * MPLD + sr] = acc[q][0];
        sP[t * MPLD + sr + 1] = acc[q][1];
        sP[(t + 8) * MPLD + sr] = acc[q][2];
        sP[(t + 8) * MPLD + sr + 1] = acc[q][3];
    }
    __syncthreads();
    // the band: G restricted to this chunk, G(t, k0 + kk) = P[t][t + 127 - kk],
    // written for the block's samples (coalesced along the lags)
    const int K1 = A.K + 1;
    float *out = A.part + (long long)blockIdx.y * VB * K1;
    for (int e = threadIdx.x; e < nb * VKT; e += blockDim.x) {
        const int t = e / VKT, kk = e - t * VKT, k = k0 + kk;
        if (k < K1) out[(long long)t * K1 + k] = sP[t * MPLD + t + (VKT - 1) - kk];
    }
}

cudaError_t prepare_vacf_kernels() {
    return cudaFuncSetAttribute(k_vacf_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, MMA_SMEM);
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
    for (int c = 0; c < A.nchunks; ++c) g += (double)p[c * stride];
    A.G[(long long)t * K1 + k] = g;
}

// H(t, k) = G(t, 0) + 2 sum_{m=1}^{k-1} G(t, m) for k = 1..K, one CTA per sample
// row: a block-wide inclusive scan of 2 G(t, m) over m = 1..K-1 in tiles of
// 1024, in a fixed order (FP64).  H(t, 0) = 0.
constexpr int SCAN_T = 1024;
__global__ void __launch_bounds__(SCAN_T) k_msd_scan(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int t = blockIdx.x;
    if (t >= (int)(te - tb)) return;
    const int K1 = A.K + 1;
    const double *g = A.G + (long long)t * K1;
    double *h = A.H + (long long)t * K1;
    __shared__ double sh[SCAN_T];
    const double g0 = g[0];
    double carry = 0.0;  // 2 sum of G(t, m) over the tiles before
    if (threadIdx.x == 0) h[0] = 0.0;
    // H(t, k) for k = 1 + m0 + i uses the scan of m = 1 .. k - 1
    for (int m0 = 0; m0 < A.K; m0 += SCAN_T) {
        const int i = threadIdx.x;
        const int m = m0 + i;  // H index k = m + 1 takes G(t, 1..m)
        double v = (m >= 1 && m < K1) ? 2.0 * g[m] : 0.0;
        sh[i] = v;
        __syncthreads();
        for (int off = 1; off < SCAN_T; off <<= 1) {
            const double add = i >= off ? sh[i - off] : 0.0;
            __syncthreads();
            sh[i] += add;
            __syncthreads();
        }
        const double incl = carry + sh[i];
        if (m + 1 < K1) h[m + 1] = g0 + incl;
        carry += sh[SCAN_T - 1];
        __syncthreads();
    }
}

// W(e, k) along the diagonals: thread d walks the block's samples e = tb + j
// with k = d - (nb - 1) + j, W(e, k) = W(e - 1, k - 1) + H(e, k) (W(., 0) = 0),
// starting from the kept W(tb - 1, .) and leaving W(te - 1, d) for the next
// block.  Writes W[j][k] for 1 <= k <= K.
__global__ void __launch_bounds__(256) k_msd_diag(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    const int K1 = A.K + 1;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;  // k at the block's last sample
    if (d < 1 || d > A.K + nb - 1) return;
    const int par = (int)(A.d_vacf[4] & 1);
    const double *prev = A.wstate + (long long)par * K1;
    double *next = A.wstate + (long long)(par ^ 1) * K1;
    int k = d - nb;  // k at sample tb - 1
    double w = k >= 1 ? prev[k] : 0.0;
    for (int j = 0; j < nb; ++j) {
        ++k;
        if (k >= 1 && k < K1) {
            w += A.H[(long long)j * K1 + k];
            A.W[(long long)j * K1 + k] = w;
        }
    }
    if (d < K1) next[d] = w;
}

// C(k) += sum_t G(t, k); M(k) += sum_{e >= k} W(e, k); pair counts (the same
// origins for both).  The last block marks the samples done and flips the
// parity of the kept W.
__global__ void __launch_bounds__(256) k_corr_acc(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    const int K1 = A.K + 1;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < K1) {
        double c = 0.0, m = 0.0;
        for (int j = 0; j < nb; ++j) {
            c += A.G[(long long)j * K1 + k];
            if (k >= 1 && tb + j >= k) m += A.W[(long long)j * K1 + k];
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
    const int K1 = s.vacf_lag + 1;
    dim3 g1((s.vacf_lag + VKT) / VKT, s.vacf_nchunks);
    k_vacf_mma<<<g1, 256, MMA_SMEM, st>>>(A);
    k_corr_gsum<<<dim3((K1 + 255) / 256, VB), 256, 0, st>>>(A);
    k_msd_scan<<<VB, SCAN_T, 0, st>>>(A);
    k_msd_diag<<<(K1 + VB + 255) / 256, 256, 0, st>>>(A);
    k_corr_acc<<<(K1 + 255) / 256, 256, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace lbp
