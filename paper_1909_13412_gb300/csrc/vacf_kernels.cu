// vacf_kernels.cu -- velocity autocorrelation accumulator of liblbp (sm_103a).
//
// C(k) = sum_i sum_{t0} V_i(t0).V_i(t0 + k) over all time origins (the VACF of
// Section 3 / Fig. 2).  The particle kernel writes every step's velocities
// (FP32) into a ring of K + B samples.  Every B = 64 samples the correlator
// adds, for the B new samples t and every lag k <= K, the products
// V(t).V(t - k): a dense contraction over the 3 n_p velocity components.
//
// k_vacf_corr : CTA = 128 lags x 1024 components; warp = 16 consecutive lags,
//               lane = one component of a 32-wide sub-chunk staged in shared
//               memory.  A lane keeps the 16 window values V(t - k) it needs
//               in registers and slides them by one sample per t, so each
//               (t, component) costs two shared loads for 16 FMAs.  Products
//               and the per-lane sums are FP32; the lane sums are combined in
//               FP64 with a fixed shuffle tree into one partial per (chunk, k).
// k_vacf_reduce : adds the chunk partials in chunk order (FP64) to the
//               running sums and pair counts, then marks the samples done.
#include <cuda_runtime.h>

#include "lbp_internal.cuh"

namespace lbp {

constexpr int VB = 64;        // samples per correlation block
constexpr int VKT = 128;      // lags per CTA
constexpr int VLW = 16;       // lags per warp
constexpr int VJ = 32;        // components per sub-chunk (one per lane)
constexpr int VJCH = 1024;    // components per CTA
constexpr int VWIN = VB + VKT - 1;

int vacf_block_samples() { return VB; }
int vacf_chunk_components() { return VJCH; }

struct VacfArgs {
    const float *ring;
    int cap;     // ring samples
    int ncomp;   // 3 n_p
    int K;
    long long *d_vacf;  // [0] t0, [1] samples done, [2] samples written, [3] block counter
    int flush;
    double *part;       // [nchunks][K+1]
    double *sum;        // [K+1]
    long long *cnt;     // [K+1]
    int np;
    unsigned int *done; // block counter of the reduce kernel
};

__device__ __forceinline__ bool vacf_range(const VacfArgs &A, long long &tb, long long &te) {
    tb = A.d_vacf[1];
    te = A.d_vacf[2];
    if (te - tb > VB) te = tb + VB;
    if (A.flush) return te > tb;
    return te - tb == VB;
}

__global__ void __launch_bounds__(256) k_vacf_corr(const VacfArgs A) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    const int nb = (int)(te - tb);
    __shared__ float sA[VB][VJ];
    __shared__ float sW[VWIN][VJ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = blockIdx.x * VKT;
    const int jc0 = blockIdx.y * VJCH;
    // absolute sample index of sW row 0
    const long long s_lo = tb - k0 - (VKT - 1);

    float acc[VLW];
#pragma unroll
    for (int m = 0; m < VLW; ++m) acc[m] = 0.f;

    // ring slots of the first rows of sA and sW (one 64-bit modulo per CTA;
    // later rows wrap by one subtraction: a block spans fewer than cap rows)
    const int cap = A.cap;
    const int slotA0 = (int)(tb % cap);
    const int slotW0 = s_lo >= 0 ? (int)(s_lo % cap) : 0;
    for (int js = 0; js < VJCH; js += VJ) {
        const int jb = jc0 + js;
        if (jb >= A.ncomp) break;
        __syncthreads();
        for (int e = threadIdx.x; e < VB * VJ; e += blockDim.x) {
            const int t = e / VJ, l = e - t * VJ;
            const int jj = jb + l;
            float v = 0.f;
            if (t < nb && jj < A.ncomp) {
                int slot = slotA0 + t;
                if (slot >= cap) slot -= cap;
                v = A.ring[(long long)slot * A.ncomp + jj];
            }
            sA[t][l] = v;
        }
        for (int e = threadIdx.x; e < VWIN * VJ; e += blockDim.x) {
            const int sr = e / VJ, l = e - sr * VJ;
            const int jj = jb + l;
            const long long s = s_lo + sr;
            float v = 0.f;
            // rows older than te - cap were overwritten; they only meet lags > K
            if (s >= 0 && s >= te - cap && s < te && jj < A.ncomp) {
                // slot of sample s: s mod cap (slotW0 + sr < 3 cap, s < 2 cap here)
                int slot = s_lo >= 0 ? slotW0 + sr : (int)s;
                while (slot >= cap) slot -= cap;
                v = A.ring[(long long)slot * A.ncomp + jj];
            }
            sW[sr][l] = v;
        }
        __syncthreads();
        // window for lags k = k0 + VLW*warp + m at sample t: sW[t + VKT-1 - VLW*warp - m].
        // 16 samples at a time: their 16 values and the 31 window values they
        // meet sit in registers with static indices, 256 FMAs per 47 loads.
        const int base0 = VKT - 1 - VLW * warp;
#pragma unroll 1
        for (int tc = 0; tc < VB; tc += VLW) {
            float a[VLW], w[2 * VLW - 1];
#pragma unroll
            for (int i = 0; i < VLW; ++i) a[i] = sA[tc + i][lane];
#pragma unroll
            for (int i = 0; i < 2 * VLW - 1; ++i) w[i] = sW[base0 + tc - (VLW - 1) + i][lane];
#pragma unroll
            for (int i = 0; i < VLW; ++i)
#pragma unroll
                for (int m = 0; m < VLW; ++m) acc[m] = fmaf(a[i], w[i - m + VLW - 1], acc[m]);
        }
    }
    // combine the lanes in FP64, fixed tree
#pragma unroll
    for (int m = 0; m < VLW; ++m) {
        double v = (double)acc[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int k = k0 + VLW * warp + m;
        if (lane == 0 && k <= A.K) A.part[(long long)blockIdx.y * (A.K + 1) + k] = v;
    }
}

__global__ void __launch_bounds__(256) k_vacf_reduce(const VacfArgs A, int nchunks) {
    long long tb, te;
    if (!vacf_range(A, tb, te)) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= A.K; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += A.part[(long long)c * (A.K + 1) + k];
        A.sum[k] += s;
        const long long first = tb > k ? tb : (long long)k;
        if (te > first) A.cnt[k] += (long long)A.np * (te - first);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int d = atomicAdd(A.done, 1u);
        if (d == gridDim.x - 1) {
            A.d_vacf[1] = te;
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
    A.sum = s.vacf_sum;
    A.cnt = s.vacf_cnt;
    A.np = s.np;
    A.done = reinterpret_cast<unsigned int *>(s.d_vacf + 3);
    dim3 g1((s.vacf_lag + VKT) / VKT, s.vacf_nchunks);
    k_vacf_corr<<<g1, 256, 0, st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int g2 = (s.vacf_lag + 1 + 255) / 256;
    k_vacf_reduce<<<g2, 256, 0, st>>>(A, s.vacf_nchunks);
    return cudaGetLastError();
}

}  // namespace lbp
