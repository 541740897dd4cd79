// vacf_noalloc.cu -- a velocity-autocorrelation entry point that allocates no
// device memory.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// want the correlation -- for example code running inside a memory pool or
// arena they do not control, a host process that has handed all device memory
// to another framework's caching allocator, or a real-time loop that must not
// risk an allocation's implicit synchronisation or failure.  They pass their
// own sample and output buffers; the only scratch this routine needs (the
// per-chunk partial sums of the correlator) lives in a fixed array compiled
// into the library, which every GPU that loads the library keeps until the
// process exits.
//
// The correlation itself is the same blocked all-origin estimator as the
// library's stateful VACF (vacf_kernels.cu): for every block of up to 64 new
// samples t and every lag k <= max_lag it adds V(t).V(t - k).  Products are
// FP32; each lane sums the products of one component over one block (at most
// 64 terms) in FP32 and adds that to an FP64 accumulator, and everything
// above that (components, chunks, blocks) is summed in FP64.  Here the
// samples are the caller's whole trajectory instead of the library's ring.
#include <cuda_runtime.h>

#include <mutex>

#include "lbp_internal.cuh"

namespace {

constexpr int NB = 64;       // samples per correlation block
constexpr int NKT = 128;     // lags per CTA
constexpr int NLW = 16;      // lags per warp
constexpr int NJ = 32;       // components per sub-chunk (one per lane)
constexpr int NJCH = 1024;   // components per CTA
constexpr int NWIN = NB + NKT - 1;

// Scratch: partial sums [chunks][max_lag + 1], 4 MiB.
constexpr long long SCRATCH_DOUBLES = 524288;
static __device__ __align__(256) double g_vacf_scratch[SCRATCH_DOUBLES];

// Address of g_vacf_scratch per device, looked up once per device.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_scratch_ptr[MAX_DEVICES] = {};

__global__ void __launch_bounds__(256) k_corr_noalloc(const float *__restrict__ samples,
                                                      long long T, int ncomp, int K,
                                                      long long tb, long long te, double *part) {
    const int nb = (int)(te - tb);
    __shared__ float sA[NB][NJ];
    __shared__ float sW[NWIN][NJ];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int k0 = blockIdx.x * NKT;
    const int jc0 = blockIdx.y * NJCH;
    const long long s_lo = tb - k0 - (NKT - 1);
    double dacc[NLW];
#pragma unroll
    for (int m = 0; m < NLW; ++m) dacc[m] = 0.0;
    for (int js = 0; js < NJCH; js += NJ) {
        const int jb = jc0 + js;
        if (jb >= ncomp) break;
        __syncthreads();
        for (int e = threadIdx.x; e < NB * NJ; e += blockDim.x) {
            const int t = e / NJ, l = e - t * NJ;
            const int jj = jb + l;
            sA[t][l] = (t < nb && jj < ncomp) ? samples[(tb + t) * ncomp + jj] : 0.f;
        }
        for (int e = threadIdx.x; e < NWIN * NJ; e += blockDim.x) {
            const int sr = e / NJ, l = e - sr * NJ;
            const int jj = jb + l;
            const long long s = s_lo + sr;
            sW[sr][l] = (s >= 0 && s < te && jj < ncomp) ? samples[s * ncomp + jj] : 0.f;
        }
        __syncthreads();
        // 16 samples at a time against the 31 window values they meet, in
        // registers with static indices
        const int base0 = NKT - 1 - NLW * warp;
        // FP32 holds one component's products over this block only
        float acc[NLW];
#pragma unroll
        for (int m = 0; m < NLW; ++m) acc[m] = 0.f;
#pragma unroll 1
        for (int tc = 0; tc < NB; tc += NLW) {
            float a[NLW], w[2 * NLW - 1];
#pragma unroll
            for (int i = 0; i < NLW; ++i) a[i] = sA[tc + i][lane];
#pragma unroll
            for (int i = 0; i < 2 * NLW - 1; ++i) w[i] = sW[base0 + tc - (NLW - 1) + i][lane];
#pragma unroll
            for (int i = 0; i < NLW; ++i)
#pragma unroll
                for (int m = 0; m < NLW; ++m) acc[m] = fmaf(a[i], w[i - m + NLW - 1], acc[m]);
        }
#pragma unroll
        for (int m = 0; m < NLW; ++m) dacc[m] += (double)acc[m];
    }
#pragma unroll
    for (int m = 0; m < NLW; ++m) {
        double v = dacc[m];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int k = k0 + NLW * warp + m;
        if (lane == 0 && k <= K) part[(long long)blockIdx.y * (K + 1) + k] = v;
    }
    (void)T;
}

__global__ void __launch_bounds__(256) k_reduce_noalloc(const double *part, int nchunks, int K,
                                                        long long tb, long long te, int npairs,
                                                        double *csum, long long *counts) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += part[(long long)c * (K + 1) + k];
        csum[k] += s;
        const long long first = tb > k ? tb : (long long)k;
        if (te > first) counts[k] += (long long)npairs * (te - first);
    }
}

}  // namespace

// sets the thread's lbp_last_error message (lbp_api.cu)
lbp_status lbp_set_error_for_noalloc(lbp_status st, const char *msg);

// One-time set-up per device happens inside the first call on that device
// (cudaGetSymbolAddress with the device current): make that first call
// before any CUDA graph capture that includes this routine.  The address is
// kept for the life of the process, so the routine must not be used on a
// device after cudaDeviceReset has torn down its context.
extern "C" lbp_status lbp_vacf_correlate_noalloc(const float *samples, int64_t T, int ncomp,
                                                 int max_lag, int npairs, double *csum,
                                                 int64_t *counts, void *stream) {
    if (T < 0 || ncomp < 1 || max_lag < 0 || npairs < 0)
        return lbp_set_error_for_noalloc(LBP_EINVAL,
                                         "lbp_vacf_correlate_noalloc: need T >= 0, ncomp >= 1, max_lag >= 0, npairs >= 0");
    if (!csum || !counts || (T > 0 && !samples))
        return lbp_set_error_for_noalloc(LBP_EINVAL, "lbp_vacf_correlate_noalloc: null pointer");
    const long long nchunks = ((long long)ncomp + NJCH - 1) / NJCH;
    // both factors are at least 1, so this also bounds max_lag (and with it the
    // grid sizes below) by the scratch size
    if (nchunks * ((long long)max_lag + 1) > SCRATCH_DOUBLES)
        return lbp_set_error_for_noalloc(
            LBP_EINVAL,
            "lbp_vacf_correlate_noalloc: ceil(ncomp / 1024) * (max_lag + 1) exceeds the 524288-entry scratch");
    if (nchunks > 65535)
        return lbp_set_error_for_noalloc(LBP_EINVAL,
                                         "lbp_vacf_correlate_noalloc: ncomp > 65535 * 1024 (one grid row per chunk)");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lbp_set_error_for_noalloc(LBP_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES)
        return lbp_set_error_for_noalloc(LBP_EINVAL, "lbp_vacf_correlate_noalloc: device index >= 64");
    double *part = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_vacf_scratch);
            if (e != cudaSuccess)
                return lbp_set_error_for_noalloc(LBP_ECUDA, cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double *>(p);
        }
        part = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(csum, 0, sizeof(double) * ((size_t)max_lag + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * ((size_t)max_lag + 1), st);
    for (long long tb = 0; tb < T && e == cudaSuccess; tb += NB) {
        const long long te = tb + NB < T ? tb + NB : T;
        const dim3 g1((max_lag + NKT) / NKT, (unsigned)nchunks);
        k_corr_noalloc<<<g1, 256, 0, st>>>(samples, T, ncomp, max_lag, tb, te, part);
        e = cudaGetLastError();
        if (e != cudaSuccess) break;
        k_reduce_noalloc<<<(max_lag + 1 + 255) / 256, 256, 0, st>>>(part, (int)nchunks, max_lag, tb,
                                                                    te, npairs, csum,
                                                                    (long long *)counts);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return lbp_set_error_for_noalloc(LBP_ECUDA, cudaGetErrorString(e));
    return LBP_OK;
}
