// lbm_kernels.cu -- D3Q15 lattice kernels of liblbp (sm_103a).
//
// Storage: 15 planes (structure of arrays, x fastest), plane stride P >= N,
// holding the deviation g_a = fhat_a - w_a of the post-collision populations
// from the rest state.  With sum_a w_a = 1 and sum_a w_a e_a = 0 the moments
// of Eqs. 12-13 are rho~ - 1 = sum_a g_a and u = sum_a e_a g_a, and the
// collision of Eqs. 15, 17 and 19 becomes, exactly,
//     g'_a = g_a + (geq_a - g_a)/tau,
//     geq_a = w_a [(rho~ - 1) + 3 e_a.u + 9/2 (e_a.u)^2 - 3/2 u.u],
// so FP32 arithmetic acts on the small deviations instead of on O(0.1)
// populations.
#include <cuda_runtime.h>

#include "lbp_internal.cuh"

namespace lbp {

// ---------------------------------------------------------------------------
// Fused pull-stream + moments + BGK collision (Eqs. 20, 12, 13, 15, 17, 19).
// One thread per node and one block per 128-node segment of an x-row (a full
// grid, not a persistent loop: the hardware block scheduler keeps the blocks
// in flight on a narrow window of consecutive rows, which keeps the 15 read
// and 15 write streams local in DRAM, and balances the tail).  The 15 loads
// of a node are independent, so every thread has 60 bytes in flight.  The
// body-force term of Eqs. 18-19 is added by k_stream_collide_forced below.
// ---------------------------------------------------------------------------
template <int BX>
__global__ void __launch_bounds__(BX) k_stream_collide(const float *__restrict__ src,
                                                       float *__restrict__ dst, int nx, int ny,
                                                       int nz, long long P, float omega,
                                                       int nchunks, long long *bump) {
    const unsigned item = blockIdx.x;
    const unsigned row = item / (unsigned)nchunks;
    const int chunk = (int)(item - row * (unsigned)nchunks);
    const int x = chunk * BX + threadIdx.x;
    if (item == 0 && threadIdx.x == 0) *bump += 1;
    if (x >= nx) return;
    const int z = (int)(row / (unsigned)ny);
    const int y = (int)(row - (unsigned)z * ny);
    // source coordinate x - e for e = -1, 0, +1 (index e + 1), periodic
    const int X[3] = {x == nx - 1 ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
    const int Y[3] = {y == ny - 1 ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};
    const int Z[3] = {z == nz - 1 ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};
    float g[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const long long s = (long long)a * P +
                            ((long long)Z[ez(a) + 1] * ny + Y[ey(a) + 1]) * nx + X[ex(a) + 1];
        g[a] = __ldg(src + s);
    }
    float drho = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        drho += g[a];
        if (ex(a)) ux += ex(a) > 0 ? g[a] : -g[a];
        if (ey(a)) uy += ey(a) > 0 ? g[a] : -g[a];
        if (ez(a)) uz += ez(a) > 0 ? g[a] : -g[a];
    }
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const long long d = (long long)row * nx + x;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const float eu = (float)ex(a) * ux + (float)ey(a) * uy + (float)ez(a) * uz;
        const float geq = wgtf(a) * (drho + 3.f * eu + 4.5f * eu * eu - usq15);
        dst[(long long)a * P + d] = g[a] + omega * (geq - g[a]);
    }
}

// ---------------------------------------------------------------------------
// The same pass with the body force of Eqs. 18-19 (particles present).
// Each block is one SEG-node segment of a row and owns one force record
// (lbp_internal.cuh) filled by this step's particle kernel.  Every warp loads
// the 256-byte record -- one 8-byte word per lane -- together with its
// population loads (its address depends only on the block index, so no load
// waits on another), then each lane sums, exactly in 64-bit fixed point, the
// entries whose x is its own and adds 3 w_a F.e_a to its post-collision
// populations.  A record that overflowed (count > REC_SLOTS) is not applied
// here: warp 0 moves its entries to the dense accumulator, where the
// particle kernel already put the rest, and k_apply_overflow applies the
// whole sum.  The block also clears the count of its record of the previous
// step (which the next step's particle kernel refills) and the previous
// step's overflow flag.
// ---------------------------------------------------------------------------
template <int BX>
__global__ void __launch_bounds__(BX) k_stream_collide_forced(
    const float *__restrict__ src, float *__restrict__ dst, int nx, int ny, int nz, long long P,
    float omega, int nchunks, const unsigned long long *__restrict__ rec_cur,
    unsigned long long *rec_prev, int *oflow_cur, int *oflow_prev, unsigned long long *fq,
    unsigned int *mask, int mwords, long long *bump) {
    static_assert(BX == SEG, "one block per force-record segment");
    const unsigned item = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const unsigned row = item / (unsigned)nchunks;
    const int chunk = (int)(item - row * (unsigned)nchunks);
    if (item == 0 && threadIdx.x == 0) {
        *bump += 1;
        *oflow_prev = 0;
    }
    if (threadIdx.x == 0) rec_prev[(size_t)item * REC_WORDS] = 0ull;
    const int xw = chunk * BX + (threadIdx.x & ~31);
    if (xw >= nx) return;  // whole warp past the end of the row (never warp 0)
    const int x0 = xw + lane;
    const bool act = x0 < nx;
    const int x = act ? x0 : nx - 1;
    const int z = (int)(row / (unsigned)ny);
    const int y = (int)(row - (unsigned)z * ny);
    const int X[3] = {x == nx - 1 ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
    const int Y[3] = {y == ny - 1 ? 0 : y + 1, y, y == 0 ? ny - 1 : y - 1};
    const int Z[3] = {z == nz - 1 ? 0 : z + 1, z, z == 0 ? nz - 1 : z - 1};
    float g[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const long long s = (long long)a * P +
                            ((long long)Z[ez(a) + 1] * ny + Y[ey(a) + 1]) * nx + X[ex(a) + 1];
        g[a] = __ldg(src + s);
    }
    const unsigned long long rw = __ldg(rec_cur + (size_t)item * REC_WORDS + lane);
    const int cnt = (int)(unsigned)(__shfl_sync(0xffffffffu, rw, 0) & 0xffffffffull);
    float F0 = 0.f, F1 = 0.f, F2 = 0.f;
    if (cnt > 0) {
        if (cnt <= REC_SLOTS) {
            long long a0 = 0, a1 = 0, a2 = 0;
            for (int sl = 0; sl < cnt; ++sl) {
                const unsigned long long xw2 = __shfl_sync(0xffffffffu, rw, REC_X0 + (sl >> 1));
                const int xs = (int)(unsigned)(xw2 >> (32 * (sl & 1)));
                const long long v0 = (long long)__shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl);
                const long long v1 = (long long)__shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl + 1);
                const long long v2 = (long long)__shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl + 2);
                if (xs == x) {
                    a0 += v0;
                    a1 += v1;
                    a2 += v2;
                }
            }
            const float inv = 1.3877787807814457e-17f;  // 2^-56
            F0 = 3.f * inv * __ll2float_rn(a0);
            F1 = 3.f * inv * __ll2float_rn(a1);
            F2 = 3.f * inv * __ll2float_rn(a2);
        } else if (threadIdx.x < 32) {
#pragma unroll
            for (int sl = 0; sl < REC_SLOTS; ++sl) {
                const unsigned long long xw2 = __shfl_sync(0xffffffffu, rw, REC_X0 + (sl >> 1));
                const int xs = (int)(unsigned)(xw2 >> (32 * (sl & 1)));
                const unsigned long long v0 = __shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl);
                const unsigned long long v1 = __shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl + 1);
                const unsigned long long v2 = __shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl + 2);
                if (lane == sl) {
                    const long long node = (long long)row * nx + xs;
                    const long long N = (long long)nx * ny * nz;
                    atomicAdd(fq + node, v0);
                    atomicAdd(fq + N + node, v1);
                    atomicAdd(fq + 2 * N + node, v2);
                    atomicOr(mask + (long long)row * mwords + (xs >> 5), 1u << (xs & 31));
                }
            }
            if (lane == 0) *oflow_cur = 1;
        }
    }
    if (!act) return;
    float drho = 0.f, ux = 0.f, uy = 0.f, uz = 0.f;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        drho += g[a];
        if (ex(a)) ux += ex(a) > 0 ? g[a] : -g[a];
        if (ey(a)) uy += ey(a) > 0 ? g[a] : -g[a];
        if (ez(a)) uz += ez(a) > 0 ? g[a] : -g[a];
    }
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    const long long d = (long long)row * nx + x;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const float eu = (float)ex(a) * ux + (float)ey(a) * uy + (float)ez(a) * uz;
        const float geq = wgtf(a) * (drho + 3.f * eu + 4.5f * eu * eu - usq15);
        const float G = wgtf(a) * ((float)ex(a) * F0 + (float)ey(a) * F1 + (float)ez(a) * F2);
        dst[(long long)a * P + d] = g[a] + omega * (geq - g[a]) + G;
    }
}

constexpr int SC_BX = SEG;

cudaError_t prepare_lbm_kernels() { return cudaSuccess; }

cudaError_t launch_stream_collide(Sim &s, const float *src, float *dst, cudaStream_t st) {
    constexpr int BX = SC_BX;
    const int nchunks = (s.nx + BX - 1) / BX;
    const long long items = (long long)s.ny * s.nz * nchunks;
    k_stream_collide<BX><<<(unsigned)items, BX, 0, st>>>(src, dst, s.nx, s.ny, s.nz, s.P,
                                                          (float)(1.0 / s.tau), nchunks, s.d_step);
    return cudaGetLastError();
}

cudaError_t launch_stream_collide_forced(Sim &s, const float *src, float *dst, int parity,
                                         cudaStream_t st) {
    constexpr int BX = SC_BX;
    const int nchunks = (s.nx + BX - 1) / BX;
    const long long items = (long long)s.ny * s.nz * nchunks;
    k_stream_collide_forced<BX><<<(unsigned)items, BX, 0, st>>>(
        src, dst, s.nx, s.ny, s.nz, s.P, (float)(1.0 / s.tau), nchunks, s.rec[parity],
        s.rec[parity ^ 1], s.d_oflow + parity, s.d_oflow + (parity ^ 1), s.fq, s.mask, s.mwords,
        s.d_step);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 <-> deviation storage.  f is [15][N] FP64 (the ABI layout).
// ---------------------------------------------------------------------------
__global__ void k_from_f64(const double *__restrict__ f, float *__restrict__ g, long long N,
                           long long P) {
    const long long total = (long long)Q * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long long i = t - (long long)a * N;
        g[(long long)a * P + i] = (float)(f[t] - wgt(a));
    }
}

__global__ void k_to_f64(const float *__restrict__ g, double *__restrict__ f, long long N,
                         long long P) {
    const long long total = (long long)Q * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long long i = t - (long long)a * N;
        f[t] = wgt(a) + (double)g[(long long)a * P + i];
    }
}

static unsigned grid_for(long long work, int threads, int num_sms) {
    long long g = (work + threads - 1) / threads;
    const long long cap = (long long)num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_fill_rest(Sim &s, float *dst, cudaStream_t st) {
    return cudaMemsetAsync(dst, 0, sizeof(float) * Q * s.P, st);
}

cudaError_t launch_from_f64(Sim &s, const double *f, float *dst, cudaStream_t st) {
    k_from_f64<<<grid_for(Q * s.N, 256, s.num_sms), 256, 0, st>>>(f, dst, s.N, s.P);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(Sim &s, const float *src, double *f, cudaStream_t st) {
    k_to_f64<<<grid_for(Q * s.N, 256, s.num_sms), 256, 0, st>>>(src, f, s.N, s.P);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Moments of the streamed populations (Eqs. 12-13) and p = rho~/3, in FP64.
// ---------------------------------------------------------------------------
__global__ void k_fields(const float *__restrict__ src, double *rho, double *u, double *p, int nx,
                         int ny, int nz, long long P) {
    const long long N = (long long)nx * ny * nz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long yz = i / nx;
        const int y = (int)(yz % ny);
        const int z = (int)(yz / ny);
        double drho = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            int xs = x - ex(a), ys = y - ey(a), zs = z - ez(a);
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            const double g = (double)src[(long long)a * P + ((long long)zs * ny + ys) * nx + xs];
            drho += g;
            ux += ex(a) * g;
            uy += ey(a) * g;
            uz += ez(a) * g;
        }
        if (rho) rho[i] = 1.0 + drho;
        if (u) {
            u[i] = ux;
            u[N + i] = uy;
            u[2 * N + i] = uz;
        }
        if (p) p[i] = (1.0 + drho) / 3.0;
    }
}

cudaError_t launch_fields(Sim &s, const float *src, double *rho, double *u, double *p,
                          cudaStream_t st) {
    k_fields<<<grid_for(s.N, 256, s.num_sms), 256, 0, st>>>(src, rho, u, p, s.nx, s.ny, s.nz,
                                                            s.P);
    return cudaGetLastError();
}

}  // namespace lbp
