// particle_kernels.cu -- two-way coupling kernel of liblbp (sm_103a).
//
// k_particles: one thread per particle.  It gathers u^N at the eight corners
// of the particle's cell from the stored populations (a pull, i.e. the
// streamed f^n of Eq. 20), fits the Stokeslet flow of Eq. 8, draws the Philox
// random force (Eqs. 4-5), advances V and r (Eqs. 1-2) and adds the reaction
// force -F_H W_p (Eq. 9) to the nodes of its cell.
//
// Why a thread, not a warp, per particle: GB300 issues FP64 at 1/64 of the
// FP32 rate, so a warp-wide FP64 instruction costs the same whether one lane
// or 32 lanes need it.  Packing 32 particles into a warp divides the FP64
// instruction count per particle by 32; with one particle per warp the FP64
// work of the fit dominated the whole time step.  Precision split: corner
// geometry (d_p, 1/r_p, the Stokeslet basis a_p and the unit vector e^N) in
// FP32; relative velocities w_p, the normal-equation sums sum w.a and
// sum |a|^2, U_inf, F_H, the random force, the trilinear weights and the
// Langevin update in FP64.
//
// Reaction forces go to a dense per-node accumulator of 64-bit fixed-point
// integers (scale 2^56), added with integer atomics: the per-node sum is exact
// and independent of the order in which particles add to it (no
// floating-point atomics).  A bit per node in `mask` marks the nodes that
// received a force; the stream-collide kernel reads the mask, applies the
// body-force term of Eqs. 18-19 at those nodes and clears both.
#include <cuda_runtime.h>

#include "lbp_internal.cuh"

namespace lbp {

struct ParticleArgs {
    const float *g;  // deviation populations fhat^{n-1}
    int nx, ny, nz;
    long long P;
    long long N;
    double *r, *v, *fh, *fr;
    const double *fext, *mass, *gamma, *radius, *sig;
    const unsigned char *pinned;
    int cap, np;
    const long long *d_step;
    unsigned long long seed;
    double sqrt3;
    int mode, exclude_inside;
    unsigned long long *fq;  // [3][N] fixed-point reaction force
    unsigned int *mask;      // [rows][mwords]
    int mwords;
    float *ring;
    int ring_cap;
    long long *d_vacf;  // [0] first sampled step, [2] samples written
    int *err;
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__global__ void __launch_bounds__(128) k_particles(const ParticleArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = *A.d_step;
    if (A.ring && i == 0) {
        const long long m = step - A.d_vacf[0];
        if (m >= 0) A.d_vacf[2] = m + 1;
    }
    if (i >= A.np) return;
    const int cap = A.cap;
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const double r0 = A.r[i], r1 = A.r[cap + i], r2 = A.r[2 * cap + i];
    const double V0 = A.v[i], V1 = A.v[cap + i], V2 = A.v[2 * cap + i];

    // cell: base = floor(r), q = r - base (exact), corners base + {0,1}
    const double b0 = floor(r0), b1 = floor(r1), b2 = floor(r2);
    const double q0 = r0 - b0, q1 = r1 - b1, q2 = r2 - b2;
    const int ib0 = (int)b0, ib1 = (int)b1, ib2 = (int)b2;
    // source coordinates base + o for o = -1, 0, 1, 2 (index o + 1), periodic
    const int xs[4] = {wrapi(ib0 - 1, nx), ib0, wrapi(ib0 + 1, nx), wrapi(ib0 + 2, nx)};
    const int ys[4] = {wrapi(ib1 - 1, ny), ib1, wrapi(ib1 + 1, ny), wrapi(ib1 + 2, ny)};
    const int zs[4] = {wrapi(ib2 - 1, nz), ib2, wrapi(ib2 + 1, nz), wrapi(ib2 + 2, nz)};

    // pass 1: u at the eight corners, u = sum_a e_a g_a(x_p - e_a) (FP32)
    float ux[8], uy[8], uz[8];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
        const int c0 = p & 1, c1 = (p >> 1) & 1, c2 = (p >> 2) & 1;
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            const long long src = (long long)a * A.P +
                                  ((long long)zs[c2 - ez(a) + 1] * ny + ys[c1 - ey(a) + 1]) * nx +
                                  xs[c0 - ex(a) + 1];
            const float gv = __ldg(A.g + src);
            if (ex(a)) sx += ex(a) > 0 ? gv : -gv;
            if (ey(a)) sy += ey(a) > 0 ? gv : -gv;
            if (ez(a)) sz += ez(a) > 0 ? gv : -gv;
        }
        ux[p] = sx;
        uy[p] = sy;
        uz[p] = sz;
    }

    // trilinear weights of the corners (Eq. 9 reading), FP64, same expression as the oracle
    const double wx[2] = {1.0 - q0, q0}, wy[2] = {1.0 - q1, q1}, wz[2] = {1.0 - q2, q2};

    const double gam = A.gamma[i];
    double F0 = 0.0, F1 = 0.0, F2 = 0.0;
    bool spread = true;
    if (A.mode == LBP_STOKESLET) {
        // e^N: direction of the mean relative velocity w-bar = mean(u_p) - V
        float su0 = 0.f, su1 = 0.f, su2 = 0.f;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            su0 += ux[p];
            su1 += uy[p];
            su2 += uz[p];
        }
        const double m0 = (double)(su0 * 0.125f) - V0;
        const double m1 = (double)(su1 * 0.125f) - V1;
        const double m2 = (double)(su2 * 0.125f) - V2;
        const double n2 = m0 * m0 + m1 * m1 + m2 * m2;
        if (n2 > 0.0) {
            const double inv = 1.0 / sqrt(n2);
            const float e0 = (float)(m0 * inv), e1 = (float)(m1 * inv), e2 = (float)(m2 * inv);
            const float R = (float)A.radius[i];
            const float R2 = R * R, R34 = 0.75f * R;
            // corner offsets d_p = c - q
            const float dx[2] = {(float)(-q0), (float)(1.0 - q0)};
            const float dy[2] = {(float)(-q1), (float)(1.0 - q1)};
            const float dz[2] = {(float)(-q2), (float)(1.0 - q2)};
            double num = 0.0, den = 0.0;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const float d0 = dx[p & 1], d1 = dy[(p >> 1) & 1], d2 = dz[(p >> 2) & 1];
                const float rr = d0 * d0 + d1 * d1 + d2 * d2;
                if (rr < 1e-24f) continue;
                if (A.exclude_inside && rr < R2) continue;
                const float ir = rsqrtf(rr);
                const float x = e0 * d0 + e1 * d1 + e2 * d2;
                const float k1 = 1.f - R34 * ir;
                const float k2 = R34 * x * ir * ir * ir;
                const double a0 = (double)(k1 * e0 - k2 * d0);
                const double a1 = (double)(k1 * e1 - k2 * d1);
                const double a2 = (double)(k1 * e2 - k2 * d2);
                // normal equations of the one-parameter least-squares fit, FP64
                num += ((double)ux[p] - V0) * a0 + ((double)uy[p] - V1) * a1 + ((double)uz[p] - V2) * a2;
                den += a0 * a0 + a1 * a1 + a2 * a2;
            }
            const double U = den > 0.0 ? num / den : 0.0;
            const double gU = gam * U;
            F0 = gU * (double)e0;
            F1 = gU * (double)e1;
            F2 = gU * (double)e2;
        }
    } else if (A.mode == LBP_POINTWISE) {
        // Eq. 7 with u(r_i) = sum_p W_p u^N_p
        double ur0 = 0.0, ur1 = 0.0, ur2 = 0.0;
#pragma unroll
        for (int p = 0; p < 8; ++p) {
            const double Wp = __dmul_rn(__dmul_rn(wx[p & 1], wy[(p >> 1) & 1]), wz[(p >> 2) & 1]);
            ur0 += Wp * (double)ux[p];
            ur1 += Wp * (double)uy[p];
            ur2 += Wp * (double)uz[p];
        }
        F0 = -gam * (V0 - ur0);
        F1 = -gam * (V1 - ur1);
        F2 = -gam * (V2 - ur2);
    } else {
        // Eq. 6: friction against a fluid at rest; nothing is returned to the fluid
        F0 = -gam * V0;
        F1 = -gam * V1;
        F2 = -gam * V2;
        spread = false;
    }

    // Eq. 9: reaction force -F_H W_p at the eight corners, fixed point, exact sums
    if (spread) {
        const double s0 = -F0 * FIX_SCALE, s1 = -F1 * FIX_SCALE, s2 = -F2 * FIX_SCALE;
        const bool ok = fabs(F0) < FIX_LIMIT && fabs(F1) < FIX_LIMIT && fabs(F2) < FIX_LIMIT;
        if (!ok) atomicOr(A.err, ERR_RANGE);
        if (ok) {
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const int c0 = p & 1, c1 = (p >> 1) & 1, c2 = (p >> 2) & 1;
                const double Wp = __dmul_rn(__dmul_rn(wx[c0], wy[c1]), wz[c2]);
                const int X = xs[c0 + 1], Y = ys[c1 + 1], Z = zs[c2 + 1];
                const long long row = (long long)Z * ny + Y;
                const long long node = row * nx + X;
                atomicAdd(A.fq + node, (unsigned long long)__double2ll_rn(s0 * Wp));
                atomicAdd(A.fq + A.N + node, (unsigned long long)__double2ll_rn(s1 * Wp));
                atomicAdd(A.fq + 2 * A.N + node, (unsigned long long)__double2ll_rn(s2 * Wp));
                atomicOr(A.mask + row * A.mwords + (X >> 5), 1u << (X & 31));
            }
        }
    }

    // Eqs. 4-5: F_R = sqrt(2 gamma kT) xi, xi = sqrt3 (2u - 1) with
    // u = ((x >> 11) + 1/2) 2^-53 from Philox(counter = (step, i, 0, 0), key = (seed, 0)).
    // 2u - 1 is formed as fma((double)(2k + 1), 2^-53, -1): the same correctly
    // rounded value as 2 ((double)k + 1/2) 2^-53 - 1, so F_R is bit-identical
    // to the oracle's.
    unsigned long long c[4] = {(unsigned long long)step, (unsigned long long)i, 0ull, 0ull};
    philox4x64_10(c, A.seed, 0ull);
    const double sg = A.sig[i];
    double R3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double t = __fma_rn(__ull2double_rn(2ull * (c[k] >> 11) + 1ull), 0x1.0p-53, -1.0);
        R3[k] = __dmul_rn(sg, __dmul_rn(A.sqrt3, t));
    }
    const double FH3[3] = {F0, F1, F2};
    const double Vo[3] = {V0, V1, V2};
    const double ro[3] = {r0, r1, r2};
    const int L[3] = {nx, ny, nz};
    double Vn[3] = {V0, V1, V2};
    const bool pin = A.pinned[i] != 0;
    const double invM = 1.0 / A.mass[i];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        A.fh[k * cap + i] = FH3[k];
        A.fr[k * cap + i] = R3[k];
        if (!pin) {
            // Eqs. 1-2, dt = 1: V += (F_H + F_R + F_ext)/M; r += V; periodic wrap
            Vn[k] = Vo[k] + (FH3[k] + R3[k] + A.fext[k * cap + i]) * invM;
            double rn = ro[k] + Vn[k];
            if (rn < 0.0) rn += (double)L[k];
            if (rn >= (double)L[k]) rn -= (double)L[k];
            const bool b = !isfinite(Vn[k]) || !(rn >= 0.0) || !(rn < (double)L[k]);
            if (b) rn = 0.0;  // keep the next gather inside the box; reported as LBP_ENAN
            bad |= b;
            A.v[k * cap + i] = Vn[k];
            A.r[k * cap + i] = rn;
        }
    }
    if (bad) atomicOr(A.err, ERR_NAN);
    if (A.ring) {
        const long long m = step - A.d_vacf[0];
        if (m >= 0) {
            float *dst = A.ring + (m % A.ring_cap) * 3 * (long long)A.np;
            dst[i] = (float)Vn[0];
            dst[A.np + i] = (float)Vn[1];
            dst[2 * A.np + i] = (float)Vn[2];
        }
    }
}

cudaError_t launch_particles(Sim &s, const float *src, cudaStream_t st) {
    if (s.np == 0) return cudaSuccess;
    ParticleArgs A;
    A.g = src;
    A.nx = s.nx;
    A.ny = s.ny;
    A.nz = s.nz;
    A.P = s.P;
    A.N = s.N;
    A.r = s.r;
    A.v = s.v;
    A.fh = s.fh;
    A.fr = s.fr;
    A.fext = s.fext;
    A.mass = s.mass;
    A.gamma = s.gamma;
    A.radius = s.radius;
    A.sig = s.sig;
    A.pinned = s.pinned;
    A.cap = s.cap;
    A.np = s.np;
    A.d_step = s.d_step;
    A.seed = s.seed;
    A.sqrt3 = s.sqrt3;
    A.mode = s.mode;
    A.exclude_inside = s.exclude_inside;
    A.fq = s.fq;
    A.mask = s.mask;
    A.mwords = s.mwords;
    A.ring = s.vacf_lag >= 0 ? s.ring : nullptr;
    A.ring_cap = s.vacf_cap;
    A.d_vacf = s.d_vacf;
    A.err = s.d_err;
    const int threads = 128;
    const unsigned grid = (unsigned)((s.np + threads - 1) / threads);
    k_particles<<<grid, threads, 0, st>>>(A);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout helpers: ABI arrays are [n][3]; device state is [3][ld].
// ---------------------------------------------------------------------------
__global__ void k_aos_to_soa(const double *aos, double *soa, int n, int ld, int offset) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * n; t += gridDim.x * blockDim.x) {
        const int i = t / 3, k = t - 3 * i;
        soa[(long long)k * ld + offset + i] = aos[t];
    }
}

__global__ void k_soa_to_aos(const double *soa, double *aos, int n, int ld) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * n; t += gridDim.x * blockDim.x) {
        const int i = t / 3, k = t - 3 * i;
        aos[t] = soa[(long long)k * ld + i];
    }
}

cudaError_t launch_aos_to_soa(const double *aos, double *soa, int n, int ld, int offset,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_aos_to_soa<<<(3 * n + 255) / 256, 256, 0, st>>>(aos, soa, n, ld, offset);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double *soa, double *aos, int n, int ld, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_soa_to_aos<<<(3 * n + 255) / 256, 256, 0, st>>>(soa, aos, n, ld);
    return cudaGetLastError();
}

// Cell base index and trilinear weights of the current positions, with the
// same expressions k_particles uses (for bit-exact checks of the indexing).
__global__ void k_cells(const double *r, int cap, int np, int *base, double *weights) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double r0 = r[i], r1 = r[cap + i], r2 = r[2 * cap + i];
    const double b0 = floor(r0), b1 = floor(r1), b2 = floor(r2);
    const double q0 = r0 - b0, q1 = r1 - b1, q2 = r2 - b2;
    base[3 * i] = (int)b0;
    base[3 * i + 1] = (int)b1;
    base[3 * i + 2] = (int)b2;
    const double wx[2] = {1.0 - q0, q0}, wy[2] = {1.0 - q1, q1}, wz[2] = {1.0 - q2, q2};
    for (int p = 0; p < 8; ++p)
        weights[8 * i + p] = __dmul_rn(__dmul_rn(wx[p & 1], wy[(p >> 1) & 1]), wz[(p >> 2) & 1]);
}

cudaError_t launch_cells(Sim &s, int *base, double *weights, cudaStream_t st) {
    if (s.np == 0) return cudaSuccess;
    k_cells<<<(s.np + 127) / 128, 128, 0, st>>>(s.r, s.cap, s.np, base, weights);
    return cudaGetLastError();
}

__global__ void k_philox(const unsigned long long *ctr, const unsigned long long *key,
                         unsigned long long *out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
        philox4x64_10(c, key[0], key[1]);
        for (int k = 0; k < 4; ++k) out[4 * i + k] = c[k];
    }
}

cudaError_t launch_philox(const unsigned long long *ctr, const unsigned long long *key,
                          unsigned long long *out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    long long grid = (n + 255) / 256;
    if (grid > 4096) grid = 4096;
    k_philox<<<(unsigned)grid, 256, 0, st>>>(ctr, key, out, n);
    return cudaGetLastError();
}

}  // namespace lbp
