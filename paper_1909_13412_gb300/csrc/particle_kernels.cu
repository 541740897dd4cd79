// particle_kernels.cu -- two-way coupling kernels of liblbp (sm_103a).
//
//  k_particles : one warp per particle.  Gathers u^N at the eight corners of
//                the particle's cell from the stored populations (pull, i.e.
//                the streamed f^n of Eq. 20), fits the Stokeslet flow of Eq. 8
//                with warp-shuffle reductions, draws the Philox random force
//                (Eqs. 4-5), advances V and r (Eqs. 1-2) in FP64 and adds the
//                reaction force -F_H W_p (Eq. 9) to a per-node accumulator.
//  k_apply     : adds the body-force term 3 w_a F.e_a of Eqs. 18-19 to the
//                post-collision populations at every node that received a
//                reaction force, then clears the accumulator.
//
// Determinism: per-node reaction forces are summed as 64-bit fixed-point
// integers (scale 2^56) with integer atomics, so the sum is exact and does not
// depend on the order in which particles add to it; no floating-point atomics
// are used.  The accumulator is an open-addressing hash of node index ->
// (Fx, Fy, Fz) sized to at least twice the 8 n_p nodes particles can touch,
// with a list of the slots in use, so no dense force field is read or cleared.
#include <cuda_runtime.h>

#include "lbp_internal.cuh"

namespace lbp {

struct ParticleArgs {
    const float *g;  // deviation populations fhat^{n-1}
    int nx, ny, nz;
    long long P;
    double *r, *v, *fh, *fr;
    const double *fext, *mass, *gamma, *radius, *sig;
    const unsigned char *pinned;
    int cap, np;
    const long long *d_step;
    unsigned long long seed;
    double sqrt3;
    int mode, exclude_inside;
    unsigned long long *hkey, *hacc;
    unsigned int *hlist, *hcount;
    int hash_bits;
    float *ring;
    int ring_cap;
    const long long *d_vacf;  // [0] = first sampled step, or null
    int *err;
};

__device__ __forceinline__ double wsum8(double x) {
    // sum over the eight corners (lane bits 2..4); every lane ends with the sum
    x += __shfl_xor_sync(0xffffffffu, x, 4);
    x += __shfl_xor_sync(0xffffffffu, x, 8);
    x += __shfl_xor_sync(0xffffffffu, x, 16);
    return x;
}

__device__ __forceinline__ void hash_add(const ParticleArgs &A, unsigned long long node,
                                         long long q0, long long q1, long long q2) {
    const unsigned int H = 1u << A.hash_bits;
    const unsigned int mask = H - 1u;
    unsigned int h = (unsigned int)((node * 0x9E3779B97F4A7C15ull) >> (64 - A.hash_bits));
    for (unsigned int probe = 0; probe < H; ++probe) {
        const unsigned long long prev = atomicCAS(&A.hkey[h], HASH_EMPTY, node);
        if (prev == HASH_EMPTY) {
            const unsigned int idx = atomicAdd(&A.hcount[0], 1u);
            A.hlist[idx] = h;
        }
        if (prev == HASH_EMPTY || prev == node) {
            atomicAdd(&A.hacc[h], (unsigned long long)q0);
            atomicAdd(&A.hacc[H + h], (unsigned long long)q1);
            atomicAdd(&A.hacc[2 * (size_t)H + h], (unsigned long long)q2);
            return;
        }
        h = (h + 1u) & mask;
    }
    atomicOr(A.err, ERR_HASH);
}

__device__ __forceinline__ long long to_fixed(double x, int *err) {
    if (!(fabs(x) < FIX_LIMIT)) {
        atomicOr(err, ERR_RANGE);
        return 0;
    }
    return __double2ll_rn(x * FIX_SCALE);
}

__global__ void __launch_bounds__(256) k_particles(const ParticleArgs A) {
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    if (i >= A.np) return;  // uniform per warp
    const int cap = A.cap;
    const double r0 = A.r[i], r1 = A.r[cap + i], r2 = A.r[2 * cap + i];
    const double V0 = A.v[i], V1 = A.v[cap + i], V2 = A.v[2 * cap + i];
    const long long step = *A.d_step;

    // cell of the particle: base = floor(r), frac = r - base (exact)
    const double b0 = floor(r0), b1 = floor(r1), b2 = floor(r2);
    const double q0 = r0 - b0, q1 = r1 - b1, q2 = r2 - b2;
    const int p = lane >> 2, j = lane & 3;
    const int c0 = p & 1, c1 = (p >> 1) & 1, c2 = (p >> 2) & 1;
    int X = (int)b0 + c0, Y = (int)b1 + c1, Z = (int)b2 + c2;
    if (X >= A.nx) X -= A.nx;
    if (Y >= A.ny) Y -= A.ny;
    if (Z >= A.nz) Z -= A.nz;

    // u^N at corner p: sum_a e_a g_a(x_p - e_a); lane j of the corner takes a = j mod 4
    double ux = 0.0, uy = 0.0, uz = 0.0;
#pragma unroll
    for (int a = 1; a < Q; ++a) {
        if ((a & 3) == j) {
            int xs = X - ex(a), ys = Y - ey(a), zs = Z - ez(a);
            xs = xs < 0 ? xs + A.nx : (xs >= A.nx ? xs - A.nx : xs);
            ys = ys < 0 ? ys + A.ny : (ys >= A.ny ? ys - A.ny : ys);
            zs = zs < 0 ? zs + A.nz : (zs >= A.nz ? zs - A.nz : zs);
            const double gv =
                (double)__ldg(A.g + (long long)a * A.P + ((long long)zs * A.ny + ys) * A.nx + xs);
            if (ex(a)) ux += ex(a) > 0 ? gv : -gv;
            if (ey(a)) uy += ey(a) > 0 ? gv : -gv;
            if (ez(a)) uz += ez(a) > 0 ? gv : -gv;
        }
    }
#pragma unroll
    for (int m = 1; m <= 2; m <<= 1) {
        ux += __shfl_xor_sync(0xffffffffu, ux, m);
        uy += __shfl_xor_sync(0xffffffffu, uy, m);
        uz += __shfl_xor_sync(0xffffffffu, uz, m);
    }

    // corner offset d_p = x_p - r and trilinear weight W_p (same expressions as Eq. 9 reading)
    const double d0 = c0 ? 1.0 - q0 : -q0;
    const double d1 = c1 ? 1.0 - q1 : -q1;
    const double d2 = c2 ? 1.0 - q2 : -q2;
    const double Wp = __dmul_rn(__dmul_rn(__dmul_rn(1.0, c0 ? q0 : 1.0 - q0), c1 ? q1 : 1.0 - q1),
                                c2 ? q2 : 1.0 - q2);
    const double gam = A.gamma[i];
    const double w0 = ux - V0, w1 = uy - V1, w2 = uz - V2;

    double F0, F1, F2;
    bool spread = true;
    if (A.mode == LBP_STOKESLET) {
        // Eq. 8: e^N from the mean relative velocity, then one-parameter least squares
        const double m0 = wsum8(w0) / 8.0, m1 = wsum8(w1) / 8.0, m2 = wsum8(w2) / 8.0;
        const double nw = sqrt(m0 * m0 + m1 * m1 + m2 * m2);
        double U = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
        if (nw != 0.0) {
            e0 = m0 / nw;
            e1 = m1 / nw;
            e2 = m2 / nw;
            const double R = A.radius[i];
            const double rp = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            double num = 0.0, den = 0.0;
            if (!(rp < 1e-12) && !(A.exclude_inside && rp < R)) {
                const double xx = e0 * d0 + e1 * d1 + e2 * d2;
                const double k1 = 1.0 - 3.0 * R / (4.0 * rp);
                const double k2 = 3.0 * R * xx / (4.0 * rp * rp * rp);
                const double a0 = k1 * e0 - k2 * d0, a1 = k1 * e1 - k2 * d1, a2 = k1 * e2 - k2 * d2;
                num = w0 * a0 + w1 * a1 + w2 * a2;
                den = a0 * a0 + a1 * a1 + a2 * a2;
            }
            num = wsum8(num);
            den = wsum8(den);
            U = den == 0.0 ? 0.0 : num / den;
        }
        F0 = gam * U * e0;
        F1 = gam * U * e1;
        F2 = gam * U * e2;
    } else if (A.mode == LBP_POINTWISE) {
        // Eq. 7 with u(r_i) = sum_p W_p u^N_p
        const double ur0 = wsum8(Wp * ux), ur1 = wsum8(Wp * uy), ur2 = wsum8(Wp * uz);
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

    // Eq. 9: reaction force -F_H W_p at corner p (one lane per corner)
    if (spread && j == 0) {
        const unsigned long long node =
            (unsigned long long)(((long long)Z * A.ny + Y) * A.nx + X);
        const long long a0 = to_fixed(-F0 * Wp, A.err);
        const long long a1 = to_fixed(-F1 * Wp, A.err);
        const long long a2 = to_fixed(-F2 * Wp, A.err);
        hash_add(A, node, a0, a1, a2);
    }

    if (lane == 0) {
        // Eqs. 4-5: F_R = sqrt(2 gamma kT) xi, xi = sqrt3 (2u - 1), u from 53 Philox bits
        unsigned long long c[4] = {(unsigned long long)step, (unsigned long long)i, 0ull, 0ull};
        philox4x64_10(c, A.seed, 0ull);
        const double sg = A.sig[i];
        double R3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double u = __dmul_rn(__dadd_rn(__ull2double_rn(c[k] >> 11), 0.5), 0x1.0p-53);
            const double xi = __dmul_rn(A.sqrt3, __dsub_rn(__dmul_rn(2.0, u), 1.0));
            R3[k] = __dmul_rn(sg, xi);
        }
        const double FH3[3] = {F0, F1, F2};
        double Vn[3] = {V0, V1, V2};
        const double Vo[3] = {V0, V1, V2};
        const double ro[3] = {r0, r1, r2};
        const int L[3] = {A.nx, A.ny, A.nz};
        const bool pin = A.pinned[i] != 0;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            A.fh[k * cap + i] = FH3[k];
            A.fr[k * cap + i] = R3[k];
            if (!pin) {
                // Eqs. 1-2, dt = 1: V += (F_H + F_R + F_ext)/M; r += V; periodic wrap
                const double acc = __ddiv_rn(__dadd_rn(__dadd_rn(FH3[k], R3[k]), A.fext[k * cap + i]),
                                             A.mass[i]);
                Vn[k] = __dadd_rn(Vo[k], acc);
                double rn = __dadd_rn(ro[k], Vn[k]);
                if (rn < 0.0) rn = __dadd_rn(rn, (double)L[k]);
                if (rn >= (double)L[k]) rn = __dsub_rn(rn, (double)L[k]);
                bad |= !isfinite(Vn[k]) || !isfinite(rn) || !(rn >= 0.0) || !(rn < (double)L[k]);
                if (bad) rn = 0.0;  // keep the next gather inside the box
                A.v[k * cap + i] = Vn[k];
                A.r[k * cap + i] = rn;
            }
        }
        if (bad) atomicOr(A.err, ERR_NAN);
        if (A.ring) {
            const long long m = step - A.d_vacf[0];
            if (m >= 0) {
                const long long slot = m % A.ring_cap;
                float *dst = A.ring + slot * 3 * (long long)A.np;
                dst[i] = (float)Vn[0];
                dst[A.np + i] = (float)Vn[1];
                dst[2 * A.np + i] = (float)Vn[2];
            }
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
    A.hkey = s.hkey;
    A.hacc = s.hacc;
    A.hlist = s.hlist;
    A.hcount = s.hcount;
    A.hash_bits = s.hash_bits;
    A.ring = s.vacf_lag >= 0 ? s.ring : nullptr;
    A.ring_cap = s.vacf_cap;
    A.d_vacf = s.d_vacf;
    A.err = s.d_err;
    const int warps_per_block = 8;
    const unsigned grid = (unsigned)((s.np + warps_per_block - 1) / warps_per_block);
    k_particles<<<grid, 32 * warps_per_block, 0, st>>>(A);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Body-force term at the nodes that received reaction forces, then clear.
// The last block to finish resets the slot counter and advances the step.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_apply(float *g, long long P, unsigned long long *hkey,
                                               unsigned long long *hacc, const unsigned int *hlist,
                                               unsigned int *hcount, int hash_bits,
                                               long long *d_step) {
    const unsigned int H = 1u << hash_bits;
    const unsigned int count = hcount[0];
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < count;
         t += gridDim.x * blockDim.x) {
        const unsigned int h = hlist[t];
        const long long node = (long long)hkey[h];
        const double F0 = (double)(long long)hacc[h] * FIX_INV;
        const double F1 = (double)(long long)hacc[H + h] * FIX_INV;
        const double F2 = (double)(long long)hacc[2 * (size_t)H + h] * FIX_INV;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double G = wgt(a) * (3.0 * (ex(a) * F0 + ey(a) * F1 + ez(a) * F2));
            float *q = g + (long long)a * P + node;
            *q = (float)((double)*q + G);
        }
        hkey[h] = HASH_EMPTY;
        hacc[h] = 0ull;
        hacc[H + h] = 0ull;
        hacc[2 * (size_t)H + h] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(&hcount[1], 1u);
        if (done == gridDim.x - 1) {
            hcount[0] = 0u;
            hcount[1] = 0u;
            *d_step += 1;
            __threadfence();
        }
    }
}

cudaError_t launch_apply_forces(Sim &s, float *dst, cudaStream_t st) {
    long long work = 8ll * s.np;
    long long grid = (work + 255) / 256;
    if (grid > 4ll * s.num_sms) grid = 4ll * s.num_sms;
    if (grid < 1) grid = 1;
    k_apply<<<(unsigned)grid, 256, 0, st>>>(dst, s.P, s.hkey, s.hacc, s.hlist, s.hcount,
                                            s.hash_bits, s.d_step);
    return cudaGetLastError();
}

__global__ void k_hash_clear(unsigned long long *hkey, unsigned long long *hacc, unsigned int H) {
    for (unsigned int t = blockIdx.x * blockDim.x + threadIdx.x; t < H; t += gridDim.x * blockDim.x) {
        hkey[t] = HASH_EMPTY;
        hacc[t] = 0ull;
        hacc[H + t] = 0ull;
        hacc[2 * (size_t)H + t] = 0ull;
    }
}

cudaError_t launch_hash_clear(Sim &s, cudaStream_t st) {
    const unsigned int H = 1u << s.hash_bits;
    k_hash_clear<<<(H + 255) / 256, 256, 0, st>>>(s.hkey, s.hacc, H);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(s.hcount, 0, 2 * sizeof(unsigned int), st);
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
    for (int p = 0; p < 8; ++p) {
        const int c0 = p & 1, c1 = (p >> 1) & 1, c2 = (p >> 2) & 1;
        weights[8 * i + p] =
            __dmul_rn(__dmul_rn(__dmul_rn(1.0, c0 ? q0 : 1.0 - q0), c1 ? q1 : 1.0 - q1),
                      c2 ? q2 : 1.0 - q2);
    }
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
