// adjoint_kernels.cu -- reverse-mode derivative (adjoint) of one coupled time
// step of liblbp (sm_103a).
//
// The forward step n (lbm_kernels.cu, particle_kernels.cu) maps the
// post-collision populations fhat^{n-1} and the particle state (r^n, V^n) to
// fhat^n and (r^{n+1}, V^{n+1}):
//   f_a(x)   = fhat^{n-1}_a(x - e_a)                               (Eq. 20)
//   rho~, u  = sum_a f_a, sum_a e_a f_a                            (Eqs. 12-13)
//   F_H      = gamma U_inf e^N from u at the 8 cell corners        (Eq. 8; or Eq. 7 / Eq. 6)
//   F(x_p)  += -F_H W_p(q)                                          (Eq. 9)
//   V' = V + (F_H + F_R + F_ext)/M,  r' = r + V'                   (Eqs. 1-2)
//   fhat_a   = (1 - w) f_a + w f^eq_a(rho~, u) + 3 w_a F.e_a,  w = 1/tau   (Eqs. 15, 17-19)
// Given the adjoints lam = dL/dfhat^n (FP32 planes), dL/dV^{n+1}, dL/dr^{n+1},
// these kernels produce dL/dfhat^{n-1}, dL/dV^n, dL/dr^n and add this step's
// share of dL/domega, dL/dgamma_i, dL/dR_i, dL/dM_i and dL/dkT.
//
// k_adj_gather + k_adj_fp64 : eight threads per particle gather u(x_p) and
//   lam_F(x_p) = sum_a 3 w_a e_a lam_a(x_p) at its corners (the adjoint of the
//   body-force term) into a small scratch array; then one thread per particle,
//   in 64-thread blocks so that many warps share each SM's FP64 pipe (the FP64
//   chain is long and latency-bound), re-evaluates the particle's forward step
//   in FP64 from the recorded state and runs
//   the chain rule backwards through the update, the random force, the
//   spreading weights and the Stokeslet fit.  What the fit sends back to the
//   fluid is lam_u(x_p), the adjoint of the node velocity at each corner: it
//   is appended, as (x, 3 FP64 values), to the 256-byte record of the corner's
//   row segment (the same records the forward step uses for forces).
// k_adj_lattice : the fused adjoint of collision, moments and streaming, one
//   thread per node, one block per 128-node row segment:
//     lam_feq_a = w lam_a
//     lam_rho   = w sum_a w_a lam_a
//     lam_u     = w sum_a w_a lam_a (3 e_a + 9 (e_a.u) e_a - 3 u) + lam_u(particles)
//     lam_f_a   = (1 - w) lam_a + lam_rho + e_a.lam_u
//     dL/dw    += sum_a lam_a (f^eq_a - f_a)
//   and, streaming being a permutation, dL/dfhat^{n-1}_a(x - e_a) = lam_f_a(x).
//   The adjoint buffer holds dL/df (the streamed populations) rather than
//   dL/dfhat, so that every node stores its 15 results at its own address
//   (aligned, like the forward pass) and reads dL/dfhat^n_a(x) as the value at
//   x + e_a (a shifted read, which the forward pass shows costs nothing).  It
//   reads that, the populations fhat^{n-1} (pulled, as forward) and writes
//   the result: 180 bytes per node in FP32.  The record entries of a node are summed in an order fixed by
//   their values, so the result does not depend on which particle appended
//   first; entries that did not fit a record go to a dense FP64 buffer (FP64
//   atomics, order-dependent in that rare case).  dL/dw is summed per block in
//   FP32 and added in FP64 to the block's own accumulator slot (no atomics).
#include <cuda_runtime.h>

#include <cstring>

#include "lbp_internal.cuh"

namespace lbp {

constexpr int APB = 32;  // particles per block (8 threads each)

struct AdjPArgs {
    const void *g;           // fhat^{n-1}, storage type St, 15 planes of P
    const float *lam;        // dL/dfhat^n, FP32, 15 planes of P
    long long P, N;
    const int *prep;         // box of each particle (batches)
    const double *r, *v;     // r^n, V^n, [3][cap]
    int cap, np;
    const double *fext, *inv_mass, *gamma, *radius, *sig;
    const unsigned char *pinned;
    double kT;
    unsigned long long seed;
    long long step;          // Philox counter of step n
    double sqrt3;
    int mode, exclude_inside;
    const double *gv, *gr;   // dL/dV^{n+1}, dL/dr^{n+1}: [np][3] or null
    double *lam_v, *lam_r;   // in: adjoint of V^{n+1}, r^{n+1}; out: of V^n, r^n ([3][cap])
    double *acc;             // [4][np]: dL/dgamma, dL/dR, dL/dM, dL/dkT (added)
    unsigned long long *rec; // records of this adjoint step
    double *fqd;             // [3][N] overflow accumulator (FP64)
    float *ug;               // [np][8][6] scratch: u(x_p) and lam_F(x_p) per corner
};

__device__ __forceinline__ int wrap_i(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Gathers (eight threads per particle): u(x_p) of the streamed f (pull) and
// lam_F(x_p) = sum_a 3 w_a e_a lam_a(x_p) (aligned) at the eight corners, to
// A.ug[i][p][0..2] and A.ug[i][p][3..5].
template <typename St, int MAXR>
__global__ void __launch_bounds__(256) k_adj_gather(const AdjPArgs A, const RepTable<MAXR> rt) {
    const typename St::T *G = static_cast<const typename St::T *>(A.g);
    __shared__ int s_base[APB][3];
    const int t = threadIdx.x, lane = t & 31;
    const int i0 = blockIdx.x * APB;
    const int cap = A.cap;
    const int ip = i0 + lane;
    if (t < 32 && ip < A.np) {
#pragma unroll
        for (int k = 0; k < 3; ++k) s_base[lane][k] = (int)floor(A.r[k * cap + ip]);
    }
    __syncthreads();

    // ---- gathers: u(x_p) of the streamed f (pull) and lam_F(x_p) (aligned)
    const int j = t >> 3, p = t & 7;
    const int ij = i0 + j;
    int X = 0, Y = 0, Z = 0;
    const Rep &rj = rt.rep[MAXR == 1 || ij >= A.np ? 0 : A.prep[ij]];
    const int nx = rj.nx, ny = rj.ny, nz = rj.nz;
    const long long off = rj.node_off;
    if (ij < A.np) {
        X = wrap_i(s_base[j][0] + (p & 1), nx);
        Y = wrap_i(s_base[j][1] + ((p >> 1) & 1), ny);
        Z = wrap_i(s_base[j][2] + ((p >> 2) & 1), nz);
        const int xs[3] = {wrap_i(X + 1, nx), X, wrap_i(X - 1, nx)};
        const int ys[3] = {wrap_i(Y + 1, ny), Y, wrap_i(Y - 1, ny)};
        const int zs[3] = {wrap_i(Z + 1, nz), Z, wrap_i(Z - 1, nz)};
        float sx = 0.f, sy = 0.f, sz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            const long long src = (long long)a * A.P + off + ((long long)zs[ez(a) + 1] * ny + ys[ey(a) + 1]) * nx +
                                  xs[ex(a) + 1];
            const float gv = St::load(G + src, a);
            // dL/dfhat_a(x_p) = dL/df^{n+1}_a(x_p + e_a) (the buffer's layout)
            const long long lnode = off + ((long long)zs[1 - ez(a)] * ny + ys[1 - ey(a)]) * nx + xs[1 - ex(a)];
            const float lv = (3.f * wgtf(a)) * __ldg(A.lam + (long long)a * A.P + lnode);
            if (ex(a)) { sx += ex(a) > 0 ? gv : -gv; lx += ex(a) > 0 ? lv : -lv; }
            if (ey(a)) { sy += ey(a) > 0 ? gv : -gv; ly += ey(a) > 0 ? lv : -lv; }
            if (ez(a)) { sz += ez(a) > 0 ? gv : -gv; lz += ez(a) > 0 ? lv : -lv; }
        }
        float *o = A.ug + ((size_t)ij * 8 + p) * 6;
        o[0] = sx;
        o[1] = sy;
        o[2] = sz;
        o[3] = lx;
        o[4] = ly;
        o[5] = lz;
    }
}

// Sum over the eight lanes of a particle (an aligned group of 8 lanes): every
// lane gets the same value (the butterfly adds the same pairs in every lane).
__device__ __forceinline__ double grp8_sum(double v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

// The FP64 adjoint of one particle's step with eight lanes per particle, one
// per corner of its cell: the per-corner terms of the fit (its forward
// re-evaluation and its adjoint) and of the spreading run in parallel and meet
// in group sums, which cuts the serial FP64 chain of a particle about
// fourfold; the per-particle scalars (the Langevin update, the random force)
// are evaluated in every lane of the group.  Blocks of 64 threads (8
// particles), so that many warps share the narrow FP64 pipe.  Each lane
// appends its corner's lam_u(x_p) to the record of that corner's row segment.
template <int MAXR>
__global__ void __launch_bounds__(64) k_adj_fp64(const AdjPArgs A, const RepTable<MAXR> rt) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = (tid >> 3) < A.np;
    const int i = valid ? tid >> 3 : A.np - 1;  // lanes past the last particle shadow it (no stores)
    const int c = tid & 7;                      // the lane's corner: offsets (c & 1, c >> 1 & 1, c >> 2)
    const int cap = A.cap;
    double r[3], V[3], q[3], lV[3], lr[3], fe[3];
    int base[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        r[k] = A.r[k * cap + i];
        V[k] = A.v[k * cap + i];
        base[k] = (int)floor(r[k]);
        q[k] = r[k] - (double)base[k];
        fe[k] = A.fext[k * cap + i];
        lV[k] = A.lam_v[k * cap + i] + (A.gv ? A.gv[3 * i + k] : 0.0);
        lr[k] = A.lam_r[k * cap + i] + (A.gr ? A.gr[3 * i + k] : 0.0);
    }
    const double gam = A.gamma[i], R = A.radius[i], invM = A.inv_mass[i], sg = A.sig[i];
    const bool pin = A.pinned[i] != 0;
    // this corner's gathered u(x_p) and lam_F(x_p), and its trilinear weight
    double u[3], lF[3], Wp = 1.0;
    {
        const float *g = A.ug + ((size_t)i * 8 + c) * 6;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            u[k] = (double)g[k];
            lF[k] = (double)g[3 + k];
            Wp *= ((c >> k) & 1) ? q[k] : 1.0 - q[k];
        }
    }
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = (double)((c >> k) & 1) - q[k];
    // forward re-evaluation of F_H
    double FH[3] = {0.0, 0.0, 0.0}, e[3] = {0.0, 0.0, 0.0};
    double U = 0.0, num = 0.0, den = 0.0, nw = 0.0, inw = 0.0, iden = 0.0;
    double ur[3] = {0.0, 0.0, 0.0};
    bool fit = false;
    // this corner's fit geometry (used by the forward and the adjoint fit)
    bool use = false;
    double rp = 0.0, ir = 0.0, ir3 = 0.0, x = 0.0, k1 = 0.0, k2 = 0.0, av[3] = {0.0, 0.0, 0.0};
    const double cR = 0.75 * R;
    if (A.mode == LBP_STOKESLET) {
        double m[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) m[k] = grp8_sum(u[k] - V[k]) * 0.125;
        // reciprocal square roots instead of square roots and divisions (the
        // FP64 pipe is narrow and divisions are long sequences on it)
        const double mm = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
        if (mm > 0.0) {
            inw = rsqrt(mm);
            nw = mm * inw;
#pragma unroll
            for (int k = 0; k < 3; ++k) e[k] = m[k] * inw;
        }
        const double rr = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        ir = rr > 0.0 ? rsqrt(rr) : 0.0;
        rp = rr * ir;
        use = nw > 0.0 && !(rp < 1e-12 || (A.exclude_inside && rp < R));
        double pn = 0.0, pd = 0.0;
        if (use) {
            ir3 = ir * ir * ir;
            x = e[0] * d[0] + e[1] * d[1] + e[2] * d[2];
            k1 = 1.0 - cR * ir;
            k2 = cR * x * ir3;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                av[k] = k1 * e[k] - k2 * d[k];
                pn += (u[k] - V[k]) * av[k];
                pd += av[k] * av[k];
            }
        }
        num = grp8_sum(pn);
        den = grp8_sum(pd);
        if (nw > 0.0 && den != 0.0) {
            iden = 1.0 / den;
            U = num * iden;
            fit = true;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) FH[k] = gam * U * e[k];
    } else if (A.mode == LBP_POINTWISE) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ur[k] = grp8_sum(Wp * u[k]);
            FH[k] = -gam * (V[k] - ur[k]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) FH[k] = -gam * V[k];
    }
    // the random force of this step (same Philox numbers as the forward step)
    unsigned long long ctr[4] = {(unsigned long long)A.step, (unsigned long long)i, 0ull, 0ull};
    philox4x64_10(ctr, A.seed, 0ull);
    double xi[3], FR[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double tt = __fma_rn(__ull2double_rn(2ull * (ctr[k] >> 11) + 1ull), 0x1.0p-53, -1.0);
        xi[k] = __dmul_rn(A.sqrt3, tt);
        FR[k] = __dmul_rn(sg, xi[k]);
    }

    // ---- backward
    double lFH[3] = {0.0, 0.0, 0.0}, lq[3] = {0.0, 0.0, 0.0};
    double gG = 0.0, gR = 0.0, gM = 0.0, gK = 0.0;
    if (!pin) {
        // r' = r + V'  then  V' = V + (F_H + F_R + F_ext)/M
        double lFR_xi = 0.0, lF_tot = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lV[k] += lr[k];
            lFH[k] = lV[k] * invM;
            lFR_xi += lV[k] * invM * xi[k];
            lF_tot += lV[k] * (FH[k] + FR[k] + fe[k]);
        }
        gM = -lF_tot * invM * invM;
        // F_R = sigma xi, sigma = sqrt(2 gamma kT)
        if (sg > 0.0) {
            const double isg = 1.0 / sg;
            gG += lFR_xi * (A.kT * isg);
            gK += lFR_xi * (gam * isg);
        }
    }
    const bool spread = A.mode != LBP_BROWNIAN;
    // dW_p/dq_k of this corner
    double dw[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dw[k] = ((c >> k) & 1) ? 1.0 : -1.0;
#pragma unroll
        for (int j2 = 0; j2 < 3; ++j2)
            if (j2 != k) dw[k] *= ((c >> j2) & 1) ? q[j2] : 1.0 - q[j2];
    }
    if (spread) {
        // F(x_p) += -F_H W_p(q)
        const double fl = FH[0] * lF[0] + FH[1] * lF[1] + FH[2] * lF[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lFH[k] -= grp8_sum(Wp * lF[k]);
            lq[k] -= grp8_sum(fl * dw[k]);
        }
    }
    double lu[3] = {0.0, 0.0, 0.0};  // this corner's lam_u(x_p)
    if (A.mode == LBP_STOKESLET) {
        // the adjoint of the fit, with zero terms where there was none
        const double eF = e[0] * lFH[0] + e[1] * lFH[1] + e[2] * lFH[2];
        const double lU = fit ? gam * eF : 0.0;
        if (fit) gG += U * eF;
        double le[3] = {gam * U * lFH[0], gam * U * lFH[1], gam * U * lFH[2]};
        const double lnum = fit ? lU * iden : 0.0, lden = fit ? -lU * num * iden * iden : 0.0;
        double ple[3] = {0.0, 0.0, 0.0}, pq[3] = {0.0, 0.0, 0.0}, plc = 0.0;
        if (use && fit) {
            const double ir5 = ir3 * ir * ir;
            double la[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                lu[k] += lnum * av[k];
                la[k] = lnum * (u[k] - V[k]) + 2.0 * lden * av[k];
            }
            const double dla = d[0] * la[0] + d[1] * la[1] + d[2] * la[2];
            const double lk1 = e[0] * la[0] + e[1] * la[1] + e[2] * la[2];
            const double lk2 = -dla;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                ple[k] = k1 * la[k] - cR * ir3 * d[k] * dla;
                pq[k] = -k2 * la[k] + lk1 * cR * ir3 * d[k] + lk2 * cR * (ir3 * e[k] - 3.0 * x * ir5 * d[k]);
            }
            plc = -lk1 * ir + lk2 * x * ir3;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            le[k] += grp8_sum(ple[k]);
            lq[k] -= grp8_sum(pq[k]);
        }
        const double lc = grp8_sum(plc);
        if (fit) {
            gR += 0.75 * lc;
            // e = m/|m| with m the mean of the w_p
            const double ee = e[0] * le[0] + e[1] * le[1] + e[2] * le[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) lu[k] += (le[k] - e[k] * ee) * inw * 0.125;
        }
        // w_p = u_p - V
#pragma unroll
        for (int k = 0; k < 3; ++k) lV[k] -= grp8_sum(lu[k]);
    } else if (A.mode == LBP_POINTWISE) {
        gG += -((V[0] - ur[0]) * lFH[0] + (V[1] - ur[1]) * lFH[1] + (V[2] - ur[2]) * lFH[2]);
        const double ul = u[0] * lFH[0] + u[1] * lFH[1] + u[2] * lFH[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lV[k] -= gam * lFH[k];
            lu[k] = gam * Wp * lFH[k];
            lq[k] += grp8_sum(gam * ul * dw[k]);
        }
    } else {
        gG += -(V[0] * lFH[0] + V[1] * lFH[1] + V[2] * lFH[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) lV[k] -= gam * lFH[k];
    }
    if (!valid) return;  // past the shuffles: shadow lanes leave
    if (c == 0) {
        // q = r - floor(r)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lr[k] += lq[k];
            A.lam_v[k * cap + i] = lV[k];
            A.lam_r[k * cap + i] = lr[k];
        }
        A.acc[i] += gG;
        A.acc[A.np + i] += gR;
        A.acc[2 * A.np + i] += gM;
        A.acc[3 * A.np + i] += gK;
    }
    // lam_u(x_p) of this corner to the record of its row segment
    if (spread && !(lu[0] == 0.0 && lu[1] == 0.0 && lu[2] == 0.0)) {
        const Rep &ri = rt.rep[MAXR == 1 ? 0 : A.prep[i]];
        const int nx = ri.nx, ny = ri.ny, nz = ri.nz;
        const int X = wrap_i(base[0] + (c & 1), nx);
        const int Y = wrap_i(base[1] + ((c >> 1) & 1), ny);
        const int Z = wrap_i(base[2] + ((c >> 2) & 1), nz);
        const long long row = (long long)Z * ny + Y;
        unsigned long long *rec = A.rec + (size_t)(ri.seg_off + row * ri.nchunks + X / SEG) * REC_WORDS;
        const unsigned int slot = atomicAdd(reinterpret_cast<unsigned int *>(rec), 1u);
        if (slot < (unsigned)REC_SLOTS) {
            reinterpret_cast<int *>(rec + REC_X0)[slot] = X;
            rec[REC_F0 + 3 * slot] = (unsigned long long)__double_as_longlong(lu[0]);
            rec[REC_F0 + 3 * slot + 1] = (unsigned long long)__double_as_longlong(lu[1]);
            rec[REC_F0 + 3 * slot + 2] = (unsigned long long)__double_as_longlong(lu[2]);
        } else {
            const long long node = ri.node_off + row * nx + X;
            atomicAdd(A.fqd + node, lu[0]);
            atomicAdd(A.fqd + A.N + node, lu[1]);
            atomicAdd(A.fqd + 2 * A.N + node, lu[2]);
        }
    }
}

// Sum the record entries whose x is this node's in ascending order of their
// value bits (a fixed order whatever the order of the appends).
__device__ __forceinline__ void adj_record_sum(const unsigned long long *rec, unsigned mask,
                                               double &a0, double &a1, double &a2) {
    while (mask) {
        int best = -1;
        unsigned long long b0 = 0, b1 = 0, b2 = 0;
        for (unsigned m = mask; m; m &= m - 1) {
            const int sl = __ffs(m) - 1;
            const unsigned long long v0 = rec[REC_F0 + 3 * sl], v1 = rec[REC_F0 + 3 * sl + 1],
                                     v2 = rec[REC_F0 + 3 * sl + 2];
            if (best < 0 || v0 < b0 || (v0 == b0 && (v1 < b1 || (v1 == b1 && v2 < b2)))) {
                best = sl;
                b0 = v0;
                b1 = v1;
                b2 = v2;
            }
        }
        a0 += __longlong_as_double((long long)b0);
        a1 += __longlong_as_double((long long)b1);
        a2 += __longlong_as_double((long long)b2);
        mask &= ~(1u << best);
    }
}

// At least 6 blocks per SM: 80 registers (32 bytes spilled) instead of 96,
// measured 6.5% faster at 256^3 (more bytes in flight per SM).
template <typename St, int MAXR>
__global__ void __launch_bounds__(SEG, 6) k_adj_lattice(const typename St::T *__restrict__ G,
                                                     const float *__restrict__ lam, float *lam_out,
                                                     long long P, const RepTable<MAXR> rt,
                                                     const unsigned long long *rec_cur,
                                                     unsigned long long *rec_prev, double *fqd,
                                                     long long N, double *acc_omega) {
    __shared__ float s_red[SEG / 32];
    // the block's box (batches: one block per row segment of every box, in box order)
    const int rb = find_block_rep(rt, blockIdx.x);
    const Rep &rp = rt.rep[rb];
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz, nchunks = rp.nchunks;
    const float omega = rp.omega;
    const unsigned item = blockIdx.x - rt.item_off[rb];
    const unsigned row = divide(item, rp.dchunks);
    const int chunk = (int)(item - row * (unsigned)nchunks);
    const size_t seg = (size_t)rp.seg_off + (size_t)row * nchunks + chunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) rec_prev[seg * REC_WORDS] = 0ull;
    const int x0 = chunk * SEG + threadIdx.x;
    const bool act = x0 < nx;
    const int x = act ? x0 : nx - 1;
    // node index and the offsets of x - e (index e + 1), periodic
    const int z = (int)divide(row, rp.dny), y = (int)(row - (unsigned)z * ny);
    const int slab = nx * ny;
    const int d = (int)rp.node_off + (int)row * nx + x;
    const int ox[3] = {x == nx - 1 ? 1 - nx : 1, 0, x == 0 ? nx - 1 : -1};
    const int oy[3] = {y == ny - 1 ? (1 - ny) * nx : nx, 0, y == 0 ? (ny - 1) * nx : -nx};
    const int oz[3] = {z == nz - 1 ? (1 - nz) * slab : slab, 0, z == 0 ? (nz - 1) * slab : -slab};
    float g[Q], l[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        const int o = ox[ex(a) + 1] + oy[ey(a) + 1] + oz[ez(a) + 1];   // x - e_a
        const int op = ox[1 - ex(a)] + oy[1 - ey(a)] + oz[1 - ez(a)];  // x + e_a
        g[a] = St::load(G + (long long)a * P + d + o, a);
        // dL/dfhat^n_a(x) = dL/df^{n+1}_a(x + e_a): the buffer holds the latter
        l[a] = __ldg(lam + (long long)a * P + d + op);
    }
    const unsigned long long rw = __ldg(rec_cur + seg * REC_WORDS + lane);
    // particle contributions lam_u(x)
    float pu0 = 0.f, pu1 = 0.f, pu2 = 0.f;
    const int cnt = (int)(unsigned)(__shfl_sync(0xffffffffu, rw, 0) & 0xffffffffull);
    if (cnt > 0) {
        const int used = cnt < REC_SLOTS ? cnt : REC_SLOTS;
        unsigned mask = 0;
        for (int sl = 0; sl < used; ++sl) {
            const unsigned long long xw2 = __shfl_sync(0xffffffffu, rw, REC_X0 + (sl >> 1));
            if ((int)(unsigned)(xw2 >> (32 * (sl & 1))) == x) mask |= 1u << sl;
        }
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        if (mask && act)
            adj_record_sum(rec_cur + seg * REC_WORDS, mask, a0, a1, a2);
        if (cnt > REC_SLOTS && act) {
            a0 += fqd[d];
            a1 += fqd[N + d];
            a2 += fqd[2 * N + d];
            fqd[d] = 0.0;
            fqd[N + d] = 0.0;
            fqd[2 * N + d] = 0.0;
        }
        pu0 = (float)a0;
        pu1 = (float)a1;
        pu2 = (float)a2;
    }
    // forward moments and equilibrium (deviation form, as the forward kernel)
    float drho = 0.f;
#pragma unroll
    for (int a = 0; a < Q; ++a) drho += g[a];
    const float c78 = g[7] - g[8], c910 = g[9] - g[10], c1112 = g[11] - g[12], c1314 = g[13] - g[14];
    const float ux = (g[1] - g[2]) + c78 + c910 + c1112 - c1314;
    const float uy = (g[3] - g[4]) + c78 + c910 - c1112 + c1314;
    const float uz = (g[5] - g[6]) + c78 - c910 + c1112 + c1314;
    const float base = drho - 1.5f * (ux * ux + uy * uy + uz * uz);
    // dL/domega partial and the equilibrium-part adjoints, per opposite pair
    float dom = l[0] * ((2.f / 9.f) * base - g[0]);
    float swl = (2.f / 9.f) * l[0];  // sum_a w_a lam_a
    float lx = 0.f, ly = 0.f, lz = 0.f;  // sum_pairs W e (3 d + 9 eu s)
#define LBP_ADJ_PAIR(A, W, EX, EY, EZ)                                              \
    {                                                                               \
        const float eu = (EX) * ux + (EY) * uy + (EZ) * uz;                         \
        const float sym = (W) * (base + 4.5f * eu * eu);                            \
        const float anti = (3.f * (W)) * eu;                                        \
        dom += l[A] * (sym + anti - g[A]) + l[A + 1] * (sym - anti - g[A + 1]);     \
        const float s = l[A] + l[A + 1], dd = l[A] - l[A + 1];                      \
        swl += (W) * s;                                                             \
        const float c = (W) * (3.f * dd + 9.f * eu * s);                            \
        lx += (EX) * c;                                                             \
        ly += (EY) * c;                                                             \
        lz += (EZ) * c;                                                             \
    }
    LBP_ADJ_PAIR(1, 1.f / 9.f, 1.f, 0.f, 0.f)
    LBP_ADJ_PAIR(3, 1.f / 9.f, 0.f, 1.f, 0.f)
    LBP_ADJ_PAIR(5, 1.f / 9.f, 0.f, 0.f, 1.f)
    LBP_ADJ_PAIR(7, 1.f / 72.f, 1.f, 1.f, 1.f)
    LBP_ADJ_PAIR(9, 1.f / 72.f, 1.f, 1.f, -1.f)
    LBP_ADJ_PAIR(11, 1.f / 72.f, 1.f, -1.f, 1.f)
    LBP_ADJ_PAIR(13, 1.f / 72.f, -1.f, 1.f, 1.f)
#undef LBP_ADJ_PAIR
    const float lrho = omega * swl;
    const float lux = omega * lx - 3.f * ux * lrho + pu0;
    const float luy = omega * ly - 3.f * uy * lrho + pu1;
    const float luz = omega * lz - 3.f * uz * lrho + pu2;
    const float om1 = 1.f - omega;
    if (act) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const float v = om1 * l[a] + lrho + (float)ex(a) * lux + (float)ey(a) * luy + (float)ez(a) * luz;
            lam_out[(long long)a * P + d] = v;  // dL/df^n_a(x), aligned
        }
    }
    // dL/domega: the block's 128 terms summed in FP32 (fixed tree), added in
    // FP64 to the block's own slot.  (A tree of FP64 shuffles kept the narrow
    // FP64 pipe of this GPU busy at every block's end.)
    float v = act ? dom : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
#pragma unroll
        for (int w = 0; w < SEG / 32; ++w) s += s_red[w];
        acc_omega[blockIdx.x] += (double)s;
    }
}

template <typename F>
static cudaError_t by_storage_adj(int precision, F &&f) {
    switch (precision) {
        case LBP_BF16: return f(StoreBF16{});
        case LBP_F16: return f(StoreF16{});
        default: return f(StoreF32{});
    }
}

// The box table of an adjoint launch: every box with its blocks of one
// 128-node row segment each (item_off, for the lattice kernel) -- one entry
// for a single box.
template <int MAXR>
static RepTable<MAXR> adj_table(const Sim &s) {
    RepTable<MAXR> t;
    memset(&t, 0, sizeof(t));
    t.nrep = s.nrep;
    unsigned off = 0;
    for (int r = 0; r < s.nrep; ++r) {
        t.rep[r] = s.reps[r];
        t.item_off[r] = off;
        off += (unsigned)s.reps[r].ny * (unsigned)s.reps[r].nz * (unsigned)s.reps[r].nchunks;
    }
    t.item_off[s.nrep] = off;
    return t;
}

// Run f(RepTable<1 or MAX_BATCH>) for a single box or a batch.
template <typename F>
static cudaError_t by_batch_adj(const Sim &s, F &&f) {
    if (s.nrep == 1) return f(adj_table<1>(s));
    return f(adj_table<MAX_BATCH>(s));
}

cudaError_t launch_adj_particles(Sim &s, const void *g, const float *lam, const double *r,
                                 const double *v, long long step, const double *gv,
                                 const double *gr, double *lam_v, double *lam_r, double *acc,
                                 int parity, float *ug, cudaStream_t st) {
    if (s.np == 0) return cudaSuccess;
    AdjPArgs A;
    A.g = g;
    A.lam = lam;
    A.P = s.P;
    A.N = s.N;
    A.prep = s.prep;
    A.r = r;
    A.v = v;
    A.cap = s.cap;
    A.np = s.np;
    A.fext = s.fext;
    A.inv_mass = s.inv_mass;
    A.gamma = s.gamma;
    A.radius = s.radius;
    A.sig = s.sig;
    A.pinned = s.pinned;
    A.kT = s.kT;
    A.seed = s.seed;
    A.step = step;
    A.sqrt3 = s.sqrt3;
    A.mode = s.mode;
    A.exclude_inside = s.exclude_inside;
    A.gv = gv;
    A.gr = gr;
    A.lam_v = lam_v;
    A.lam_r = lam_r;
    A.acc = acc;
    A.rec = s.rec[parity];
    A.fqd = reinterpret_cast<double *>(s.fq);
    A.ug = ug;
    const unsigned grid = (unsigned)((s.np + APB - 1) / APB);
    return by_batch_adj(s, [&](const auto &rt) {
        constexpr int MAXR = sizeof(rt.rep) / sizeof(Rep);
        cudaError_t e = by_storage_adj(s.precision, [&](auto tag) {
            using St = decltype(tag);
            k_adj_gather<St, MAXR><<<grid, 8 * APB, 0, st>>>(A, rt);
            return cudaGetLastError();
        });
        if (e != cudaSuccess) return e;
        k_adj_fp64<MAXR><<<(unsigned)((8 * s.np + 63) / 64), 64, 0, st>>>(A, rt);
        return cudaGetLastError();
    });
}

cudaError_t launch_adj_lattice(Sim &s, const void *g, const float *lam, float *lam_out, int parity,
                               double *acc_omega, cudaStream_t st) {
    const unsigned grid = (unsigned)adj_lattice_blocks(s);
    return by_batch_adj(s, [&](const auto &rt) {
        constexpr int MAXR = sizeof(rt.rep) / sizeof(Rep);
        return by_storage_adj(s.precision, [&](auto tag) {
            using St = decltype(tag);
            k_adj_lattice<St, MAXR><<<grid, SEG, 0, st>>>(static_cast<const typename St::T *>(g), lam, lam_out,
                                                          s.P, rt, s.rec[parity], s.rec[parity ^ 1],
                                                          reinterpret_cast<double *>(s.fq), s.N, acc_omega);
            return cudaGetLastError();
        });
    });
}

int adj_lattice_blocks(const Sim &s) {
    int n = 0;
    for (int r = 0; r < s.nrep; ++r) n += s.reps[r].ny * s.reps[r].nz * s.reps[r].nchunks;
    return n;
}

int adj_lattice_first_block(const Sim &s, int replica) {
    int n = 0;
    for (int r = 0; r < replica; ++r) n += s.reps[r].ny * s.reps[r].nz * s.reps[r].nchunks;
    return n;
}

// dL/dfhat_a(y) of the first recorded state = dL/df_a(y + e_a) of its first
// step (the buffer's layout), to the FP64 [15][N] ABI layout, every box periodic on its own
template <int MAXR>
__global__ void k_adj_out(const float *src, double *dst, const RepTable<MAXR> rt, long long N, long long P) {
    const long long total = (long long)Q * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long long gi = t - (long long)a * N;
        const Rep &rp = rt.rep[find_node_rep(rt, gi)];
        const int nx = rp.nx, ny = rp.ny, nz = rp.nz;
        const long long i = gi - rp.node_off;
        const int x = (int)(i % nx);
        const long long yz = i / nx;
        const int y = (int)(yz % ny), z = (int)(yz / ny);
        int xs = x + ex(a), ys = y + ey(a), zs = z + ez(a);
        xs = xs == nx ? 0 : (xs < 0 ? nx - 1 : xs);
        ys = ys == ny ? 0 : (ys < 0 ? ny - 1 : ys);
        zs = zs == nz ? 0 : (zs < 0 ? nz - 1 : zs);
        dst[t] = (double)src[(long long)a * P + rp.node_off + ((long long)zs * ny + ys) * nx + xs];
    }
}

cudaError_t launch_f32_to_f64(Sim &s, const float *src, double *dst, cudaStream_t st) {
    long long g = ((long long)Q * s.N + 255) / 256;
    if (g > (long long)s.num_sms * 16) g = (long long)s.num_sms * 16;
    return by_batch_adj(s, [&](const auto &rt) {
        constexpr int MAXR = sizeof(rt.rep) / sizeof(Rep);
        k_adj_out<MAXR><<<(unsigned)(g < 1 ? 1 : g), 256, 0, st>>>(src, dst, rt, s.N, s.P);
        return cudaGetLastError();
    });
}

}  // namespace lbp
