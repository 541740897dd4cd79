// particle_kernels.cu -- two-way coupling kernel of liblbp (sm_103a).
//
// k_particles: a block of 8 PB threads serves PB particles in three phases.
//   A. eight threads per particle (one per corner) gather u^N at the corners
//      of the particle's cell from the stored populations (a pull, i.e. the
//      streamed f^n of Eq. 20): 14 independent loads per thread;
//   B. the Stokeslet flow of Eq. 8 is fitted -- by one thread per particle
//      (PB = 32), or with few particles by its eight corner lanes (PB = 8) --
//      and one thread per particle draws the Philox random force (Eqs. 4-5)
//      and advances V and r (Eqs. 1-2);
//   C. eight threads per particle append the shares of the reaction force
//      -F_H (Eq. 9) at the corner nodes to the force records of the row
//      segments holding those nodes; the stream-collide kernel applies them.
//
// Why one thread per particle in phase B: GB300 issues FP64 at 1/64 of the
// FP32 rate, so a warp-wide FP64 instruction costs the same whether one lane
// or 32 lanes need it.  Packing 32 particles into the warp that does the FP64
// work divides its FP64 instruction count per particle by 32; with one
// particle per warp the FP64 work of the fit dominated the whole time step.
// That holds while the FP64 pipe is the limit; with a warp or two of
// particles per SM the fit's dependent chain is, and the lane-per-corner
// layout shortens it (see PB_WIDE / PB_NARROW below).
//
// Exchange I/O (lbp_step_exchange with device buffers or page-locked host
// buffers, seen through their device views): warp 1 reads the block's
// external forces from the caller's [n][3] buffer and keeps them; the new
// positions and velocities go to the caller's buffers after phase B, as one
// contiguous span per block read back from the state arrays (PB = 32) or
// straight from the update's registers (PB = 8).  For host buffers the last
// block to finish then sets a completion flag in page-locked memory after a
// system-scope fence, and the host returns without waiting for the lattice
// pass.
//
// Precision split.  FP32: the gathered u^N (the lattice arithmetic is FP32).
// FP64: everything after the gather -- positions, velocities, the cell and
// fraction of r, the relative velocities w_p = u_p - V, e^N, the corner
// geometry, the basis a_p and the eight-point sums of the normal equation
// with its solve U_inf = (sum w.a)/(sum |a|^2), F_H, the random force and the
// Langevin update.
//
// Reaction forces are 64-bit fixed-point integers (scale 2^56).  -F_H is
// converted once and split over the eight corners by the trilinear fractions
// with integer arithmetic (the 1 - q share is the remainder), so the eight
// shares sum to -F_H exactly and the momentum the fluid receives is exactly
// what the particle lost.  Each share is appended to the record of its row
// segment (slot index from an integer atomic on the record's count).  The
// per-node force is the integer sum of the matching entries, so it is exact
// and independent of the order in which particles appended them (no
// floating-point atomics).  When a record is full the share goes to a dense
// per-node accumulator (integer atomics), which the stream-collide block of
// an overflowed segment adds to the record sum; the total is the same exact
// integer sum whichever shares found a slot.
#include <cuda_runtime.h>

#include "lbp_internal.cuh"

namespace lbp {

struct ParticleArgs {
    const void *g;   // deviation populations fhat^{n-1} (storage type of the handle)
    const int *prep; // replica (box) of each particle
    long long P;
    long long N;
    double *r, *v, *fh, *fr;
    double *fext;  // written only when fext_in is given (lbp_step_exchange)
    const double *inv_mass, *gamma, *radius, *sig;
    const unsigned char *pinned;
    int cap, np;
    const long long *d_step;
    unsigned long long seed;
    double sqrt3;
    int mode, exclude_inside;
    unsigned long long *rec; // force records of this step's parity
    unsigned long long *fq;  // [3][N] fixed-point overflow accumulator
    float *ring;        // per-particle VACF ring (FP32), or null
    __half *ring16;     // ensemble VACF/MSD ring (fp16 hi/lo planes), or null
    int ring_ld, ring_dup;
    int ring_cap;
    long long *d_vacf;  // [0] first sampled step, [2] samples written
    int *err;
    double *inj;        // [3] momentum put in by F_R + F_ext (null: not tracked)
    // lbp_step_exchange with page-locked host buffers ([n][3] FP64, device views
    // of host memory; null: none): the external forces to use (and keep), and
    // the positions and velocities after the update; done_flag (host memory) is
    // set to the step index once every block has written them
    const double *fext_in;
    double *r_out, *v_out;
    unsigned *done_ticket;
    long long *done_flag;
};

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Eq. 8 in FP64, shared by both layouts of the fit below.  Every operation is
// rounded explicitly (no contraction left to the compiler), and the eight
// corners' terms are summed as the tree ((0 + 1) + (2 + 3)) + ((4 + 5) + (6 + 7)),
// which is also the order of a butterfly over eight lanes: one thread per
// particle and one lane per corner give the same bits.
//
// e^N = m/|m| of the mean relative velocity m (times 8); false if m = 0.
__device__ __forceinline__ bool fit_direction(double m0, double m1, double m2, double &e0, double &e1,
                                              double &e2) {
    if (m0 == 0.0 && m1 == 0.0 && m2 == 0.0) return false;
    double mm = __fma_rn(m2, m2, __fma_rn(m1, m1, __dmul_rn(m0, m0)));
    if (!(mm > 1e-280)) {
        // tiny mean: rescale before the norm so that it does not underflow
        const double sc = 1.0 / fmax(fabs(m0), fmax(fabs(m1), fabs(m2)));
        m0 = __dmul_rn(m0, sc);
        m1 = __dmul_rn(m1, sc);
        m2 = __dmul_rn(m2, sc);
        mm = __fma_rn(m2, m2, __fma_rn(m1, m1, __dmul_rn(m0, m0)));
    }
    const double inrm = rsqrt(mm);
    e0 = __dmul_rn(m0, inrm);
    e1 = __dmul_rn(m1, inrm);
    e2 = __dmul_rn(m2, inrm);
    return true;
}

// The terms of one corner: t_n = w.a and t_d = |a|^2 with d = x_p - r_i (the
// corner minus the cell fraction, exact), w = u_p - V and the basis
// a = (1 - 3R/(4 r)) e^N - 3R (e^N.d)/(4 r^3) d; zero for a corner the fit
// skips (r < 1e-12, or r < R with exclude).
__device__ __forceinline__ void fit_corner(double d0, double d1, double d2, double e0, double e1, double e2,
                                           double R34, double R2, int exclude, double w0, double w1, double w2,
                                           double &tn, double &td) {
    tn = 0.0;
    td = 0.0;
    const double rr = __fma_rn(d2, d2, __fma_rn(d1, d1, __dmul_rn(d0, d0)));
    if (rr < 1e-24 || (exclude && rr < R2)) return;
    const double ir = rsqrt(rr);
    const double x = __fma_rn(e2, d2, __fma_rn(e1, d1, __dmul_rn(e0, d0)));
    const double k1 = __fma_rn(-R34, ir, 1.0);
    const double k2 = __dmul_rn(__dmul_rn(R34, x), __dmul_rn(__dmul_rn(ir, ir), ir));
    const double a0 = __fma_rn(k1, e0, -__dmul_rn(k2, d0));
    const double a1 = __fma_rn(k1, e1, -__dmul_rn(k2, d1));
    const double a2 = __fma_rn(k1, e2, -__dmul_rn(k2, d2));
    tn = __fma_rn(w2, a2, __fma_rn(w1, a1, __dmul_rn(w0, a0)));
    td = __fma_rn(a2, a2, __fma_rn(a1, a1, __dmul_rn(a0, a0)));
}

// Sum of v over the eight lanes of a particle (lanes 8j .. 8j + 7), in the
// tree order above; every lane of the group gets the same sum.
__device__ __forceinline__ double sum8(double v) {
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Particles per block: 32 (256 threads) with the fit one thread per particle
// (FIT8 = false); 8 (64 threads) with the fit one lane per corner (FIT8 =
// true).  An FP64 warp instruction occupies the SM's narrow FP64 pipe for 16
// cycles whatever its active lanes, and the fit is ~480 of them per particle.
// With many particles the pipe is the limit and one thread per particle uses
// every lane of each instruction.  With few particles (a warp or two per SM)
// the fit is one warp's chain of dependent FP64 instructions; spreading the
// eight corners over eight lanes, and the particles over more blocks, cuts
// that chain about fourfold.
constexpr int PB_WIDE = 32, PB_NARROW = 8;

// 64 registers (four blocks of 256 threads per SM) keep the 16384-particle
// grid of the 256^3 workload (512 blocks) in a single wave on 152 SMs (at 80
// registers, three blocks per SM, it took two).
template <typename St, int MAXR, int PB, bool FIT8>
__global__ void __launch_bounds__(8 * PB, PB == PB_WIDE ? 4 : 16) k_particles(const ParticleArgs A,
                                                                            const RepTable<MAXR> rt) {
    const typename St::T *G = static_cast<const typename St::T *>(A.g);
    __shared__ int s_base[PB][3];
    __shared__ int s_rep[PB];
    // u^N of each corner: summed in FP32 by its gather thread, which also
    // converts it to FP64 (exact), while the FP64 pipe is otherwise idle
    __shared__ double s_u[PB][8][3];
    __shared__ long long s_fix[PB][3];
    __shared__ long long s_frac[PB][3];
    __shared__ int s_spread[PB];
    // state read only by the Langevin update, staged by warp 1 so that warp 0
    // (the FP64 fit) carries fewer registers across the gather
    __shared__ double s_fe[3][PB];
    __shared__ double s_invM[PB], s_sg[PB];
    __shared__ unsigned char s_pin[PB];
    // one lane per corner: the particle state the corner lanes read, and the fit
    __shared__ double s_q[FIT8 ? PB : 1][4], s_V[FIT8 ? PB : 1][3];
    __shared__ double s_e[FIT8 ? PB : 1][3], s_nd[FIT8 ? PB : 1][2];
    __shared__ int s_eok[FIT8 ? PB : 1];
    const int t = threadIdx.x, lane = t & 31;
    const int i0 = blockIdx.x * PB;
    const long long step = *A.d_step;
    // the step's lattice pass may launch now: it waits for this grid's
    // completion before it reads anything this kernel writes (or bumps the step)
    grid_dependents_launch();
    const int cap = A.cap;
    if ((A.ring || A.ring16) && blockIdx.x == 0 && t == 0) {
        const long long m = step - A.d_vacf[0];
        if (m >= 0) A.d_vacf[2] = m + 1;
    }

    // ---- cell of each particle (warp 0): base = floor(r), q = r - base (exact).
    // Warp 0 also loads all the particle state phase B needs now, so that its
    // loads overlap this step's other memory round trips.
    const int ip = i0 + lane;
    double r0 = 0.0, r1 = 0.0, r2 = 0.0, q0 = 0.0, q1 = 0.0, q2 = 0.0;
    double V0 = 0.0, V1 = 0.0, V2 = 0.0, gam = 0.0, Rd = 0.0;
    if (t >= 32 && t < 32 + PB && ip < A.np) {
        s_invM[lane] = A.inv_mass[ip];
        s_sg[lane] = A.sig[ip];
        if (A.fext_in) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double f = A.fext_in[3 * (size_t)ip + k];
                s_fe[k][lane] = f;
                A.fext[k * cap + ip] = f;  // kept for the steps that follow
            }
        } else {
            s_fe[0][lane] = A.fext[ip];
            s_fe[1][lane] = A.fext[cap + ip];
            s_fe[2][lane] = A.fext[2 * cap + ip];
        }
        s_pin[lane] = A.pinned[ip];
    }
    if (t < PB && ip < A.np) {
        r0 = A.r[ip];
        r1 = A.r[cap + ip];
        r2 = A.r[2 * cap + ip];
        V0 = A.v[ip];
        V1 = A.v[cap + ip];
        V2 = A.v[2 * cap + ip];
        gam = A.gamma[ip];
        Rd = A.radius[ip];
        s_rep[lane] = MAXR == 1 ? 0 : A.prep[ip];
        const double b0 = floor(r0), b1 = floor(r1), b2 = floor(r2);
        q0 = r0 - b0;
        q1 = r1 - b1;
        q2 = r2 - b2;
        s_base[lane][0] = (int)b0;
        s_base[lane][1] = (int)b1;
        s_base[lane][2] = (int)b2;
        if (FIT8) {
            s_q[lane][0] = q0;
            s_q[lane][1] = q1;
            s_q[lane][2] = q2;
            s_q[lane][3] = Rd;
            s_V[lane][0] = V0;
            s_V[lane][1] = V1;
            s_V[lane][2] = V2;
        }
    }
    __syncthreads();

    // ---- phase A: u at corner p, u = sum_a e_a g_a(x_p - e_a) (FP32)
    const int j = t >> 3, p = t & 7;
    const int ij = i0 + j;
    const int c0 = p & 1, c1 = (p >> 1) & 1, c2 = (p >> 2) & 1;
    int X = 0, Y = 0, Z = 0;
    const Rep &rj = rt.rep[MAXR == 1 || ij >= A.np ? 0 : s_rep[j]];
    const int nx = rj.nx, ny = rj.ny, nz = rj.nz;
    if (ij < A.np) {
        X = wrapi(s_base[j][0] + c0, nx);
        Y = wrapi(s_base[j][1] + c1, ny);
        Z = wrapi(s_base[j][2] + c2, nz);
        const int xs[3] = {wrapi(X + 1, nx), X, wrapi(X - 1, nx)};  // x - e for e = -1, 0, 1
        const int ys[3] = {wrapi(Y + 1, ny), Y, wrapi(Y - 1, ny)};
        const int zs[3] = {wrapi(Z + 1, nz), Z, wrapi(Z - 1, nz)};
        float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int a = 1; a < Q; ++a) {
            const long long src = (long long)a * A.P + rj.node_off +
                                  ((long long)zs[ez(a) + 1] * ny + ys[ey(a) + 1]) * nx + xs[ex(a) + 1];
            const float gv = St::load(G + src, a);
            if (ex(a)) sx += ex(a) > 0 ? gv : -gv;
            if (ey(a)) sy += ey(a) > 0 ? gv : -gv;
            if (ez(a)) sz += ez(a) > 0 ? gv : -gv;
        }
        s_u[j][p][0] = (double)sx;
        s_u[j][p][1] = (double)sy;
        s_u[j][p][2] = (double)sz;
    }
    __syncthreads();

    // ---- the fit of Eq. 8 with one lane per corner (all threads): the mean
    // relative velocity and e^N in every lane of the particle (sum8 gives all
    // eight the same sum), the corner's terms, their sums to s_nd
    if (FIT8 && A.mode == LBP_STOKESLET) {
        const bool live = ij < A.np;
        double V[3] = {0.0, 0.0, 0.0}, m[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (live) V[k] = s_V[j][k];
            m[k] = __fma_rn(-8.0, V[k], sum8(live ? s_u[j][p][k] : 0.0));
        }
        double e0 = 0.0, e1 = 0.0, e2 = 0.0;
        const bool eok = live && fit_direction(m[0], m[1], m[2], e0, e1, e2);
        double tn = 0.0, td = 0.0;
        if (eok) {
            const double q0p = s_q[j][0], q1p = s_q[j][1], q2p = s_q[j][2], Rp = s_q[j][3];
            const double d0 = c0 ? __dsub_rn(1.0, q0p) : -q0p;
            const double d1 = c1 ? __dsub_rn(1.0, q1p) : -q1p;
            const double d2 = c2 ? __dsub_rn(1.0, q2p) : -q2p;
            fit_corner(d0, d1, d2, e0, e1, e2, 0.75 * Rp, Rp * Rp, A.exclude_inside,
                       __dsub_rn(s_u[j][p][0], V[0]), __dsub_rn(s_u[j][p][1], V[1]),
                       __dsub_rn(s_u[j][p][2], V[2]), tn, td);
        }
        tn = sum8(tn);
        td = sum8(td);
        if (live && p == 0) {
            s_eok[j] = eok;
            s_e[j][0] = e0;
            s_e[j][1] = e1;
            s_e[j][2] = e2;
            s_nd[j][0] = tn;
            s_nd[j][1] = td;
        }
        __syncthreads();
    }

    // ---- phase B (warp 0): fit, random force, Langevin update
    if (t < PB && ip < A.np) {
        const int i = ip;
        double F0 = 0.0, F1 = 0.0, F2 = 0.0;
        bool spread = true;
        if (A.mode == LBP_STOKESLET) {
            // Eq. 8 in FP64 from the FP32 corner velocities: w_p = u_p - V,
            // e^N = mean(w)/|mean(w)|, d_p = x_p - r_i (exact: corner minus
            // cell fraction), basis a_p = (1 - 3R/(4 r_p)) e^N - 3R (e^N.d_p)/(4 r_p^3) d_p,
            // and the normal equation U_inf sum|a_p|^2 = sum w_p.a_p, solved
            // for U_inf; F_H = gamma U_inf e^N (Eq. 7 with u_inf = U_inf e^N + V).
            double num = 0.0, den = 0.0, e0 = 0.0, e1 = 0.0, e2 = 0.0;
            bool eok;
            if (FIT8) {
                eok = s_eok[lane];
                e0 = s_e[lane][0];
                e1 = s_e[lane][1];
                e2 = s_e[lane][2];
                num = s_nd[lane][0];
                den = s_nd[lane][1];
            } else {
                // the same operations as the lane-per-corner layout, in one
                // thread: w_p is formed again in the corner loop from the shared
                // corner velocities (holding all 24 would spill)
                double m[3];
                const double Vk[3] = {V0, V1, V2};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    asm volatile("" ::: "memory");
                    double h[4];
#pragma unroll
                    for (int c = 0; c < 8; c += 2)
                        h[c >> 1] = __dadd_rn(s_u[lane][c][k], s_u[lane][c + 1][k]);
                    m[k] = __fma_rn(-8.0, Vk[k], __dadd_rn(__dadd_rn(h[0], h[1]), __dadd_rn(h[2], h[3])));
                }
                eok = fit_direction(m[0], m[1], m[2], e0, e1, e2);
                if (eok) {
                    const double R34 = 0.75 * Rd, R2 = Rd * Rd;
                    const double dx[2] = {-q0, __dsub_rn(1.0, q0)}, dy[2] = {-q1, __dsub_rn(1.0, q1)},
                                 dz[2] = {-q2, __dsub_rn(1.0, q2)};
                    double hn[4], hd[4];
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        // load each pair's corner velocities where they are used
                        // (hoisting all 24 doubles would spill)
                        asm volatile("" ::: "memory");
                        double tn0, td0, tn1, td1;
                        fit_corner(dx[0], dy[(c >> 1) & 1], dz[(c >> 2) & 1], e0, e1, e2, R34, R2, A.exclude_inside,
                                   __dsub_rn(s_u[lane][c][0], V0), __dsub_rn(s_u[lane][c][1], V1),
                                   __dsub_rn(s_u[lane][c][2], V2), tn0, td0);
                        fit_corner(dx[1], dy[(c >> 1) & 1], dz[(c >> 2) & 1], e0, e1, e2, R34, R2, A.exclude_inside,
                                   __dsub_rn(s_u[lane][c + 1][0], V0),
                                   __dsub_rn(s_u[lane][c + 1][1], V1),
                                   __dsub_rn(s_u[lane][c + 1][2], V2), tn1, td1);
                        hn[c >> 1] = __dadd_rn(tn0, tn1);
                        hd[c >> 1] = __dadd_rn(td0, td1);
                    }
                    num = __dadd_rn(__dadd_rn(hn[0], hn[1]), __dadd_rn(hn[2], hn[3]));
                    den = __dadd_rn(__dadd_rn(hd[0], hd[1]), __dadd_rn(hd[2], hd[3]));
                }
            }
            if (eok) {
                const double U = den > 0.0 ? num / den : 0.0;
                const double gU = gam * U;
                F0 = gU * e0;
                F1 = gU * e1;
                F2 = gU * e2;
            }
        } else if (A.mode == LBP_POINTWISE) {
            // Eq. 7 with u(r_i) = sum_p W_p u^N_p (trilinear weights of the cell
            // fraction), in FP64
            const double wx[2] = {1.0 - q0, q0}, wy[2] = {1.0 - q1, q1}, wz[2] = {1.0 - q2, q2};
            double ur0 = 0.0, ur1 = 0.0, ur2 = 0.0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const double Wp = wx[c & 1] * wy[(c >> 1) & 1] * wz[(c >> 2) & 1];
                ur0 += Wp * s_u[lane][c][0];
                ur1 += Wp * s_u[lane][c][1];
                ur2 += Wp * s_u[lane][c][2];
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
        if (spread) {
            const bool ok = fabs(F0) < FIX_LIMIT && fabs(F1) < FIX_LIMIT && fabs(F2) < FIX_LIMIT;
            if (!ok) {
                atomicOr(A.err, ERR_RANGE);
                spread = false;
            } else {
                s_fix[lane][0] = __double2ll_rn(-F0 * FIX_SCALE);
                s_fix[lane][1] = __double2ll_rn(-F1 * FIX_SCALE);
                s_fix[lane][2] = __double2ll_rn(-F2 * FIX_SCALE);
                // q as 31-bit fractions q31 = floor(q 2^31) in bits 32..62
                s_frac[lane][0] = (long long)((unsigned long long)__double2uint_rz(q0 * 2147483648.0) << 32);
                s_frac[lane][1] = (long long)((unsigned long long)__double2uint_rz(q1 * 2147483648.0) << 32);
                s_frac[lane][2] = (long long)((unsigned long long)__double2uint_rz(q2 * 2147483648.0) << 32);
            }
        }
        s_spread[lane] = spread ? 1 : 0;

        // Eqs. 4-5: F_R = sqrt(2 gamma kT) xi, xi = sqrt3 (2u - 1) with
        // u = ((x >> 11) + 1/2) 2^-53 from Philox(counter = (step, i, 0, 0), key = (seed, 0)).
        // 2u - 1 is formed as fma((double)(2k + 1), 2^-53, -1): the same correctly
        // rounded value as 2 ((double)k + 1/2) 2^-53 - 1, so F_R is bit-identical
        // to the oracle's.
        unsigned long long ctr[4] = {(unsigned long long)step, (unsigned long long)i, 0ull, 0ull};
        philox4x64_10(ctr, A.seed, 0ull);
        double R3[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double tt = __fma_rn(__ull2double_rn(2ull * (ctr[k] >> 11) + 1ull), 0x1.0p-53, -1.0);
            R3[k] = __dmul_rn(s_sg[lane], __dmul_rn(A.sqrt3, tt));
        }
        const double FH3[3] = {F0, F1, F2};
        const double Vo[3] = {V0, V1, V2};
        const double ro[3] = {r0, r1, r2};
        const double invM = s_invM[lane];
        const bool pin = s_pin[lane] != 0;
        const Rep &ri = rt.rep[MAXR == 1 ? 0 : s_rep[lane]];
        const int L[3] = {ri.nx, ri.ny, ri.nz};
        double Vn[3] = {V0, V1, V2};
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            A.fh[k * cap + i] = FH3[k];
            A.fr[k * cap + i] = R3[k];
            double rw = ro[k];
            if (!pin) {
                // Eqs. 1-2, dt = 1: V += (F_H + F_R + F_ext)/M; r += V; periodic wrap
                Vn[k] = Vo[k] + (FH3[k] + R3[k] + s_fe[k][lane]) * invM;
                double rn = ro[k] + Vn[k];
                if (rn < 0.0) rn += (double)L[k];
                if (rn >= (double)L[k]) rn -= (double)L[k];
                const bool b = !isfinite(Vn[k]) || !(rn >= 0.0) || !(rn < (double)L[k]);
                if (b) rn = 0.0;  // keep the next gather inside the box; reported as LBP_ENAN
                bad |= b;
                A.v[k * cap + i] = Vn[k];
                A.r[k * cap + i] = rn;
                rw = rn;
            }
            if (FIT8) {  // few particles: straight from the update's registers
                if (A.r_out) A.r_out[3 * (size_t)i + k] = rw;
                if (A.v_out) A.v_out[3 * (size_t)i + k] = Vn[k];
            }
        }
        if (FIT8 && A.done_flag) __threadfence_system();  // the host copies before the flag
        if (bad) atomicOr(A.err, ERR_NAN);
        if (A.inj)
#pragma unroll
            for (int k = 0; k < 3; ++k) s_fe[k][lane] = pin ? 0.0 : R3[k] + s_fe[k][lane];
        if (A.ring) {
            const long long m = step - A.d_vacf[0];
            if (m >= 0) {
                float *dst = A.ring + (m % A.ring_cap) * 3 * (long long)A.np;
                dst[i] = (float)Vn[0];
                dst[A.np + i] = (float)Vn[1];
                dst[2 * A.np + i] = (float)Vn[2];
            }
        }
        if (A.ring16) {
            // the sample as fp16 hi/lo of 4096 V (the tensor-core correlator's
            // operands), at its ring row and, for the first rows, once more
            // after the end of the ring
            const long long m = step - A.d_vacf[0];
            if (m >= 0) {
                const int row = (int)(m % A.ring_cap);
                bool big = false;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double a = Vn[k] * (double)VACF_RING_SCALE;
                    big |= !(fabs(a) < 65504.0);
                    const __half hi = __double2half(a);
                    const __half lo = __double2half(a - (double)__half2float(hi));
                    const long long j = (long long)k * A.np + i;
                    __half *p = A.ring16 + (long long)row * 2 * A.ring_ld + j;
                    p[0] = hi;
                    p[A.ring_ld] = lo;
                    if (row < A.ring_dup) {
                        __half *p2 = p + (long long)A.ring_cap * 2 * A.ring_ld;
                        p2[0] = hi;
                        p2[A.ring_ld] = lo;
                    }
                }
                if (big) atomicOr(A.err, ERR_RANGE);
            }
        }
    }
    __syncthreads();

    // With many particles (one thread per particle), positions and velocities
    // go to the caller's buffers ([n][3], host memory seen through its device
    // mapping) as one contiguous span per block, read back from the state
    // arrays the update above wrote (a pinned particle's entries there are its
    // unchanged ones), before phase C so that their round trip overlaps it.
    // (With one lane per corner the update's threads write them directly: the
    // 64-register budget of that layout has no room for this step beside
    // phase C's live values.)
    if (!FIT8 && (A.r_out || A.v_out) && t < 3 * PB && 3LL * i0 + t < 3LL * A.np) {
        const int pi = i0 + t / 3, k = t - 3 * (t / 3);
        if (A.r_out) A.r_out[3LL * i0 + t] = A.r[k * cap + pi];
        if (A.v_out) A.v_out[3LL * i0 + t] = A.v[k * cap + pi];
    }

    if (A.inj && t < 32) {
        // conservation budget: the momentum F_R + F_ext put into the block's
        // unpinned particles (left in s_fe by phase B), summed over the warp,
        // one FP64 atomic per component
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double vk = lane < PB && ip < A.np ? s_fe[k][lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vk += __shfl_xor_sync(0xffffffffu, vk, o);
            if (lane == 0) atomicAdd(A.inj + k, vk);
        }
    }

    // ---- phase C: share of corner p of the fixed-point reaction force -F_H.
    // Per axis the far corner (c = 1) takes floor(v q) -- the signed high half
    // of (2 v) (q31 2^32) -- and the near corner the rest, so the eight shares
    // add up to v exactly.  |v| < 2^61 (|F_H| < 32), so 2 v stays within int64.
    if (ij < A.np && s_spread[j]) {
        const int cc[3] = {c0, c1, c2};
        long long sh[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            long long v = s_fix[j][k];
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const long long far = __mul64hi(2 * v, s_frac[j][ax]);
                v = cc[ax] ? far : v - far;
            }
            sh[k] = v;
        }
        const long long row = (long long)Z * ny + Y;
        unsigned long long *rec =
            A.rec + (size_t)(rj.seg_off + row * rj.nchunks + X / SEG) * REC_WORDS;
        const unsigned int slot = atomicAdd(reinterpret_cast<unsigned int *>(rec), 1u);
        if (slot < (unsigned)REC_SLOTS) {
            reinterpret_cast<int *>(rec + REC_X0)[slot] = X;
            rec[REC_F0 + 3 * slot] = (unsigned long long)sh[0];
            rec[REC_F0 + 3 * slot + 1] = (unsigned long long)sh[1];
            rec[REC_F0 + 3 * slot + 2] = (unsigned long long)sh[2];
        } else {
            const long long node = rj.node_off + row * nx + X;
            atomicAdd(A.fq + node, (unsigned long long)sh[0]);
            atomicAdd(A.fq + A.N + node, (unsigned long long)sh[1]);
            atomicAdd(A.fq + 2 * A.N + node, (unsigned long long)sh[2]);
        }
    }

    // the last block to finish tells the host that every position and velocity
    // is in its buffers (the lattice pass may still run)
    if (A.done_flag) {
        // the writes to the host buffers, made visible before the block's ticket
        if (!FIT8 && t < 3 * PB) __threadfence_system();
        __syncthreads();
        if (t == 0) {
            const unsigned ticket = atomicAdd(A.done_ticket, 1u);
            if (ticket == gridDim.x - 1) {
                *A.done_ticket = 0u;
                __threadfence_system();
                *reinterpret_cast<volatile long long *>(A.done_flag) = step;
            }
        }
    }
}

template <int MAXR, int PB, bool FIT8>
static void launch_particles_pb(const Sim &s, const ParticleArgs &A, const RepTable<MAXR> &t, cudaStream_t st) {
    const unsigned grid = (unsigned)((s.np + PB - 1) / PB);
    switch (s.precision) {
        case LBP_BF16: k_particles<StoreBF16, MAXR, PB, FIT8><<<grid, 8 * PB, 0, st>>>(A, t); break;
        case LBP_F16: k_particles<StoreF16, MAXR, PB, FIT8><<<grid, 8 * PB, 0, st>>>(A, t); break;
        default: k_particles<StoreF32, MAXR, PB, FIT8><<<grid, 8 * PB, 0, st>>>(A, t); break;
    }
}

// The fit one lane per corner while the one-thread-per-particle layout would
// leave the FP64 pipe mostly idle (fewer than ~50 particles per SM: its
// dependent chain, not the pipe, sets the time); both give the same bits.
bool particles_fit_per_corner(const Sim &s) { return s.np < 48 * (s.num_sms > 0 ? s.num_sms : 1); }

template <int MAXR>
static void launch_particles_t(const Sim &s, const ParticleArgs &A, const RepTable<MAXR> &t, cudaStream_t st) {
    if (particles_fit_per_corner(s))
        launch_particles_pb<MAXR, PB_NARROW, true>(s, A, t, st);
    else
        launch_particles_pb<MAXR, PB_WIDE, false>(s, A, t, st);
}

cudaError_t launch_particles(Sim &s, const void *src, int parity, cudaStream_t st, const ParticleIO *io) {
    if (s.np == 0) return cudaSuccess;
    ParticleArgs A;
    A.g = src;
    A.prep = s.prep;
    A.P = s.P;
    A.N = s.N;
    A.r = s.r;
    A.v = s.v;
    A.fh = s.fh;
    A.fr = s.fr;
    A.fext = s.fext;
    A.inv_mass = s.inv_mass;
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
    A.rec = s.rec[parity];
    A.ring = s.vacf_lag >= 0 && s.vacf_pp ? s.ring : nullptr;
    A.ring16 = s.vacf_lag >= 0 && !s.vacf_pp ? static_cast<__half *>(s.ring16) : nullptr;
    A.ring_ld = s.ring_ld;
    A.ring_dup = vacf_ring_dup_rows();
    A.ring_cap = s.vacf_cap;
    A.d_vacf = s.d_vacf;
    A.err = s.d_err;
    A.inj = s.inj;
    A.fext_in = io ? io->fext_in : nullptr;
    A.r_out = io ? io->r_out : nullptr;
    A.v_out = io ? io->v_out : nullptr;
    A.done_ticket = io && io->signal ? s.d_xticket : nullptr;
    A.done_flag = io && io->signal ? s.h_xflag_dev : nullptr;
    if (s.nrep == 1) {
        RepTable<1> t;
        t.nrep = 1;
        t.item_off[0] = 0;
        t.item_off[1] = 0;
        t.rep[0] = s.reps[0];
        launch_particles_t(s, A, t, st);
    } else {
        RepTable<MAX_BATCH> t;  // kernel parameter
        t.nrep = s.nrep;
        for (int r = 0; r <= s.nrep; ++r) t.item_off[r] = 0;
        for (int r = 0; r < s.nrep; ++r) t.rep[r] = s.reps[r];
        launch_particles_t(s, A, t, st);
    }
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

// Cell base index and cell fraction of the current positions, with the same
// expressions k_particles uses (for bit-exact checks of the indexing).
__global__ void k_cells(const double *r, int cap, int np, int *base, double *frac) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    for (int k = 0; k < 3; ++k) {
        const double rk = r[(long long)k * cap + i];
        const double b = floor(rk);
        base[3 * i + k] = (int)b;
        frac[3 * i + k] = rk - b;
    }
}

cudaError_t launch_cells(Sim &s, int *base, double *frac, cudaStream_t st) {
    if (s.np == 0) return cudaSuccess;
    k_cells<<<(s.np + 127) / 128, 128, 0, st>>>(s.r, s.cap, s.np, base, frac);
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
