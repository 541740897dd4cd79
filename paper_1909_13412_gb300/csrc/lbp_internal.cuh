// lbp_internal.cuh -- device-side definitions shared by the liblbp translation
// units: the D3Q15 table, the Philox-4x64-10 block function, the handle layout
// and the kernel launchers.  Written for sm_103a (GB300).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lbp.h"

namespace lbp {

constexpr int Q = 15;

// D3Q15 velocity set in the order the ABI documents (Section 2.2, Succi's
// fifteen-velocity set): rest, 6 faces, 8 corners; opposite pairs adjacent.
__host__ __device__ constexpr int ex(int a) {
    return a == 1 ? 1 : a == 2 ? -1 : (a == 7 || a == 9 || a == 11 || a == 14) ? 1
         : (a == 8 || a == 10 || a == 12 || a == 13) ? -1 : 0;
}
__host__ __device__ constexpr int ey(int a) {
    return a == 3 ? 1 : a == 4 ? -1 : (a == 7 || a == 9 || a == 12 || a == 13) ? 1
         : (a == 8 || a == 10 || a == 11 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int ez(int a) {
    return a == 5 ? 1 : a == 6 ? -1 : (a == 7 || a == 10 || a == 11 || a == 13) ? 1
         : (a == 8 || a == 9 || a == 12 || a == 14) ? -1 : 0;
}
// weights: 2/9 rest, 1/9 faces, 1/72 corners
__host__ __device__ constexpr double wgt(int a) {
    return a == 0 ? 2.0 / 9.0 : a <= 6 ? 1.0 / 9.0 : 1.0 / 72.0;
}
__host__ __device__ constexpr float wgtf(int a) {
    return a == 0 ? 2.0f / 9.0f : a <= 6 ? 1.0f / 9.0f : 1.0f / 72.0f;
}

// ------------------------------------------------------------ storage
// The populations are stored as deviations g_a = f_a - w_a from the rest
// state; arithmetic is always FP32.  Three storage types:
//   F32  : g_a as float (120 bytes per node update);
//   BF16 : g_a rounded to bfloat16 (60 bytes);
//   F16  : g_a * (F16_SCALE / w_a) rounded to binary16 (60 bytes).  The
//          per-population scale keeps the deviations of slow flows inside
//          binary16's normal range (|g/w| down to ~6e-8 stays normal) while
//          |g/w| up to 64 still fits.
constexpr float F16_SCALE = 1024.f;

// load/store: the deviation g.  cload/cstore (and cload_shared): the values
// the lattice kernels' collision works on (collide_st): g itself for F32 and
// BF16; for F16 the stored variable h = g F16_SCALE / w_a, on which the
// collision is written directly (collide_values_scaled), so the lattice pass
// does not scale its 15 loads and 15 stores per node.
struct StoreF32 {
    using T = float;
    static constexpr bool SCALED = false;
    static __device__ __forceinline__ float load(const T *p, int) { return __ldg(p); }
    static __device__ __forceinline__ float load_shared(const T *p, int) { return *p; }
    static __device__ __forceinline__ void store(T *p, int, float v) { *p = v; }
    static __device__ __forceinline__ float cload(const T *p, int a) { return load(p, a); }
    static __device__ __forceinline__ float cload_shared(const T *p, int a) { return load_shared(p, a); }
    static __device__ __forceinline__ void cstore(T *p, int a, float v) { store(p, a, v); }
};
struct StoreBF16 {
    using T = __nv_bfloat16;
    static constexpr bool SCALED = false;
    static __device__ __forceinline__ float load(const T *p, int) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float load_shared(const T *p, int) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void store(T *p, int, float v) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ float cload(const T *p, int a) { return load(p, a); }
    static __device__ __forceinline__ float cload_shared(const T *p, int a) { return load_shared(p, a); }
    static __device__ __forceinline__ void cstore(T *p, int a, float v) { store(p, a, v); }
};
struct StoreF16 {
    using T = __half;
    static constexpr bool SCALED = true;
    static __device__ __forceinline__ float load(const T *p, int a) {
        return __half2float(__ldg(p)) * (wgtf(a) * (1.f / F16_SCALE));
    }
    static __device__ __forceinline__ float load_shared(const T *p, int a) {
        return __half2float(*p) * (wgtf(a) * (1.f / F16_SCALE));
    }
    static __device__ __forceinline__ void store(T *p, int a, float v) {
        *p = __float2half_rn(v * (F16_SCALE / wgtf(a)));
    }
    static __device__ __forceinline__ float cload(const T *p, int) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float cload_shared(const T *p, int) { return __half2float(*p); }
    static __device__ __forceinline__ void cstore(T *p, int, float v) { *p = __float2half_rn(v); }
};

__host__ __device__ constexpr int storage_bytes(int precision) { return precision == LBP_F32 ? 4 : 2; }

// ------------------------------------------------------------ collision
// Per-population plane pointers of the source (pulled from) and destination
// buffers of one lattice pass.
template <typename St>
struct Planes {
    const typename St::T *s[Q];
    typename St::T *d[Q];
};

// Collision of one node (Eqs. 15, 17-19 in deviation form, see
// lbm_kernels.cu): the 15 post-collision deviations of the node whose
// pulled deviations are g; (F0, F1, F2) is the body force of Eq. 18 at the
// node (zero if none).  Per opposite pair (A, A+1), e_{A+1} = -e_A, weight W:
//     o_A, o_{A+1} = (1 - omega) g + S +- X,
//     S = omega W (base + 9/2 (e.u)^2),   X = 3 omega W e.u + 3 W e.F,
// with base = (rho~ - 1) - 3/2 u.u, and o_0 = (1 - omega) g_0 + (2/9) omega base:
// omega is folded into the per-class constants omega W, so a pair costs eight
// operations.  Every operation is written out with its rounding (no
// contraction left to the compiler), so that every kernel that inlines this
// function performs the same operations in the same order, bit for bit.
__device__ __forceinline__ void collide_values(const float g[Q], float omega, float F0, float F1,
                                               float F2, float o[Q]) {
    float drho = g[0];
#pragma unroll
    for (int a = 1; a < Q; ++a) drho = __fadd_rn(drho, g[a]);
    const float c78 = __fsub_rn(g[7], g[8]), c910 = __fsub_rn(g[9], g[10]),
                c1112 = __fsub_rn(g[11], g[12]), c1314 = __fsub_rn(g[13], g[14]);
    const float ux = __fsub_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fsub_rn(g[1], g[2]), c78), c910), c1112), c1314);
    const float uy = __fadd_rn(__fsub_rn(__fadd_rn(__fadd_rn(__fsub_rn(g[3], g[4]), c78), c910), c1112), c1314);
    const float uz = __fadd_rn(__fadd_rn(__fsub_rn(__fadd_rn(__fsub_rn(g[5], g[6]), c78), c910), c1112), c1314);
    const float uu = __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmul_rn(ux, ux)));
    const float base = __fmaf_rn(-1.5f, uu, drho);
    const float om1 = __fsub_rn(1.f, omega);
    // per-class constants (uniform over the box)
    const float wo_f = __fmul_rn(omega, 1.f / 9.f), wo_c = __fmul_rn(omega, 1.f / 72.f);
    const float s_f = __fmul_rn(wo_f, base), s_c = __fmul_rn(wo_c, base);
    o[0] = __fmaf_rn(om1, g[0], __fmul_rn(__fmul_rn(omega, 2.f / 9.f), base));
    // pair (A, A+1): velocity e_A with e.u = EU and e.F = FE, class constants WO
    // (omega W), SB (omega W base) and W
#define LBP_PAIR(A, W, WO, SB, EU, FE)                                                     \
    {                                                                                      \
        const float eu = (EU);                                                             \
        const float S = __fmaf_rn(__fmul_rn(4.5f, (WO)), __fmul_rn(eu, eu), (SB));         \
        const float X = __fmaf_rn(__fmul_rn(3.f, (WO)), eu, __fmul_rn(3.f * (W), (FE)));   \
        o[A] = __fmaf_rn(om1, g[A], __fadd_rn(S, X));                                      \
        o[A + 1] = __fmaf_rn(om1, g[A + 1], __fsub_rn(S, X));                              \
    }
    LBP_PAIR(1, 1.f / 9.f, wo_f, s_f, ux, F0)
    LBP_PAIR(3, 1.f / 9.f, wo_f, s_f, uy, F1)
    LBP_PAIR(5, 1.f / 9.f, wo_f, s_f, uz, F2)
    LBP_PAIR(7, 1.f / 72.f, wo_c, s_c, __fadd_rn(__fadd_rn(ux, uy), uz), __fadd_rn(__fadd_rn(F0, F1), F2))
    LBP_PAIR(9, 1.f / 72.f, wo_c, s_c, __fsub_rn(__fadd_rn(ux, uy), uz), __fsub_rn(__fadd_rn(F0, F1), F2))
    LBP_PAIR(11, 1.f / 72.f, wo_c, s_c, __fadd_rn(__fsub_rn(ux, uy), uz), __fadd_rn(__fsub_rn(F0, F1), F2))
    LBP_PAIR(13, 1.f / 72.f, wo_c, s_c, __fadd_rn(__fsub_rn(uy, ux), uz), __fadd_rn(__fsub_rn(F1, F0), F2))
#undef LBP_PAIR
}

// The same collision on the scaled variables h_a = g_a F16_SCALE / w_a of the
// FP16 storage (in and out).  The moments take the weights back, per class:
//     rho~ - 1 = (2/9 h_0 + 1/9 sum_faces h + 1/72 sum_corners h) / F16_SCALE,
//     u = (1/9 sum_faces e h + 1/72 sum_corners e h) / F16_SCALE;
// in the outputs the weights cancel against the scale:
//     h'_0 = (1 - omega) h_0 + F16_SCALE omega base,
//     h'_A, h'_{A+1} = (1 - omega) h + S' +- X',
//     S' = F16_SCALE omega (base + 9/2 (e.u)^2),  X' = 3 F16_SCALE (omega e.u + e.F),
// the same for every velocity class.  Every operation is rounded explicitly, so
// every FP16 lattice kernel gives the same bits.
__device__ __forceinline__ void collide_values_scaled(const float h[Q], float omega, float F0, float F1,
                                                      float F2, float o[Q]) {
    constexpr float kr = (2.f / 9.f) / F16_SCALE, kf = (1.f / 9.f) / F16_SCALE, kc = (1.f / 72.f) / F16_SCALE;
    const float sf = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(h[1], h[2]), h[3]), h[4]), h[5]), h[6]);
    float sc = h[7];
#pragma unroll
    for (int a = 8; a < Q; ++a) sc = __fadd_rn(sc, h[a]);
    const float drho = __fmaf_rn(kc, sc, __fmaf_rn(kf, sf, __fmul_rn(kr, h[0])));
    const float c78 = __fsub_rn(h[7], h[8]), c910 = __fsub_rn(h[9], h[10]),
                c1112 = __fsub_rn(h[11], h[12]), c1314 = __fsub_rn(h[13], h[14]);
    const float a78 = __fadd_rn(c78, c910), b78 = __fsub_rn(c78, c910);
    const float ux = __fmaf_rn(kc, __fsub_rn(__fadd_rn(a78, c1112), c1314), __fmul_rn(kf, __fsub_rn(h[1], h[2])));
    const float uy = __fmaf_rn(kc, __fadd_rn(__fsub_rn(a78, c1112), c1314), __fmul_rn(kf, __fsub_rn(h[3], h[4])));
    const float uz = __fmaf_rn(kc, __fadd_rn(__fadd_rn(b78, c1112), c1314), __fmul_rn(kf, __fsub_rn(h[5], h[6])));
    const float uu = __fmaf_rn(uz, uz, __fmaf_rn(uy, uy, __fmul_rn(ux, ux)));
    const float base = __fmaf_rn(-1.5f, uu, drho);
    const float om1 = __fsub_rn(1.f, omega);
    const float so = __fmul_rn(F16_SCALE, omega);   // F16_SCALE omega
    const float sb = __fmul_rn(so, base);
    const float s45 = __fmul_rn(4.5f, so), s3 = __fmul_rn(3.f, so);
    o[0] = __fmaf_rn(om1, h[0], sb);
#define LBP_PAIR_S(A, EU, FE)                                                              \
    {                                                                                      \
        const float eu = (EU);                                                             \
        const float S = __fmaf_rn(s45, __fmul_rn(eu, eu), sb);                             \
        const float X = __fmaf_rn(s3, eu, __fmul_rn(3.f * F16_SCALE, (FE)));               \
        o[A] = __fmaf_rn(om1, h[A], __fadd_rn(S, X));                                      \
        o[A + 1] = __fmaf_rn(om1, h[A + 1], __fsub_rn(S, X));                              \
    }
    LBP_PAIR_S(1, ux, F0)
    LBP_PAIR_S(3, uy, F1)
    LBP_PAIR_S(5, uz, F2)
    LBP_PAIR_S(7, __fadd_rn(__fadd_rn(ux, uy), uz), __fadd_rn(__fadd_rn(F0, F1), F2))
    LBP_PAIR_S(9, __fsub_rn(__fadd_rn(ux, uy), uz), __fsub_rn(__fadd_rn(F0, F1), F2))
    LBP_PAIR_S(11, __fadd_rn(__fsub_rn(ux, uy), uz), __fadd_rn(__fsub_rn(F0, F1), F2))
    LBP_PAIR_S(13, __fadd_rn(__fsub_rn(uy, ux), uz), __fadd_rn(__fsub_rn(F1, F0), F2))
#undef LBP_PAIR_S
}

// The collision of the lattice kernels on their collision-space values (cload).
template <typename St>
__device__ __forceinline__ void collide_st(const float g[Q], float omega, float F0, float F1, float F2,
                                           float o[Q]) {
    if constexpr (St::SCALED)
        collide_values_scaled(g, omega, F0, F1, F2, o);
    else
        collide_values(g, omega, F0, F1, F2, o);
}

// Programmatic dependent launch.  A step's lattice pass is launched as the
// programmatic dependent of the step's particle kernel: the particle kernel
// lets it start early, and the lattice kernel issues its population loads
// (which do not depend on the particle kernel) before it waits for the
// particle kernel to complete and its writes (force records, overflow
// accumulator) to be visible.  Both are no-ops for ordinary launches.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// The float nearest (within one unit in the last place) to a 64-bit integer,
// from its two 32-bit halves: the direct 64-bit conversion runs on the FP64
// pipe, which is narrow on this GPU.  Every lattice kernel converts its
// fixed-point force sums with this one function.
__device__ __forceinline__ float fix_to_float(long long a) {
    const unsigned long long m = a < 0 ? 0ull - (unsigned long long)a : (unsigned long long)a;
    const float f = __fmaf_rn((float)(unsigned)(m >> 32), 4294967296.f, (float)(unsigned)m);
    return a < 0 ? -f : f;
}

// Reaction forces are summed per node in 64-bit fixed point so that the sum
// is exact and independent of the order in which particles add to it.
constexpr double FIX_SCALE = 72057594037927936.0;  // 2^56
constexpr double FIX_LIMIT = 32.0;                 // |F_H| < 2^5 per particle

// Per-segment force records.  Every 128-node segment of an x-row (the block
// of the stream-collide kernel) owns a 256-byte record: a count and up to
// REC_SLOTS (x, fixed-point force share) entries appended by the particle
// kernel.  The stream-collide kernel loads its record together with the
// populations and adds the force term in registers.  Entries beyond the
// capacity go to a dense per-node accumulator instead (see the kernels).
constexpr int SEG = 128;                 // nodes per segment (stream-collide block)
constexpr int REC_SLOTS = 8;
constexpr int REC_WORDS = 32;            // 8-byte words per record (256 bytes)
// layout (8-byte words): [0] count | pad, [1..4] x of slots 0..7 (two int32
// per word), [5 + 3 s + k] fixed-point share k of slot s.
constexpr int REC_X0 = 1;
constexpr int REC_F0 = 5;

// error bits in Sim::d_err
constexpr int ERR_NAN = 1;
constexpr int ERR_RANGE = 2;
constexpr int ERR_TIMEOUT = 4;  // a bounded wait on an mbarrier ran out
constexpr int ERR_LATTICE = 8;  // a collided population became non-finite
constexpr float VACF_RING_SCALE = 4096.f;  // the fp16 ring holds hi/lo of 4096 V; |V| < 16 fits

// True when the collided rest population of a node is not finite.  Every
// population of the node enters it through rho~ - 1 and u.u (collide_values),
// so a NaN or an infinity anywhere among the node's pulled values, or an
// overflow of u.u, shows here: one comparison per node.
__device__ __forceinline__ bool nonfinite_node(const float o[Q]) { return !(fabsf(o[0]) <= 3.4028234663852886e38f); }

// ------------------------------------------------------------------ Philox
// Philox-4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 64x64->128 multiplications with the published multipliers; the key is
// bumped by the published Weyl constants between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0,
                                              unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += W0;
            k1 += W1;
        }
        const unsigned long long lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
        const unsigned long long lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
        const unsigned long long n0 = hi1 ^ c[1] ^ k0;
        const unsigned long long n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

// ------------------------------------------------------------ replicas
// A handle holds one or more independent periodic boxes ("replicas", the
// batched ensemble).  Their populations are concatenated node-wise in the same
// 15 planes; every kernel gets the replica table by value (a kernel parameter,
// so the per-block lookup reads the constant bank, not global memory).
// Division by a divisor fixed per box, for numerators below 2^31, by one
// multiplication (Granlund & Montgomery, PLDI 1994, Theorem 4.2 with N = 31):
// with l = ceil(log2 d) and m = ceil(2^(31 + l) / d) (m < 2^32),
// floor(n / d) = floor(n m / 2^(31 + l)) for 0 <= n < 2^31.
struct Divisor {
    unsigned m;
    int l;
};
__host__ __device__ __forceinline__ unsigned divide(unsigned n, Divisor d) {
    return (unsigned)(((unsigned long long)n * d.m) >> (31 + d.l));
}
inline Divisor make_divisor(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long p = 1ull << (31 + l);
    return Divisor{(unsigned)((p + d - 1) / d), l};
}

struct Rep {
    int nx, ny, nz, nchunks;  // box and SEG-node segments per row
    long long node_off;       // first global node of the box
    long long seg_off;        // first global force-record segment
    float omega;              // 1 / tau
    float gx, gy, gz;         // uniform body force density on every node of the box (Eq. 18)
    int pad;                  // rows per item of the staged lattice kernel (set per launch)
    Divisor dchunks, dny;     // division by nchunks and by ny (row -> z) in the lattice kernels
};

constexpr int MAX_BATCH = 256;

// default bound of a device-side wait on an mbarrier, in SM clock cycles
// (~0.5 s at 2 GHz)
constexpr long long DEFAULT_WAIT_CYCLES = 1ll << 30;

template <int MAXR>
struct RepTable {
    int nrep;
    unsigned item_off[MAXR + 1];  // first block of each box in the launch, and the total
    Rep rep[MAXR];
};

// replica of a block / of a global node: last r with off[r] <= v (uniform per block)
template <int MAXR>
__device__ __forceinline__ int find_block_rep(const RepTable<MAXR> &t, unsigned b) {
    if (MAXR == 1) return 0;
    int lo = 0, hi = t.nrep - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.item_off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int MAXR>
__device__ __forceinline__ int find_node_rep(const RepTable<MAXR> &t, long long node) {
    if (MAXR == 1) return 0;
    int lo = 0, hi = t.nrep - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.rep[mid].node_off <= node) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ adjoint tape
// What a recorded forward run keeps for its reverse sweep: a checkpoint of the
// populations and of the particle positions and velocities every C steps.
struct Tape {
    int64_t T = 0;           // recorded steps (0: no tape)
    int C = 0;               // steps between checkpoints
    int64_t step0 = 0;       // step index of the first recorded step
    int cur0 = 0;            // buffer parity at the first recorded step
    int np = 0;              // particles during the recording
    uint64_t edits = 0;      // the handle's edit count when the recording ended
    int64_t nck = 0;         // checkpoints
    char *ck_f = nullptr;    // [nck][15 P] populations (storage type)
    double *ck_p = nullptr;  // [nck][6][cap]: r then V, [3][cap] each
};

// --------------------------------------------------------------- handle
struct Sim {
    int nx = 0, ny = 0, nz = 0;  // box of replica 0
    int64_t N = 0;  // nodes of all replicas
    int nrep = 1;
    Rep reps[MAX_BATCH] = {};
    double taus[MAX_BATCH] = {};
    int64_t P = 0;  // plane stride (elements), N rounded up to 64
    double tau = 1.0;
    int precision = LBP_F32;
    int rows = 1;  // rows of SEG nodes per lattice-kernel block (1, 2 or 4)
    int variant = 0;  // lattice kernel: 0 one node per thread, 1 two nodes, 2 bulk-copy staged
    int dev = 0;
    int num_sms = 0;
    long long wait_cycles = DEFAULT_WAIT_CYCLES;  // bound of every device-side wait (SM cycles)
    int wait_probe = 0;  // 1: the staged kernel's waits run out on purpose (tests of the error path)

    cudaStream_t user = nullptr;  // caller's stream
    cudaStream_t s0 = nullptr;    // library main stream (non-blocking)
    cudaStream_t s1 = nullptr;    // library side stream (particles, VACF)
    cudaEvent_t ev_in = nullptr, ev_fork = nullptr, ev_join = nullptr, ev_out = nullptr;

    void *f[2] = {nullptr, nullptr};   // deviation populations, 15 planes of P (storage type)
    int cur = 0;                       // f[cur] holds fhat^n
    int64_t step = 0;                  // host mirror of the step index
    long long *d_step = nullptr;       // device step index (Philox counter)
    int *d_err = nullptr;

    // particles, FP64 structure of arrays, 3 planes of cap for vectors
    int np = 0, cap = 0;
    double *r = nullptr, *v = nullptr, *fh = nullptr, *fr = nullptr, *fext = nullptr;
    double *mass = nullptr, *inv_mass = nullptr, *gamma = nullptr, *radius = nullptr, *sig = nullptr;
    int *prep = nullptr;  // replica of each particle
    unsigned char *pinned = nullptr;
    double kT = 0.0;
    unsigned long long seed = 0;
    int mode = LBP_STOKESLET;
    int exclude_inside = 0;
    double sqrt3 = 0.0;

    // force records and their overflow: a fixed-point accumulator per node that
    // the stream-collide block of an overflowed segment reads and clears
    unsigned long long *fq = nullptr;  // [3][N], allocated with the first particle
    unsigned long long *rec[2] = {nullptr, nullptr};  // [segments][REC_WORDS], by step parity
    long long nseg = 0;                                // segments of all replicas

    // VACF
    int vacf_lag = -1;
    int vacf_pp = 0;              // 1: sums per particle ([np][K + 1])
    int vacf_cap = 0;             // ring length in samples
    float *ring = nullptr;        // per-particle VACF: FP32 [vacf_cap][3 n_p]
    // ensemble VACF and MSD: fp16 hi/lo of 4096 V, [vacf_cap + dup rows][2][ring_ld]
    void *ring16 = nullptr;
    int ring_ld = 0;
    alignas(64) unsigned char tmaps[2][128];  // TMA tensor maps of ring16 (window, new samples)
    long long *d_vacf = nullptr;  // [0] t0 step, [1] samples correlated, [2] samples written,
                                  // [3] block counter of the reduce kernel
    long long vacf_done_host = 0; // host mirror of d_vacf[1]
    long long vacf_t0 = 0;        // step index of sample 0
    double *vacf_sum = nullptr;   // [K + 1]
    long long *vacf_cnt = nullptr;
    float *vacf_part = nullptr;   // [nchunks][64][K + 1] per-chunk G(t, k) of a block
    int vacf_nchunks = 0;
    // mean squared displacement (with the ensemble VACF, not per particle)
    double *corr_g = nullptr;     // [64][K + 1] G(t, k) of the block
    double *corr_h = nullptr;     // [64][K + 1] H(t, k)
    double *corr_w = nullptr;     // [64][K + 1] W(e, k)
    double *msd_state = nullptr;  // [2][K + 1] W(last sample, k), by parity
    double *msd_sum = nullptr;    // [K + 1]

    Tape tape;
    uint64_t edits = 0;  // state-changing calls other than steps (set_*, add)

    // conservation budget: momentum put into the unpinned particles by F_R and
    // F_ext since tracking began (FP64, [3]; null: not tracked)
    double *inj = nullptr;
    double *budget_part = nullptr;  // [budget_blocks][4]

    double *xbuf = nullptr;  // [9][cap]: f_ext, r, V of lbp_step_exchange (array-of-structures)
    // lbp_step_exchange with page-locked buffers: a block counter and a flag in
    // page-locked host memory that the particle kernel sets to the step index
    // once r and V are in the host buffers
    unsigned *d_xticket = nullptr;
    long long *h_xflag = nullptr;      // host address
    long long *h_xflag_dev = nullptr;  // its device view
    int xbuf_cap = 0;

    // scratch for host <-> device conversions
    double *stage = nullptr;
    size_t stage_bytes = 0;

    // graphs
    int use_graphs = 1;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // one step, by buffer parity
    // lbp_step_exchange with page-locked host or device buffers: the step whose
    // particle kernel does the I/O, by parity, with the buffer addresses, their
    // side and the particle count it was captured for
    cudaGraphExec_t xgraph[2] = {nullptr, nullptr};
    const void *xkey[2][3] = {};
    int xkey_np[2] = {0, 0};
    int xkey_dev[2] = {0, 0};
    int vacf_pending = 0;  // a VACF block runs on s1 (ev_join marks its end)

    // kernel timing
    int timing = 0;
    int ntimed = 0;
    static constexpr int MAX_TIMED = 4096;
    cudaEvent_t tev[2 * MAX_TIMED] = {};
    double timed_ms = 0.0;
    int64_t timed_launches = 0;
};

// ------------------------------------------------------------ launchers
// lbm_kernels.cu
cudaError_t prepare_lbm_kernels();
cudaError_t launch_stream_collide(Sim &s, const void *src, void *dst, cudaStream_t st);
// the lattice kernels with an explicit step counter, force records and rows per block
cudaError_t launch_stream_collide_cfg(Sim &s, const void *src, void *dst, long long *bump,
                                      int rows, int variant, cudaStream_t st);
cudaError_t launch_stream_collide_forced_cfg(Sim &s, const void *src, void *dst,
                                             const unsigned long long *rec_cur,
                                             unsigned long long *rec_prev, long long *bump, int rows,
                                             int variant, cudaStream_t st);
void default_shape(const Sim &s, int &rows, int &variant);  // before lbp_autotune
bool pair_kernel_ok(const Sim &s);  // 2-byte storage and every box with even nx
bool variant_ok(const Sim &s, int variant);
// pdl: launched right after the step's particle kernel on `st`, as its
// programmatic dependent
cudaError_t launch_stream_collide_forced(Sim &s, const void *src, void *dst, int parity,
                                         cudaStream_t st, bool pdl);
cudaError_t launch_fill_rest(Sim &s, void *dst, cudaStream_t st);
cudaError_t launch_from_f64(Sim &s, const double *f, void *dst, cudaStream_t st);
cudaError_t launch_to_f64(Sim &s, const void *src, double *f, cudaStream_t st);
cudaError_t launch_set_equilibrium(Sim &s, const double *rho, const double *u, void *dst,
                                   cudaStream_t st);
cudaError_t launch_fields(Sim &s, const void *src, double *rho, double *u, double *p,
                          cudaStream_t st);
int budget_blocks(const Sim &s);
cudaError_t launch_budget(Sim &s, const void *src, double *out, cudaStream_t st);  // [budget_blocks][4]
// particle_kernels.cu
// the I/O of one lbp_step_exchange step, done by the particle kernel itself
// ([n][3] FP64: device buffers, or the device views of page-locked host
// buffers; null: none); `signal`: raise the completion flag for a host
// waiting on page-locked buffers
struct ParticleIO {
    const double *fext_in;
    double *r_out, *v_out;
    bool signal;
};
cudaError_t launch_particles(Sim &s, const void *src, int parity, cudaStream_t st, const ParticleIO *io = nullptr);
bool particles_fit_per_corner(const Sim &s);  // the fit of Eq. 8 one lane per corner (few particles)
cudaError_t launch_aos_to_soa(const double *aos, double *soa, int n, int ld, int offset,
                              cudaStream_t st);
cudaError_t launch_soa_to_aos(const double *soa, double *aos, int n, int ld, cudaStream_t st);
cudaError_t launch_cells(Sim &s, int *base, double *frac, cudaStream_t st);
cudaError_t launch_philox(const unsigned long long *ctr, const unsigned long long *key,
                          unsigned long long *out, int64_t n, cudaStream_t st);
// lbm_staged.cu
template <typename St, int MAXR, bool FORCED>
cudaError_t launch_staged_t(const Planes<St> &pl, const RepTable<MAXR> &rt, const unsigned long long *rec_cur,
                            unsigned long long *rec_prev, unsigned long long *fq, long long Ntot, long long *bump,
                            int *err, long long wait_cycles, int probe, int num_sms, cudaStream_t st,
                            bool pdl = false);
bool staged_kernel_ok(const Sim &s);  // every box: nx a multiple of 16 bytes of storage, nx <= STAGED_NODES
int staged_rows(int nx, int ny);      // rows per item of the staged kernel
constexpr int STAGED_NODES = 512;     // nodes per item (whole rows) of the staged kernel
constexpr int STAGED_RECS = 16;       // force records per item of the staged kernel
constexpr int STAGED_THREADS = 256;
// adjoint_kernels.cu
cudaError_t launch_adj_particles(Sim &s, const void *g, const float *lam, const double *r,
                                 const double *v, long long step, const double *gv,
                                 const double *gr, double *lam_v, double *lam_r, double *acc,
                                 int parity, float *ug, cudaStream_t st);
cudaError_t launch_adj_lattice(Sim &s, const void *g, const float *lam, float *lam_out, int parity,
                               double *acc_omega, cudaStream_t st);
int adj_lattice_blocks(const Sim &s);
int adj_lattice_first_block(const Sim &s, int replica);  // first block of a box in the adjoint lattice launch
cudaError_t launch_f32_to_f64(Sim &s, const float *src, double *dst, cudaStream_t st);
// vacf_kernels.cu
int vacf_block_samples();
cudaError_t prepare_vacf_kernels();  // opt-in shared memory of the tensor-core correlator
int vacf_chunk_components();
int vacf_ring_dup_rows();                  // rows of ring16 kept twice (its first rows again after cap)
cudaError_t encode_vacf_tensor_maps(Sim &s);
cudaError_t launch_vacf_block(Sim &s, bool flush, cudaStream_t st);

}  // namespace lbp
