// lbm_kernels.cu -- D3Q15 lattice kernels of liblbp (sm_103a).
//
// Storage: 15 planes (structure of arrays, x fastest), plane stride P >= N,
// holding the deviation g_a = fhat_a - w_a of the post-collision populations
// from the rest state, as FP32, BF16 or scaled FP16 (the Store* types of
// lbp_internal.cuh); every kernel is a template on the storage type.  With sum_a w_a = 1 and sum_a w_a e_a = 0 the moments
// of Eqs. 12-13 are rho~ - 1 = sum_a g_a and u = sum_a e_a g_a, and the
// collision of Eqs. 15, 17 and 19 becomes, exactly,
//     g'_a = g_a + (geq_a - g_a)/tau,
//     geq_a = w_a [(rho~ - 1) + 3 e_a.u + 9/2 (e_a.u)^2 - 3/2 u.u],
// so FP32 arithmetic acts on the small deviations instead of on O(0.1)
// populations.
#include <cuda_runtime.h>

#include <type_traits>

#include <cstring>

#include "lbp_internal.cuh"

namespace lbp {

// ---------------------------------------------------------------------------
// Fused pull-stream + moments + BGK collision (Eqs. 20, 12, 13, 15, 17, 19).
//
// One thread per node and one block per SEG-node segment of an x-row: a full
// grid, not a persistent loop, so the hardware block scheduler keeps the
// blocks in flight on a narrow window of consecutive rows (the 15 read and 15
// write streams stay local in DRAM) and balances the tail.  The 15 loads of a
// node are independent, so every thread keeps 60 bytes in flight.  Address
// arithmetic is 32-bit offsets from per-population plane pointers passed as
// kernel parameters, and the collision (collide_values) is written per
// opposite pair (a, a+1), e_{a+1} = -e_a, with 1/tau folded into per-class
// constants: eight operations a pair.  The FP32 kernel stays bound by DRAM
// bandwidth (measured on GB300 at 256^3: within 2% of a plain copy); the
// 2-byte kernels, which move half the bytes, are bound by instruction issue.
// ---------------------------------------------------------------------------
template <typename St>
__device__ __forceinline__ void collide_store(const float g[Q], const Planes<St> &pl, int d,
                                              float omega, float F0, float F1, float F2, bool &bad) {
    float o[Q];
    collide_st<St>(g, omega, F0, F1, F2, o);
    bad |= nonfinite_node(o);
#pragma unroll
    for (int a = 0; a < Q; ++a) St::cstore(pl.d[a] + d, a, o[a]);
}

// Index arithmetic shared by both variants: node d of (x, row) and the
// offsets of the pull sources x - e, y - e, z - e (index e + 1), periodic.
struct NodeIdx {
    int d;
    int ox[3], oy[3], oz[3];
};

template <bool MUL_DIV = true>
__device__ __forceinline__ NodeIdx node_index(int x, unsigned row, int nx, int ny, int nz, Divisor dny) {
    NodeIdx n;
    const int z = MUL_DIV ? (int)divide(row, dny) : (int)(row / (unsigned)ny);
    const int y = (int)(row - (unsigned)z * ny);
    const int slab = nx * ny;
    n.d = (int)row * nx + x;
    n.ox[0] = x == nx - 1 ? 1 - nx : 1;
    n.ox[1] = 0;
    n.ox[2] = x == 0 ? nx - 1 : -1;
    n.oy[0] = y == ny - 1 ? (1 - ny) * nx : nx;
    n.oy[1] = 0;
    n.oy[2] = y == 0 ? (ny - 1) * nx : -nx;
    n.oz[0] = z == nz - 1 ? (1 - nz) * slab : slab;
    n.oz[1] = 0;
    n.oz[2] = z == 0 ? (nz - 1) * slab : -slab;
    return n;
}

// Each block serves R rows (consecutive in y) of one SEG-node x-segment of one
// replica box: a thread issues the 15 R loads of its R nodes before any
// arithmetic.  R = 2 for the 2-byte storage types, whose 15 loads per node
// alone keep too few bytes in flight; R = 1 for FP32.  The block finds its box
// in the replica table (a kernel parameter; one entry for a single box).
// Two rows per block are held to 64 registers (eight blocks of 128 threads per
// SM): the batched ensemble's short rows need the occupancy (0.793 ms per
// launch there, against 0.833 ms at the compiler's 72 registers).
template <int BX, typename St, int R, int MAXR>
__global__ void __launch_bounds__(BX, R == 2 ? 8 : 1) k_stream_collide(Planes<St> pl, const RepTable<MAXR> rt,
                                                       long long *bump, int *err) {
    const int r = find_block_rep(rt, blockIdx.x);
    const Rep &rp = rt.rep[r];
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz, nchunks = rp.nchunks;
    const unsigned nrows = (unsigned)ny * (unsigned)nz;
    const unsigned item = blockIdx.x - rt.item_off[r];
    const unsigned grp = divide(item, rp.dchunks);
    const int chunk = (int)(item - grp * (unsigned)nchunks);
    const int x = chunk * BX + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *bump += 1;
    if (x >= nx) return;
    const int base = (int)rp.node_off;
    NodeIdx n[R];
    float g[R][Q];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
        n[h] = node_index(x, row, nx, ny, nz, rp.dny);
        n[h].d += base;
#pragma unroll
        for (int a = 0; a < Q; ++a)
            g[h][a] = St::cload(pl.s[a] + (n[h].d + n[h].ox[ex(a) + 1] + n[h].oy[ey(a) + 1] +
                                          n[h].oz[ez(a) + 1]), a);
    }
    bool bad = false;
#pragma unroll
    for (int h = 0; h < R; ++h)
        if (grp * R + h < nrows) collide_store<St>(g[h], pl, n[h].d, rp.omega, rp.gx, rp.gy, rp.gz, bad);
    if (bad) atomicOr(err, ERR_LATTICE);
}

// Sum, exactly in 64-bit fixed point, the record entries whose x is this
// lane's x; rw is this lane's word of the 256-byte record (see lbp_internal.cuh).
__device__ __forceinline__ void record_sum(unsigned long long rw, int cnt, int x, long long &a0,
                                           long long &a1, long long &a2) {
    const int used = cnt < REC_SLOTS ? cnt : REC_SLOTS;
    for (int sl = 0; sl < used; ++sl) {
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
}

// ---------------------------------------------------------------------------
// The same pass with the body force of Eqs. 18-19 (particles present).
// Every SEG-node segment of a row owns one force record (lbp_internal.cuh)
// filled by this step's particle kernel.  Every warp loads the 256-byte
// record of each of its rows -- one 8-byte word per lane -- together with its
// population loads (the address depends only on the block index, so no load
// waits on another), then each lane sums, exactly in 64-bit fixed point, the
// entries whose x is its own and adds 3 w_a F.e_a to its post-collision
// populations.  If a record overflowed (count > REC_SLOTS) the particle kernel
// put the shares that did not fit into the dense per-node accumulator: the
// lanes of that (rare) segment also read and clear their node's accumulator
// and add it to the record sum -- still an exact integer sum of all the node's
// shares.  The block clears the counts of its rows' records of the previous
// step, which the next step's particle kernel refills.
// ---------------------------------------------------------------------------
template <int BX, typename St, int R, int MAXR>
__global__ void __launch_bounds__(BX, R == 2 ? 8 : 1) k_stream_collide_forced(
    Planes<St> pl, const RepTable<MAXR> rt, const unsigned long long *__restrict__ rec_cur,
    unsigned long long *rec_prev, unsigned long long *fq, long long Ntot, long long *bump, int *err) {
    static_assert(BX == SEG, "one block per force-record segment");
    const int r = find_block_rep(rt, blockIdx.x);
    const Rep &rp = rt.rep[r];
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz, nchunks = rp.nchunks;
    const unsigned nrows = (unsigned)ny * (unsigned)nz;
    const int lane = threadIdx.x & 31;
    const unsigned item = blockIdx.x - rt.item_off[r];
    const unsigned grp = divide(item, rp.dchunks);
    const int chunk = (int)(item - grp * (unsigned)nchunks);
    const size_t seg0 = (size_t)rp.seg_off;
    // the previous step's records (this step's particle kernel writes the others)
    if (threadIdx.x < R && grp * R + threadIdx.x < nrows)
        rec_prev[(seg0 + (size_t)(grp * R + threadIdx.x) * nchunks + chunk) * REC_WORDS] = 0ull;
    const int xw = chunk * BX + (threadIdx.x & ~31);
    if (xw >= nx) return;  // whole warp past the end of the row
    const int x0 = xw + lane;
    const bool act = x0 < nx;
    const int x = act ? x0 : nx - 1;
    const int base = (int)rp.node_off;
    NodeIdx n[R];
    float g[R][Q];
    unsigned long long rw[R];
    bool bad = false;
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
        n[h] = node_index(x, row, nx, ny, nz, rp.dny);
        n[h].d += base;
#pragma unroll
        for (int a = 0; a < Q; ++a)
            g[h][a] = St::cload(pl.s[a] + (n[h].d + n[h].ox[ex(a) + 1] + n[h].oy[ey(a) + 1] +
                                          n[h].oz[ez(a) + 1]), a);
    }
    // the loads above do not depend on this step's particle kernel; what follows does
    // (a no-op unless launched as its programmatic dependent)
    grid_dependency_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) *bump += 1;
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
        rw[h] = __ldg(rec_cur + (seg0 + (size_t)row * nchunks + chunk) * REC_WORDS + lane);
    }
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const int cnt = (int)(unsigned)(__shfl_sync(0xffffffffu, rw[h], 0) & 0xffffffffull);
        float F0 = rp.gx, F1 = rp.gy, F2 = rp.gz;  // uniform body force of the box
        if (cnt > 0 && grp * R + h < nrows) {
            long long a0 = 0, a1 = 0, a2 = 0;
            record_sum(rw[h], cnt, x, a0, a1, a2);
            if (cnt > REC_SLOTS && act) {
                const int d = n[h].d;
                a0 += (long long)fq[d];
                a1 += (long long)fq[Ntot + d];
                a2 += (long long)fq[2 * Ntot + d];
                fq[d] = 0ull;
                fq[Ntot + d] = 0ull;
                fq[2 * Ntot + d] = 0ull;
            }
            const float inv = 1.3877787807814457e-17f;  // 2^-56
            F0 = __fmaf_rn(inv, fix_to_float(a0), F0);
            F1 = __fmaf_rn(inv, fix_to_float(a1), F1);
            F2 = __fmaf_rn(inv, fix_to_float(a2), F2);
        }
        if (act && grp * R + h < nrows) collide_store<St>(g[h], pl, n[h].d, rp.omega, F0, F1, F2, bad);
    }
    if (bad) atomicOr(err, ERR_LATTICE);
}

// ---------------------------------------------------------------------------
// Paired-node variant for the 2-byte storage types (every box with even nx).
// A thread owns two neighbouring nodes (x, x + 1), x even, and moves each
// plane's pair of 2-byte deviations with one 4-byte load and one 4-byte store;
// a 64-thread block covers one SEG-node segment of R rows.  The pull streaming
// in x is done in registers: for e_x = +1 the pair (x - 1, x) is the high
// half of the left lane's pair and the low half of the lane's own, for
// e_x = -1 the pair (x + 1, x + 2) is the high half of its own and the low
// half of the right lane's (warp shuffles); the lanes at a warp's or a row's
// end load the neighbouring pair themselves (periodic in x).  This halves the
// load and store instructions per node and leaves the conversions packed, so
// the kernel is no longer bound by instruction issue.  Per node the
// arithmetic is that of collide_st: results equal the one-node kernels'
// bit for bit.
// ---------------------------------------------------------------------------
template <typename St>
__device__ __forceinline__ void unpack2(unsigned v, int a, float &lo, float &hi);
template <>
__device__ __forceinline__ void unpack2<StoreBF16>(unsigned v, int, float &lo, float &hi) {
    lo = __uint_as_float(v << 16);
    hi = __uint_as_float(v & 0xffff0000u);
}
// FP16: the collision-space values h (StoreF16::cload), not scaled
template <>
__device__ __forceinline__ void unpack2<StoreF16>(unsigned v, int, float &lo, float &hi) {
    lo = __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
    hi = __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}
template <typename St>
__device__ __forceinline__ unsigned pack2(float lo, float hi, int a);
template <>
__device__ __forceinline__ unsigned pack2<StoreBF16>(float lo, float hi, int) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&p);
}
template <>
__device__ __forceinline__ unsigned pack2<StoreF16>(float lo, float hi, int) {
    const __half2 p = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&p);
}

constexpr int PAIR_BX = SEG / 2;  // threads per block of the paired kernel

// True if either 2-byte value of a packed pair is a NaN or an infinity (its
// exponent field all ones: 0x7f80 for bfloat16, 0x7c00 for binary16).
template <typename St>
__device__ __forceinline__ bool packed_nonfinite(unsigned v);
template <>
__device__ __forceinline__ bool packed_nonfinite<StoreBF16>(unsigned v) {
    return (v & 0x7f80u) == 0x7f80u || (v & 0x7f800000u) == 0x7f800000u;
}
template <>
__device__ __forceinline__ bool packed_nonfinite<StoreF16>(unsigned v) {
    return (v & 0x7c00u) == 0x7c00u || (v & 0x7c000000u) == 0x7c000000u;
}

template <typename St, int R, int MAXR, bool FORCED>
__global__ void __launch_bounds__(PAIR_BX) k_stream_collide_pair(
    Planes<St> pl, const RepTable<MAXR> rt, const unsigned long long *__restrict__ rec_cur,
    unsigned long long *rec_prev, unsigned long long *fq, long long Ntot, long long *bump, int *err) {
    const int r = find_block_rep(rt, blockIdx.x);
    const Rep &rp = rt.rep[r];
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz, nchunks = rp.nchunks;
    const unsigned nrows = (unsigned)ny * (unsigned)nz;
    const int lane = threadIdx.x & 31;
    const unsigned item = blockIdx.x - rt.item_off[r];
    const unsigned grp = divide(item, rp.dchunks);
    const int chunk = (int)(item - grp * (unsigned)nchunks);
    const size_t seg0 = (size_t)rp.seg_off;
    if (FORCED && threadIdx.x < R && grp * R + threadIdx.x < nrows)
        rec_prev[(seg0 + (size_t)(grp * R + threadIdx.x) * nchunks + chunk) * REC_WORDS] = 0ull;
    if (!FORCED && blockIdx.x == 0 && threadIdx.x == 0) *bump += 1;
    const int xw = chunk * SEG + 2 * (threadIdx.x & ~31);  // first node of the warp
    if (xw >= nx) return;
    const int x0 = xw + 2 * lane;
    const bool act = x0 < nx;
    const int x = act ? x0 : nx - 2;       // even; inactive lanes read a valid pair
    const int xl = x == 0 ? nx - 2 : x - 2;  // left and right pairs, periodic
    const int xr = x + 2 == nx ? 0 : x + 2;
    const bool own_left = lane == 0;               // no left lane in the warp
    const bool own_right = lane == 31 || x0 + 2 >= nx;  // no (active) right lane
    const int base = (int)rp.node_off;
    float g[R][2][Q];
    unsigned long long rw[R];
    int drow[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
        const NodeIdx n = node_index(0, row, nx, ny, nz, rp.dny);
        drow[h] = base + n.d;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const int rb = drow[h] + n.oy[ey(a) + 1] + n.oz[ez(a) + 1];  // source row start
            const unsigned *src = reinterpret_cast<const unsigned *>(pl.s[a] + rb);
            const unsigned v = __ldg(src + (x >> 1));
            unsigned w = v;
            if (ex(a) > 0) {
                // pull from x - 1: (x - 1, x) = (hi of left pair, lo of own)
                unsigned left = __shfl_up_sync(0xffffffffu, v, 1);
                if (own_left) left = __ldg(src + (xl >> 1));
                w = __byte_perm(left, v, 0x5432);
            } else if (ex(a) < 0) {
                // pull from x + 1: (x + 1, x + 2) = (hi of own, lo of right pair)
                unsigned right = __shfl_down_sync(0xffffffffu, v, 1);
                if (own_right) right = __ldg(src + (xr >> 1));
                w = __byte_perm(v, right, 0x5432);
            }
            unpack2<St>(w, a, g[h][0][a], g[h][1][a]);
        }
    }
    if (FORCED) {
        grid_dependency_wait();  // the records come from this step's particle kernel
        if (blockIdx.x == 0 && threadIdx.x == 0) *bump += 1;
#pragma unroll
        for (int h = 0; h < R; ++h) {
            const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
            rw[h] = __ldg(rec_cur + (seg0 + (size_t)row * nchunks + chunk) * REC_WORDS + lane);
        }
    }
#pragma unroll
    for (int h = 0; h < R; ++h) {
        float F[2][3] = {{rp.gx, rp.gy, rp.gz}, {rp.gx, rp.gy, rp.gz}};
        if (FORCED) {
            const int cnt = (int)(unsigned)(__shfl_sync(0xffffffffu, rw[h], 0) & 0xffffffffull);
            if (cnt > 0 && grp * R + h < nrows) {
                long long s0[3] = {0, 0, 0}, s1[3] = {0, 0, 0};
                record_sum(rw[h], cnt, x, s0[0], s0[1], s0[2]);
                record_sum(rw[h], cnt, x + 1, s1[0], s1[1], s1[2]);
                if (cnt > REC_SLOTS && act) {
                    const int d = drow[h] + x;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        s0[k] += (long long)fq[k * Ntot + d];
                        s1[k] += (long long)fq[k * Ntot + d + 1];
                        fq[k * Ntot + d] = 0ull;
                        fq[k * Ntot + d + 1] = 0ull;
                    }
                }
                const float inv = 1.3877787807814457e-17f;  // 2^-56
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    F[0][k] = __fmaf_rn(inv, fix_to_float(s0[k]), F[0][k]);
                    F[1][k] = __fmaf_rn(inv, fix_to_float(s1[k]), F[1][k]);
                }
            }
        }
        if (act && grp * R + h < nrows) {
            float o0[Q], o1[Q];
            collide_st<St>(g[h][0], rp.omega, F[0][0], F[0][1], F[0][2], o0);
            collide_st<St>(g[h][1], rp.omega, F[1][0], F[1][1], F[1][2], o1);
            if (nonfinite_node(o0) || nonfinite_node(o1)) atomicOr(err, ERR_LATTICE);
#pragma unroll
            for (int a = 0; a < Q; ++a)
                reinterpret_cast<unsigned *>(pl.d[a] + drow[h])[x >> 1] = pack2<St>(o0[a], o1[a], a);
        }
    }
}

// Sum, exactly, the record entries whose x is one of x .. x + 3 (one pass
// over the slots for four nodes; the same integer sums as record_sum).
__device__ __forceinline__ void record_sum4(unsigned long long rw, int cnt, int x, long long s[4][3]) {
    const int used = cnt < REC_SLOTS ? cnt : REC_SLOTS;
    for (int sl = 0; sl < used; ++sl) {
        const unsigned long long xw2 = __shfl_sync(0xffffffffu, rw, REC_X0 + (sl >> 1));
        const int k = (int)(unsigned)(xw2 >> (32 * (sl & 1))) - x;
        const long long v0 = (long long)__shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl);
        const long long v1 = (long long)__shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl + 1);
        const long long v2 = (long long)__shfl_sync(0xffffffffu, rw, REC_F0 + 3 * sl + 2);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
            if (k == kk) {
                s[kk][0] += v0;
                s[kk][1] += v1;
                s[kk][2] += v2;
            }
    }
}

// ---------------------------------------------------------------------------
// Four-node variant for the 2-byte storage types (every box with nx a
// multiple of 4).  One warp per SEG-node row segment (and R rows): lane l owns
// the nodes x .. x + 3, x = segment start + 4 l, and moves each plane's four
// 2-byte deviations with one 8-byte load and one 8-byte store, so a warp
// touches the segment's 256 contiguous bytes per plane.  The pull in x is done
// in registers as in the paired kernel: for e_x = +1 the node left of x is the
// top element of the left lane's group, for e_x = -1 the node right of x + 3
// is the bottom element of the right lane's group (warp shuffles); the lanes
// at a warp's or a row's end load that one element themselves (periodic in
// x).  A thread keeps 15 R 8-byte loads in flight in 30 R registers, twice the
// bytes per register of the paired kernel, and collides the pairs (x, x + 1)
// and (x + 2, x + 3) in turn, packing the results over the pulled values.
// Per node the arithmetic is that of collide_st, and the force sums are
// the same exact integer sums: results equal the other kernels' bit for bit.
// ---------------------------------------------------------------------------
constexpr int QUAD_WARPS = 4;  // row segments (warps) per block
// With one row the kernel is bound by instruction issue and latency, so it is
// held to 80 registers for six blocks (24 warps) per SM: measured 4% (BF16)
// and 7% (FP16) faster at 256^3 than the compiler's 94 registers and five
// blocks, against 48 bytes of spills.  More rows keep more loads in flight
// and need the registers.

template <typename St>
__device__ __forceinline__ unsigned load_elem(const typename St::T *p) {
    return (unsigned)__ldg(reinterpret_cast<const unsigned short *>(p));
}

template <typename St, int R, int MAXR, bool FORCED>
__global__ void __launch_bounds__(32 * QUAD_WARPS, R == 1 ? 6 : 1) k_stream_collide_quad(
    Planes<St> pl, const RepTable<MAXR> rt, const unsigned long long *__restrict__ rec_cur,
    unsigned long long *rec_prev, unsigned long long *fq, long long Ntot, long long *bump, int *err) {
    if (!FORCED && blockIdx.x == 0 && threadIdx.x == 0) *bump += 1;
    const unsigned item = blockIdx.x * QUAD_WARPS + (threadIdx.x >> 5);
    if (item >= rt.item_off[MAXR == 1 ? 1 : rt.nrep]) return;  // whole warp past the last segment
    const int r = find_block_rep(rt, item);
    const Rep &rp = rt.rep[r];
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz, nchunks = rp.nchunks;
    const unsigned nrows = (unsigned)ny * (unsigned)nz;
    const int lane = threadIdx.x & 31;
    const unsigned it = item - rt.item_off[r];
    // the row segment by one multiplication (Divisor); the FP16 instantiation
    // keeps the hardware division, measured faster there (0.1798 vs 0.1861 ms
    // at 256^3), while BF16 gains (0.1740 -> 0.1707 ms)
    constexpr bool MUL_DIV = !std::is_same<St, StoreF16>::value;
    const unsigned grp = MUL_DIV ? divide(it, rp.dchunks) : it / (unsigned)nchunks;
    const int chunk = (int)(it - grp * (unsigned)nchunks);
    const size_t seg0 = (size_t)rp.seg_off;
    if (FORCED && lane < R && grp * R + lane < nrows)
        rec_prev[(seg0 + (size_t)(grp * R + lane) * nchunks + chunk) * REC_WORDS] = 0ull;
    const int x0 = chunk * SEG + 4 * lane;
    const bool act = x0 < nx;
    const int x = act ? x0 : nx - 4;         // inactive lanes read a valid group
    const int xl = x == 0 ? nx - 1 : x - 1;  // periodic neighbours of the group
    const int xr = x + 4 == nx ? 0 : x + 4;
    const bool own_left = lane == 0;                    // no left lane in the warp
    const bool own_right = lane == 31 || x0 + 4 >= nx;  // no (active) right lane
    const int base = (int)rp.node_off;
    uint2 p[R][Q];
    unsigned long long rw[R];
    int drow[R];
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
        const NodeIdx n = node_index<MUL_DIV>(0, row, nx, ny, nz, rp.dny);
        drow[h] = base + n.d;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const typename St::T *src = pl.s[a] + (drow[h] + n.oy[ey(a) + 1] + n.oz[ez(a) + 1]);
            const uint2 v = __ldg(reinterpret_cast<const uint2 *>(src + x));
            if (ex(a) > 0) {
                // pull from x - 1: (x - 1, x, x + 1, x + 2)
                const unsigned e = own_left ? load_elem<St>(src + xl) : 0u;
                unsigned left = __shfl_up_sync(0xffffffffu, v.y, 1);
                if (own_left) left = e << 16;
                p[h][a] = make_uint2(__byte_perm(left, v.x, 0x5432), __byte_perm(v.x, v.y, 0x5432));
            } else if (ex(a) < 0) {
                // pull from x + 1: (x + 1, x + 2, x + 3, x + 4)
                const unsigned e = own_right ? load_elem<St>(src + xr) : 0u;
                unsigned right = __shfl_down_sync(0xffffffffu, v.x, 1);
                if (own_right) right = e;
                p[h][a] = make_uint2(__byte_perm(v.x, v.y, 0x5432), __byte_perm(v.y, right, 0x5432));
            } else {
                p[h][a] = v;
            }
        }
    }
    if (FORCED) {
        grid_dependency_wait();  // the records come from this step's particle kernel
        if (blockIdx.x == 0 && threadIdx.x == 0) *bump += 1;
#pragma unroll
        for (int h = 0; h < R; ++h) {
            const unsigned row = grp * R + h < nrows ? grp * R + h : nrows - 1;
            rw[h] = __ldg(rec_cur + (seg0 + (size_t)row * nchunks + chunk) * REC_WORDS + lane);
        }
    }
#pragma unroll
    for (int h = 0; h < R; ++h) {
        const bool row_ok = grp * R + h < nrows;
        float F[4][3];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            F[k][0] = rp.gx;
            F[k][1] = rp.gy;
            F[k][2] = rp.gz;
        }
        // no force anywhere in this warp's row segment (no record entry, no body
        // force): the collision with literal zero forces, whose force terms the
        // compiler folds away -- the same operations on the same values as with
        // F = 0 passed in, so the results are the same bits
        bool unforced = rp.gx == 0.f && rp.gy == 0.f && rp.gz == 0.f;
        if (FORCED) {
            const int cnt = (int)(unsigned)(__shfl_sync(0xffffffffu, rw[h], 0) & 0xffffffffull);
            unforced = unforced && cnt == 0;
            if (cnt > 0 && row_ok) {
                long long sum[4][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                record_sum4(rw[h], cnt, x, sum);
                if (cnt > REC_SLOTS && act) {
                    const int d = drow[h] + x;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            sum[k][c] += (long long)fq[c * Ntot + d + k];
                            fq[c * Ntot + d + k] = 0ull;
                        }
                }
                const float inv = 1.3877787807814457e-17f;  // 2^-56
#pragma unroll
                for (int k = 0; k < 4; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) F[k][c] = __fmaf_rn(inv, fix_to_float(sum[k][c]), F[k][c]);
            }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float g0[Q], g1[Q], o0[Q], o1[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) unpack2<St>(j ? p[h][a].y : p[h][a].x, a, g0[a], g1[a]);
            if (unforced) {
                collide_st<St>(g0, rp.omega, 0.f, 0.f, 0.f, o0);
                collide_st<St>(g1, rp.omega, 0.f, 0.f, 0.f, o1);
            } else {
                collide_st<St>(g0, rp.omega, F[2 * j][0], F[2 * j][1], F[2 * j][2], o0);
                collide_st<St>(g1, rp.omega, F[2 * j + 1][0], F[2 * j + 1][1], F[2 * j + 1][2], o1);
            }
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const unsigned w = pack2<St>(o0[a], o1[a], a);
                if (j) p[h][a].y = w; else p[h][a].x = w;
            }
        }
        if (act && row_ok) {
            // the packed collided rest populations of the four nodes: a NaN or an
            // infinity (also one from the rounding to 2 bytes) has an all-ones exponent
            if (packed_nonfinite<St>(p[h][0].x) || packed_nonfinite<St>(p[h][0].y)) atomicOr(err, ERR_LATTICE);
#pragma unroll
            for (int a = 0; a < Q; ++a) *reinterpret_cast<uint2 *>(pl.d[a] + drow[h] + x) = p[h][a];
        }
    }
}

constexpr int SC_BX = SEG;

cudaError_t prepare_lbm_kernels() { return cudaSuccess; }

template <typename St>
static Planes<St> planes_of(const Sim &s, const void *src, void *dst) {
    Planes<St> pl;
    const typename St::T *a0 = static_cast<const typename St::T *>(src);
    typename St::T *b0 = static_cast<typename St::T *>(dst);
    for (int a = 0; a < Q; ++a) {
        pl.s[a] = a0 + (long long)a * s.P;
        pl.d[a] = b0 + (long long)a * s.P;
    }
    return pl;
}

// Run f(StoreX{}) for the handle's storage type.
template <typename F>
static cudaError_t by_storage(const Sim &s, F &&f) {
    switch (s.precision) {
        case LBP_BF16: return f(StoreBF16{});
        case LBP_F16: return f(StoreF16{});
        default: return f(StoreF32{});
    }
}

bool quad_kernel_ok(const Sim &s);

// The lattice kernel's shape before any lbp_autotune: the autotuner's pick on
// GB300 at 256^3 and for the 68-box ensemble -- one node per thread with two
// rows of SEG nodes per block for FP32 (0.302 ms against 0.315-0.322 with one
// row at 256^3; 0.769 against 0.957 ms for the ensemble), four nodes per
// thread with one row for the 2-byte types (0.172 ms against 0.245 ms for one
// node per thread with two rows) where every box's nx is a multiple of 4, else
// one node per thread with two rows.
void default_shape(const Sim &s, int &rows, int &variant) {
    if (s.precision != LBP_F32 && quad_kernel_ok(s)) {
        variant = 3;
        rows = 1;
    } else {
        variant = 0;
        rows = 2;
    }
}

template <typename F>
static cudaError_t by_rows(int R, F &&f) {
    switch (R) {
        case 2: return f(std::integral_constant<int, 2>{});
        case 4: return f(std::integral_constant<int, 4>{});
        default: return f(std::integral_constant<int, 1>{});
    }
}

// Replica table for a launch whose blocks cover R rows of SEG nodes.
template <int MAXR>
static RepTable<MAXR> rep_table(const Sim &s, int R) {
    RepTable<MAXR> t;
    memset(&t, 0, sizeof(t));
    t.nrep = s.nrep;
    unsigned off = 0;
    for (int r = 0; r < s.nrep; ++r) {
        t.rep[r] = s.reps[r];
        t.item_off[r] = off;
        const unsigned rows = (unsigned)s.reps[r].ny * (unsigned)s.reps[r].nz;
        off += (rows + R - 1) / R * (unsigned)s.reps[r].nchunks;
    }
    t.item_off[s.nrep] = off;
    return t;
}

// Run f(RepTable<1 or MAX_BATCH>) for a single box or a batch.
template <typename F>
static cudaError_t by_batch(const Sim &s, int R, F &&f) {
    if (s.nrep == 1) return f(rep_table<1>(s, R));
    return f(rep_table<MAX_BATCH>(s, R));
}

bool pair_kernel_ok(const Sim &s) {
    if (s.precision == LBP_F32) return false;
    for (int r = 0; r < s.nrep; ++r)
        if (s.reps[r].nx % 2) return false;
    return true;
}

bool quad_kernel_ok(const Sim &s) {
    if (s.precision == LBP_F32) return false;
    for (int r = 0; r < s.nrep; ++r)
        if (s.reps[r].nx % 4) return false;
    return true;
}

bool staged_kernel_ok(const Sim &s) {
    const int H = 16 / storage_bytes(s.precision);
    for (int r = 0; r < s.nrep; ++r)
        if (s.reps[r].nx % H || s.reps[r].nx > STAGED_NODES) return false;
    return true;
}

// Replica table of the staged kernel: items of whole rows (Rep::pad = rows per item).
template <int MAXR>
static RepTable<MAXR> rep_table_staged(const Sim &s) {
    RepTable<MAXR> t;
    memset(&t, 0, sizeof(t));
    t.nrep = s.nrep;
    unsigned off = 0;
    for (int r = 0; r < s.nrep; ++r) {
        t.rep[r] = s.reps[r];
        const int rows = staged_rows(s.reps[r].nx, s.reps[r].ny);
        t.rep[r].pad = rows;
        t.item_off[r] = off;
        off += (unsigned)s.reps[r].nz * (unsigned)((s.reps[r].ny + rows - 1) / rows);
    }
    t.item_off[s.nrep] = off;
    return t;
}

bool variant_ok(const Sim &s, int variant) {
    return variant == 0 || (variant == 1 && pair_kernel_ok(s)) || (variant == 2 && staged_kernel_ok(s)) ||
           (variant == 3 && quad_kernel_ok(s));
}

// Launch `kern` on `st`; with `pdl` as the programmatic dependent of the
// kernel launched before it on that stream (see grid_dependency_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                            bool pdl, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// variant 0: one node per thread; 1: two nodes per thread (2-byte storage,
// even nx); 2: bulk-copy staged persistent kernel (lbm_staged.cu); 3: four
// nodes per thread, one warp per row segment (2-byte storage, nx % 4 == 0).
// pdl: launched right after the step's particle kernel, as its programmatic
// dependent (forced passes only).
template <bool FORCED>
static cudaError_t launch_sc(Sim &s, const void *src, void *dst, const unsigned long long *rec_cur,
                             unsigned long long *rec_prev, long long *bump, int rows, int variant,
                             cudaStream_t st, bool pdl = false) {
    constexpr int BX = SC_BX;
    if (!variant_ok(s, variant)) variant = 0;
    if (variant == 2) {
        return by_storage(s, [&](auto tag) {
            using St = decltype(tag);
            if (s.nrep == 1)
                return launch_staged_t<St, 1, FORCED>(planes_of<St>(s, src, dst), rep_table_staged<1>(s), rec_cur,
                                                      rec_prev, s.fq, s.N, bump, s.d_err, s.wait_cycles, s.wait_probe,
                                                      s.num_sms, st, pdl);
            return launch_staged_t<St, MAX_BATCH, FORCED>(planes_of<St>(s, src, dst), rep_table_staged<MAX_BATCH>(s),
                                                          rec_cur, rec_prev, s.fq, s.N, bump, s.d_err,
                                                          s.wait_cycles, s.wait_probe, s.num_sms, st, pdl);
        });
    }
    const bool use_pair = variant == 1, use_quad = variant == 3;
    return by_storage(s, [&](auto tag) {
        using St = decltype(tag);
        return by_rows(rows, [&](auto rc) {
            constexpr int R = decltype(rc)::value;
            return by_batch(s, R, [&](const auto &rt) {
                constexpr int MAXR = sizeof(rt.rep) / sizeof(Rep);
                const unsigned grid = rt.item_off[rt.nrep];
                if constexpr (!std::is_same<St, StoreF32>::value) {
                    if (use_pair)
                        return launch_k(k_stream_collide_pair<St, R, MAXR, FORCED>, grid, PAIR_BX, 0, st, pdl,
                                        planes_of<St>(s, src, dst), rt, rec_cur, rec_prev, s.fq, s.N, bump, s.d_err);
                    if (use_quad)
                        return launch_k(k_stream_collide_quad<St, R, MAXR, FORCED>, (grid + QUAD_WARPS - 1) / QUAD_WARPS,
                                        32 * QUAD_WARPS, 0, st, pdl, planes_of<St>(s, src, dst), rt, rec_cur, rec_prev,
                                        s.fq, s.N, bump, s.d_err);
                }
                if constexpr (FORCED)
                    return launch_k(k_stream_collide_forced<BX, St, R, MAXR>, grid, BX, 0, st, pdl,
                                    planes_of<St>(s, src, dst), rt, rec_cur, rec_prev, s.fq, s.N, bump, s.d_err);
                else
                    k_stream_collide<BX, St, R, MAXR><<<grid, BX, 0, st>>>(planes_of<St>(s, src, dst), rt, bump,
                                                                           s.d_err);
                return cudaGetLastError();
            });
        });
    });
}

cudaError_t launch_stream_collide_cfg(Sim &s, const void *src, void *dst, long long *bump,
                                      int rows, int variant, cudaStream_t st) {
    return launch_sc<false>(s, src, dst, nullptr, nullptr, bump, rows, variant, st);
}

cudaError_t launch_stream_collide_forced_cfg(Sim &s, const void *src, void *dst,
                                             const unsigned long long *rec_cur,
                                             unsigned long long *rec_prev, long long *bump, int rows,
                                             int variant, cudaStream_t st) {
    return launch_sc<true>(s, src, dst, rec_cur, rec_prev, bump, rows, variant, st);
}

cudaError_t launch_stream_collide(Sim &s, const void *src, void *dst, cudaStream_t st) {
    return launch_stream_collide_cfg(s, src, dst, s.d_step, s.rows, s.variant, st);
}

cudaError_t launch_stream_collide_forced(Sim &s, const void *src, void *dst, int parity,
                                         cudaStream_t st, bool pdl) {
    return launch_sc<true>(s, src, dst, s.rec[parity], s.rec[parity ^ 1], s.d_step, s.rows, s.variant, st, pdl);
}

// ---------------------------------------------------------------------------
// FP64 <-> deviation storage.  f is [15][N] FP64 (the ABI layout).
// ---------------------------------------------------------------------------
template <typename St>
__global__ void k_from_f64(const double *__restrict__ f, typename St::T *__restrict__ g,
                           long long N, long long P) {
    const long long total = (long long)Q * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long long i = t - (long long)a * N;
        St::store(g + (long long)a * P + i, a, (float)(f[t] - wgt(a)));
    }
}

template <typename St>
__global__ void k_to_f64(const typename St::T *__restrict__ g, double *__restrict__ f, long long N,
                         long long P) {
    const long long total = (long long)Q * N;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(t / N);
        const long long i = t - (long long)a * N;
        f[t] = wgt(a) + (double)St::load(g + (long long)a * P + i, a);
    }
}

// Eq. 17 at every node: g_a = f^eq_a(rho~, u) - w_a, computed in FP64 and
// stored in the handle's storage type.  rho: [N] or null (1); u: [3][N] or null (0).
template <typename St>
__global__ void k_set_equilibrium(const double *__restrict__ rho, const double *__restrict__ u,
                                  typename St::T *__restrict__ g, long long N, long long P) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const double dr = rho ? rho[i] - 1.0 : 0.0;
        const double ux = u ? u[i] : 0.0, uy = u ? u[N + i] : 0.0, uz = u ? u[2 * N + i] : 0.0;
        const double uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double eu = ex(a) * ux + ey(a) * uy + ez(a) * uz;
            St::store(g + (long long)a * P + i, a, (float)(wgt(a) * (dr + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu)));
        }
    }
}

static unsigned grid_for(long long work, int threads, int num_sms) {
    long long g = (work + threads - 1) / threads;
    const long long cap = (long long)num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

cudaError_t launch_fill_rest(Sim &s, void *dst, cudaStream_t st) {
    // all three storage types encode 0 as all-zero bits
    return cudaMemsetAsync(dst, 0, (size_t)storage_bytes(s.precision) * Q * s.P, st);
}

cudaError_t launch_from_f64(Sim &s, const double *f, void *dst, cudaStream_t st) {
    return by_storage(s, [&](auto tag) {
        using St = decltype(tag);
        k_from_f64<St><<<grid_for(Q * s.N, 256, s.num_sms), 256, 0, st>>>(
            f, static_cast<typename St::T *>(dst), s.N, s.P);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_equilibrium(Sim &s, const double *rho, const double *u, void *dst,
                                   cudaStream_t st) {
    return by_storage(s, [&](auto tag) {
        using St = decltype(tag);
        k_set_equilibrium<St><<<grid_for(s.N, 256, s.num_sms), 256, 0, st>>>(
            rho, u, static_cast<typename St::T *>(dst), s.N, s.P);
        return cudaGetLastError();
    });
}

cudaError_t launch_to_f64(Sim &s, const void *src, double *f, cudaStream_t st) {
    return by_storage(s, [&](auto tag) {
        using St = decltype(tag);
        k_to_f64<St><<<grid_for(Q * s.N, 256, s.num_sms), 256, 0, st>>>(
            static_cast<const typename St::T *>(src), f, s.N, s.P);
        return cudaGetLastError();
    });
}

// ---------------------------------------------------------------------------
// Totals of the stored populations for the conservation budget: per block, in
// FP64, the sums over its nodes of sum_a g_a (mass minus the node count) and
// sum_a e_a g_a (momentum; sum_a w_a e_a = 0), so out[4 b + k], k = 0..3.
// Streaming permutes the populations, so these are also the totals of the
// streamed f; the collision conserves the mass and adds exactly the body
// force (Eqs. 15, 18-19).  A fixed grid and a fixed reduction order: the
// result is the same on every call for the same state.
// ---------------------------------------------------------------------------
constexpr int BUDGET_THREADS = 256;

template <typename St>
__global__ void __launch_bounds__(BUDGET_THREADS) k_budget(const typename St::T *__restrict__ g, long long N,
                                                           long long P, double *out) {
    __shared__ double sh[4][BUDGET_THREADS];
    double m = 0.0, p0 = 0.0, p1 = 0.0, p2 = 0.0;
    for (long long i = blockIdx.x * (long long)BUDGET_THREADS + threadIdx.x; i < N;
         i += (long long)gridDim.x * BUDGET_THREADS) {
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            const double v = (double)St::load(g + (long long)a * P + i, a);
            m += v;
            if (ex(a)) p0 += ex(a) > 0 ? v : -v;
            if (ey(a)) p1 += ey(a) > 0 ? v : -v;
            if (ez(a)) p2 += ez(a) > 0 ? v : -v;
        }
    }
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = p0;
    sh[2][threadIdx.x] = p1;
    sh[3][threadIdx.x] = p2;
    __syncthreads();
    for (int w = BUDGET_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) out[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}

int budget_blocks(const Sim &s) { return 2 * s.num_sms; }

cudaError_t launch_budget(Sim &s, const void *src, double *out, cudaStream_t st) {
    return by_storage(s, [&](auto tag) {
        using St = decltype(tag);
        k_budget<St><<<budget_blocks(s), BUDGET_THREADS, 0, st>>>(static_cast<const typename St::T *>(src), s.N,
                                                                 s.P, out);
        return cudaGetLastError();
    });
}

// ---------------------------------------------------------------------------
// Moments of the streamed populations (Eqs. 12-13) and p = rho~/3, in FP64.
// ---------------------------------------------------------------------------
template <typename St, int MAXR>
__global__ void k_fields(const typename St::T *__restrict__ src, double *rho, double *u, double *p,
                         const RepTable<MAXR> rt, long long N, long long P) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const Rep &rp = rt.rep[find_node_rep(rt, i)];
        const int nx = rp.nx, ny = rp.ny, nz = rp.nz;
        const long long li = i - rp.node_off;
        const int x = (int)(li % nx);
        const long long yz = li / nx;
        const int y = (int)(yz % ny);
        const int z = (int)(yz / ny);
        double drho = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
#pragma unroll
        for (int a = 0; a < Q; ++a) {
            int xs = x - ex(a), ys = y - ey(a), zs = z - ez(a);
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
            zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
            const long long sidx = rp.node_off + ((long long)zs * ny + ys) * nx + xs;
            const double g = (double)St::load(src + (long long)a * P + sidx, a);
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

cudaError_t launch_fields(Sim &s, const void *src, double *rho, double *u, double *p,
                          cudaStream_t st) {
    return by_storage(s, [&](auto tag) {
        using St = decltype(tag);
        return by_batch(s, 1, [&](const auto &rt) {
            constexpr int MAXR = sizeof(rt.rep) / sizeof(Rep);
            k_fields<St, MAXR><<<grid_for(s.N, 256, s.num_sms), 256, 0, st>>>(
                static_cast<const typename St::T *>(src), rho, u, p, rt, s.N, s.P);
            return cudaGetLastError();
        });
    });
}

}  // namespace lbp
