// lbm_staged.cu -- the fused stream-collide pass with bulk asynchronous copies
// (the TMA engine's cp.async.bulk) staging the pulled populations in shared
// memory (sm_103a).
//
// Same update as lbm_kernels.cu (pull streaming of Eq. 20, moments of
// Eqs. 12-13, BGK collision with the force term of Eqs. 15, 17-19, per node
// the arithmetic of collide_st, so results are identical bit for bit), but
// the loads no longer come from registers.  A persistent CTA walks the items
// of the lattice -- an item is R whole x-rows of one z-plane (R nx <= STAGED_NODES)
// -- through a pipeline of shared-memory stages.  A producer warp refills a
// stage as soon as the eight consumer warps release it (an "empty" mbarrier);
// for each item its lane 0 issues, per population plane a, one bulk copy of
// the item's source rows (the
// rows shifted by -e_y, -e_z; two copies where the shift wraps around in y)
// and one copy of the rows' force records; they complete on the stage's
// "full" mbarrier with a byte count.  The consumer warps wait on it, read their 15
// pulled values from shared memory -- the x-shift, periodic, is an index
// there, since whole rows are staged -- collide and store to global memory.
// Stages of ~15 KB (2-byte storage) or ~30 KB (FP32), several per SM, keep
// ~150 KB per SM in flight without registers held for them; copies of whole
// rows (1-2 KB) keep the number of bulk operations low.
//
// Requirements (checked on the host): every box has nx <= STAGED_NODES and
// nx a multiple of 16 bytes of storage, so that every copy starts and ends on
// a 16-byte boundary.  Every wait on an mbarrier is bounded by `wait_cycles`
// SM clock cycles (a kernel parameter).  A wait that runs out sets ERR_TIMEOUT
// and a CTA-wide abort flag in shared memory; every other wait of the CTA
// then gives up at its next poll and the producer stops issuing copies.
// Before the producer thread leaves, in every case, it waits for the "full"
// barrier of the last copy it issued into each stage, so that no bulk copy is
// still writing into shared memory when the CTA exits.  Those last waits use
// the fixed, long DRAIN_CYCLES bound (copies that were issued land within
// microseconds).
#include <cuda_runtime.h>

#include <type_traits>

#include "lbp_async.cuh"
#include "lbp_internal.cuh"

namespace lbp {

using namespace async;

template <typename St>
struct StagedGeom {
    static constexpr int E = (int)sizeof(typename St::T);
    static constexpr int STAGES = E == 4 ? 3 : 4;
    static constexpr int PLANE_BYTES = STAGED_NODES * E;
    static constexpr int REC_BYTES = STAGED_RECS * REC_WORDS * 8;  // records of an item's rows
    static constexpr int STAGE_BYTES = Q * PLANE_BYTES + REC_BYTES;
    // + full and empty barriers, and one barrier that nothing ever completes (the probe)
    static constexpr int SMEM = STAGES * STAGE_BYTES + (2 * STAGES + 1) * 8;
};

// Item i -> (replica, z, first row y0, rows R) of the staged launch.
template <int MAXR>
__device__ __forceinline__ void staged_item(const RepTable<MAXR> &rt, unsigned item, int &r, int &z,
                                            int &y0, int &R) {
    r = find_block_rep(rt, item);
    const Rep &rp = rt.rep[r];
    const unsigned it = item - rt.item_off[r];
    const int rows = rp.pad;  // rows per item of this box
    const int per_plane = (rp.ny + rows - 1) / rows;
    z = (int)(it / (unsigned)per_plane);
    y0 = (int)(it - (unsigned)z * per_plane) * rows;
    R = rp.ny - y0 < rows ? rp.ny - y0 : rows;
}

// issue the copies of one item into one stage (one thread)
template <typename St, int MAXR, bool FORCED>
__device__ __forceinline__ void issue_item(const Planes<St> &pl, const RepTable<MAXR> &rt,
                                           const unsigned long long *rec_cur, unsigned item, char *stage,
                                           unsigned bar) {
    using G = StagedGeom<St>;
    constexpr int E = G::E;
    int r, z, y0, R;
    staged_item(rt, item, r, z, y0, R);
    const Rep &rp = rt.rep[r];
    const int nx = rp.nx, ny = rp.ny, nz = rp.nz;
    const unsigned row_bytes = (unsigned)(nx * E);
    unsigned bytes = Q * R * row_bytes;
    if (FORCED) bytes += (unsigned)(R * rp.nchunks * REC_WORDS * 8);
    mbar_expect_tx(bar, bytes);  // every byte expected before any lands
#pragma unroll
    for (int a = 0; a < Q; ++a) {
        int zs = z - ez(a);
        zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
        int ys = y0 - ey(a);  // first source row, periodic
        ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
        const typename St::T *plane = pl.s[a] + rp.node_off + (long long)zs * ny * nx;
        const unsigned dst = smem_addr(stage + a * G::PLANE_BYTES);
        const int first = ny - ys < R ? ny - ys : R;  // rows before the wrap
        bulk_g2s(dst, plane + (long long)ys * nx, (unsigned)first * row_bytes, bar);
        if (first < R) bulk_g2s(dst + first * row_bytes, plane, (unsigned)(R - first) * row_bytes, bar);
    }
    if (FORCED) {
        const unsigned long long *rec =
            rec_cur + ((size_t)rp.seg_off + ((size_t)z * ny + y0) * rp.nchunks) * REC_WORDS;
        bulk_g2s(smem_addr(stage + Q * G::PLANE_BYTES), rec, (unsigned)(R * rp.nchunks * REC_WORDS * 8), bar);
    }
}

template <typename St, int MAXR, bool FORCED>
__global__ void __launch_bounds__(STAGED_THREADS + 32) k_stream_collide_staged(
    Planes<St> pl, const RepTable<MAXR> rt, const unsigned long long *__restrict__ rec_cur,
    unsigned long long *rec_prev, unsigned long long *fq, long long Ntot, long long *bump, int *err,
    long long wait_cycles, int probe) {
    using G = StagedGeom<St>;
    constexpr int STAGES = G::STAGES;
    constexpr int NCW = STAGED_THREADS / 32;  // consumer warps; warp NCW is the producer
    extern __shared__ __align__(128) char smem[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem + STAGES * G::STAGE_BYTES);
    unsigned long long *empty = full + STAGES;
    unsigned long long *never = empty + STAGES;  // the probe: no arrival ever completes it
    __shared__ volatile int s_abort;  // set by the first wait of the CTA that runs out
    const unsigned total = rt.item_off[rt.nrep];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (FORCED) grid_dependency_wait();  // everything below may read this step's particle kernel's output
    if (blockIdx.x == 0 && t == 0) *bump += 1;
    if (t == 0) {
        s_abort = 0;
        for (int st = 0; st < STAGES; ++st) {
            mbar_init(smem_addr(full + st), 1);
            mbar_init(smem_addr(empty + st), NCW);
        }
        mbar_init(smem_addr(never), 1);
        fence_barrier_init();
    }
    __syncthreads();  // the only CTA-wide barrier

    if (warp == NCW) {
        // ---- producer: refill a stage as soon as the consumers release it
        if (lane == 0) {
            unsigned k = 0;  // items issued
            for (unsigned item = blockIdx.x; item < total; item += gridDim.x, ++k) {
                const int st = (int)(k % STAGES);
                if (s_abort) break;
                if (k >= (unsigned)STAGES &&
                    !mbar_wait(smem_addr(empty + st), ((k / STAGES) - 1) & 1u, wait_cycles, &s_abort)) {
                    atomicOr(err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                fence_proxy_async();
                issue_item<St, MAXR, FORCED>(pl, rt, rec_cur, item, smem + st * G::STAGE_BYTES,
                                             smem_addr(full + st));
            }
            // drain, whether or not a wait ran out: the last issue into each
            // stage (at most STAGES items) has landed before the thread that
            // issued it returns, so no copy is in flight once every thread of
            // the CTA has left (a consumer may give up on a stage after this
            // thread finished issuing)
            const unsigned first = k > (unsigned)STAGES ? k - STAGES : 0u;
            for (unsigned j = first; j < k; ++j)
                mbar_wait(smem_addr(full + (j % STAGES)), (j / STAGES) & 1u, DRAIN_CYCLES, nullptr);
        }
        return;
    }

    // ---- consumers
    unsigned k = 0;
    bool bad = false;
    if (probe && !mbar_wait(smem_addr(never), 0u, wait_cycles, &s_abort)) {
        // the failure path on purpose: a bounded wait on a barrier that nothing
        // completes runs out (lbp_set_wait_probe, for tests of the error path)
        atomicOr(err, ERR_TIMEOUT);
        s_abort = 1;
        k = 0xffffffffu;  // skip every item
    }
    for (unsigned item = blockIdx.x; item < total && k != 0xffffffffu; item += gridDim.x, ++k) {
        const int st = (int)(k % STAGES);
        const unsigned parity = (k / STAGES) & 1u;
        char *stage = smem + st * G::STAGE_BYTES;
        if (!mbar_wait(smem_addr(full + st), parity, wait_cycles, &s_abort)) {
            // the producer drains the copies in flight before the CTA ends
            atomicOr(err, ERR_TIMEOUT);
            s_abort = 1;
            break;
        }
        int r, z, y0, R;
        staged_item(rt, item, r, z, y0, R);
        const Rep &rp = rt.rep[r];
        const int nx = rp.nx, nch = rp.nchunks;
        const long long row0 = (long long)z * rp.ny + y0;  // first row of the item in its box
        if (FORCED && t < R * nch) rec_prev[((size_t)rp.seg_off + (size_t)row0 * nch + t) * REC_WORDS] = 0ull;
        const unsigned long long *recs = reinterpret_cast<const unsigned long long *>(stage + Q * G::PLANE_BYTES);
        for (int n = t; n < R * nx; n += STAGED_THREADS) {
            const int yy = n / nx, x = n - yy * nx;
            const int xp = x == nx - 1 ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
            const int rb = yy * nx;
            float g[Q];
#pragma unroll
            for (int a = 0; a < Q; ++a) {
                const typename St::T *p = reinterpret_cast<const typename St::T *>(stage + a * G::PLANE_BYTES);
                g[a] = St::cload_shared(p + rb + (ex(a) > 0 ? xm : (ex(a) < 0 ? xp : x)), a);
            }
            float F0 = rp.gx, F1 = rp.gy, F2 = rp.gz;
            const long long d = rp.node_off + (row0 + yy) * nx + x;
            if (FORCED) {
                const unsigned long long *rec = recs + (size_t)(yy * nch + x / SEG) * REC_WORDS;
                const int cnt = (int)(unsigned)(rec[0] & 0xffffffffull);
                if (cnt > 0) {
                    long long a0 = 0, a1 = 0, a2 = 0;
                    const int used = cnt < REC_SLOTS ? cnt : REC_SLOTS;
                    const int *xs = reinterpret_cast<const int *>(rec + REC_X0);
                    for (int sl = 0; sl < used; ++sl)
                        if (xs[sl] == x) {
                            a0 += (long long)rec[REC_F0 + 3 * sl];
                            a1 += (long long)rec[REC_F0 + 3 * sl + 1];
                            a2 += (long long)rec[REC_F0 + 3 * sl + 2];
                        }
                    if (cnt > REC_SLOTS) {
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
            }
            float o[Q];
            collide_st<St>(g, rp.omega, F0, F1, F2, o);
            bad |= nonfinite_node(o);
#pragma unroll
            for (int a = 0; a < Q; ++a) St::cstore(pl.d[a] + d, a, o[a]);
        }
        // this warp is done with the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(empty + st));
    }
    if (bad) atomicOr(err, ERR_LATTICE);
}

// The launcher: one persistent CTA per free slot (occupancy of this kernel).
template <typename St, int MAXR, bool FORCED>
cudaError_t launch_staged_t(const Planes<St> &pl, const RepTable<MAXR> &rt, const unsigned long long *rec_cur,
                            unsigned long long *rec_prev, unsigned long long *fq, long long Ntot, long long *bump,
                            int *err, long long wait_cycles, int probe, int num_sms, cudaStream_t st, bool pdl) {
    using G = StagedGeom<St>;
    auto kern = k_stream_collide_staged<St, MAXR, FORCED>;
    static int per_sm = 0;  // per instantiation
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, STAGED_THREADS + 32, G::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
    }
    const unsigned total = rt.item_off[rt.nrep];
    unsigned grid = (unsigned)(per_sm * num_sms);
    if (grid > total) grid = total;
    if (grid == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STAGED_THREADS + 32);
    cfg.dynamicSmemBytes = G::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, pl, rt, rec_cur, rec_prev, fq, Ntot, bump, err, wait_cycles, probe);
}

// rows per item of a box: as many whole rows as fit STAGED_NODES nodes and
// STAGED_RECS force records (at most ny)
int staged_rows(int nx, int ny) {
    const int nch = (nx + SEG - 1) / SEG;
    int r = STAGED_NODES / nx;
    if (r * nch > STAGED_RECS) r = STAGED_RECS / nch;
    if (r < 1) r = 1;
    return r < ny ? r : ny;
}

#define LBP_STAGED_INST(ST, MAXR, F)                                                                        \
    template cudaError_t launch_staged_t<ST, MAXR, F>(const Planes<ST> &, const RepTable<MAXR> &,          \
                                                      const unsigned long long *, unsigned long long *,     \
                                                      unsigned long long *, long long, long long *, int *, \
                                                      long long, int, int, cudaStream_t, bool);
LBP_STAGED_INST(StoreF32, 1, true)
LBP_STAGED_INST(StoreF32, 1, false)
LBP_STAGED_INST(StoreF32, MAX_BATCH, true)
LBP_STAGED_INST(StoreF32, MAX_BATCH, false)
LBP_STAGED_INST(StoreBF16, 1, true)
LBP_STAGED_INST(StoreBF16, 1, false)
LBP_STAGED_INST(StoreBF16, MAX_BATCH, true)
LBP_STAGED_INST(StoreBF16, MAX_BATCH, false)
LBP_STAGED_INST(StoreF16, 1, true)
LBP_STAGED_INST(StoreF16, 1, false)
LBP_STAGED_INST(StoreF16, MAX_BATCH, true)
LBP_STAGED_INST(StoreF16, MAX_BATCH, false)
#undef LBP_STAGED_INST

}  // namespace lbp
