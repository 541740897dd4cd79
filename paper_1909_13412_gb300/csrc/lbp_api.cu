// lbp_api.cu -- the C ABI of liblbp (declared in include/lbp.h).
//
// Host side of the library: argument validation, device allocation, layout
// conversion for the ABI arrays, and the per-step launch sequence
//
//      s0:  k_particles (fhat^{n-1} -> F_H, V, r, force records)
//           -> k_stream_collide_forced (fhat^{n-1} + records -> fhat^n)
//      s1:  after every 64th step the VACF block, which overlaps the next
//           steps; s0 waits for it only before the following block is forked.
//
// A step is captured into a CUDA graph per buffer parity and replayed; the
// VACF fork stays outside the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <chrono>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbp_internal.cuh"

using namespace lbp;

struct lbp_sim : public lbp::Sim {
    std::vector<double> h_gamma, h_radius;  // host copies for parameter updates
    std::vector<double> h_mass;             // host copy for the momentum budget
    std::vector<int> h_prep;                // replica of each particle
};

namespace {

// NVTX range for profilers and tracers (a no-op unless a tool is attached):
// every ABI entry point that queues GPU work, and the step's launches, are
// named on the host timeline
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

thread_local std::string g_err;

lbp_status fail(lbp_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            if (e_ == cudaErrorMemoryAllocation) {                                       \
                (void)cudaGetLastError();                                                \
                return fail(LBP_ENOMEM, "%s: %s", #call, cudaGetErrorString(e_));       \
            }                                                                            \
            return fail(LBP_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));            \
        }                                                                                \
    } while (0)

#define CHECK_SIM(s)                                                   \
    do {                                                               \
        if (!(s)) return fail(LBP_EINVAL, "null lbp_sim handle");      \
    } while (0)

const double kSqrt3Bound = 1.7320508075688772;  // R must stay below sqrt(3) dx (Section 2.2)

lbp_status enter(lbp_sim *s) {
    CK(cudaEventRecord(s->ev_in, s->user));
    CK(cudaStreamWaitEvent(s->s0, s->ev_in, 0));
    return LBP_OK;
}

lbp_status leave(lbp_sim *s) {
    CK(cudaEventRecord(s->ev_out, s->s0));
    CK(cudaStreamWaitEvent(s->user, s->ev_out, 0));
    return LBP_OK;
}

void drop_graphs(lbp_sim *s) {
    for (int i = 0; i < 2; ++i) {
        if (s->graph[i]) {
            cudaGraphExecDestroy(s->graph[i]);
            s->graph[i] = nullptr;
        }
        if (s->xgraph[i]) {
            cudaGraphExecDestroy(s->xgraph[i]);
            s->xgraph[i] = nullptr;
        }
    }
}

lbp_status stage(lbp_sim *s, size_t bytes) {
    if (s->stage_bytes >= bytes) return LBP_OK;
    if (s->stage) {
        CK(cudaStreamSynchronize(s->s0));
        cudaFree(s->stage);
        s->stage = nullptr;
        s->stage_bytes = 0;
    }
    CK(cudaMalloc(&s->stage, bytes));
    s->stage_bytes = bytes;
    return LBP_OK;
}

template <typename T>
lbp_status dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    CK(cudaMalloc((void **)p, sizeof(T) * count));
    return LBP_OK;
}

#define TRY(x)                              \
    do {                                    \
        lbp_status st_ = (x);               \
        if (st_ != LBP_OK) return st_;      \
    } while (0)

bool radius_ok(double R, int exclude) {
    if (!(R > 0.0) || !std::isfinite(R)) return false;
    return exclude ? R < 0.5 * kSqrt3Bound : R < kSqrt3Bound;
}

double nu_of(double tau) { return (tau - 0.5) / 3.0; }

// one time step (see the sequence at the top of this file).  With `io` (the
// buffers of lbp_step_exchange: device buffers, or the device views of
// page-locked host buffers) the particle kernel reads the external forces and
// writes the positions and velocities itself, and for host buffers raises the
// step's completion flag.
lbp_status enqueue_step(lbp_sim *s, bool timed, const ParticleIO *io = nullptr) {
    Range range("lbp step: particles + lattice pass");
    const void *src = s->f[s->cur];
    void *dst = s->f[s->cur ^ 1];
    const int parity = s->cur;
    if (s->np > 0) CK(launch_particles(*s, src, parity, s->s0, io));
    if (timed) CK(cudaEventRecord(s->tev[2 * s->ntimed], s->s0));
    // the lattice pass as the programmatic dependent of the particle kernel
    // (its population loads overlap the particle kernel's tail); not when
    // events around it time the lattice kernel alone
    if (s->np > 0)
        CK(launch_stream_collide_forced(*s, src, dst, parity, s->s0, !timed));
    else
        CK(launch_stream_collide(*s, src, dst, s->s0));
    if (timed) {
        CK(cudaEventRecord(s->tev[2 * s->ntimed + 1], s->s0));
        s->ntimed += 1;
    }
    return LBP_OK;
}

// The VACF block of samples just completed runs on the side stream s1 while
// s0 goes on stepping; s0 waits for it only when the next block is due, i.e.
// before the step whose sample would overwrite the oldest sample it reads (the
// ring holds max_lag + 2 blocks).
lbp_status join_vacf(lbp_sim *s) {
    if (s->vacf_pending) {
        CK(cudaStreamWaitEvent(s->s0, s->ev_join, 0));
        s->vacf_pending = 0;
    }
    return LBP_OK;
}

lbp_status fork_vacf(lbp_sim *s) {
    Range range("lbp VACF/MSD block");
    TRY(join_vacf(s));
    CK(cudaEventRecord(s->ev_fork, s->s0));
    CK(cudaStreamWaitEvent(s->s1, s->ev_fork, 0));
    CK(launch_vacf_block(*s, false, s->s1));
    CK(cudaEventRecord(s->ev_join, s->s1));
    s->vacf_pending = 1;
    return LBP_OK;
}

lbp_status fold_timing(lbp_sim *s) {
    if (s->ntimed == 0) return LBP_OK;
    CK(cudaEventSynchronize(s->tev[2 * s->ntimed - 1]));
    for (int i = 0; i < s->ntimed; ++i) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, s->tev[2 * i], s->tev[2 * i + 1]));
        s->timed_ms += ms;
    }
    s->timed_launches += s->ntimed;
    s->ntimed = 0;
    return LBP_OK;
}

lbp_status capture(lbp_sim *s, int parity) {
    cudaGraph_t g = nullptr;
    const int saved = s->cur;
    s->cur = parity;
    CK(cudaStreamBeginCapture(s->s0, cudaStreamCaptureModeThreadLocal));
    lbp_status st = enqueue_step(s, false);
    cudaError_t e = cudaStreamEndCapture(s->s0, &g);
    s->cur = saved;
    if (st != LBP_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    CK(e);
    e = cudaGraphInstantiate(&s->graph[parity], g, 0);
    cudaGraphDestroy(g);
    CK(e);
    return LBP_OK;
}

// one time step on s0 (graph replay, timed or plain launches); `whole`, when
// given, is a graph that holds this step with its host exchange and replaces
// the step graph of this parity
lbp_status step_once(lbp_sim *s, cudaGraphExec_t whole = nullptr) {
    // the VACF correlator runs when the step completes a block of B samples
    const int B = vacf_block_samples();
    bool due = false;
    if (s->vacf_lag >= 0 && s->np > 0) {
        const long long written = s->step - s->vacf_t0 + 1;
        if (written - s->vacf_done_host >= B) {
            due = true;
            s->vacf_done_host += B;
        }
    }
    if (whole) {
        CK(cudaGraphLaunch(whole, s->s0));
    } else if (s->timing) {
        if (s->ntimed == lbp::Sim::MAX_TIMED) TRY(fold_timing(s));
        TRY(enqueue_step(s, true));
    } else if (s->use_graphs) {
        if (!s->graph[s->cur]) TRY(capture(s, s->cur));
        CK(cudaGraphLaunch(s->graph[s->cur], s->s0));
    } else {
        TRY(enqueue_step(s, false));
    }
    if (due) TRY(fork_vacf(s));
    s->cur ^= 1;
    s->step += 1;
    return LBP_OK;
}

// the exchange's copies and conversions before and after one step, on s0, for
// buffers the particle kernel cannot address directly (pageable, another
// device's, not 8-byte aligned); the others take exchange_graph
lbp_status exchange_in(lbp_sim *s, const double *f_ext, cudaMemcpyKind kind) {
    const int n = s->np;
    if (n > 0 && f_ext) {
        CK(cudaMemcpyAsync(s->xbuf, f_ext, sizeof(double) * 3 * n, kind, s->s0));
        CK(launch_aos_to_soa(s->xbuf, s->fext, n, s->cap, 0, s->s0));
    }
    return LBP_OK;
}

lbp_status exchange_out(lbp_sim *s, double *r, double *v, cudaMemcpyKind kind, cudaStream_t st) {
    const int n = s->np;
    if (n > 0 && r) {
        CK(launch_soa_to_aos(s->r, s->xbuf + 3 * (size_t)n, n, s->cap, st));
        CK(cudaMemcpyAsync(r, s->xbuf + 3 * (size_t)n, sizeof(double) * 3 * n, kind, st));
    }
    if (n > 0 && v) {
        CK(launch_soa_to_aos(s->v, s->xbuf + 6 * (size_t)n, n, s->cap, st));
        CK(cudaMemcpyAsync(v, s->xbuf + 6 * (size_t)n, sizeof(double) * 3 * n, kind, st));
    }
    return LBP_OK;
}

// the device address of a mapped page-locked host buffer (null stays null)
lbp_status device_view(double *&p) {
    if (!p) return LBP_OK;
    cudaPointerAttributes at;
    CK(cudaPointerGetAttributes(&at, p));
    p = static_cast<double *>(at.devicePointer);
    return LBP_OK;
}

// [forces in, step, positions and velocities out] from and to page-locked host
// buffers or device buffers as one graph for the current buffer parity, kept
// while the same buffers come back: the particle kernel reads and writes the
// buffers directly, so the graph holds the step's two kernels only
lbp_status exchange_graph(lbp_sim *s, const double *f_ext, double *r, double *v, int on_device,
                          cudaGraphExec_t *out) {
    const int par = s->cur;
    const void *key[3] = {f_ext, r, v};
    bool same = s->xgraph[par] && s->xkey_np[par] == s->np && s->xkey_dev[par] == on_device;
    for (int k = 0; k < 3 && same; ++k) same = s->xkey[par][k] == key[k];
    if (!same) {
        if (s->xgraph[par]) {
            cudaGraphExecDestroy(s->xgraph[par]);
            s->xgraph[par] = nullptr;
        }
        if (!on_device && !s->d_xticket) {
            TRY(dalloc(&s->d_xticket, 1));
            CK(cudaMemset(s->d_xticket, 0, sizeof(unsigned)));
            CK(cudaHostAlloc((void **)&s->h_xflag, sizeof(long long), cudaHostAllocMapped));
            *s->h_xflag = -1;
            CK(cudaHostGetDevicePointer((void **)&s->h_xflag_dev, s->h_xflag, 0));
        }
        double *f_dev = const_cast<double *>(f_ext), *r_dev = r, *v_dev = v;
        if (!on_device) {
            TRY(device_view(f_dev));
            TRY(device_view(r_dev));
            TRY(device_view(v_dev));
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(s->s0, cudaStreamCaptureModeThreadLocal));
        const ParticleIO io{f_dev, r_dev, v_dev, !on_device};
        lbp_status st = enqueue_step(s, false, &io);
        cudaError_t e = cudaStreamEndCapture(s->s0, &g);
        if (st != LBP_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        CK(e);
        e = cudaGraphInstantiate(&s->xgraph[par], g, 0);
        cudaGraphDestroy(g);
        CK(e);
        for (int k = 0; k < 3; ++k) s->xkey[par][k] = key[k];
        s->xkey_np[par] = s->np;
        s->xkey_dev[par] = on_device;
    }
    *out = s->xgraph[par];
    return LBP_OK;
}

// Wait until the particle kernel of step `step` has written the positions and
// velocities to the host buffers (its completion flag in page-locked memory),
// without waiting for the step's lattice pass.  Bounded: if the stream fails,
// or is idle without the flag, or nothing happens for a minute, give up with
// an error instead of spinning on.
lbp_status wait_exchange_flag(lbp_sim *s, long long step) {
    const auto t0 = std::chrono::steady_clock::now();
    for (long long spin = 1;; ++spin) {
        if (__atomic_load_n(s->h_xflag, __ATOMIC_ACQUIRE) == step) return LBP_OK;
        if (spin % 4096 == 0) {
            const cudaError_t q = cudaStreamQuery(s->s0);
            if (q != cudaSuccess && q != cudaErrorNotReady)
                return fail(LBP_ECUDA, "lbp_step_exchange: %s", cudaGetErrorString(q));
            if (q == cudaSuccess && __atomic_load_n(s->h_xflag, __ATOMIC_ACQUIRE) != step)
                return fail(LBP_ECUDA, "lbp_step_exchange: the step finished without its completion flag");
            if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(60))
                return fail(LBP_ETIMEOUT, "lbp_step_exchange: no completion flag within 60 s");
        }
    }
}

// page-locked (or registered) host memory mapped into the device's address
// space, which kernels can read and write directly (FP64 elements: 8-byte
// aligned; anything else takes the copies, which accept any alignment)
bool host_pinned(const void *p) {
    if (!p) return true;
    if (reinterpret_cast<uintptr_t>(p) % sizeof(double) != 0) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost && at.devicePointer != nullptr;
}

// memory of the current device that its kernels can read and write directly
// (8-byte aligned, as host_pinned)
bool device_memory(const void *p) {
    if (!p) return true;
    if (reinterpret_cast<uintptr_t>(p) % sizeof(double) != 0) return false;
    int dev = 0;
    cudaPointerAttributes at;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}


void free_tape(lbp_sim *s) {
    if (s->tape.ck_f) cudaFree(s->tape.ck_f);
    if (s->tape.ck_p) cudaFree(s->tape.ck_p);
    s->tape = lbp::Tape();
}

lbp_status host_to_device(lbp_sim *s, void *dst, const void *src, size_t bytes, int on_device) {
    CK(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       s->s0));
    return LBP_OK;
}

}  // namespace

// Error hook for entry points defined in other translation units.
lbp_status lbp_set_error_for_noalloc(lbp_status st, const char *msg) { return fail(st, "%s", msg); }

extern "C" {

int lbp_version(void) { return 100; }

const char *lbp_last_error(void) { return g_err.c_str(); }

lbp_status lbp_create(const lbp_lattice_desc *desc, void *stream, lbp_sim **out) {
    if (!desc || !out) return fail(LBP_EINVAL, "lbp_create: null argument");
    return lbp_create_batch(desc, 1, stream, out);
}

lbp_status lbp_create_batch(const lbp_lattice_desc *descs, int nrep, void *stream, lbp_sim **out) {
    if (!descs || !out) return fail(LBP_EINVAL, "lbp_create: null argument");
    *out = nullptr;
    if (nrep < 1 || nrep > MAX_BATCH)
        return fail(LBP_EINVAL, "lbp_create_batch: nrep must be in [1, %d] (got %d)", MAX_BATCH, nrep);
    long long N = 0, nseg = 0;
    for (int r = 0; r < nrep; ++r) {
        const lbp_lattice_desc *desc = descs + r;
        if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1)
            return fail(LBP_EINVAL, "lbp_create: box %d sizes must be >= 1 (got %d %d %d)", r,
                        desc->nx, desc->ny, desc->nz);
        if (!(desc->tau > 0.5) || !std::isfinite(desc->tau))
            return fail(LBP_EINVAL, "lbp_create: box %d: tau must be finite and > 1/2 (nu = (tau-1/2)/3 > 0)", r);
        if (desc->precision != LBP_F32 && desc->precision != LBP_BF16 && desc->precision != LBP_F16)
            return fail(LBP_EINVAL, "lbp_create: unsupported precision %d", desc->precision);
        if (desc->precision != descs[0].precision)
            return fail(LBP_EINVAL, "lbp_create_batch: all boxes must share one precision");
        N += (long long)desc->nx * desc->ny * desc->nz;
        nseg += (long long)desc->ny * desc->nz * ((desc->nx + SEG - 1) / SEG);
        if (N > 2147483647ll)
            return fail(LBP_EINVAL, "lbp_create: %lld nodes in total exceed 2^31-1", N);
    }

    lbp_sim *s = new lbp_sim();
    s->nrep = nrep;
    long long noff = 0, soff = 0;
    for (int r = 0; r < nrep; ++r) {
        const lbp_lattice_desc &d = descs[r];
        Rep &rp = s->reps[r];
        rp.nx = d.nx;
        rp.ny = d.ny;
        rp.nz = d.nz;
        rp.nchunks = (d.nx + SEG - 1) / SEG;
        rp.node_off = noff;
        rp.seg_off = soff;
        rp.omega = (float)(1.0 / d.tau);
        rp.gx = rp.gy = rp.gz = 0.f;
        rp.pad = 0;
        rp.dchunks = make_divisor((unsigned)rp.nchunks);
        rp.dny = make_divisor((unsigned)d.ny);
        // the lattice kernels divide row-segment and row indices by these; check
        // the one-multiplication division on the edges of both ranges
        const unsigned rows = (unsigned)d.ny * (unsigned)d.nz, items = rows * (unsigned)rp.nchunks;
        const unsigned dv[2] = {(unsigned)rp.nchunks, (unsigned)d.ny}, top[2] = {items, rows};
        const Divisor dd[2] = {rp.dchunks, rp.dny};
        for (int k = 0; k < 2; ++k) {
            const unsigned probe[] = {0u, 1u, dv[k] - 1, dv[k], dv[k] + 1, 2 * dv[k] - 1, top[k] - 1, top[k],
                                      0x7fffffffu};
            for (unsigned n : probe)
                if (divide(n, dd[k]) != n / dv[k]) {
                    delete s;
                    return fail(LBP_EINVAL, "lbp_create: internal check of the index division failed");
                }
        }
        s->taus[r] = d.tau;
        noff += (long long)d.nx * d.ny * d.nz;
        soff += (long long)d.ny * d.nz * rp.nchunks;
    }
    s->nx = descs[0].nx;
    s->ny = descs[0].ny;
    s->nz = descs[0].nz;
    s->N = N;
    s->P = (N + 63) / 64 * 64;
    s->nseg = nseg;
    s->tau = descs[0].tau;
    s->precision = descs[0].precision;
    // the measured best on GB300 without tuning (lbp_autotune measures the rest)
    default_shape(*s, s->rows, s->variant);
    s->user = (cudaStream_t)stream;
    s->sqrt3 = std::sqrt(3.0);
    auto bail = [&](lbp_status st) {
        std::string keep = g_err;
        lbp_destroy(s);
        g_err = keep;
        return st;
    };
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->dev);
    if (e == cudaSuccess) e = prepare_lbm_kernels();
    if (e == cudaSuccess) e = prepare_vacf_kernels();
    // the step's own kernels at the highest stream priority, the side stream (the
    // VACF correlator, compute-bound) at the lowest: when both have blocks
    // waiting, the HBM-bound lattice pass gets the SM slots first and the
    // correlator fills what it leaves idle
    int prio_low = 0, prio_high = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->s0, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&s->s1, cudaStreamNonBlocking, prio_low);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        fail(LBP_ECUDA, "lbp_create: %s", cudaGetErrorString(e));
        return bail(LBP_ECUDA);
    }
    lbp_status st = LBP_OK;
    for (int i = 0; i < 2 && st == LBP_OK; ++i) {
        char *buf = nullptr;
        st = dalloc(&buf, (size_t)storage_bytes(s->precision) * Q * s->P);
        s->f[i] = buf;
    }
    if (st == LBP_OK) st = dalloc(&s->d_step, 1);
    if (st == LBP_OK) st = dalloc(&s->d_err, 1);
    if (st == LBP_OK) st = dalloc(&s->d_vacf, 8);

    if (st != LBP_OK) return bail(st);
    e = cudaSuccess;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = launch_fill_rest(*s, s->f[i], s->s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_step, 0, sizeof(long long), s->s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_err, 0, sizeof(int), s->s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_vacf, 0, 8 * sizeof(long long), s->s0);

    if (e == cudaSuccess) e = cudaStreamSynchronize(s->s0);
    if (e != cudaSuccess) {
        fail(LBP_ECUDA, "lbp_create: %s", cudaGetErrorString(e));
        return bail(LBP_ECUDA);
    }
    *out = s;
    return LBP_OK;
}

lbp_status lbp_destroy(lbp_sim *s) {
    if (!s) return LBP_OK;
    if (s->s0) cudaStreamSynchronize(s->s0);
    if (s->s1) cudaStreamSynchronize(s->s1);
    drop_graphs(s);
    free_tape(s);
    void *bufs[] = {s->f[0], s->f[1], s->d_step, s->d_err, s->r, s->v, s->fh, s->fr, s->fext, s->xbuf,
                    s->mass, s->inv_mass, s->gamma, s->radius, s->sig, s->pinned, s->prep, s->fq, s->rec[0],
                    s->rec[1], s->ring,
                    s->d_vacf, s->vacf_sum, s->vacf_cnt, s->vacf_part, s->stage, s->inj, s->budget_part,
                    s->corr_g, s->corr_h, s->corr_w, s->msd_state, s->msd_sum, s->ring16, s->d_xticket};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (s->h_xflag) cudaFreeHost(s->h_xflag);
    for (int i = 0; i < 2 * lbp::Sim::MAX_TIMED; ++i)
        if (s->tev[i]) cudaEventDestroy(s->tev[i]);
    cudaEvent_t evs[] = {s->ev_in, s->ev_out, s->ev_fork, s->ev_join};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    if (s->s0) cudaStreamDestroy(s->s0);
    if (s->s1) cudaStreamDestroy(s->s1);
    delete s;
    return LBP_OK;
}

lbp_status lbp_set_populations(lbp_sim *s, const double *f, int on_device) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (!f) return fail(LBP_EINVAL, "lbp_set_populations: null f");
    TRY(enter(s));
    void *dst = s->f[s->cur];
    if (on_device) {
        CK(launch_from_f64(*s, f, dst, s->s0));
    } else {
        TRY(stage(s, sizeof(double) * Q * s->N));
        CK(cudaMemcpyAsync(s->stage, f, sizeof(double) * Q * s->N, cudaMemcpyHostToDevice, s->s0));
        CK(launch_from_f64(*s, s->stage, dst, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    }
    return leave(s);
}

lbp_status lbp_set_fluid(lbp_sim *s, const double *rho, const double *u, int on_device) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    TRY(enter(s));
    void *dst = s->f[s->cur];
    if (on_device || (!rho && !u)) {
        CK(launch_set_equilibrium(*s, rho, u, dst, s->s0));
    } else {
        TRY(stage(s, sizeof(double) * 4 * s->N));
        const double *dr = nullptr, *du = nullptr;
        if (rho) {
            CK(cudaMemcpyAsync(s->stage, rho, sizeof(double) * s->N, cudaMemcpyHostToDevice, s->s0));
            dr = s->stage;
        }
        if (u) {
            CK(cudaMemcpyAsync(s->stage + s->N, u, sizeof(double) * 3 * s->N, cudaMemcpyHostToDevice, s->s0));
            du = s->stage + s->N;
        }
        CK(launch_set_equilibrium(*s, dr, du, dst, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    }
    return leave(s);
}

lbp_status lbp_read_populations(lbp_sim *s, double *f, int on_device) {
    CHECK_SIM(s);
    if (!f) return fail(LBP_EINVAL, "lbp_read_populations: null f");
    TRY(enter(s));
    const void *src = s->f[s->cur];
    if (on_device) {
        CK(launch_to_f64(*s, src, f, s->s0));
    } else {
        TRY(stage(s, sizeof(double) * Q * s->N));
        CK(launch_to_f64(*s, src, s->stage, s->s0));
        CK(cudaMemcpyAsync(f, s->stage, sizeof(double) * Q * s->N, cudaMemcpyDeviceToHost, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    }
    return leave(s);
}

lbp_status lbp_read_fields(lbp_sim *s, double *rho, double *u, double *p, int on_device) {
    CHECK_SIM(s);
    if (!rho && !u && !p) return LBP_OK;
    TRY(enter(s));
    const void *src = s->f[s->cur];
    if (on_device) {
        CK(launch_fields(*s, src, rho, u, p, s->s0));
    } else {
        TRY(stage(s, sizeof(double) * 5 * s->N));
        double *drho = s->stage, *du = s->stage + s->N, *dp = s->stage + 4 * s->N;
        CK(launch_fields(*s, src, rho ? drho : nullptr, u ? du : nullptr, p ? dp : nullptr, s->s0));
        if (rho) CK(cudaMemcpyAsync(rho, drho, sizeof(double) * s->N, cudaMemcpyDeviceToHost, s->s0));
        if (u) CK(cudaMemcpyAsync(u, du, sizeof(double) * 3 * s->N, cudaMemcpyDeviceToHost, s->s0));
        if (p) CK(cudaMemcpyAsync(p, dp, sizeof(double) * s->N, cudaMemcpyDeviceToHost, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    }
    return leave(s);
}

static lbp_status fetch_host(lbp_sim *s, std::vector<double> &dst, const double *src, size_t count,
                             int on_device) {
    dst.resize(count);
    if (count == 0) return LBP_OK;
    if (on_device) {
        CK(cudaMemcpyAsync(dst.data(), src, sizeof(double) * count, cudaMemcpyDeviceToHost, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    } else {
        std::memcpy(dst.data(), src, sizeof(double) * count);
    }
    return LBP_OK;
}

lbp_status lbp_particles_add(lbp_sim *s, int n, const double *r, const double *v,
                             const double *mass, const double *gamma, const double *radius,
                             int on_device) {
    return lbp_particles_add_to(s, 0, n, r, v, mass, gamma, radius, on_device);
}

lbp_status lbp_particles_add_to(lbp_sim *s, int replica, int n, const double *r, const double *v,
                                const double *mass, const double *gamma, const double *radius,
                                int on_device) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (replica < 0 || replica >= s->nrep)
        return fail(LBP_EINVAL, "lbp_particles_add: replica %d outside [0, %d)", replica, s->nrep);
    if (n < 0) return fail(LBP_EINVAL, "lbp_particles_add: n < 0");
    if (n == 0) return LBP_OK;
    if (!r || !v || !mass || !gamma)
        return fail(LBP_EINVAL, "lbp_particles_add: r, v, mass and gamma are required");
    if ((long long)s->np + n > (1 << 26))
        return fail(LBP_EINVAL, "lbp_particles_add: more than 2^26 particles");
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    CK(cudaStreamSynchronize(s->s1));
    std::vector<double> hr, hv, hm, hg, hR;
    TRY(fetch_host(s, hr, r, 3 * (size_t)n, on_device));
    TRY(fetch_host(s, hv, v, 3 * (size_t)n, on_device));
    TRY(fetch_host(s, hm, mass, n, on_device));
    TRY(fetch_host(s, hg, gamma, n, on_device));
    if (radius) TRY(fetch_host(s, hR, radius, n, on_device));
    const int L[3] = {s->reps[replica].nx, s->reps[replica].ny, s->reps[replica].nz};
    const double nu = nu_of(s->taus[replica]);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k) {
            const double x = hr[3 * i + k];
            if (!(x >= 0.0) || !(x < (double)L[k]))
                return fail(LBP_EINVAL, "lbp_particles_add: r[%d][%d] = %g outside [0, %d)", i, k, x, L[k]);
            if (!std::isfinite(hv[3 * i + k]))
                return fail(LBP_EINVAL, "lbp_particles_add: v[%d][%d] is not finite", i, k);
        }
        if (!(hm[i] > 0.0) || !std::isfinite(hm[i]))
            return fail(LBP_EINVAL, "lbp_particles_add: mass[%d] must be > 0", i);
        if (!(hg[i] >= 0.0) || !std::isfinite(hg[i]))
            return fail(LBP_EINVAL, "lbp_particles_add: gamma[%d] must be >= 0", i);
        if (!radius) hR.push_back(hg[i] / (6.0 * M_PI * nu));
        if (!radius_ok(hR[i], s->exclude_inside))
            return fail(LBP_EINVAL,
                        "lbp_particles_add: radius[%d] = %g must be > 0 and < %s dx (Section 2.2)",
                        i, hR[i], s->exclude_inside ? "sqrt(3)/2" : "sqrt(3)");
    }

    // grow the device arrays
    const int np_new = s->np + n;
    if (np_new > s->cap) {
        int cap = s->cap ? s->cap : 64;
        while (cap < np_new) cap *= 2;
        CK(cudaStreamSynchronize(s->s0));
        CK(cudaStreamSynchronize(s->s1));
        double **vec[] = {&s->r, &s->v, &s->fh, &s->fr, &s->fext};
        for (double **pp : vec) {
            double *nb = nullptr;
            TRY(dalloc(&nb, 3 * (size_t)cap));
            CK(cudaMemset(nb, 0, sizeof(double) * 3 * cap));
            if (*pp) {
                for (int k = 0; k < 3; ++k)
                    CK(cudaMemcpy(nb + (size_t)k * cap, *pp + (size_t)k * s->cap,
                                  sizeof(double) * s->np, cudaMemcpyDeviceToDevice));
                cudaFree(*pp);
            }
            *pp = nb;
        }
        double **sca[] = {&s->mass, &s->inv_mass, &s->gamma, &s->radius, &s->sig};
        for (double **pp : sca) {
            double *nb = nullptr;
            TRY(dalloc(&nb, (size_t)cap));
            CK(cudaMemset(nb, 0, sizeof(double) * cap));
            if (*pp) {
                CK(cudaMemcpy(nb, *pp, sizeof(double) * s->np, cudaMemcpyDeviceToDevice));
                cudaFree(*pp);
            }
            *pp = nb;
        }
        unsigned char *np8 = nullptr;
        TRY(dalloc(&np8, (size_t)cap));
        CK(cudaMemset(np8, 0, cap));
        if (s->pinned) {
            CK(cudaMemcpy(np8, s->pinned, s->np, cudaMemcpyDeviceToDevice));
            cudaFree(s->pinned);
        }
        s->pinned = np8;
        int *nrp = nullptr;
        TRY(dalloc(&nrp, (size_t)cap));
        CK(cudaMemset(nrp, 0, sizeof(int) * cap));
        if (s->prep) {
            CK(cudaMemcpy(nrp, s->prep, sizeof(int) * s->np, cudaMemcpyDeviceToDevice));
            cudaFree(s->prep);
        }
        s->prep = nrp;

        // force records (two step parities) and the dense overflow
        // accumulator (3 x 64-bit per node), allocated with the first particle
        if (!s->fq) {
            TRY(dalloc(&s->fq, 3 * (size_t)s->N));
            CK(cudaMemset(s->fq, 0, sizeof(unsigned long long) * 3 * (size_t)s->N));
            for (int q = 0; q < 2; ++q) {
                TRY(dalloc(&s->rec[q], (size_t)s->nseg * REC_WORDS));
                CK(cudaMemset(s->rec[q], 0, sizeof(unsigned long long) * (size_t)s->nseg * REC_WORDS));
            }
        }
        s->cap = cap;
    }
    // upload the new particles into the SoA planes
    std::vector<double> plane(n);
    for (int k = 0; k < 3; ++k) {
        for (int i = 0; i < n; ++i) plane[i] = hr[3 * i + k];
        CK(cudaMemcpy(s->r + (size_t)k * s->cap + s->np, plane.data(), sizeof(double) * n,
                      cudaMemcpyHostToDevice));
        for (int i = 0; i < n; ++i) plane[i] = hv[3 * i + k];
        CK(cudaMemcpy(s->v + (size_t)k * s->cap + s->np, plane.data(), sizeof(double) * n,
                      cudaMemcpyHostToDevice));
    }
    std::vector<double> sg(n);
    for (int i = 0; i < n; ++i) sg[i] = std::sqrt(2.0 * hg[i] * s->kT);
    CK(cudaMemcpy(s->mass + s->np, hm.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    std::vector<double> him(n);
    for (int i = 0; i < n; ++i) him[i] = 1.0 / hm[i];
    CK(cudaMemcpy(s->inv_mass + s->np, him.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->gamma + s->np, hg.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->radius + s->np, hR.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->sig + s->np, sg.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    std::vector<int> hp(n, replica);
    CK(cudaMemcpy(s->prep + s->np, hp.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    s->h_gamma.insert(s->h_gamma.end(), hg.begin(), hg.end());
    s->h_mass.insert(s->h_mass.end(), hm.begin(), hm.end());
    s->h_radius.insert(s->h_radius.end(), hR.begin(), hR.end());
    s->h_prep.insert(s->h_prep.end(), hp.begin(), hp.end());
    s->np = np_new;
    // the VACF ring is laid out per particle count: adding particles turns it off
    s->vacf_lag = -1;
    drop_graphs(s);
    return leave(s);
}

lbp_status lbp_replica_info(lbp_sim *s, int replica, int *dims, double *tau, int64_t *node_offset) {
    CHECK_SIM(s);
    if (replica < 0 || replica >= s->nrep)
        return fail(LBP_EINVAL, "lbp_replica_info: replica %d outside [0, %d)", replica, s->nrep);
    const Rep &rp = s->reps[replica];
    if (dims) {
        dims[0] = rp.nx;
        dims[1] = rp.ny;
        dims[2] = rp.nz;
    }
    if (tau) *tau = s->taus[replica];
    if (node_offset) *node_offset = rp.node_off;
    return LBP_OK;
}

lbp_status lbp_replica_count(lbp_sim *s, int *nrep) {
    CHECK_SIM(s);
    if (!nrep) return fail(LBP_EINVAL, "lbp_replica_count: null nrep");
    *nrep = s->nrep;
    return LBP_OK;
}

lbp_status lbp_particles_count(lbp_sim *s, int *n) {
    CHECK_SIM(s);
    if (!n) return fail(LBP_EINVAL, "lbp_particles_count: null n");
    *n = s->np;
    return LBP_OK;
}

lbp_status lbp_volume_fraction(lbp_sim *s, int replica, double *phi) {
    CHECK_SIM(s);
    if (!phi) return fail(LBP_EINVAL, "lbp_volume_fraction: null phi");
    if (replica < -1 || replica >= s->nrep)
        return fail(LBP_EINVAL, "lbp_volume_fraction: replica %d outside [-1, %d)", replica, s->nrep);
    // sphere volumes per box, from the host copies of the radii
    std::vector<double> vol(s->nrep, 0.0);
    for (size_t i = 0; i < s->h_radius.size(); ++i) {
        const double R = s->h_radius[i];
        vol[s->h_prep[i]] += 4.0 / 3.0 * M_PI * R * R * R;
    }
    double best = 0.0;
    for (int r = 0; r < s->nrep; ++r) {
        const Rep &rp = s->reps[r];
        const double f = vol[r] / ((double)rp.nx * rp.ny * rp.nz);
        if (r == replica) best = f;
        if (replica < 0) best = std::max(best, f);
    }
    *phi = best;
    return LBP_OK;
}

lbp_status lbp_particles_set_params(lbp_sim *s, const lbp_particle_params *prm) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (!prm) return fail(LBP_EINVAL, "lbp_particles_set_params: null params");
    if (!(prm->kT >= 0.0) || !std::isfinite(prm->kT))
        return fail(LBP_EINVAL, "lbp_particles_set_params: kT must be finite and >= 0");
    if (prm->mode < LBP_STOKESLET || prm->mode > LBP_BROWNIAN)
        return fail(LBP_EINVAL, "lbp_particles_set_params: unknown coupling mode %d", prm->mode);
    for (int i = 0; i < s->np; ++i)
        if (!radius_ok(s->h_radius[i], prm->fit_exclude_inside))
            return fail(LBP_EINVAL,
                        "lbp_particles_set_params: radius[%d] = %g too large for fit_exclude_inside=%d",
                        i, s->h_radius[i], prm->fit_exclude_inside);
    TRY(enter(s));
    s->kT = prm->kT;
    s->seed = prm->seed;
    s->mode = prm->mode;
    s->exclude_inside = prm->fit_exclude_inside ? 1 : 0;
    if (s->np) {
        std::vector<double> sg(s->np);
        for (int i = 0; i < s->np; ++i) sg[i] = std::sqrt(2.0 * s->h_gamma[i] * s->kT);
        CK(cudaMemcpyAsync(s->sig, sg.data(), sizeof(double) * s->np, cudaMemcpyHostToDevice, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    }
    drop_graphs(s);
    return leave(s);
}

static lbp_status upload_vec3(lbp_sim *s, double *dst_soa, const double *src_aos, int on_device) {
    const int n = s->np;
    if (on_device) {
        CK(launch_aos_to_soa(src_aos, dst_soa, n, s->cap, 0, s->s0));
        return LBP_OK;
    }
    std::vector<double> plane(3 * (size_t)n);
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < n; ++i) plane[(size_t)k * n + i] = src_aos[3 * i + k];
    for (int k = 0; k < 3; ++k)
        CK(cudaMemcpyAsync(dst_soa + (size_t)k * s->cap, plane.data() + (size_t)k * n,
                           sizeof(double) * n, cudaMemcpyHostToDevice, s->s0));
    CK(cudaStreamSynchronize(s->s0));
    return LBP_OK;
}

lbp_status lbp_particles_set_external_force(lbp_sim *s, const double *f_ext, const uint8_t *pinned,
                                            int on_device) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (s->np == 0) return LBP_OK;
    TRY(enter(s));
    if (f_ext) {
        TRY(upload_vec3(s, s->fext, f_ext, on_device));
    } else {
        CK(cudaMemsetAsync(s->fext, 0, sizeof(double) * 3 * s->cap, s->s0));
    }
    if (pinned) {
        TRY(host_to_device(s, s->pinned, pinned, s->np, on_device));
        if (!on_device) CK(cudaStreamSynchronize(s->s0));
    } else {
        CK(cudaMemsetAsync(s->pinned, 0, s->cap, s->s0));
    }
    return leave(s);
}

lbp_status lbp_particles_set_state(lbp_sim *s, const double *r, const double *v, int on_device) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (s->np == 0) return LBP_OK;
    if (r) {
        std::vector<double> hr;
        TRY(fetch_host(s, hr, r, 3 * (size_t)s->np, on_device));
        for (int i = 0; i < s->np; ++i)
            for (int k = 0; k < 3; ++k) {
                const Rep &rp = s->reps[s->h_prep[i]];
                const int L[3] = {rp.nx, rp.ny, rp.nz};
                if (!(hr[3 * i + k] >= 0.0) || !(hr[3 * i + k] < (double)L[k]))
                    return fail(LBP_EINVAL, "lbp_particles_set_state: r[%d][%d] outside the box", i, k);
            }
    }
    if (v) {
        std::vector<double> hv;
        TRY(fetch_host(s, hv, v, 3 * (size_t)s->np, on_device));
        for (double x : hv)
            if (!std::isfinite(x)) return fail(LBP_EINVAL, "lbp_particles_set_state: non-finite v");
    }
    TRY(enter(s));
    if (r) TRY(upload_vec3(s, s->r, r, on_device));
    if (v) TRY(upload_vec3(s, s->v, v, on_device));
    return leave(s);
}

lbp_status lbp_particles_read(lbp_sim *s, double *r, double *v, double *f_h, double *f_r,
                              int on_device) {
    CHECK_SIM(s);
    if (s->np == 0) return LBP_OK;
    TRY(enter(s));
    const double *srcs[4] = {s->r, s->v, s->fh, s->fr};
    double *dsts[4] = {r, v, f_h, f_r};
    if (!on_device) TRY(stage(s, sizeof(double) * 12 * (size_t)s->np));
    for (int q = 0; q < 4; ++q) {
        if (!dsts[q]) continue;
        double *tgt = on_device ? dsts[q] : s->stage + (size_t)q * 3 * s->np;
        CK(launch_soa_to_aos(srcs[q], tgt, s->np, s->cap, s->s0));
        if (!on_device)
            CK(cudaMemcpyAsync(dsts[q], tgt, sizeof(double) * 3 * s->np, cudaMemcpyDeviceToHost,
                               s->s0));
    }
    if (!on_device) CK(cudaStreamSynchronize(s->s0));
    return leave(s);
}

lbp_status lbp_particles_read_cells(lbp_sim *s, int32_t *base, double *frac, int on_device) {
    CHECK_SIM(s);
    if (!base || !frac) return fail(LBP_EINVAL, "lbp_particles_read_cells: null output");
    if (s->np == 0) return LBP_OK;
    TRY(enter(s));
    if (on_device) {
        CK(launch_cells(*s, base, frac, s->s0));
    } else {
        TRY(stage(s, sizeof(double) * 6 * (size_t)s->np));
        double *df = s->stage;
        int *db = reinterpret_cast<int *>(s->stage + 3 * (size_t)s->np);
        CK(launch_cells(*s, db, df, s->s0));
        CK(cudaMemcpyAsync(base, db, sizeof(int) * 3 * s->np, cudaMemcpyDeviceToHost, s->s0));
        CK(cudaMemcpyAsync(frac, df, sizeof(double) * 3 * s->np, cudaMemcpyDeviceToHost, s->s0));
        CK(cudaStreamSynchronize(s->s0));
    }
    return leave(s);
}

lbp_status lbp_step(lbp_sim *s, int64_t nsteps) {
    Range range("lbp_step");
    CHECK_SIM(s);
    if (nsteps < 0) return fail(LBP_EINVAL, "lbp_step: nsteps < 0");
    if (nsteps == 0) return LBP_OK;
    TRY(enter(s));
    for (int64_t n = 0; n < nsteps; ++n) TRY(step_once(s));
    return leave(s);
}


lbp_status lbp_step_exchange(lbp_sim *s, const double *f_ext, double *r, double *v, int on_device) {
    Range range("lbp_step_exchange");
    CHECK_SIM(s);
    TRY(enter(s));
    const int n = s->np;
    if (n > 0 && (f_ext || r || v)) {
        if (s->xbuf_cap < s->cap) {
            CK(cudaStreamSynchronize(s->s0));
            if (s->xbuf) cudaFree(s->xbuf);
            s->xbuf = nullptr;
            s->xbuf_cap = 0;
            drop_graphs(s);  // the particle capacity grew: captured anew
            TRY(dalloc(&s->xbuf, (size_t)9 * s->cap));
            s->xbuf_cap = s->cap;
        }
    }
    if (n > 0 && f_ext) s->edits += 1;  // as lbp_particles_set_external_force
    const bool as_graph = n > 0 && s->use_graphs && !s->timing &&
                          (on_device ? device_memory(f_ext) && device_memory(r) && device_memory(v)
                                     : host_pinned(f_ext) && host_pinned(r) && host_pinned(v));
    if (as_graph && on_device) {
        // the particle kernel reads f_ext and writes r, v in device memory;
        // stream-ordered like any other step
        cudaGraphExec_t whole = nullptr;
        TRY(exchange_graph(s, f_ext, r, v, 1, &whole));
        TRY(step_once(s, whole));
        return leave(s);
    }
    if (as_graph) {
        // returns once f_ext has been consumed and r, v are on the host; the
        // step's lattice pass may still run, and later work on s0 follows it
        cudaGraphExec_t whole = nullptr;
        TRY(exchange_graph(s, f_ext, r, v, 0, &whole));
        const long long step = s->step;
        // the flag may hold this step index from before a lbp_set_step_index or a
        // checkpoint load; the previous call's kernel has finished writing it
        __atomic_store_n(s->h_xflag, -1ll, __ATOMIC_RELEASE);
        TRY(step_once(s, whole));
        TRY(wait_exchange_flag(s, step));
        return leave(s);
    }
    const cudaMemcpyKind in = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TRY(exchange_in(s, f_ext, in));
    TRY(step_once(s));
    TRY(exchange_out(s, r, v, out, s->s0));
    if (!on_device) CK(cudaStreamSynchronize(s->s0));
    return leave(s);
}

lbp_status lbp_set_step_index(lbp_sim *s, int64_t step) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (step < 0) return fail(LBP_EINVAL, "lbp_set_step_index: step < 0");
    TRY(enter(s));
    long long v = step;
    CK(cudaMemcpyAsync(s->d_step, &v, sizeof(long long), cudaMemcpyHostToDevice, s->s0));
    CK(cudaStreamSynchronize(s->s0));
    s->step = step;
    s->vacf_lag = -1;
    drop_graphs(s);
    return leave(s);
}

lbp_status lbp_get_step_index(lbp_sim *s, int64_t *step) {
    CHECK_SIM(s);
    if (!step) return fail(LBP_EINVAL, "lbp_get_step_index: null step");
    *step = s->step;
    return LBP_OK;
}

lbp_status lbp_vacf_configure(lbp_sim *s, int max_lag) {
    return lbp_vacf_configure_ex(s, max_lag, 0);
}

lbp_status lbp_vacf_configure_ex(lbp_sim *s, int max_lag, int per_particle) {
    CHECK_SIM(s);
    if (max_lag < -1) return fail(LBP_EINVAL, "lbp_vacf_configure: max_lag < -1");
    TRY(enter(s));
    TRY(join_vacf(s));
    CK(cudaStreamSynchronize(s->s0));
    drop_graphs(s);
    s->vacf_lag = -1;
    void **bufs[] = {(void **)&s->ring,   (void **)&s->ring16,   (void **)&s->vacf_sum, (void **)&s->vacf_cnt,
                     (void **)&s->vacf_part, (void **)&s->corr_g, (void **)&s->corr_h,
                     (void **)&s->corr_w, (void **)&s->msd_state, (void **)&s->msd_sum};
    for (void **b : bufs)
        if (*b) {
            cudaFree(*b);
            *b = nullptr;
        }
    if (max_lag < 0) return leave(s);
    if (s->np == 0) return fail(LBP_ESTATE, "lbp_vacf_configure: add particles first");
    const int B = vacf_block_samples();
    const long long ncomp = 3ll * s->np;
    // per particle: FP32 ring of max_lag + 2 blocks (one block more than the
    // window, see join_vacf); ensemble: fp16 hi/lo ring of max_lag + 320
    // samples plus the duplicated first rows (see vacf_kernels.cu)
    const int ld = (int)((ncomp + 7) / 8 * 8);
    const long long cap = per_particle ? (long long)max_lag + 2 * B : (long long)max_lag + 320;
    const size_t K1 = (size_t)max_lag + 1;
    const size_t nsum = (per_particle ? (size_t)s->np : 1) * K1;
    const int nchunks = (int)((ncomp + vacf_chunk_components() - 1) / vacf_chunk_components());
    // every size check before the first allocation: a refused call allocates nothing
    if (per_particle && (nsum > ((size_t)1 << 28) || s->np > 65535))
        return fail(LBP_EINVAL,
                    "lbp_vacf_configure_ex: per particle needs n_particles <= 65535 and n_particles * (max_lag + 1) <= 2^28");
    if (!per_particle && cap + vacf_ring_dup_rows() > 2147483647ll)
        return fail(LBP_EINVAL, "lbp_vacf_configure: max_lag too large");
    const size_t ring_bytes = per_particle ? sizeof(float) * (size_t)cap * (size_t)ncomp
                                           : 4 * (size_t)(cap + vacf_ring_dup_rows()) * (size_t)ld;
    // sums and counts; the ensemble's block partials, G, H, W and MSD state and sums
    size_t total = ring_bytes + sizeof(double) * nsum + sizeof(long long) * K1;
    if (!per_particle) total += sizeof(double) * K1 * ((size_t)nchunks * B + 3 * (size_t)B + 3);
    if (total > ((size_t)64 << 30))
        return fail(LBP_EINVAL, "lbp_vacf_configure: %zu bytes of VACF buffers exceed 64 GiB", total);
    s->vacf_cap = (int)cap;
    s->ring_ld = ld;
    s->vacf_nchunks = nchunks;
    if (per_particle) {
        TRY(dalloc(&s->ring, (size_t)s->vacf_cap * ncomp));
    } else {
        TRY(dalloc(reinterpret_cast<char **>(&s->ring16), ring_bytes));
        CK(cudaMemsetAsync(s->ring16, 0, ring_bytes, s->s0));
        CK(encode_vacf_tensor_maps(*s));
    }
    TRY(dalloc(&s->vacf_sum, nsum));
    TRY(dalloc(&s->vacf_cnt, K1));
    CK(cudaMemsetAsync(s->vacf_sum, 0, sizeof(double) * nsum, s->s0));
    CK(cudaMemsetAsync(s->vacf_cnt, 0, sizeof(long long) * K1, s->s0));
    if (!per_particle) {
        const int B = vacf_block_samples();
        TRY(dalloc(&s->vacf_part, (size_t)s->vacf_nchunks * B * K1));
        TRY(dalloc(&s->corr_g, (size_t)B * K1));
        TRY(dalloc(&s->corr_h, (size_t)B * K1));
        TRY(dalloc(&s->corr_w, (size_t)B * K1));
        TRY(dalloc(&s->msd_state, 2 * K1));
        TRY(dalloc(&s->msd_sum, K1));
        CK(cudaMemsetAsync(s->msd_state, 0, sizeof(double) * 2 * K1, s->s0));
        CK(cudaMemsetAsync(s->msd_sum, 0, sizeof(double) * K1, s->s0));
    }
    long long hv[8] = {s->step, 0, 0, 0, 0, 0, 0, 0};
    CK(cudaMemcpyAsync(s->d_vacf, hv, sizeof(hv), cudaMemcpyHostToDevice, s->s0));
    CK(cudaStreamSynchronize(s->s0));
    s->vacf_lag = max_lag;
    s->vacf_pp = per_particle ? 1 : 0;
    s->vacf_t0 = s->step;
    s->vacf_done_host = 0;
    return leave(s);
}

static lbp_status vacf_read_impl(lbp_sim *s, double *csum, int64_t *counts, int on_device,
                                 int nsets) {
    Range range("lbp_vacf_read (flush)");
    TRY(enter(s));
    TRY(join_vacf(s));
    CK(launch_vacf_block(*s, true, s->s0));
    s->vacf_done_host = s->step - s->vacf_t0;
    const size_t K1 = (size_t)s->vacf_lag + 1;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (csum) CK(cudaMemcpyAsync(csum, s->vacf_sum, sizeof(double) * K1 * (size_t)nsets, kind, s->s0));
    if (counts) CK(cudaMemcpyAsync(counts, s->vacf_cnt, sizeof(long long) * K1, kind, s->s0));
    if (!on_device) CK(cudaStreamSynchronize(s->s0));
    return leave(s);
}

lbp_status lbp_vacf_read(lbp_sim *s, double *csum, int64_t *counts, int on_device) {
    CHECK_SIM(s);
    if (s->vacf_lag < 0) return fail(LBP_ESTATE, "lbp_vacf_read: VACF not configured");
    if (s->vacf_pp) return fail(LBP_ESTATE, "lbp_vacf_read: configured per particle; use lbp_vacf_read_per_particle");
    return vacf_read_impl(s, csum, counts, on_device, 1);
}

lbp_status lbp_msd_read(lbp_sim *s, double *msum, int64_t *counts, int on_device) {
    Range range("lbp_msd_read (flush)");
    CHECK_SIM(s);
    if (s->vacf_lag < 0) return fail(LBP_ESTATE, "lbp_msd_read: VACF not configured (lbp_vacf_configure)");
    if (s->vacf_pp) return fail(LBP_ESTATE, "lbp_msd_read: not kept when the VACF is configured per particle");
    TRY(enter(s));
    TRY(join_vacf(s));
    CK(launch_vacf_block(*s, true, s->s0));
    s->vacf_done_host = s->step - s->vacf_t0;
    const size_t K1 = (size_t)s->vacf_lag + 1;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (msum) CK(cudaMemcpyAsync(msum, s->msd_sum, sizeof(double) * K1, kind, s->s0));
    if (counts) CK(cudaMemcpyAsync(counts, s->vacf_cnt, sizeof(long long) * K1, kind, s->s0));
    if (!on_device) CK(cudaStreamSynchronize(s->s0));
    return leave(s);
}

lbp_status lbp_vacf_read_per_particle(lbp_sim *s, double *csum, int64_t *counts, int on_device) {
    CHECK_SIM(s);
    if (s->vacf_lag < 0 || !s->vacf_pp)
        return fail(LBP_ESTATE, "lbp_vacf_read_per_particle: VACF not configured per particle");
    return vacf_read_impl(s, csum, counts, on_device, s->np);
}

lbp_status lbp_set_body_force(lbp_sim *s, int replica, const double *g) {
    CHECK_SIM(s);
    s->edits += 1;  // invalidates an adjoint recording
    if (!g) return fail(LBP_EINVAL, "lbp_set_body_force: null g");
    if (replica < -1 || replica >= s->nrep)
        return fail(LBP_EINVAL, "lbp_set_body_force: replica %d outside [-1, %d)", replica, s->nrep);
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(g[k])) return fail(LBP_EINVAL, "lbp_set_body_force: non-finite component");
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    for (int r = 0; r < s->nrep; ++r)
        if (replica < 0 || r == replica) {
            s->reps[r].gx = (float)g[0];
            s->reps[r].gy = (float)g[1];
            s->reps[r].gz = (float)g[2];
        }
    drop_graphs(s);  // the graphs hold the replica table by value
    return leave(s);
}

lbp_status lbp_set_block_shape(lbp_sim *s, int rows, int variant) {
    CHECK_SIM(s);
    if (rows != 1 && rows != 2 && rows != 4) return fail(LBP_EINVAL, "lbp_set_block_shape: rows must be 1, 2 or 4");
    if (variant < 0 || variant > 3 || !variant_ok(*s, variant))
        return fail(LBP_EINVAL,
                    "lbp_set_block_shape: variant %d does not apply (1 needs 2-byte storage and even nx, 2 needs nx a "
                    "multiple of 16 bytes of storage, 3 needs 2-byte storage and nx a multiple of 4, in every box)",
                    variant);
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    s->rows = variant == 2 ? 1 : rows;
    s->variant = variant;
    drop_graphs(s);
    return leave(s);
}

lbp_status lbp_set_block_rows(lbp_sim *s, int rows) {
    CHECK_SIM(s);
    return lbp_set_block_shape(s, rows, s->variant == 2 ? 0 : s->variant);
}

lbp_status lbp_autotune(lbp_sim *s, int launches, int *rows, int *variant, double *ms) {
    Range range("lbp_autotune");
    CHECK_SIM(s);
    if (launches < 1 || launches > 1000) return fail(LBP_EINVAL, "lbp_autotune: launches must be in [1, 1000]");
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    // candidates k = 0..9: (variant, rows) = (0: 1, 2, 4 rows), (1: 1, 2, 4),
    // (2: one shape), (3: 1, 2, 4)
    constexpr int NC = LBP_AUTOTUNE_CANDIDATES;
    static const int cand_v[NC] = {0, 0, 0, 1, 1, 1, 2, 3, 3, 3};
    static const int cand_r[NC] = {1, 2, 4, 1, 2, 4, 1, 1, 2, 4};
    bool apply[NC];
    for (int k = 0; k < NC; ++k) apply[k] = variant_ok(*s, cand_v[k]);
    // scratch: a copy of the force records of the last step (all zero before
    // the first), so that the candidates sum the particle forces a step sums,
    // an all-zero record set for the counts they clear, and a step counter to
    // bump.  The dense overflow accumulator is all zero between steps (each
    // lattice pass clears what it reads), so its reads and clears by the
    // candidates change nothing.
    const size_t rec_words = s->np > 0 ? (size_t)s->nseg * REC_WORDS : 0;
    unsigned long long *scr = nullptr;
    TRY(dalloc(&scr, 2 * rec_words + 1));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double t[NC];
    for (int k = 0; k < NC; ++k) t[k] = -1.0;
    cudaError_t e = cudaMemsetAsync(scr, 0, sizeof(unsigned long long) * (2 * rec_words + 1), s->s0);
    if (e == cudaSuccess && rec_words)
        e = cudaMemcpyAsync(scr, s->rec[s->cur ^ 1], sizeof(unsigned long long) * rec_words,
                            cudaMemcpyDeviceToDevice, s->s0);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    long long *bump = reinterpret_cast<long long *>(scr + 2 * rec_words);
    // reads the current populations, writes the other buffer, which the next
    // step overwrites whole: the handle's state is unchanged
    const void *src = s->f[s->cur];
    void *dst = s->f[s->cur ^ 1];
    auto one = [&](int R, int V) {
        return s->np > 0 ? launch_stream_collide_forced_cfg(*s, src, dst, scr, scr + rec_words, bump, R, V, s->s0)
                         : launch_stream_collide_cfg(*s, src, dst, bump, R, V, s->s0);
    };
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass)
        for (int k = 0; k < NC && e == cudaSuccess; ++k) {
            if (!apply[k]) continue;
            const int V = cand_v[k], R = cand_r[k];
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = one(R, V);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s->s0);
            for (int l = 0; l < launches && e == cudaSuccess; ++l) e = one(R, V);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s->s0);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float el = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&el, e0, e1);
            const double per = (double)el / launches;
            if (e == cudaSuccess) t[k] = pass == 0 ? per : std::min(t[k], per);
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(scr);
    if (e != cudaSuccess) return fail(LBP_ECUDA, "lbp_autotune: %s", cudaGetErrorString(e));
    // a bounded wait inside the staged kernel that ran out shows in the error flag
    int err = 0;
    CK(cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err & ERR_TIMEOUT) return fail(LBP_ETIMEOUT, "lbp_autotune: a bounded wait in the staged kernel ran out");
    int best = -1;
    for (int k = 0; k < NC; ++k)
        if (t[k] > 0 && (best < 0 || t[k] < t[best])) best = k;
    s->variant = cand_v[best];
    s->rows = cand_r[best];
    drop_graphs(s);
    if (rows) *rows = s->rows;
    if (variant) *variant = s->variant;
    if (ms)
        for (int k = 0; k < NC; ++k) ms[k] = t[k];
    return leave(s);
}

lbp_status lbp_adjoint_record(lbp_sim *s, int64_t nsteps, int checkpoint_every, double *v_traj,
                              double *r_traj, int on_device) {
    Range range("lbp_adjoint_record");
    CHECK_SIM(s);
    if (nsteps < 1 || checkpoint_every < 1)
        return fail(LBP_EINVAL, "lbp_adjoint_record: need nsteps >= 1 and checkpoint_every >= 1");
    if (s->np < 1) return fail(LBP_ESTATE, "lbp_adjoint_record: add particles first (the recorded outputs are their trajectories)");
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    free_tape(s);
    lbp::Tape &tp = s->tape;
    const size_t pop_bytes = (size_t)storage_bytes(s->precision) * Q * s->P;
    const int64_t nck = (nsteps + checkpoint_every - 1) / checkpoint_every;
    const size_t pcount = (size_t)6 * (s->cap > 0 ? s->cap : 1);
    TRY(dalloc(&tp.ck_f, pop_bytes * (size_t)nck));
    TRY(dalloc(&tp.ck_p, pcount * (size_t)nck));
    const size_t traj = (size_t)nsteps * s->np * 3;
    double *vt = v_traj, *rt = r_traj;
    if (!on_device && (v_traj || r_traj) && traj > 0) {
        TRY(stage(s, sizeof(double) * 2 * traj));
        vt = v_traj ? s->stage : nullptr;
        rt = r_traj ? s->stage + traj : nullptr;
    }
    tp.step0 = s->step;
    tp.cur0 = s->cur;
    tp.C = checkpoint_every;
    tp.np = s->np;
    tp.nck = nck;
    for (int64_t n = 0; n < nsteps; ++n) {
        if (n % checkpoint_every == 0) {
            const int64_t k = n / checkpoint_every;
            CK(cudaMemcpyAsync(tp.ck_f + (size_t)k * pop_bytes, s->f[s->cur], pop_bytes,
                               cudaMemcpyDeviceToDevice, s->s0));
            if (s->np > 0) {
                CK(cudaMemcpyAsync(tp.ck_p + (size_t)k * pcount, s->r, sizeof(double) * 3 * s->cap,
                                   cudaMemcpyDeviceToDevice, s->s0));
                CK(cudaMemcpyAsync(tp.ck_p + (size_t)k * pcount + 3 * s->cap, s->v,
                                   sizeof(double) * 3 * s->cap, cudaMemcpyDeviceToDevice, s->s0));
            }
        }
        TRY(step_once(s));
        if (vt) CK(launch_soa_to_aos(s->v, vt + (size_t)n * s->np * 3, s->np, s->cap, s->s0));
        if (rt) CK(launch_soa_to_aos(s->r, rt + (size_t)n * s->np * 3, s->np, s->cap, s->s0));
    }
    if (!on_device && traj > 0) {
        if (v_traj) CK(cudaMemcpyAsync(v_traj, vt, sizeof(double) * traj, cudaMemcpyDeviceToHost, s->s0));
        if (r_traj) CK(cudaMemcpyAsync(r_traj, rt, sizeof(double) * traj, cudaMemcpyDeviceToHost, s->s0));
    }
    CK(cudaStreamSynchronize(s->s0));
    tp.T = nsteps;
    tp.edits = s->edits;
    return leave(s);
}

lbp_status lbp_adjoint_backward(lbp_sim *s, const double *g_v, const double *g_r, int on_device,
                                const lbp_gradients *out) {
    Range range("lbp_adjoint_backward");
    CHECK_SIM(s);
    if (!out) return fail(LBP_EINVAL, "lbp_adjoint_backward: null grads");
    const lbp::Tape &tp = s->tape;
    if (tp.T == 0) return fail(LBP_ESTATE, "lbp_adjoint_backward: nothing recorded (lbp_adjoint_record)");
    if (s->step != tp.step0 + tp.T || s->edits != tp.edits || s->np != tp.np)
        return fail(LBP_ESTATE, "lbp_adjoint_backward: the handle changed since lbp_adjoint_record");
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    const int np = s->np, cap = s->cap > 0 ? s->cap : 1, C = tp.C;
    const int64_t T = tp.T;
    const size_t pop_bytes = (size_t)storage_bytes(s->precision) * Q * s->P;
    const size_t pcount = (size_t)6 * cap;
    const size_t traj = (size_t)T * np * 3;
    const int nblk = adj_lattice_blocks(*s);
    const size_t rec_bytes = sizeof(unsigned long long) * REC_WORDS * (size_t)s->nseg;

    // work buffers, freed on every exit path
    char *seg = nullptr;
    float *lam = nullptr;
    double *dwork = nullptr;
    struct Guard {
        std::vector<void *> p;
        ~Guard() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } guard;
    // the states of a segment after its first (the first is the checkpoint itself)
    TRY(dalloc(&seg, pop_bytes * (size_t)(C > 1 ? C - 1 : 1)));
    guard.p.push_back(seg);
    TRY(dalloc(&lam, (size_t)2 * Q * s->P));
    guard.p.push_back(lam);
    float *ug = nullptr;  // per-corner gathers of the particle adjoint
    TRY(dalloc(&ug, (size_t)48 * (np > 0 ? np : 1)));
    guard.p.push_back(ug);
    // doubles: seg_p [C][6 cap] | lam_v, lam_r [3 cap] | acc [4 np] | acc_om [nblk] |
    //          save (r, v, fh, fr) [12 cap] | g_v, g_r staged [traj] each
    const size_t n_segp = (size_t)C * pcount, n_lvr = (size_t)6 * cap, n_acc = (size_t)4 * (np > 0 ? np : 1),
                 n_om = (size_t)nblk, n_save = (size_t)12 * cap;
    const bool stage_g = !on_device && traj > 0;
    const size_t n_g = stage_g ? 2 * traj : 0;
    TRY(dalloc(&dwork, n_segp + n_lvr + n_acc + n_om + n_save + n_g));
    guard.p.push_back(dwork);
    double *f0tmp = nullptr;  // FP64 staging of dL/df0 for a host destination
    if (out->f0 && !on_device) {
        TRY(dalloc(&f0tmp, (size_t)Q * s->N));
        guard.p.push_back(f0tmp);
    }
    double *seg_p = dwork, *lam_v = seg_p + n_segp, *lam_r = lam_v + 3 * (size_t)cap,
           *acc = lam_v + n_lvr, *acc_om = acc + n_acc, *save = acc_om + n_om, *gst = save + n_save;
    const double *gv = g_v, *gr = g_r;
    if (stage_g) {
        if (g_v) {
            CK(cudaMemcpyAsync(gst, g_v, sizeof(double) * traj, cudaMemcpyHostToDevice, s->s0));
            gv = gst;
        }
        if (g_r) {
            CK(cudaMemcpyAsync(gst + traj, g_r, sizeof(double) * traj, cudaMemcpyHostToDevice, s->s0));
            gr = gst + traj;
        }
    }
    CK(cudaMemsetAsync(lam, 0, sizeof(float) * 2 * Q * s->P, s->s0));
    CK(cudaMemsetAsync(lam_v, 0, sizeof(double) * (n_lvr + n_acc + n_om), s->s0));
    // the state to put back: particles (the populations are not touched)
    double *sv[4] = {s->r, s->v, s->fh, s->fr};
    if (np > 0)
        for (int k = 0; k < 4; ++k)
            CK(cudaMemcpyAsync(save + (size_t)3 * cap * k, sv[k], sizeof(double) * 3 * cap,
                               cudaMemcpyDeviceToDevice, s->s0));
    const int saved_vacf = s->vacf_lag;
    s->vacf_lag = -1;  // the replay writes no VACF samples
    auto restore = [&]() {
        s->vacf_lag = saved_vacf;
        if (np > 0)
            for (int k = 0; k < 4; ++k)
                cudaMemcpyAsync(sv[k], save + (size_t)3 * cap * k, sizeof(double) * 3 * cap,
                                cudaMemcpyDeviceToDevice, s->s0);
        if (s->rec[0]) {
            cudaMemsetAsync(s->rec[0], 0, rec_bytes, s->s0);
            cudaMemsetAsync(s->rec[1], 0, rec_bytes, s->s0);
        }
        long long st = s->step;
        cudaMemcpyAsync(s->d_step, &st, sizeof(long long), cudaMemcpyHostToDevice, s->s0);
        cudaStreamSynchronize(s->s0);
    };
    cudaError_t e = cudaSuccess;
    int L = 0;  // lam + L * 15 P holds dL/dfhat of the current step
#define ADJ_CK(x)                   \
    do {                            \
        if (e == cudaSuccess) e = (x); \
    } while (0)
    for (int64_t k = tp.nck - 1; k >= 0 && e == cudaSuccess; --k) {
        const int64_t n0 = k * C;
        const int m = (int)(T - n0 < C ? T - n0 : C);
        // replay the segment forward from its checkpoint, keeping every state
        // state j of the segment: the checkpoint for j = 0, else replay slot j - 1
        char *ck = tp.ck_f + (size_t)k * pop_bytes;
        auto state = [&](int j) -> char * { return j == 0 ? ck : seg + (size_t)(j - 1) * pop_bytes; };
        if (np > 0) {
            ADJ_CK(cudaMemcpyAsync(s->r, tp.ck_p + (size_t)k * pcount, sizeof(double) * 3 * cap,
                                   cudaMemcpyDeviceToDevice, s->s0));
            ADJ_CK(cudaMemcpyAsync(s->v, tp.ck_p + (size_t)k * pcount + 3 * cap, sizeof(double) * 3 * cap,
                                   cudaMemcpyDeviceToDevice, s->s0));
        }
        long long st0 = tp.step0 + n0;
        ADJ_CK(cudaMemcpyAsync(s->d_step, &st0, sizeof(long long), cudaMemcpyHostToDevice, s->s0));
        if (s->rec[0]) {
            ADJ_CK(cudaMemsetAsync(s->rec[0], 0, rec_bytes, s->s0));
            ADJ_CK(cudaMemsetAsync(s->rec[1], 0, rec_bytes, s->s0));
        }
        for (int j = 0; j < m && e == cudaSuccess; ++j) {
            const int64_t n = n0 + j;
            const int parity = tp.cur0 ^ (int)(n & 1);
            if (np > 0) {
                ADJ_CK(cudaMemcpyAsync(seg_p + (size_t)j * pcount, s->r, sizeof(double) * 3 * cap,
                                       cudaMemcpyDeviceToDevice, s->s0));
                ADJ_CK(cudaMemcpyAsync(seg_p + (size_t)j * pcount + 3 * cap, s->v, sizeof(double) * 3 * cap,
                                       cudaMemcpyDeviceToDevice, s->s0));
            }
            if (j == m - 1) break;
            const void *src = state(j);
            void *dst = state(j + 1);
            if (np > 0) {
                ADJ_CK(launch_particles(*s, src, parity, s->s0));
                ADJ_CK(launch_stream_collide_forced(*s, src, dst, parity, s->s0, false));
            } else {
                ADJ_CK(launch_stream_collide(*s, src, dst, s->s0));
            }
        }
        if (s->rec[0]) {
            ADJ_CK(cudaMemsetAsync(s->rec[0], 0, rec_bytes, s->s0));
            ADJ_CK(cudaMemsetAsync(s->rec[1], 0, rec_bytes, s->s0));
        }
        // step the adjoint back through the segment
        for (int j = m - 1; j >= 0 && e == cudaSuccess; --j) {
            const int64_t n = n0 + j;
            const int q = j & 1;
            const void *src = state(j);
            const float *lc = lam + (size_t)L * Q * s->P;
            float *ln = lam + (size_t)(L ^ 1) * Q * s->P;
            const double *rj = seg_p + (size_t)j * pcount, *vj = rj + 3 * cap;
            ADJ_CK(launch_adj_particles(*s, src, lc, rj, vj, tp.step0 + n, gv ? gv + (size_t)n * np * 3 : nullptr,
                                        gr ? gr + (size_t)n * np * 3 : nullptr, lam_v, lam_r, acc, q, ug, s->s0));
            const bool timed = s->timing && e == cudaSuccess;
            if (timed) {
                if (s->ntimed == lbp::Sim::MAX_TIMED && fold_timing(s) != LBP_OK) e = cudaErrorUnknown;
                ADJ_CK(cudaEventRecord(s->tev[2 * s->ntimed], s->s0));
            }
            ADJ_CK(launch_adj_lattice(*s, src, lc, ln, q, acc_om, s->s0));
            if (timed) {
                ADJ_CK(cudaEventRecord(s->tev[2 * s->ntimed + 1], s->s0));
                if (e == cudaSuccess) s->ntimed += 1;
            }
            L ^= 1;
        }
    }
#undef ADJ_CK
    // gradients
    auto collect = [&]() -> lbp_status {
        if (e != cudaSuccess) return fail(LBP_ECUDA, "lbp_adjoint_backward: %s", cudaGetErrorString(e));
        const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        std::vector<double> h_om(nblk), h_acc(4 * (size_t)np);
        CK(cudaMemcpyAsync(h_om.data(), acc_om, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s->s0));
        if (np > 0)
            CK(cudaMemcpyAsync(h_acc.data(), acc, sizeof(double) * 4 * np, cudaMemcpyDeviceToHost, s->s0));
        if (out->f0) {
            CK(launch_f32_to_f64(*s, lam + (size_t)L * Q * s->P, on_device ? out->f0 : f0tmp, s->s0));
            if (!on_device)
                CK(cudaMemcpyAsync(out->f0, f0tmp, sizeof(double) * Q * s->N, cudaMemcpyDeviceToHost, s->s0));
        }
        if (np > 0) {
            double *aos = seg_p;  // free now: C * 6 cap >= 6 np doubles
            if (out->v0) {
                CK(launch_soa_to_aos(lam_v, on_device ? out->v0 : aos, np, cap, s->s0));
                if (!on_device)
                    CK(cudaMemcpyAsync(out->v0, aos, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost, s->s0));
            }
            if (out->r0) {
                double *aos2 = aos + 3 * (size_t)np;
                CK(launch_soa_to_aos(lam_r, on_device ? out->r0 : aos2, np, cap, s->s0));
                if (!on_device)
                    CK(cudaMemcpyAsync(out->r0, aos2, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost, s->s0));
            }
            double *accs[3] = {out->gamma, out->radius, out->mass};
            for (int k = 0; k < 3; ++k)
                if (accs[k]) CK(cudaMemcpyAsync(accs[k], acc + (size_t)k * np, sizeof(double) * np, kind, s->s0));
        }
        CK(cudaStreamSynchronize(s->s0));
        // fixed-order host sums of the per-block and per-particle accumulators;
        // dL/dtau per box from the blocks of its row segments
        std::vector<double> dtau(s->nrep);
        for (int r = 0; r < s->nrep; ++r) {
            const int b1 = r + 1 < s->nrep ? adj_lattice_first_block(*s, r + 1) : nblk;
            double dom = 0.0;
            for (int b = adj_lattice_first_block(*s, r); b < b1; ++b) dom += h_om[b];
            const double omega = (double)s->reps[r].omega;
            dtau[r] = -dom * omega * omega;  // omega = 1/tau
        }
        double dkT = 0.0;
        for (int i = 0; i < np; ++i) dkT += h_acc[3 * (size_t)np + i];
        const cudaMemcpyKind hk = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        if (out->tau) CK(cudaMemcpy(out->tau, dtau.data(), sizeof(double) * s->nrep, hk));
        if (out->kT) CK(cudaMemcpy(out->kT, &dkT, sizeof(double), hk));
        return LBP_OK;
    };
    const lbp_status st = collect();
    restore();
    if (st != LBP_OK) return st;
    return leave(s);
}

lbp_status lbp_check(lbp_sim *s) {
    CHECK_SIM(s);
    CK(cudaStreamSynchronize(s->s0));
    CK(cudaStreamSynchronize(s->s1));
    int err = 0;
    CK(cudaMemcpy(&err, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err) {
        CK(cudaMemset(s->d_err, 0, sizeof(int)));
        if (err & ERR_TIMEOUT) {
            // the lattice pass that gave up left some force-record counts and
            // overflow entries of its step uncleared; between steps both are
            // disposable, so start the next step from clean ones
            if (s->fq) {
                CK(cudaMemset(s->fq, 0, sizeof(unsigned long long) * 3 * (size_t)s->N));
                for (int q = 0; q < 2; ++q)
                    CK(cudaMemset(s->rec[q], 0, sizeof(unsigned long long) * (size_t)s->nseg * REC_WORDS));
            }
            return fail(LBP_ETIMEOUT, "lbp_check: a bounded wait on an mbarrier in the staged lattice kernel ran out "
                                      "(that step's lattice pass is incomplete)");
        }
        if (err & ERR_LATTICE) return fail(LBP_ENAN, "lbp_check: a population of the lattice became non-finite");
        if (err & ERR_NAN) return fail(LBP_ENAN, "lbp_check: a particle velocity or position became non-finite or left the box");
        return fail(LBP_ERANGE, "lbp_check: a friction force exceeded the fixed-point range (|F_H| >= 32)");
    }
    return LBP_OK;
}

lbp_status lbp_diagnostics(lbp_sim *s, int64_t *out, int n) {
    CHECK_SIM(s);
    if (n < 0 || (n > 0 && !out)) return fail(LBP_EINVAL, "lbp_diagnostics: bad output");
    CK(cudaStreamSynchronize(s->s0));
    int64_t v[6] = {0, REC_SLOTS, s->nseg, s->rows, (int64_t)s->variant, particles_fit_per_corner(*s) ? 1 : 0};
    if (s->rec[0]) {
        // shares beyond the slots of the records of the last completed step
        std::vector<unsigned long long> words((size_t)s->nseg * REC_WORDS);
        CK(cudaMemcpy(words.data(), s->rec[s->cur ^ 1], sizeof(unsigned long long) * words.size(),
                      cudaMemcpyDeviceToHost));
        for (long long q = 0; q < s->nseg; ++q) {
            const long long c = (long long)(words[(size_t)q * REC_WORDS] & 0xffffffffull);
            if (c > REC_SLOTS) v[0] += c - REC_SLOTS;
        }
    }
    for (int i = 0; i < n && i < 6; ++i) out[i] = v[i];
    return LBP_OK;
}

// ------------------------------------------------------------------ checkpoints
// Layout: a header of 16 int64 words, then the populations in the storage
// format (15 planes of N deviations, plane after plane), then the particle
// positions and velocities (FP64, [3][np] each, SoA).
namespace {
constexpr int64_t CKPT_MAGIC = 0x4c42504b43503031ll;  // "LBPKCP01"
constexpr int CKPT_HEADER = 16;

size_t ckpt_bytes(const lbp_sim *s) {
    return sizeof(int64_t) * CKPT_HEADER + (size_t)storage_bytes(s->precision) * Q * (size_t)s->N +
           sizeof(double) * 6 * (size_t)s->np;
}

void ckpt_header(const lbp_sim *s, int64_t *h) {
    for (int i = 0; i < CKPT_HEADER; ++i) h[i] = 0;
    h[0] = CKPT_MAGIC;
    h[1] = s->precision;
    h[2] = s->nrep;
    h[3] = s->N;
    h[4] = s->np;
    h[5] = s->step;
    // a fingerprint of the box sizes and relaxation times
    uint64_t fp = 1469598103934665603ull;
    for (int r = 0; r < s->nrep; ++r) {
        uint64_t tb;
        std::memcpy(&tb, &s->taus[r], sizeof(tb));
        const uint64_t v[4] = {(uint64_t)s->reps[r].nx, (uint64_t)s->reps[r].ny, (uint64_t)s->reps[r].nz, tb};
        for (uint64_t x : v) fp = (fp ^ x) * 1099511628211ull;
    }
    h[6] = (int64_t)fp;
}
}  // namespace

lbp_status lbp_checkpoint_size(lbp_sim *s, size_t *bytes) {
    CHECK_SIM(s);
    if (!bytes) return fail(LBP_EINVAL, "lbp_checkpoint_size: null bytes");
    *bytes = ckpt_bytes(s);
    return LBP_OK;
}

lbp_status lbp_checkpoint_save(lbp_sim *s, void *buf, int on_device) {
    Range range("lbp_checkpoint_save");
    CHECK_SIM(s);
    if (!buf) return fail(LBP_EINVAL, "lbp_checkpoint_save: null buffer");
    TRY(enter(s));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    int64_t h[CKPT_HEADER];
    ckpt_header(s, h);
    char *out = static_cast<char *>(buf);
    CK(cudaMemcpyAsync(out, h, sizeof(h), on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s->s0));
    out += sizeof(h);
    const size_t plane = (size_t)storage_bytes(s->precision) * (size_t)s->N;
    const size_t pstride = (size_t)storage_bytes(s->precision) * (size_t)s->P;
    for (int a = 0; a < Q; ++a)
        CK(cudaMemcpyAsync(out + a * plane, static_cast<const char *>(s->f[s->cur]) + a * pstride, plane, kind, s->s0));
    out += Q * plane;
    for (int k = 0; k < 3 && s->np > 0; ++k) {
        CK(cudaMemcpyAsync(out + sizeof(double) * (size_t)k * s->np, s->r + (size_t)k * s->cap,
                           sizeof(double) * s->np, kind, s->s0));
        CK(cudaMemcpyAsync(out + sizeof(double) * (size_t)(3 + k) * s->np, s->v + (size_t)k * s->cap,
                           sizeof(double) * s->np, kind, s->s0));
    }
    CK(cudaStreamSynchronize(s->s0));
    return leave(s);
}

lbp_status lbp_checkpoint_load(lbp_sim *s, const void *buf, int on_device) {
    Range range("lbp_checkpoint_load");
    CHECK_SIM(s);
    if (!buf) return fail(LBP_EINVAL, "lbp_checkpoint_load: null buffer");
    int64_t h[CKPT_HEADER], want[CKPT_HEADER];
    CK(cudaMemcpy(h, buf, sizeof(h), on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
    ckpt_header(s, want);
    if (h[0] != CKPT_MAGIC) return fail(LBP_EINVAL, "lbp_checkpoint_load: not a checkpoint of this library");
    if (h[1] != want[1] || h[2] != want[2] || h[3] != want[3] || h[6] != want[6])
        return fail(LBP_EINVAL, "lbp_checkpoint_load: the checkpoint holds other boxes (sizes, tau) or storage");
    if (h[4] != want[4])
        return fail(LBP_EINVAL, "lbp_checkpoint_load: the checkpoint holds %lld particles, the handle %d",
                    (long long)h[4], s->np);
    if (h[5] < 0) return fail(LBP_EINVAL, "lbp_checkpoint_load: bad step index");
    s->edits += 1;  // invalidates an adjoint recording
    TRY(enter(s));
    TRY(join_vacf(s));
    CK(cudaStreamSynchronize(s->s0));
    CK(cudaStreamSynchronize(s->s1));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const char *in = static_cast<const char *>(buf) + sizeof(h);
    const size_t plane = (size_t)storage_bytes(s->precision) * (size_t)s->N;
    const size_t pstride = (size_t)storage_bytes(s->precision) * (size_t)s->P;
    for (int a = 0; a < Q; ++a)
        CK(cudaMemcpyAsync(static_cast<char *>(s->f[s->cur]) + a * pstride, in + a * plane, plane, kind, s->s0));
    in += Q * plane;
    for (int k = 0; k < 3 && s->np > 0; ++k) {
        CK(cudaMemcpyAsync(s->r + (size_t)k * s->cap, in + sizeof(double) * (size_t)k * s->np,
                           sizeof(double) * s->np, kind, s->s0));
        CK(cudaMemcpyAsync(s->v + (size_t)k * s->cap, in + sizeof(double) * (size_t)(3 + k) * s->np,
                           sizeof(double) * s->np, kind, s->s0));
    }
    long long st = h[5];
    CK(cudaMemcpyAsync(s->d_step, &st, sizeof(long long), cudaMemcpyHostToDevice, s->s0));
    CK(cudaStreamSynchronize(s->s0));
    s->step = h[5];
    s->vacf_lag = -1;  // as lbp_set_step_index: the VACF restarts from a new configure
    drop_graphs(s);
    return leave(s);
}

lbp_status lbp_set_wait_bound(lbp_sim *s, int64_t cycles) {
    CHECK_SIM(s);
    if (cycles < 0) return fail(LBP_EINVAL, "lbp_set_wait_bound: cycles < 0");
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    s->wait_cycles = cycles == 0 ? DEFAULT_WAIT_CYCLES : (long long)cycles;
    drop_graphs(s);  // the graphs hold the bound as a kernel parameter
    return leave(s);
}

lbp_status lbp_set_wait_probe(lbp_sim *s, int enable) {
    CHECK_SIM(s);
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    s->wait_probe = enable ? 1 : 0;
    drop_graphs(s);  // the graphs hold the probe flag as a kernel parameter
    return leave(s);
}

lbp_status lbp_budget_track(lbp_sim *s, int enable) {
    CHECK_SIM(s);
    TRY(enter(s));
    CK(cudaStreamSynchronize(s->s0));
    CK(cudaStreamSynchronize(s->s1));
    if (enable) {
        if (!s->inj) TRY(dalloc(&s->inj, 3));
        CK(cudaMemsetAsync(s->inj, 0, 3 * sizeof(double), s->s0));
        CK(cudaStreamSynchronize(s->s0));
    } else if (s->inj) {
        cudaFree(s->inj);
        s->inj = nullptr;
    }
    drop_graphs(s);  // the particle kernel's arguments change
    return leave(s);
}

lbp_status lbp_budget(lbp_sim *s, double *out) {
    Range range("lbp_budget");
    CHECK_SIM(s);
    if (!out) return fail(LBP_EINVAL, "lbp_budget: null out");
    TRY(enter(s));
    const int nb = budget_blocks(*s);
    if (!s->budget_part) TRY(dalloc(&s->budget_part, 4 * (size_t)nb));
    CK(launch_budget(*s, s->f[s->cur], s->budget_part, s->s0));
    std::vector<double> part(4 * (size_t)nb), v(3 * (size_t)s->np);
    double inj[3] = {0.0, 0.0, 0.0};
    CK(cudaMemcpyAsync(part.data(), s->budget_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s->s0));
    for (int k = 0; k < 3 && s->np > 0; ++k)
        CK(cudaMemcpyAsync(v.data() + (size_t)k * s->np, s->v + (size_t)k * s->cap, sizeof(double) * s->np,
                           cudaMemcpyDeviceToHost, s->s0));
    if (s->inj) CK(cudaMemcpyAsync(inj, s->inj, sizeof(inj), cudaMemcpyDeviceToHost, s->s0));
    CK(cudaStreamSynchronize(s->s0));
    // fixed-order sums on the host
    double tot[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 4; ++k) tot[k] += part[4 * (size_t)b + k];
    out[0] = (double)s->N + tot[0];
    for (int k = 0; k < 3; ++k) {
        out[1 + k] = tot[1 + k];
        double pk = 0.0;
        for (int i = 0; i < s->np; ++i) pk += s->h_mass[i] * v[(size_t)k * s->np + i];
        out[4 + k] = pk;
        out[7 + k] = s->inj ? inj[k] : 0.0;
    }
    return leave(s);
}

lbp_status lbp_set_use_graphs(lbp_sim *s, int enable) {
    CHECK_SIM(s);
    s->use_graphs = enable ? 1 : 0;
    if (!enable) drop_graphs(s);
    return LBP_OK;
}

lbp_status lbp_timing_enable(lbp_sim *s, int enable) {
    CHECK_SIM(s);
    if (enable && !s->tev[0]) {
        for (int i = 0; i < 2 * lbp::Sim::MAX_TIMED; ++i) CK(cudaEventCreate(&s->tev[i]));
    }
    if (!enable) TRY(fold_timing(s));
    s->timing = enable ? 1 : 0;
    s->timed_ms = 0.0;
    s->timed_launches = 0;
    s->ntimed = 0;
    return LBP_OK;
}

lbp_status lbp_timing_read(lbp_sim *s, double *ms_total, int64_t *launches) {
    CHECK_SIM(s);
    TRY(fold_timing(s));
    if (ms_total) *ms_total = s->timed_ms;
    if (launches) *launches = s->timed_launches;
    return LBP_OK;
}

lbp_status lbp_philox4x64_10(const uint64_t *ctr, const uint64_t *key, uint64_t *out, int64_t n,
                             void *stream) {
    if (n < 0) return fail(LBP_EINVAL, "lbp_philox4x64_10: n < 0");
    if (n > 0 && (!ctr || !key || !out)) return fail(LBP_EINVAL, "lbp_philox4x64_10: null pointer");
    CK(launch_philox((const unsigned long long *)ctr, (const unsigned long long *)key,
                     (unsigned long long *)out, n, (cudaStream_t)stream));
    return LBP_OK;
}

}  // extern "C"
