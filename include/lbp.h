/*
 * lbp.h -- C ABI of liblbp: a D3Q15 lattice-Boltzmann fluid two-way coupled to
 * Langevin point particles by the Stokeslet-fit friction estimate of
 * Yoshida, Kinjo & Washizu, "Numerical simulation method for Brownian particles
 * dispersed in incompressible fluids" (arXiv:1909.13412).
 *
 * Units: lattice units throughout, dx = dt = C = rho0 = dV = 1.
 *
 * One call of lbp_step advances the system by one time step n -> n+1, which is
 * (Section 2 of the paper, with the step order stated below):
 *   1. streaming, Eq. 20, as a pull f_a(x) = fhat_a(x - e_a) on a periodic box;
 *   2. moments rho~ = sum_a f_a (Eq. 12), u = sum_a e_a f_a (Eq. 13);
 *   3. for every particle, the friction force F_H from the least-squares fit of
 *      the Stokeslet flow of Eq. 8 to u - V at the eight corners of the cell
 *      holding r_i, F_H = gamma U_inf e^N (Section 2.1 with Eq. 7);
 *   4. the random force F_R = sqrt(2 gamma kT) xi (Eqs. 4-5), xi from a
 *      Philox-4x64-10 stream keyed by (seed) and counted by (step, particle);
 *   5. the reaction force -F_H spread onto the eight corners with trilinear
 *      weights of r_i^n (Eq. 9);
 *   6. the Langevin update V += F_H + F_R + F_ext over M, r += V (Eqs. 1-2,
 *      semi-implicit Euler, periodic wrap);
 *   7. the BGK collision with body force (Eqs. 14, 15, 17, 18, 19):
 *      fhat_a = f_a + (f^eq_a - f_a)/tau + 3 w_a F.e_a.
 * The state kept between steps is the post-collision fhat.
 *
 * Populations: D3Q15 in this order (e_x, e_y, e_z), weights w:
 *   0 ( 0, 0, 0) 2/9;  1 ( 1, 0, 0)  2 (-1, 0, 0)  3 ( 0, 1, 0)  4 ( 0,-1, 0)
 *   5 ( 0, 0, 1)  6 ( 0, 0,-1) 1/9;  7 ( 1, 1, 1)  8 (-1,-1,-1)  9 ( 1, 1,-1)
 *   10 (-1,-1, 1) 11 ( 1,-1, 1) 12 (-1, 1,-1) 13 (-1, 1, 1) 14 ( 1,-1,-1) 1/72.
 * Field arrays exchanged through this ABI are FP64, structure of arrays with x
 * fastest: f[a][z][y][x] (15 * N values, N = nx*ny*nz), rho[z][y][x],
 * u[k][z][y][x] (k = x, y, z component; 3 * N values).  Particle arrays are
 * FP64, array of structures: r[i][k], v[i][k] (3 * n values), in insertion
 * order (particle ids are 0, 1, ... in the order of lbp_particles_add calls).
 *
 * Memory and streams: the library owns its device state (allocated at create
 * and at particles_add).  Every pointer passed in is owned by the caller; it is
 * a host pointer if the call's on_device argument is 0, else a device pointer
 * on the current device.  All work is ordered after the work already queued on
 * the stream given to lbp_create, and later work on that stream is ordered
 * after it.  Calls that take host pointers return after their copies finish;
 * calls that take device pointers are asynchronous with respect to the host.
 * A handle must not be used from two host threads at once.
 *
 * Errors: every call returns an lbp_status; nothing is thrown across the ABI.
 * lbp_last_error() returns a message for the last failing call of the calling
 * thread.  Arguments are validated before any work is queued: an invalid call
 * changes nothing.
 */
#ifndef LBP_H
#define LBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBP_OK = 0,
    LBP_EINVAL = 1,   /* bad argument (size, tau <= 1/2, radius, null pointer, ...) */
    LBP_ENOMEM = 2,   /* device allocation failed */
    LBP_ECUDA = 3,    /* a CUDA call failed; the message names it */
    LBP_ETIMEOUT = 4, /* a bounded device wait ran out */
    LBP_ENAN = 5,     /* a particle velocity or position, or a lattice population, became non-finite */
    LBP_ESTATE = 6,   /* call not valid in the current state */
    LBP_ERANGE = 7    /* a friction force exceeded the fixed-point range (|F_H| >= 32) */
} lbp_status;

/* Storage of the populations on the device.  Arithmetic is FP32 in every case;
 * the stored quantity is the deviation g_a = f_a - w_a from the rest state:
 *   LBP_F32  g_a as float (120 bytes moved per node update);
 *   LBP_BF16 g_a rounded to bfloat16 (60 bytes);
 *   LBP_F16  g_a * 1024 / w_a rounded to binary16 (60 bytes; the per-population
 *            scale keeps slow-flow deviations in binary16's normal range).
 * Particle state, the fit's solve and the VACF sums stay FP64.                */
typedef enum {
    LBP_F32 = 0,
    LBP_BF16 = 1,
    LBP_F16 = 2
} lbp_precision;

/* Friction model. STOKESLET is the paper's method (Eq. 8); POINTWISE is Eq. 7
 * with u(r_i) interpolated trilinearly from the same eight corners; BROWNIAN is
 * Eq. 6 (F_H = -gamma V, fluid not coupled).                                    */
typedef enum {
    LBP_STOKESLET = 0,
    LBP_POINTWISE = 1,
    LBP_BROWNIAN = 2
} lbp_coupling;

typedef struct {
    int nx, ny, nz;  /* periodic box, each >= 1; nx*ny*nz <= 2^31 - 1          */
    double tau;      /* BGK relaxation time (Eq. 15), > 1/2: nu = (tau-1/2)/3   */
    int precision;   /* lbp_precision                                           */
} lbp_lattice_desc;

typedef struct {
    double kT;              /* thermal energy; sigma^2 = 2 gamma kT (Eq. 5); >= 0    */
    uint64_t seed;          /* Philox key word 0                                     */
    int mode;               /* lbp_coupling                                          */
    int fit_exclude_inside; /* 1: corners with r_p < R are left out of the fit       */
} lbp_particle_params;

typedef struct lbp_sim lbp_sim;

/* Create a periodic box with the fluid at rest (f_a = w_a, rho~ = 1) and no
 * particles.  stream: a cudaStream_t (NULL = the legacy default stream).
 * Section 2.2 (Eqs. 12-20).                                                    */
lbp_status lbp_create(const lbp_lattice_desc *desc, void *stream, lbp_sim **out);

/* Batched ensemble: nrep independent periodic boxes of possibly different
 * sizes and tau (one precision for all), stepped together by the same kernel
 * launches (each launch covers every box).  Populations and fields of all
 * boxes are concatenated node-wise: box r occupies global nodes
 * [node_offset_r, node_offset_r + nx_r ny_r nz_r) of every array exchanged
 * through this ABI (see lbp_replica_info).  1 <= nrep <= 256; lbp_create is
 * the case nrep = 1.  Section 3 averages the VACF over independent particles;
 * the boxes are how such an ensemble is run at once.                           */
lbp_status lbp_create_batch(const lbp_lattice_desc *descs, int nrep, void *stream, lbp_sim **out);

/* Box `replica` of a batch: dims = (nx, ny, nz), tau, first global node.     */
lbp_status lbp_replica_info(lbp_sim *sim, int replica, int *dims, double *tau, int64_t *node_offset);
lbp_status lbp_replica_count(lbp_sim *sim, int *nrep);

/* Free every device resource of the handle.  NULL is accepted.               */
lbp_status lbp_destroy(lbp_sim *sim);

/* Replace the stored post-collision populations fhat with f ([15][nz][ny][nx]
 * FP64).  Eq. 19 output state.                                                 */
lbp_status lbp_set_populations(lbp_sim *sim, const double *f, int on_device);

/* Fluid state from density and velocity fields: every node is set to the
 * equilibrium of Eq. 17, f_a = f^eq_a(rho~, u), as the current post-collision
 * populations.  rho: [N] (NULL: rho~ = 1), u: [3][N] (NULL: u = 0), FP64,
 * host or device per on_device; N counts the nodes of all boxes of a batch.  */
lbp_status lbp_set_fluid(lbp_sim *sim, const double *rho, const double *u, int on_device);

/* Read the stored post-collision populations fhat into f ([15][nz][ny][nx]).  */
lbp_status lbp_read_populations(lbp_sim *sim, double *f, int on_device);

/* Moments of the streamed populations f^{n+1}(x) = fhat(x - e_a), i.e. the
 * fields the particles see at the next step: rho~ (Eq. 12), u (Eq. 13) and
 * p = rho~/3 (pressure, Section 2.2).  Any of rho, u, p may be NULL.            */
lbp_status lbp_read_fields(lbp_sim *sim, double *rho, double *u, double *p, int on_device);

/* Append n particles (ids continue from the current count).  r in [0, L) per
 * component; mass > 0; gamma >= 0; radius > 0 (radius may be NULL: then
 * R = gamma / (6 pi nu), Stokes' law with nu = (tau - 1/2)/3).  Section 2.1.  */
lbp_status lbp_particles_add(lbp_sim *sim, int n, const double *r, const double *v,
                             const double *mass, const double *gamma, const double *radius,
                             int on_device);

/* lbp_particles_add for the box `replica` of a batch (positions in that box's
 * own coordinates); lbp_particles_add adds to box 0.  Particle ids stay global
 * (insertion order over all boxes).                                          */
lbp_status lbp_particles_add_to(lbp_sim *sim, int replica, int n, const double *r, const double *v,
                                const double *mass, const double *gamma, const double *radius,
                                int on_device);

/* Coupling parameters for all particles (Sections 2.1; Eqs. 4-8).            */
lbp_status lbp_particles_set_params(lbp_sim *sim, const lbp_particle_params *params);

/* External force per particle (adds to Eq. 1; NULL = zero) and pinned flags
 * (1 = V and r are held fixed, the particle still exerts its reaction force;
 * NULL = none pinned).                                                          */
lbp_status lbp_particles_set_external_force(lbp_sim *sim, const double *f_ext,
                                            const uint8_t *pinned, int on_device);

/* Overwrite positions and/or velocities (either may be NULL).                */
lbp_status lbp_particles_set_state(lbp_sim *sim, const double *r, const double *v, int on_device);

/* Read positions, velocities and the last step's F_H and F_R (any may be NULL). */
lbp_status lbp_particles_read(lbp_sim *sim, double *r, double *v, double *f_h, double *f_r,
                              int on_device);

/* Cell of each particle as the device computes it: base[i][k] = floor(r_i,k)
 * (int32, [n][3]) and the cell fraction q[i][k] = r_i,k - base[i][k] (FP64,
 * exact, [n][3]).  The reaction force of Eq. 9 is shared over the corners
 * base + {0,1}^3 with the trilinear weights of q (31-bit fixed-point
 * fractions; the eight shares sum to -F_H exactly).                          */
lbp_status lbp_particles_read_cells(lbp_sim *sim, int32_t *base, double *frac, int on_device);

/* Number of particles.                                                       */
lbp_status lbp_particles_count(lbp_sim *sim, int *n);

/* Volume fraction of the particles of box `replica` (-1: the largest over the
 * boxes): the sum of 4/3 pi R^3 over the box's particles divided by its
 * nx ny nz nodes.  The method was checked for volume fractions below 0.1
 * (Section 2.2, closing remarks); lbp_particles_add does not refuse a denser
 * suspension, and the Python binding warns when one is added.  Host
 * bookkeeping only: no GPU work.                                              */
lbp_status lbp_volume_fraction(lbp_sim *sim, int replica, double *phi);

/* Advance nsteps >= 0 time steps (asynchronous on the handle's stream).       */
lbp_status lbp_step(lbp_sim *sim, int64_t nsteps);

/* One step with the exchange a host-side controller needs, in one call and
 * one synchronisation: f_ext ([n][3], NULL: unchanged) becomes the external
 * force of this and later steps (as lbp_particles_set_external_force), one
 * step runs, and r and v ([n][3] each, NULL: not read) receive the positions
 * and velocities after it (as lbp_particles_read).  The call returns when the
 * host outputs are written (on_device = 0) or, for device pointers, with the
 * work queued on the handle's stream.
 * With graphs on and 8-byte aligned buffers that the device can address --
 * memory of the current device (on_device = 1), or page-locked host memory
 * mapped into the device's address space (cudaHostAlloc / cudaHostRegister
 * with unified addressing) -- the step's particle kernel itself reads f_ext
 * and writes r and v, and the step replays as one CUDA graph per buffer
 * parity, cached on the three buffer addresses.  For host buffers, positions
 * and velocities are final after the particle kernel (Eqs. 1-2), whose last
 * block then sets a completion flag in page-locked memory, so the call
 * returns (after a bounded poll of that flag: LBP_ECUDA or LBP_ETIMEOUT if
 * the stream fails or the flag does not come) while the lattice pass of the
 * same step still runs.  Every later call on the handle is ordered after it,
 * and the handle's user stream waits for it.  Other buffers (pageable, or
 * not 8-byte aligned) take plain stream-ordered copies; with host buffers
 * the call then returns after the whole step.                                 */
lbp_status lbp_step_exchange(lbp_sim *sim, const double *f_ext, double *r, double *v, int on_device);

/* Bit-exact checkpoints (no counterpart in the paper; the Philox counter of
 * Eqs. 4-5 is the step index, so a run continued from a checkpoint draws the
 * same noise as the uninterrupted run).  A checkpoint holds the stored
 * populations in their storage format (so nothing is rounded), the particle
 * positions and velocities (FP64) and the step index; the handle's
 * configuration -- boxes, storage, particles with their M, gamma, R, the
 * coupling parameters, external forces, body forces -- is the caller's to
 * recreate.  lbp_checkpoint_size gives the bytes of a checkpoint of this
 * handle; lbp_checkpoint_save writes one into buf (host or device per
 * on_device; synchronous); lbp_checkpoint_load restores one into a handle
 * with the same boxes (sizes and tau), storage and particle count (LBP_EINVAL
 * otherwise, with nothing changed).  Loading turns the VACF off, as
 * lbp_set_step_index does.  Continuing a loaded handle gives results bitwise
 * equal to continuing the handle that was saved.                             */
lbp_status lbp_checkpoint_size(lbp_sim *sim, size_t *bytes);
lbp_status lbp_checkpoint_save(lbp_sim *sim, void *buf, int on_device);
lbp_status lbp_checkpoint_load(lbp_sim *sim, const void *buf, int on_device);

/* The step index n that the next step uses as its Philox counter.            */
lbp_status lbp_set_step_index(lbp_sim *sim, int64_t step);
lbp_status lbp_get_step_index(lbp_sim *sim, int64_t *step);

/* Velocity autocorrelation (Section 3, Fig. 2): from the next step on, every
 * step's post-update velocities are samples t = 0, 1, ...; lbp_vacf_read gives
 * csum[k] = sum over particles i and origins t0 with t0 + k <= last sample of
 * V_i(t0).V_i(t0+k), and counts[k] = the number of (i, t0) pairs, k = 0..max_lag.
 * Each sample component is kept to 22 significant bits (an fp16 pair hi + lo
 * of 4096 V; |V| >= 16 is reported by lbp_check as LBP_ERANGE), the products of
 * a 64-sample block are accumulated in FP32 on the tensor cores and the sums
 * across blocks in FP64.  max_lag = -1 turns it off.  LBP_EINVAL, with nothing
 * allocated and the VACF off, if the ring, sums and correlation buffers
 * would take more than 64 GiB (about 3 * n_particles * 4 bytes per lag for the
 * ring, plus (ceil(3 n_particles / 1024) + 3) * 512 bytes per lag).           */
lbp_status lbp_vacf_configure(lbp_sim *sim, int max_lag);
lbp_status lbp_vacf_read(lbp_sim *sim, double *csum, int64_t *counts, int on_device);

/* Mean squared displacement of the particles over the same samples and lags
 * (the dispersion that accompanies the VACF of Section 3): msum[k] = sum over
 * particles i and origins t0 with t0 + k <= last sample of
 * |X_i(t0 + k) - X_i(t0)|^2, X the unwrapped position (X(t) - X(t - 1) = V(t),
 * the update of Eq. 2 before the periodic wrap), counts[k] as for
 * lbp_vacf_read.  Kept alongside the VACF of lbp_vacf_configure (not with
 * per_particle = 1); computed from the same per-sample products
 * G(t, m) = sum_i V_i(t).V_i(t - m) through the exact recurrence
 * W(e, k) = W(e - 1, k - 1) + G(e, 0) + 2 sum_{m=1}^{k-1} G(e, m) of the
 * squared window sums W, in FP64 (products FP32).  Reading flushes the
 * samples not yet correlated, as lbp_vacf_read does.                         */
lbp_status lbp_msd_read(lbp_sim *sim, double *msum, int64_t *counts, int on_device);

/* The same estimator kept per particle, for ensembles whose particles are not
 * alike (a batch of boxes of different sizes or viscosities, Section 3's
 * dependence of the VACF on L and nu): per_particle = 0 is lbp_vacf_configure;
 * per_particle = 1 keeps csum[i][k] = sum over origins t0 of V_i(t0).V_i(t0+k)
 * for each particle i (row-major [n_particles][max_lag + 1], FP64, products
 * FP32), read with lbp_vacf_read_per_particle; counts[k] is then the number of
 * origins t0, the same for every particle.  LBP_EINVAL if n_particles > 65535
 * or n_particles * (max_lag + 1) > 2^28.  Adding particles or setting the step index turns the
 * VACF off, as for lbp_vacf_configure.                                        */
lbp_status lbp_vacf_configure_ex(lbp_sim *sim, int max_lag, int per_particle);
lbp_status lbp_vacf_read_per_particle(lbp_sim *sim, double *csum, int64_t *counts, int on_device);

/* Wait for the handle's queued work and report device-side errors: LBP_ENAN if
 * a particle state became non-finite or left the box, or if a collided
 * population of the lattice became non-finite (every lattice kernel checks the
 * collided rest population of each node, which every pulled population of the
 * node enters through rho~ and u.u: a NaN or infinity anywhere in the node, or
 * an overflow of u.u, is caught in the step it appears); LBP_ERANGE on
 * fixed-point overflow; LBP_ETIMEOUT if a bounded device wait ran out.  The
 * flags are cleared by the call.                                             */
lbp_status lbp_check(lbp_sim *sim);

/* Conservation budget.  Streaming and the BGK collision conserve mass and
 * momentum (Eqs. 15, 17-20) and the fluid receives exactly -F_H (Eq. 9), so
 * only the random and external forces on the particles (and a uniform body
 * force) change the total momentum.  lbp_budget waits for the handle's work
 * and writes out[10]:
 *   out[0]    total mass, sum over all nodes and boxes of sum_a fhat_a;
 *   out[1..3] fluid momentum, sum over nodes of sum_a e_a fhat_a;
 *   out[4..6] particle momentum, sum_i M_i V_i;
 *   out[7..9] momentum that F_R + F_ext put into the unpinned particles since
 *             lbp_budget_track(sim, 1) (zero while not tracked).
 * Lattice sums in FP64 from the stored populations, in a fixed order.  With
 * no pinned particle and no body force, out[1..3] + out[4..6] - out[7..9]
 * keeps its value from when tracking began, to rounding; a uniform body force
 * g (lbp_set_body_force) adds N g per step, which the caller accounts for.
 * Tracking adds one FP64 atomic per 32 particles and component to every step;
 * lbp_budget_track(sim, 0) stops it.                                         */
lbp_status lbp_budget_track(lbp_sim *sim, int enable);
lbp_status lbp_budget(lbp_sim *sim, double *out);

/* Bound of every device-side wait on an mbarrier (the bulk-copy staged
 * lattice kernel, variant 2 of lbp_autotune), in SM clock cycles; 0 restores
 * the default 2^30 (about half a second).  A wait that runs out leaves that
 * step's lattice pass incomplete and makes lbp_check return LBP_ETIMEOUT; the
 * kernel first waits (with the default bound) for the copies it has issued,
 * so the device stays usable.  lbp_check then also resets the step's force
 * records; the populations of that step are not valid, so restore a state
 * (lbp_checkpoint_load, lbp_set_populations) before stepping on.             */
lbp_status lbp_set_wait_bound(lbp_sim *sim, int64_t cycles);

/* Failure probe for tests of the error path (no counterpart in the paper):
 * while enabled, the staged lattice kernel's consumers first wait on a
 * barrier that nothing completes, so that wait runs out after the bound of
 * lbp_set_wait_bound, the step's lattice pass is skipped and lbp_check
 * reports LBP_ETIMEOUT -- a device-side timeout made without a fault.  Other
 * kernel shapes have no device-side waits and ignore it.                    */
lbp_status lbp_set_wait_probe(lbp_sim *sim, int enable);

/* Diagnostics of the last completed step (waits for the handle's work):
 * out[0] = reaction-force shares that did not fit their row segment's record
 * and took the overflow path (both counts are implementation details of the
 * force accumulation; the results do not depend on them), out[1] = capacity of
 * a record in shares, out[2] = number of row segments, out[3] = rows of 128
 * nodes per lattice-kernel block, out[4] = its variant (see lbp_autotune),
 * out[5] = 1 if the particle kernel fits Eq. 8 with one lane per cell corner
 * (fewer than 48 particles per SM), 0 if with one thread per particle; both
 * layouts give the same bits.  n = entries of out (up to 6).                 */
lbp_status lbp_diagnostics(lbp_sim *sim, int64_t *out, int n);

/* Uniform body force density g = (gx, gy, gz) added on every node of box
 * `replica` (-1: every box) in the collision, as the force term of Eqs. 18-19
 * (3 w_a g.e_a per node, on top of the particles' reaction forces).  Used,
 * e.g., to hold a mean flow against the drag of pinned particles.  Stored
 * and applied in FP32.  Default 0.                                           */
lbp_status lbp_set_body_force(lbp_sim *sim, int replica, const double *g);

/* Kernel-shape autotuner of the fused stream-collide pass.  Times the kernel
 * this handle's steps launch (with the particle coupling if it has particles)
 * on its own lattice for each candidate and keeps the fastest for all later
 * steps.  Candidates (variant, rows):
 *   variant 0: one node per thread, 1, 2 or 4 rows of 128 nodes per block;
 *   variant 1: two neighbouring nodes per thread with 4-byte loads and stores,
 *              1, 2 or 4 rows (2-byte storage, every box with even nx);
 *   variant 2: persistent CTAs that stage each plane's source row segments in
 *              shared memory with bulk asynchronous copies (every box's nx a
 *              multiple of 16 bytes of storage: 4 for LBP_F32, 8 otherwise);
 *   variant 3: four neighbouring nodes per thread with 8-byte loads and
 *              stores, one warp per 128-node row segment, 1, 2 or 4 rows
 *              (2-byte storage, every box's nx a multiple of 4).
 * Each candidate runs `launches` back-to-back launches (1..1000) after two
 * warm-up launches, twice, best pass kept.  rows, variant (optional) receive
 * the pick; ms (optional, LBP_AUTOTUNE_CANDIDATES doubles) the mean launch
 * times in ms for (variant 0: 1, 2, 4 rows; variant 1: 1, 2, 4 rows;
 * variant 2; variant 3: 1, 2, 4 rows), -1 where a candidate does not apply.
 * The simulation state is unchanged: the launches read the current
 * populations, write only the buffer the next step overwrites, read a copy of
 * the last step's force records (all zero before the first step; run a few
 * steps first for timings that include the particle coupling) and bump a
 * scratch step counter.
 * Synchronous; LBP_ETIMEOUT if a bounded device wait ran out.  Default before
 * any call (the picks measured at 256^3): variant 0 with 2 rows for LBP_F32;
 * variant 3 with 1 row for the 2-byte types when every box's nx is a multiple
 * of 4, else variant 0 with 2 rows.                                          */
#define LBP_AUTOTUNE_CANDIDATES 10
lbp_status lbp_autotune(lbp_sim *sim, int launches, int *rows, int *variant, double *ms);

/* Fix the kernel shape by hand (LBP_EINVAL where the variant does not apply;
 * variant 2 ignores rows).  Results do not depend on the shape: each node's
 * arithmetic is the same in every variant.  lbp_set_block_rows changes the
 * rows only (leaving variant 2 for variant 0).                                */
lbp_status lbp_set_block_shape(lbp_sim *sim, int rows, int variant);
lbp_status lbp_set_block_rows(lbp_sim *sim, int rows);

/* Use CUDA graphs for lbp_step (default 1).                                  */
lbp_status lbp_set_use_graphs(lbp_sim *sim, int enable);

/* Kernel timing: while enabled, lbp_step records CUDA events around every
 * launch of the stream-collide kernel, and lbp_adjoint_backward around every
 * launch of the adjoint lattice kernel (not around its forward replay);
 * lbp_timing_read waits for them and returns the summed duration (ms) and the
 * number of launches since enable.                                           */
lbp_status lbp_timing_enable(lbp_sim *sim, int enable);
lbp_status lbp_timing_read(lbp_sim *sim, double *ms_total, int64_t *launches);

/* Philox-4x64-10 block function on the device (Salmon et al., SC'11), for
 * bit-exact checks: out[4 i + j] = word j of Philox(ctr[4 i .. 4 i + 3],
 * key[0..1]) for i < n.  All three pointers are device pointers.              */
lbp_status lbp_philox4x64_10(const uint64_t *ctr, const uint64_t *key, uint64_t *out,
                             int64_t n, void *stream);

/* VACF of a caller-supplied trajectory without any device allocation (the
 * paper has no counterpart: this is a service for callers that cannot call
 * cudaMalloc where they need the result, e.g. inside an allocator or memory
 * pool they do not control).  samples: device array [T][ncomp] of FP32
 * velocity components (any component order within a sample); outputs on the
 * device: csum[k] = sum over t0 <= T-1-k and all components of
 * samples[t0] * samples[t0 + k], counts[k] = npairs * (T - k) (0 if k >= T),
 * k = 0..max_lag -- the same estimator as lbp_vacf_read.  Products are FP32;
 * the products of one component over one block of at most 64 samples are
 * summed in FP32, every sum above that in FP64.  Scratch is a fixed 4 MiB
 * array inside the library, so ceil(ncomp / 1024) * (max_lag + 1) must not
 * exceed 524288, and ncomp must not exceed 65535 * 1024 (LBP_EINVAL
 * otherwise, with nothing queued).  The first call on a device looks up that
 * array's address and keeps it for the life of the process; make it before
 * capturing this routine into a CUDA graph, and do not use this routine on a
 * device after cudaDeviceReset (the kept address would be stale).  All calls
 * on a device share the array: calls that overlap on the GPU (different
 * streams, host threads) race and must be serialised by the caller.
 * Asynchronous on `stream`; outputs are zeroed by the call.                   */
lbp_status lbp_vacf_correlate_noalloc(const float *samples, int64_t T, int ncomp, int max_lag,
                                      int npairs, double *csum, int64_t *counts, void *stream);

/* ---------------------------------------------------------------- adjoint
 * Reverse-mode gradients of a run (no counterpart in the paper; the method's
 * step is differentiated as written: Eqs. 1-2, 4-5, 8-9, 12-20).
 *
 * lbp_adjoint_record runs nsteps >= 1 ordinary steps from the current state
 * (exactly as lbp_step would) and keeps, inside the handle, a checkpoint of the
 * populations and of the particle positions and velocities every
 * checkpoint_every >= 1 steps (memory: ceil(nsteps / checkpoint_every) copies
 * of the populations plus 48 bytes per particle each).  v_traj and r_traj
 * (optional, [nsteps][n_particles][3] FP64, host or device per on_device)
 * receive V^{n+1} and r^{n+1} after every step n: the trajectory a loss is
 * written on.  A new recording replaces the previous one.  Handles with at
 * least one particle (LBP_ESTATE without particles); single boxes and
 * batches of boxes alike.
 *
 * lbp_adjoint_backward takes dL/dV^{n+1} and dL/dr^{n+1} for every recorded
 * step (g_v, g_r: [nsteps][n_particles][3] FP64, either may be NULL = zero)
 * and returns, through the non-NULL members of grads, the gradient of L with
 * respect to the inputs of the recorded run: tau (one value per box), kT (one value),
 * each particle's gamma, radius and mass ([n_particles]), the velocities and
 * positions at the first recorded step ([n_particles][3]) and the populations
 * at the first recorded step ([15][N], ABI layout).  The reverse sweep
 * re-runs each segment between checkpoints forward from its checkpoint
 * (keeping that segment's later states: checkpoint_every - 1 population copies), then
 * steps the adjoint back through it; the handle's own state (populations,
 * particles, step index) is left as the recording left it.  Requires that no
 * step, particle change or new recording happened since lbp_adjoint_record
 * (LBP_ESTATE otherwise).  Where the method is not differentiable (a particle
 * changing cell, a corner skipped by the fit) the derivative is that of the
 * branch the forward run took.  Arithmetic: lattice adjoint in FP32, particle
 * adjoint and all accumulated gradients in FP64.  Results are bitwise
 * reproducible unless more than 8 particle-cell corners fall in one 128-node
 * row segment in one step (those extra contributions are then added with FP64
 * atomics).  Synchronous.                                                    */
typedef struct {
    double *tau;     /* [n_replicas]           dL/dtau of each box             */
    double *kT;      /* [1]                    dL/dkT                          */
    double *gamma;   /* [n_particles]          dL/dgamma_i                     */
    double *radius;  /* [n_particles]          dL/dR_i                         */
    double *mass;    /* [n_particles]          dL/dM_i                         */
    double *v0;      /* [n_particles][3]       dL/dV_i at the first step       */
    double *r0;      /* [n_particles][3]       dL/dr_i at the first step       */
    double *f0;      /* [15][N]                dL/df at the first step         */
} lbp_gradients;

lbp_status lbp_adjoint_record(lbp_sim *sim, int64_t nsteps, int checkpoint_every, double *v_traj,
                              double *r_traj, int on_device);
lbp_status lbp_adjoint_backward(lbp_sim *sim, const double *g_v, const double *g_r, int on_device,
                                const lbp_gradients *grads);

/* Message of the calling thread's last failing call ("" if none).            */
const char *lbp_last_error(void);

/* ABI version: 10000 * major + 100 * minor + patch.                          */
int lbp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBP_H */
