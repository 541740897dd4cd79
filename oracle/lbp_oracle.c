/*
 * lbp_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the
 * lattice-Boltzmann fluid coupled to Langevin point particles by the
 * Stokeslet fit (Yoshida, Kinjo & Washizu, "Numerical simulation method for
 * Brownian particles dispersed in incompressible fluids", arXiv:1909.13412).
 *
 * THIS IS TEST INFRASTRUCTURE.  It exists only to check the CUDA path.  Only
 * tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs
 * may load it.  It shares no code, header, table or helper with the CUDA
 * library; the two are written separately from the paper.
 *
 * Everything is written in the order and notation of Section 2 of the paper,
 * in lattice units dx = dt = C = rho0 = dV = 1:
 *   step n -> n+1:
 *     1. streaming (Eq. 20), pull form: f_a(x) = fhat_a(x - e_a), periodic box
 *     2. moments rho~ = sum_a f_a (Eq. 12), u = sum_a e_a f_a (Eq. 13)
 *     3. per particle, in id order: Stokeslet fit of Eq. 8 to u at the eight
 *        corners of the cell holding r_i (Section 2.1), F_H = gamma U_inf e^N
 *     4. random force F_R = sqrt(2 gamma kT) xi, xi from Philox-4x64-10
 *        (Eqs. 4-5)
 *     5. reaction force -F_H spread to the eight corners (Eq. 9) with
 *        trilinear weights of r_i^n
 *     6. Langevin update (Eqs. 1-2), semi-implicit Euler, dt = 1
 *     7. BGK collision with body force (Eqs. 14, 15, 17, 18, 19)
 *   The state kept between steps is the post-collision fhat.  The same step
 *   also runs in deviation form (or_set_deviation): the state is then
 *   g = fhat - w_a, streamed the same way, with the moments rho~ - 1 and u
 *   and the collision of or_collide_dev -- a self-check of that algebra.
 *
 * Readings where the paper is silent:
 *   D3Q15 table: e_0 = 0 (w 2/9), 6 faces (w 1/9), 8 corners (w 1/72).
 *   u is not divided by rho~ and rho~ multiplies only the leading term of
 *   f^eq (Eqs. 13, 17 literally).  The force term is plain 3 w_a F.e_a.
 *   u^N_p is the node velocity of the streamed (pre-collision) f.
 *   The "x" of Eq. 8 is e^N.d_p with d_p = x_p - r_i (unwrapped corner).
 *   If the mean relative velocity is exactly zero, U_inf = 0.
 *   Corners closer than 1e-12 to r_i are skipped; with exclude_inside set,
 *   corners with r_p < R are skipped as well.
 *   sigma^2 = 2 gamma kT; xi uniform on [-sqrt3, sqrt3] from 53-bit Philox
 *   output, independent over particles, components and steps.
 *
 * Build:  gcc -O2 -std=c11 -fPIC -shared -ffp-contract=off -fopenmp
 *         lbp_oracle.c -o liblbp_oracle.so -lm
 * (FMA contraction is off so that the noise and the cell geometry are the
 *  exact IEEE results of the expressions written here.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 15

/* ------------------------------------------------------------------ */
/* D3Q15 velocity set and weights (Section 2.2; the paper defers the   */
/* values to Succi's table).  Opposite directions are adjacent.        */
/* ------------------------------------------------------------------ */
static const int E[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0},
    {0, 1, 0}, {0, -1, 0},
    {0, 0, 1}, {0, 0, -1},
    {1, 1, 1}, {-1, -1, -1},
    {1, 1, -1}, {-1, -1, 1},
    {1, -1, 1}, {-1, 1, -1},
    {-1, 1, 1}, {1, -1, -1},
};
static const double W[Q] = {
    2.0 / 9.0,
    1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
    1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
    1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
};

void or_d3q15(int *e, double *w)
{
    for (int a = 0; a < Q; ++a) {
        for (int k = 0; k < 3; ++k) e[3 * a + k] = E[a][k];
        w[a] = W[a];
    }
}

static int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

static int64_t node(int x, int y, int z, int nx, int ny)
{
    return ((int64_t)z * ny + y) * nx + x;
}

/* ------------------------------------------------------------------ */
/* Eq. 20: streaming.  f_a(t+1, x + e_a) = fhat_a(t, x), periodic.     */
/* Written as a pull: f_a(x) = fhat_a(x - e_a).  Layout [a][z][y][x].  */
/* ------------------------------------------------------------------ */
void or_stream(const double *fhat, double *f, int nx, int ny, int nz)
{
    const int64_t N = (int64_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int a = 0; a < Q; ++a) {
                    int xs = wrap(x - E[a][0], nx);
                    int ys = wrap(y - E[a][1], ny);
                    int zs = wrap(z - E[a][2], nz);
                    f[a * N + node(x, y, z, nx, ny)] = fhat[a * N + node(xs, ys, zs, nx, ny)];
                }
}

/* Eqs. 12-13: rho~ = sum_a f_a ; u = sum_a C e_a f_a (C = 1, no 1/rho~). */
void or_moments(const double *f, double *rho, double *u, int64_t N)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0, ux = 0.0, uy = 0.0, uz = 0.0;
        for (int a = 0; a < Q; ++a) {
            double fa = f[a * N + i];
            s += fa;
            ux += E[a][0] * fa;
            uy += E[a][1] * fa;
            uz += E[a][2] * fa;
        }
        rho[i] = s;
        u[i] = ux;
        u[N + i] = uy;
        u[2 * N + i] = uz;
    }
}

/* Eq. 17: f^eq_a = w_a [rho~ + 3 u.e_a + 9/2 (u.e_a)^2 - 3/2 u.u]  (C = 1). */
void or_feq(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int a = 0; a < Q; ++a) {
        double eu = E[a][0] * u[0] + E[a][1] * u[1] + E[a][2] * u[2];
        feq[a] = W[a] * (rho + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Eqs. 14, 15, 18, 19: fhat_a = f_a + (f^eq_a - f_a)/tau + w_a G_a,
 * G_a = 3 F.e_a / (rho0 C) with rho0 = C = dt = 1.  F is the force density
 * on the fluid ([3][N], may be NULL).                                      */
void or_collide(const double *f, const double *rho, const double *u, const double *F,
                double tau, int64_t N, double *fhat)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double ui[3] = {u[i], u[N + i], u[2 * N + i]};
        double feq[Q];
        or_feq(rho[i], ui, feq);
        for (int a = 0; a < Q; ++a) {
            double G = 0.0;
            if (F) G = 3.0 * (F[i] * E[a][0] + F[N + i] * E[a][1] + F[2 * N + i] * E[a][2]);
            double Qa = (feq[a] - f[a * N + i]) / tau;
            fhat[a * N + i] = f[a * N + i] + Qa + W[a] * G;
        }
    }
}

/* The same collision in deviation form, g = f - w_a (a self-check of the
 * algebra the storage of the GPU path relies on).  With sum_a w_a = 1 and
 * sum_a w_a e_a = 0, the moments of g are rho~ - 1 (drho) and u, and
 * f^eq_a - w_a = w_a [(rho~ - 1) + 3 u.e_a + 9/2 (u.e_a)^2 - 3/2 u.u], so
 * ghat_a = g_a + (g^eq_a - g_a)/tau + w_a G_a is fhat_a - w_a exactly.   */
void or_collide_dev(const double *g, const double *drho, const double *u, const double *F,
                    double tau, int64_t N, double *ghat)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double ux = u[i], uy = u[N + i], uz = u[2 * N + i];
        double uu = ux * ux + uy * uy + uz * uz;
        for (int a = 0; a < Q; ++a) {
            double eu = E[a][0] * ux + E[a][1] * uy + E[a][2] * uz;
            double geq = W[a] * (drho[i] + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
            double G = 0.0;
            if (F) G = 3.0 * (F[i] * E[a][0] + F[N + i] * E[a][1] + F[2 * N + i] * E[a][2]);
            ghat[a * N + i] = g[a * N + i] + (geq - g[a * N + i]) / tau + W[a] * G;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Geometry of the eight corners x_p around r (Section 2.1).           */
/* base = floor(r); corner p = (cx, cy, cz) with p = cx + 2 cy + 4 cz; */
/* frac = r - base; d_p = x_p - r = c - frac (unwrapped);               */
/* trilinear weight W_p = prod_k (c_k ? frac_k : 1 - frac_k).           */
/* ------------------------------------------------------------------ */
void or_corners(const double *r, int *base, double *d, double *Wp)
{
    double frac[3];
    for (int k = 0; k < 3; ++k) {
        double b = floor(r[k]);
        base[k] = (int)b;
        frac[k] = r[k] - b;
    }
    for (int p = 0; p < 8; ++p) {
        int c[3] = {p & 1, (p >> 1) & 1, (p >> 2) & 1};
        double w = 1.0;
        for (int k = 0; k < 3; ++k) {
            d[3 * p + k] = c[k] ? 1.0 - frac[k] : -frac[k];
            w = w * (c[k] ? frac[k] : 1.0 - frac[k]);
        }
        Wp[p] = w;
    }
}

/* ------------------------------------------------------------------ */
/* Stokeslet fit, Eq. 8 and the text after it (Section 2.1).           */
/* Input: d_p (corner minus particle), u^N_p, particle V, radius R.    */
/* w_p = u^N_p - V;  e^N = mean(w_p)/|mean(w_p)|;                       */
/* u^A(d) = U [(1 - 3R/(4r)) e^N - 3R (e^N.d)/(4 r^3) d];              */
/* U_inf minimises sum_p |w_p - u^A(d_p)|^2, i.e.                       */
/*   U_inf = sum_p w_p.a_p / sum_p |a_p|^2,  a_p = u^A(d_p)/U.          */
/* Returns U_inf, writes e^N.  F_H = gamma U_inf e^N (from Eq. 7 with  */
/* u_inf = U_inf e^N + V).                                              */
/* ------------------------------------------------------------------ */
double or_stokeslet_fit(const double *d, const double *uN, const double *V, double R,
                        int exclude_inside, double *eN)
{
    double w[8][3], wm[3] = {0.0, 0.0, 0.0};
    for (int p = 0; p < 8; ++p)
        for (int k = 0; k < 3; ++k) {
            w[p][k] = uN[3 * p + k] - V[k];
            wm[k] += w[p][k];
        }
    for (int k = 0; k < 3; ++k) wm[k] = wm[k] / 8.0;
    double nw = sqrt(wm[0] * wm[0] + wm[1] * wm[1] + wm[2] * wm[2]);
    if (nw == 0.0) {
        eN[0] = eN[1] = eN[2] = 0.0;
        return 0.0;
    }
    for (int k = 0; k < 3; ++k) eN[k] = wm[k] / nw;
    double num = 0.0, den = 0.0;
    for (int p = 0; p < 8; ++p) {
        const double *dp = d + 3 * p;
        double rp = sqrt(dp[0] * dp[0] + dp[1] * dp[1] + dp[2] * dp[2]);
        if (rp < 1e-12) continue;
        if (exclude_inside && rp < R) continue;
        double x = eN[0] * dp[0] + eN[1] * dp[1] + eN[2] * dp[2];
        double c1 = 1.0 - 3.0 * R / (4.0 * rp);
        double c2 = 3.0 * R * x / (4.0 * rp * rp * rp);
        double a[3];
        for (int k = 0; k < 3; ++k) a[k] = c1 * eN[k] - c2 * dp[k];
        num += w[p][0] * a[0] + w[p][1] * a[1] + w[p][2] * a[2];
        den += a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    }
    if (den == 0.0) return 0.0;
    return num / den;
}

/* ------------------------------------------------------------------ */
/* Philox-4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11), written from   */
/* the published round function: two 64x64->128 multiplications per   */
/* round with the multipliers and Weyl key increments of that paper.   */
/* ------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    /* 64x64 -> 128 by 32-bit halves, portable C */
    uint64_t a0 = a & 0xffffffffu, a1 = a >> 32;
    uint64_t b0 = b & 0xffffffffu, b1 = b >> 32;
    uint64_t p00 = a0 * b0, p01 = a0 * b1, p10 = a1 * b0, p11 = a1 * b1;
    uint64_t mid = (p00 >> 32) + (p01 & 0xffffffffu) + (p10 & 0xffffffffu);
    *lo = (mid << 32) | (p00 & 0xffffffffu);
    *hi = p11 + (p01 >> 32) + (p10 >> 32) + (mid >> 32);
}

void or_philox4x64_10(const uint64_t *ctr_in, const uint64_t *key_in, uint64_t *out)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c[0], &hi0, &lo0);
        mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c[3] ^ k1;
        uint64_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Random force direction numbers for (step, particle): counter
 * (step, pid, 0, 0), key (seed, 0).  xi_k = sqrt3 (2 u_k - 1) with
 * u_k = ((x_k >> 11) + 1/2) 2^-53: zero mean, unit variance.             */
void or_noise_xi(uint64_t seed, uint64_t step, uint64_t pid, double *xi)
{
    uint64_t ctr[4] = {step, pid, 0, 0}, key[2] = {seed, 0}, x[4];
    or_philox4x64_10(ctr, key, x);
    const double s3 = sqrt(3.0);
    for (int k = 0; k < 3; ++k) {
        double u = ((double)(x[k] >> 11) + 0.5) * 0x1.0p-53;
        xi[k] = s3 * (2.0 * u - 1.0);
    }
}

/* ------------------------------------------------------------------ */
/* The simulated system: periodic nx*ny*nz box, relaxation time tau,  */
/* fhat (post-collision) [15][N], particles (AoS [n][3]).             */
/* ------------------------------------------------------------------ */
enum { OR_STOKESLET = 0, OR_POINTWISE = 1, OR_BROWNIAN = 2 };

typedef struct {
    int nx, ny, nz;
    int64_t N;
    double tau;
    double *fhat, *f, *rho, *u, *F;
    int np, cap;
    double *r, *V, *M, *gamma, *R, *Fext, *FH, *FR;
    unsigned char *pinned;
    double kT;
    uint64_t seed;
    int mode, exclude_inside;
    int64_t step;
    double G[3]; /* uniform body force density on every node (Eq. 18) */
    int deviation; /* fhat, f hold g = f - w_a, and rho holds rho~ - 1 */
} or_sim;

or_sim *or_create(int nx, int ny, int nz, double tau)
{
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    s->nx = nx; s->ny = ny; s->nz = nz;
    s->N = (int64_t)nx * ny * nz;
    s->tau = tau;
    s->fhat = (double *)malloc(sizeof(double) * Q * s->N);
    s->f = (double *)malloc(sizeof(double) * Q * s->N);
    s->rho = (double *)malloc(sizeof(double) * s->N);
    s->u = (double *)malloc(sizeof(double) * 3 * s->N);
    s->F = (double *)malloc(sizeof(double) * 3 * s->N);
    /* fluid at rest, rho~ = 1: f = f^eq(1, 0) = w_a */
    for (int a = 0; a < Q; ++a)
        for (int64_t i = 0; i < s->N; ++i) s->fhat[a * s->N + i] = W[a];
    return s;
}

void or_destroy(or_sim *s)
{
    if (!s) return;
    free(s->fhat); free(s->f); free(s->rho); free(s->u); free(s->F);
    free(s->r); free(s->V); free(s->M); free(s->gamma); free(s->R);
    free(s->Fext); free(s->FH); free(s->FR); free(s->pinned);
    free(s);
}

/* fhat in and out is always the full population; in deviation form the
 * state keeps fhat - w_a.                                                */
void or_set_fhat(or_sim *s, const double *fhat)
{
    for (int a = 0; a < Q; ++a)
        for (int64_t i = 0; i < s->N; ++i)
            s->fhat[a * s->N + i] = s->deviation ? fhat[a * s->N + i] - W[a] : fhat[a * s->N + i];
}
void or_get_fhat(const or_sim *s, double *fhat)
{
    for (int a = 0; a < Q; ++a)
        for (int64_t i = 0; i < s->N; ++i)
            fhat[a * s->N + i] = s->deviation ? s->fhat[a * s->N + i] + W[a] : s->fhat[a * s->N + i];
}
/* Switch the stored state between full and deviation form. */
void or_set_deviation(or_sim *s, int on)
{
    on = on != 0;
    if (on == s->deviation) return;
    for (int a = 0; a < Q; ++a)
        for (int64_t i = 0; i < s->N; ++i) s->fhat[a * s->N + i] += on ? -W[a] : W[a];
    s->deviation = on;
}
void or_set_step(or_sim *s, int64_t step) { s->step = step; }
int64_t or_get_step(const or_sim *s) { return s->step; }

/* Moments of the streamed distribution f^n = S fhat^{n-1} (what the
 * particles see at the next step), and p = C^2 rho0 rho~/3.             */
void or_get_fields(or_sim *s, double *rho, double *u, double *p)
{
    or_stream(s->fhat, s->f, s->nx, s->ny, s->nz);
    or_moments(s->f, rho, u, s->N);
    if (s->deviation)
        for (int64_t i = 0; i < s->N; ++i) rho[i] += 1.0;
    if (p)
        for (int64_t i = 0; i < s->N; ++i) p[i] = rho[i] / 3.0;
}

static void *grow(void *p, size_t bytes) { return realloc(p, bytes); }

void or_add_particles(or_sim *s, int n, const double *r, const double *V, const double *M,
                      const double *gamma, const double *R)
{
    int np = s->np + n;
    s->r = (double *)grow(s->r, sizeof(double) * 3 * np);
    s->V = (double *)grow(s->V, sizeof(double) * 3 * np);
    s->M = (double *)grow(s->M, sizeof(double) * np);
    s->gamma = (double *)grow(s->gamma, sizeof(double) * np);
    s->R = (double *)grow(s->R, sizeof(double) * np);
    s->Fext = (double *)grow(s->Fext, sizeof(double) * 3 * np);
    s->FH = (double *)grow(s->FH, sizeof(double) * 3 * np);
    s->FR = (double *)grow(s->FR, sizeof(double) * 3 * np);
    s->pinned = (unsigned char *)grow(s->pinned, np);
    for (int i = 0; i < n; ++i) {
        int j = s->np + i;
        for (int k = 0; k < 3; ++k) {
            s->r[3 * j + k] = r[3 * i + k];
            s->V[3 * j + k] = V[3 * i + k];
            s->Fext[3 * j + k] = 0.0;
            s->FH[3 * j + k] = 0.0;
            s->FR[3 * j + k] = 0.0;
        }
        s->M[j] = M[i];
        s->gamma[j] = gamma[i];
        s->R[j] = R[i];
        s->pinned[j] = 0;
    }
    s->np = np;
}

void or_set_params(or_sim *s, double kT, uint64_t seed, int mode, int exclude_inside)
{
    s->kT = kT; s->seed = seed; s->mode = mode; s->exclude_inside = exclude_inside;
}

void or_set_external(or_sim *s, const double *Fext, const unsigned char *pinned)
{
    for (int j = 0; j < s->np; ++j) {
        for (int k = 0; k < 3; ++k) s->Fext[3 * j + k] = Fext ? Fext[3 * j + k] : 0.0;
        s->pinned[j] = pinned ? pinned[j] : 0;
    }
}

/* Uniform external force density on the fluid, added to F of Eq. 18 on every
 * node (e.g. to hold a mean flow against the drag of a pinned particle). */
void or_set_body_force(or_sim *s, const double *G)
{
    for (int k = 0; k < 3; ++k) s->G[k] = G[k];
}

void or_set_particles(or_sim *s, const double *r, const double *V)
{
    if (r) memcpy(s->r, r, sizeof(double) * 3 * s->np);
    if (V) memcpy(s->V, V, sizeof(double) * 3 * s->np);
}

void or_get_particles(const or_sim *s, double *r, double *V, double *FH, double *FR)
{
    if (r) memcpy(r, s->r, sizeof(double) * 3 * s->np);
    if (V) memcpy(V, s->V, sizeof(double) * 3 * s->np);
    if (FH) memcpy(FH, s->FH, sizeof(double) * 3 * s->np);
    if (FR) memcpy(FR, s->FR, sizeof(double) * 3 * s->np);
}

/* One time step n -> n+1 in the order stated at the top of this file. */
static void one_step(or_sim *s)
{
    const int nx = s->nx, ny = s->ny, nz = s->nz;
    const int64_t N = s->N;
    const int L[3] = {nx, ny, nz};

    /* 1-2: streaming and moments of f^n */
    or_stream(s->fhat, s->f, nx, ny, nz);
    or_moments(s->f, s->rho, s->u, N);
    /* force density on the fluid: the uniform body force, then the particles' */
    for (int k = 0; k < 3; ++k)
        for (int64_t i = 0; i < N; ++i) s->F[k * N + i] = s->G[k];

    for (int i = 0; i < s->np; ++i) {
        double *r = s->r + 3 * i, *V = s->V + 3 * i;
        int base[3];
        double d[24], Wp[8], uN[24];
        or_corners(r, base, d, Wp);
        int64_t idx[8];
        for (int p = 0; p < 8; ++p) {
            int x = wrap(base[0] + (p & 1), nx);
            int y = wrap(base[1] + ((p >> 1) & 1), ny);
            int z = wrap(base[2] + ((p >> 2) & 1), nz);
            idx[p] = node(x, y, z, nx, ny);
            for (int k = 0; k < 3; ++k) uN[3 * p + k] = s->u[k * N + idx[p]];
        }
        /* 3: friction force */
        double FH[3] = {0.0, 0.0, 0.0};
        int spread = 1;
        if (s->mode == OR_STOKESLET) {
            double eN[3];
            double Uinf = or_stokeslet_fit(d, uN, V, s->R[i], s->exclude_inside, eN);
            for (int k = 0; k < 3; ++k) FH[k] = s->gamma[i] * Uinf * eN[k];
        } else if (s->mode == OR_POINTWISE) {
            /* Eq. 7 with u(r_i) interpolated trilinearly from the corners */
            for (int k = 0; k < 3; ++k) {
                double ur = 0.0;
                for (int p = 0; p < 8; ++p) ur += Wp[p] * uN[3 * p + k];
                FH[k] = -s->gamma[i] * (V[k] - ur);
            }
        } else {
            /* Eq. 6: fluid taken at rest, nothing returned to the fluid */
            for (int k = 0; k < 3; ++k) FH[k] = -s->gamma[i] * V[k];
            spread = 0;
        }
        /* 4: random force, sigma^2 = 2 gamma kT */
        double xi[3], sig = sqrt(2.0 * s->gamma[i] * s->kT);
        or_noise_xi(s->seed, (uint64_t)s->step, (uint64_t)i, xi);
        for (int k = 0; k < 3; ++k) {
            s->FH[3 * i + k] = FH[k];
            s->FR[3 * i + k] = sig * xi[k];
        }
        /* 5: reaction force density -F_H / dV spread with weights W_p */
        if (spread)
            for (int p = 0; p < 8; ++p)
                for (int k = 0; k < 3; ++k) s->F[k * N + idx[p]] += -FH[k] * Wp[p];
        /* 6: Langevin update, dt = 1: V += (F_H + F_R + F_ext)/M; r += V */
        if (!s->pinned[i]) {
            for (int k = 0; k < 3; ++k) {
                V[k] = V[k] + (FH[k] + s->FR[3 * i + k] + s->Fext[3 * i + k]) / s->M[i];
                r[k] = r[k] + V[k];
                if (r[k] < 0.0) r[k] += L[k];
                if (r[k] >= L[k]) r[k] -= L[k];
            }
        }
    }
    /* 7: collision with the body force */
    if (s->deviation)
        or_collide_dev(s->f, s->rho, s->u, s->F, s->tau, N, s->fhat);
    else
        or_collide(s->f, s->rho, s->u, s->F, s->tau, N, s->fhat);
    s->step += 1;
}

void or_step(or_sim *s, int64_t nsteps)
{
    for (int64_t n = 0; n < nsteps; ++n) one_step(s);
}

/* Force density that the particles of the current state would put on the
 * fluid at this step (step 5 alone, from the streamed u); for tests.     */
void or_spread_only(or_sim *s, double *F)
{
    const int64_t N = s->N;
    or_stream(s->fhat, s->f, s->nx, s->ny, s->nz);
    or_moments(s->f, s->rho, s->u, N);
    memset(F, 0, sizeof(double) * 3 * N);
    for (int i = 0; i < s->np; ++i) {
        int base[3];
        double d[24], Wp[8];
        or_corners(s->r + 3 * i, base, d, Wp);
        for (int p = 0; p < 8; ++p) {
            int64_t j = node(wrap(base[0] + (p & 1), s->nx), wrap(base[1] + ((p >> 1) & 1), s->ny),
                             wrap(base[2] + ((p >> 2) & 1), s->nz), s->nx, s->ny);
            for (int k = 0; k < 3; ++k) F[k * N + j] += -s->FH[3 * i + k] * Wp[p];
        }
    }
}

/* ------------------------------------------------------------------ */
/* VACF estimator (Section 3): C(k) = sum over particles i and origins */
/* t0 (every `stride`-th sample) with t0 + k < T of V_i(t0).V_i(t0+k). */
/* V is [T][np][3].  Writes the sums and the number of (i, t0) pairs.  */
/* ------------------------------------------------------------------ */
void or_vacf(const double *V, int64_t T, int np, int K, int stride, double *csum, int64_t *count)
{
    for (int k = 0; k <= K; ++k) {
        double s = 0.0;
        int64_t c = 0;
        for (int64_t t0 = 0; t0 + k < T; t0 += stride)
            for (int i = 0; i < np; ++i) {
                const double *a = V + (t0 * np + i) * 3, *b = V + ((t0 + k) * np + i) * 3;
                s += a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
                c += 1;
            }
        csum[k] = s;
        count[k] = c;
    }
}

/* ------------------------------------------------------------------ */
/* Mean squared displacement of the particles (the dispersion that the */
/* Brownian analysis of Section 3 accompanies the VACF with):          */
/* M(k) = sum over particles i and origins t0 with t0 + k < T of       */
/* |X_i(t0 + k) - X_i(t0)|^2, X [T][np][3] unwrapped positions (the    */
/* sum of the displacements r^{n+1} - r^n = V^{n+1} of Eq. 2, without  */
/* the periodic wrap).  Writes the sums and the numbers of pairs.      */
/* ------------------------------------------------------------------ */
void or_msd(const double *X, int64_t T, int np, int K, double *msum, int64_t *count)
{
    for (int k = 0; k <= K; ++k) {
        double s = 0.0;
        int64_t c = 0;
        for (int64_t t0 = 0; t0 + k < T; ++t0)
            for (int i = 0; i < np; ++i) {
                const double *a = X + (t0 * np + i) * 3, *b = X + ((t0 + k) * np + i) * 3;
                const double d0 = b[0] - a[0], d1 = b[1] - a[1], d2 = b[2] - a[2];
                s += d0 * d0 + d1 * d1 + d2 * d2;
                c += 1;
            }
        msum[k] = s;
        count[k] = c;
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the OpenMP loops over z-planes (timing only; the results do not
 * depend on it: every node and particle is computed by one thread). */
void or_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
